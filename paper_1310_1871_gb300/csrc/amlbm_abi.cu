// Host side of the C ABI declared in include/amlbm.h: validation, the device
// arena, kernel launches, CUDA-graph chunks of timesteps, read-back and
// diagnostics.  Every entry point returns a status code and never throws.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "amlbm.h"
#include "amlbm_internal.cuh"

using amlbm::InstDesc;

namespace amlbm {
// The amlbm_diag of a diagnostics result out[16] (h) after `steps` steps.
void fill_diag(const double* h, long long steps, amlbm_diag* out) {
  std::memset(out, 0, sizeof(*out));
  out->mass2d = h[0]; out->mass3d = h[1]; out->momz3d = h[2]; out->Eke = h[3]; out->umax = h[4];
  out->a2 = h[5]; out->A = h[6]; out->neck = h[7]; out->p_in = h[8]; out->p_out = h[9];
  out->dp = h[10]; out->bad = h[11]; out->sumS = h[12];
  out->steps = (double)steps;
}

// The diagnostics parameters used when the caller passes none.
amlbm_diag_params diag_defaults(const InstDesc& d) {
  amlbm_diag_params p;
  p.zc = d.Nz / 2.0; p.R = 1.0; p.rho_l = 2.0; p.rho_v = 0.1;
  return p;
}

// The same error for a state whose diagnostics found bad sites, from every
// diagnostics entry point.
std::string unstable_message(double bad) {
  return "non-finite or non-positive density at " + std::to_string((long long)bad) + " sites";
}
}  // namespace amlbm
using amlbm::diag_defaults;
using amlbm::fill_diag;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define AMLBM_CK(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(AMLBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int pitch_of(int Nz) { return (Nz + 31) / 32 * 32; }
size_t elem_bytes(int storage) {
  return storage == AMLBM_STORE_F64 ? 8 : storage == AMLBM_STORE_F32 ? 4 : 2;
}
size_t compute_bytes(int storage) { return storage == AMLBM_STORE_F64 ? 8 : 4; }

amlbm_bc default_bc() {
  amlbm_bc b;
  b.wall_r = AMLBM_WALL_FREESLIP;
  b.axisym = 1;
  b.src_mode = AMLBM_SRC_LOCAL;
  b.storage = AMLBM_STORE_F64;
  b.shift = AMLBM_SHIFT_DEFAULT;
  b.rounding = AMLBM_ROUND_DEFAULT;
  b.g_z = 0.0;
  b.rho_ref = 1.0;
  b.z_bc = AMLBM_Z_PERIODIC;
  b.r_lo = AMLBM_RLO_AXIS;
  b.r_off = 0.0;
  b.rho_out = 1.0;
  b.forcing = AMLBM_FORCE_SHIFT;
  return b;
}

// A lattice with walls in z, an inlet or an outlet, or with the Guo forcing:
// the fused schedule only.
bool bounded(const amlbm_bc& bc) {
  return bc.z_bc != AMLBM_Z_PERIODIC || bc.r_lo != AMLBM_RLO_AXIS || bc.wall_r == AMLBM_WALL_OUTLET ||
         bc.forcing != AMLBM_FORCE_SHIFT;
}

// A lattice the pair schedule takes: periodic in z with an even Nz, the axis
// below row 0, a reflecting or bounce-back outer wall, the source at the
// departure site, and element offsets of all nine planes within 32 bits.
bool pair_ok(const amlbm_instance& I) {
  return I.bc.z_bc == AMLBM_Z_PERIODIC && I.bc.r_lo == AMLBM_RLO_AXIS &&
         (I.bc.wall_r == AMLBM_WALL_FREESLIP || I.bc.wall_r == AMLBM_WALL_NOSLIP) &&
         I.bc.src_mode == AMLBM_SRC_LOCAL && I.Nz % 2 == 0 &&
         9LL * pitch_of(I.Nz) * I.Nr < (1LL << 31);
}
bool all_pair_ok(const std::vector<amlbm_instance>& inst) {
  for (const auto& I : inst)
    if (!pair_ok(I)) return false;
  return true;
}

// Schedule and tile when the caller gives none (fastest on the 64-drop sweep on
// GB300): the FP32-arithmetic forms take the pair schedule where every lattice
// allows it (else the fused one), with the first tile of a preference list that
// still gives every SM two CTAs over the whole batch; the FP64 form, bound by
// FP64 arithmetic, takes the split schedule (less recomputation).
void pick_tile(int storage, const std::vector<amlbm_instance>& inst, int* sched, int* tz, int* tr) {
  static const int pref64[][2] = {{32, 16}, {32, 8}, {32, 8}};
  static const int pref64f[][2] = {{32, 8}, {32, 8}, {32, 8}};  // fused, for bounded lattices
  static const int pref32[][2] = {{26, 16}, {64, 8}, {32, 8}};
  static const int prefpair[][2] = {{64, 24}, {40, 24}, {24, 16}};
  bool any_bounded = false;
  for (const auto& I : inst) any_bounded = any_bounded || bounded(I.bc);
  const bool f64 = storage == AMLBM_STORE_F64;
  const bool pair = !f64 && all_pair_ok(inst);
  const int(*pref)[2] = f64 ? (any_bounded ? pref64f : pref64) : pair ? prefpair : pref32;
  *sched = f64 && !any_bounded ? amlbm::SCHED_SPLIT : pair ? amlbm::SCHED_PAIR : amlbm::SCHED_FUSED;
  for (int c = 0; c < 3; ++c) {
    const int z = pref[c][0], r = pref[c][1];
    long long tiles = 0;
    for (const auto& I : inst) tiles += (long long)((I.Nz + z - 1) / z) * ((I.Nr + r - 1) / r);
    if (tiles >= 2 * 152) { *tz = z; *tr = r; return; }
  }
  *sched = f64 && !any_bounded ? amlbm::SCHED_SPLIT : amlbm::SCHED_FUSED;
  *tz = 32;
  *tr = 8;
}

// Shift code the kernels use: 0 none, 1 global rho_ref, 2 local (from psi),
// 3 equilibrium (local s and the stored velocity).
int resolve_shift(const amlbm_bc& bc) {
  if (bc.storage == AMLBM_STORE_F64) return 0;
  switch (bc.shift) {
    case AMLBM_SHIFT_NONE: return 0;
    case AMLBM_SHIFT_GLOBAL: return 1;
    case AMLBM_SHIFT_LOCAL: return 2;
    case AMLBM_SHIFT_EQUILIBRIUM: return 3;
    default: return bc.storage == AMLBM_STORE_F32 ? 0 : 2;
  }
}
// Planes of the compute type per psi copy: psi, and v_z, v_r for the equilibrium shift.
int psi_planes(int shift_code) { return shift_code == 3 ? 3 : 1; }

int validate(const amlbm_instance& I, int idx) {
  const std::string w = "instance " + std::to_string(idx) + ": ";
  if (I.Nz < 1 || I.Nr < 4 || I.Nz > (1 << 20) || I.Nr > (1 << 20) ||
      (long long)I.Nz * I.Nr > (1LL << 30))
    return fail(AMLBM_EINVAL, w + "need 1 <= Nz, 4 <= Nr, Nz*Nr <= 2^30");
  if (!(I.tau > 0.5) || !std::isfinite(I.tau)) return fail(AMLBM_EINVAL, w + "tau must exceed 1/2");
  if (!(I.rho0 > 0) || !std::isfinite(I.rho0)) return fail(AMLBM_EINVAL, w + "rho0 must be positive");
  if (!(I.G >= -6.5) || !std::isfinite(I.G))
    return fail(AMLBM_EINVAL, w + "G below -6.5 (the Shan-Chen model is unstable beyond G ~ -6)");
  if (I.bc.wall_r != AMLBM_WALL_FREESLIP && I.bc.wall_r != AMLBM_WALL_NOSLIP &&
      I.bc.wall_r != AMLBM_WALL_OUTLET)
    return fail(AMLBM_EINVAL, w + "bad wall_r");
  if (I.bc.z_bc != AMLBM_Z_PERIODIC && I.bc.z_bc != AMLBM_Z_NOSLIP) return fail(AMLBM_EINVAL, w + "bad z_bc");
  if (I.bc.forcing != AMLBM_FORCE_SHIFT && I.bc.forcing != AMLBM_FORCE_GUO)
    return fail(AMLBM_EINVAL, w + "bad forcing");
  if (I.bc.r_lo != AMLBM_RLO_AXIS && I.bc.r_lo != AMLBM_RLO_INLET) return fail(AMLBM_EINVAL, w + "bad r_lo");
  if (!(I.bc.r_off >= 0.0) || !std::isfinite(I.bc.r_off) || I.bc.r_off > 1e6)
    return fail(AMLBM_EINVAL, w + "r_off must be finite, >= 0 and <= 1e6");
  if (I.bc.r_lo == AMLBM_RLO_AXIS && I.bc.r_off != 0.0)
    return fail(AMLBM_EINVAL, w + "a lattice on the axis has r_off = 0");
  if (I.bc.wall_r == AMLBM_WALL_OUTLET && (!(I.bc.rho_out > 0) || !std::isfinite(I.bc.rho_out)))
    return fail(AMLBM_EINVAL, w + "the outlet density rho_out must be positive and finite");
  if (I.bc.z_bc == AMLBM_Z_NOSLIP && I.Nz < 4) return fail(AMLBM_EINVAL, w + "z walls need Nz >= 4");
  if ((I.bc.r_lo == AMLBM_RLO_INLET || I.bc.wall_r == AMLBM_WALL_OUTLET) && I.Nr < 6)
    return fail(AMLBM_EINVAL, w + "inlet or outlet rows need Nr >= 6");
  if (I.bc.axisym != 0 && I.bc.axisym != 1) return fail(AMLBM_EINVAL, w + "axisym must be 0 or 1");
  if (I.bc.src_mode != AMLBM_SRC_LOCAL && I.bc.src_mode != AMLBM_SRC_LINK)
    return fail(AMLBM_EINVAL, w + "bad src_mode");
  if (I.bc.storage < AMLBM_STORE_F64 || I.bc.storage > AMLBM_STORE_BF16)
    return fail(AMLBM_EINVAL, w + "bad storage");
  if (I.bc.shift < AMLBM_SHIFT_DEFAULT || I.bc.shift > AMLBM_SHIFT_EQUILIBRIUM)
    return fail(AMLBM_EINVAL, w + "bad shift");
  if (I.bc.storage == AMLBM_STORE_F64 && I.bc.shift > AMLBM_SHIFT_NONE)
    return fail(AMLBM_EINVAL, w + "FP64 storage is not shifted");
  if (I.bc.rounding < AMLBM_ROUND_DEFAULT || I.bc.rounding > AMLBM_ROUND_STOCHASTIC)
    return fail(AMLBM_EINVAL, w + "bad rounding");
  if (!std::isfinite(I.bc.g_z) || !std::isfinite(I.bc.rho_ref))
    return fail(AMLBM_EINVAL, w + "g_z and rho_ref must be finite");
  return AMLBM_OK;
}

struct Layout {
  size_t total = 0;
  size_t desc = 0, tiles = 0, rb_tiles = 0, ctr = 0, diag_part = 0, diag_cols = 0, diag_out = 0, upload = 0,
         unpack = 0, site_off = 0, diag_jobs = 0, diag_blkjob = 0;
  std::vector<size_t> f0, f1, p0, p1, uv, rho, uz, ur, inlet;
  int ntiles = 0, rb_ntiles = 0, maxN = 0, maxNz = 0, diag_nblk = 1;
  int all_nblk = 0;  // partial-sum blocks of a diagnostics pass over every instance
  long long sumN = 0, sumNz = 0;
};

// Tile of the read-back kernel: a pair batch reads back with the pair schedule's
// kernel on its step tile, every other batch with the fused read-back (rb_tile()).
void rb_tiling(int storage, int sched, int tz, int tr, int* rz, int* rr) {
  if (sched == amlbm::SCHED_PAIR) {
    *rz = tz;
    *rr = tr;
  } else {
    amlbm::rb_tile(storage, rz, rr);
  }
}

Layout make_layout(const std::vector<amlbm_instance>& inst, int storage, int tz, int tr, int sched) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes); return at; };
  const size_t n = inst.size();
  for (const auto& I : inst) {
    L.ntiles += ((I.Nz + tz - 1) / tz) * ((I.Nr + tr - 1) / tr);
    int rz, rr;
    rb_tiling(storage, sched, tz, tr, &rz, &rr);
    L.rb_ntiles += ((I.Nz + rz - 1) / rz) * ((I.Nr + rr - 1) / rr);
    L.maxN = std::max(L.maxN, I.Nz * I.Nr);
    L.maxNz = std::max(L.maxNz, I.Nz);
    L.diag_nblk = std::max(L.diag_nblk, amlbm::diag_blocks(I.Nz, I.Nr));
    L.all_nblk += amlbm::diag_blocks(I.Nz, I.Nr);
    L.sumN += (long long)I.Nz * I.Nr;
    L.sumNz += I.Nz;
  }
  L.desc = take(n * sizeof(InstDesc));
  L.tiles = take((size_t)L.ntiles * sizeof(int));
  L.rb_tiles = take((size_t)L.rb_ntiles * sizeof(int));
  L.ctr = take(5 * sizeof(int));  // two tile counters, two step counters, the init check count
  L.diag_part = take((size_t)std::max(L.diag_nblk, L.all_nblk) * 8 * sizeof(double));
  L.diag_cols = take((size_t)L.sumNz * sizeof(double));
  L.diag_out = take(16 * n * sizeof(double));
  L.diag_jobs = take(n * sizeof(amlbm::DiagJob));
  L.diag_blkjob = take((size_t)std::max(1, L.all_nblk) * sizeof(int));
  L.site_off = take((n + 1) * sizeof(long long));
  L.upload = take((size_t)3 * L.sumN * sizeof(double));
  L.unpack = take((size_t)9 * L.maxN * sizeof(double));
  for (const auto& I : inst) {
    const size_t plane = (size_t)pitch_of(I.Nz) * I.Nr;
    L.f0.push_back(take(9 * plane * elem_bytes(storage)));
    L.f1.push_back(take(9 * plane * elem_bytes(storage)));
    const size_t pp = plane * compute_bytes(storage) * psi_planes(resolve_shift(I.bc));
    L.p0.push_back(take(pp));
    L.p1.push_back(take(pp));
    L.uv.push_back(take(4 * plane * compute_bytes(storage)));
    L.rho.push_back(take((size_t)I.Nz * I.Nr * sizeof(double)));
    L.uz.push_back(take((size_t)I.Nz * I.Nr * sizeof(double)));
    L.ur.push_back(take((size_t)I.Nz * I.Nr * sizeof(double)));
    L.inlet.push_back(take((size_t)2 * I.Nz * sizeof(double)));
  }
  L.total = o;
  return L;
}

}  // namespace

struct amlbm_batch {
  int n = 0, storage = 0, sched = 0, tz = 0, tr = 0, graph_chunk = 0;
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool owns = false;
  Layout L;
  std::vector<InstDesc> desc;
  std::vector<long long> steps;  // per instance, since its fields were set
  InstDesc* d_desc = nullptr;
  int* d_tiles = nullptr;
  int* d_rb_tiles = nullptr;
  int* d_ctr = nullptr;  // tile counters of the persistent step (one per parity)
  int parity = 0;
  long long sites = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // pinned host staging of the whole-batch diagnostics (jobs, then 16 doubles per
  // instance), allocated on first use; the jobs last uploaded
  char* pin = nullptr;
  std::vector<amlbm::DiagJob> last_jobs;
};

struct amlbm_ctx {
  amlbm_batch* b;
};

namespace {

int launch_steps_direct(amlbm_batch* b, int n) {
  for (int s = 0; s < n; ++s) {
    const cudaError_t e = amlbm::launch_step(b->storage, b->sched, b->tz, b->tr, b->d_desc, b->d_tiles,
                                             b->L.ntiles, 0, b->parity, b->stream, b->d_ctr);
    if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("step kernel: ") + cudaGetErrorString(e));
    b->parity ^= 1;
  }
  return AMLBM_OK;
}

int ensure_graph(amlbm_batch* b, int parity) {
  if (b->graph[parity]) return AMLBM_OK;
  cudaGraph_t g = nullptr;
  AMLBM_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int p = parity;
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < b->graph_chunk && e == cudaSuccess; ++s) {
    e = amlbm::launch_step(b->storage, b->sched, b->tz, b->tr, b->d_desc, b->d_tiles, b->L.ntiles, 0, p,
                           b->stream, b->d_ctr);
    p ^= 1;
  }
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(AMLBM_ECUDA, std::string("graph capture: ") +
                                 cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  const cudaError_t e3 = cudaGraphInstantiate(&b->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) return fail(AMLBM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
  return AMLBM_OK;
}

int batch_build(const std::vector<amlbm_instance>& inst, const amlbm_tune* tune, void* stream,
                void* workspace, size_t ws_bytes, amlbm_batch** out) {
  if (!out) return fail(AMLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (inst.empty()) return fail(AMLBM_EINVAL, "need at least one instance");
  for (size_t i = 0; i < inst.size(); ++i) {
    const int rc = validate(inst[i], (int)i);
    if (rc) return rc;
  }
  const int storage = inst[0].bc.storage;
  int tz = 0, tr = 0, sched = 0;
  if (tune && (tune->tile_z || tune->tile_r || tune->schedule)) {
    tz = tune->tile_z;
    tr = tune->tile_r;
    bool any_bounded = false;
    for (const auto& I : inst) any_bounded = any_bounded || bounded(I.bc);
    sched = tune->schedule ? tune->schedule : (any_bounded ? AMLBM_SCHED_FUSED : AMLBM_SCHED_SPLIT);
    if (sched != AMLBM_SCHED_FUSED && sched != AMLBM_SCHED_SPLIT && sched != AMLBM_SCHED_PAIR)
      return fail(AMLBM_EINVAL, "bad schedule");
    if (sched == AMLBM_SCHED_PAIR && !all_pair_ok(inst))
      return fail(AMLBM_EINVAL,
                  "the pair schedule takes periodic lattices on the axis with an even Nz, a free-slip or "
                  "no-slip wall and the source at the departure site");
    if (sched == AMLBM_SCHED_SPLIT)
      for (const auto& I : inst)
        if (bounded(I.bc))
          return fail(AMLBM_EINVAL,
                      "the split schedule takes periodic lattices on the axis with the velocity shift only");
    if (!tz && !tr) {
      int s2;
      pick_tile(storage, inst, &s2, &tz, &tr);
      if (!amlbm::tile_supported(storage, sched, tz, tr)) { tz = 32; tr = 8; }
    }
    if (!amlbm::tile_supported(storage, sched, tz, tr))
      return fail(AMLBM_EINVAL, "tile " + std::to_string(tz) + "x" + std::to_string(tr) +
                                    " is not compiled for this storage and schedule (see amlbm_tiles)");
  } else {
    pick_tile(storage, inst, &sched, &tz, &tr);
  }
  amlbm_batch* b = new (std::nothrow) amlbm_batch();
  if (!b) return fail(AMLBM_ENOMEM, "host allocation failed");
  b->n = (int)inst.size();
  b->storage = storage;
  b->sched = sched;
  b->tz = tz;
  b->tr = tr;
  b->graph_chunk = tune ? std::max(0, tune->graph_chunk) : 0;
  if (b->graph_chunk % 2) b->graph_chunk += 1;  // even: a chunk returns to its parity
  b->stream = static_cast<cudaStream_t>(stream);
  if (!b->stream) b->graph_chunk = 0;  // the legacy stream cannot be captured
  b->L = make_layout(inst, storage, tz, tr, sched);
  if (workspace) {
    if (ws_bytes < b->L.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) {
      delete b;
      return fail(AMLBM_ENOMEM, "workspace too small or not 256-byte aligned: need " +
                                    std::to_string(b->L.total) + " bytes");
    }
    b->arena = static_cast<char*>(workspace);
    b->arena_bytes = ws_bytes;
  } else {
    const cudaError_t e = cudaMalloc(&b->arena, b->L.total);
    if (e != cudaSuccess) {
      delete b;
      return fail(AMLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->owns = true;
    b->arena_bytes = b->L.total;
  }
  const Layout& L = b->L;
  std::vector<int> tiles, rb_tiles;
  tiles.reserve(L.ntiles);
  rb_tiles.reserve(L.rb_ntiles);
  for (int i = 0; i < b->n; ++i) {
    const amlbm_instance& I = inst[i];
    InstDesc d;
    std::memset(&d, 0, sizeof(d));
    d.Nz = I.Nz;
    d.Nr = I.Nr;
    d.P = pitch_of(I.Nz);
    d.wall = I.bc.wall_r;
    d.axisym = I.bc.axisym;
    d.src = I.bc.src_mode;
    d.shift = resolve_shift(I.bc);
    d.zbc = I.bc.z_bc;
    d.rlo = I.bc.r_lo;
    d.forcing = I.bc.forcing;
    // 1 = stochastic rounding of the 16-bit stores.  Default: stochastic for BF16
    // with the W_i s shifts (measured: an order of magnitude more accurate there),
    // to nearest for FP16 and for the equilibrium shift (no gain measured)
    const bool sr_default = storage == AMLBM_STORE_BF16 && d.shift != 3;
    d.rounding = (storage != AMLBM_STORE_F16 && storage != AMLBM_STORE_BF16) ? 0
               : I.bc.rounding == AMLBM_ROUND_STOCHASTIC ? 1
               : I.bc.rounding == AMLBM_ROUND_NEAREST ? 0 : (sr_default ? 1 : 0);
    d.tiles_z = (I.Nz + tz - 1) / tz;
    d.tiles_r = (I.Nr + tr - 1) / tr;
    d.tile_base = (int)tiles.size();
    int rz, rr;
    rb_tiling(storage, sched, tz, tr, &rz, &rr);
    d.rb_tiles_z = (I.Nz + rz - 1) / rz;
    d.rb_tiles_r = (I.Nr + rr - 1) / rr;
    d.rb_tile_base = (int)rb_tiles.size();
    d.tau = I.tau;
    d.G = I.G;
    d.rho0 = I.rho0;
    d.gz = I.bc.g_z;
    d.rho_ref = I.bc.rho_ref;
    const double k[12] = {I.tau, 1.0 / I.tau, -I.G, -I.G / 18.0, I.bc.g_z, I.rho0, 1.0 / I.rho0,
                          (I.tau - 0.5) / 3.0, I.bc.rho_ref, I.bc.r_off + 0.5,
                          I.bc.wall_r == AMLBM_WALL_OUTLET ? I.bc.rho_out : 1.0, 1.0 - 0.5 / I.tau};
    for (int c = 0; c < 12; ++c) {
      d.k64[c] = k[c];
      d.k32[c] = (float)k[c];
    }
    d.f[0] = b->arena + L.f0[i];
    d.f[1] = b->arena + L.f1[i];
    d.psi[0] = b->arena + L.p0[i];
    d.psi[1] = b->arena + L.p1[i];
    d.uv = b->arena + L.uv[i];
    d.rho_out = b->arena + L.rho[i];
    d.uz_out = b->arena + L.uz[i];
    d.ur_out = b->arena + L.ur[i];
    d.inlet = reinterpret_cast<const double*>(b->arena + L.inlet[i]);
    for (int t = 0; t < d.tiles_z * d.tiles_r; ++t) tiles.push_back(i);
    for (int t = 0; t < d.rb_tiles_z * d.rb_tiles_r; ++t) rb_tiles.push_back(i);
    b->desc.push_back(d);
    b->sites += (long long)I.Nz * I.Nr;
  }
  b->steps.assign(b->n, 0);
  b->d_desc = reinterpret_cast<InstDesc*>(b->arena + L.desc);
  b->d_tiles = reinterpret_cast<int*>(b->arena + L.tiles);
  b->d_rb_tiles = reinterpret_cast<int*>(b->arena + L.rb_tiles);
  b->d_ctr = reinterpret_cast<int*>(b->arena + L.ctr);
  cudaError_t e = cudaMemcpyAsync(b->d_desc, b->desc.data(), b->desc.size() * sizeof(InstDesc),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_rb_tiles, rb_tiles.data(), rb_tiles.size() * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctr, 0, 5 * sizeof(int), b->stream);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(b->arena + L.inlet[i], 0, (size_t)2 * inst[i].Nz * sizeof(double), b->stream);
  std::vector<long long> off(b->n + 1, 0);
  for (int i = 0; i < b->n; ++i) off[i + 1] = off[i] + (long long)inst[i].Nz * inst[i].Nr;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->arena + L.site_off, off.data(), off.size() * sizeof(long long),
                        cudaMemcpyHostToDevice, b->stream);
  // the instance of every block of a whole-batch diagnostics pass
  std::vector<int> blkjob;
  blkjob.reserve(L.all_nblk);
  for (int i = 0; i < b->n; ++i)
    for (int q = 0; q < amlbm::diag_blocks(inst[i].Nz, inst[i].Nr); ++q) blkjob.push_back(i);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->arena + L.diag_blkjob, blkjob.data(), blkjob.size() * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    if (b->owns) cudaFree(b->arena);
    delete b;
    return fail(AMLBM_ECUDA, std::string("descriptor upload: ") + cudaGetErrorString(e));
  }
  // the allocation-free diagnostics' scratch: looked up now, in a call that
  // allocates anyway (its failure surfaces at that entry point, not here)
  amlbm::noalloc_prepare(storage);
  // the pair read-back's code, loaded now for the same reason (its first use
  // may be an allocation-free diagnostics call)
  if (sched == amlbm::SCHED_PAIR) amlbm::readback_pair_preload(storage, tz, tr);
  *out = b;
  return AMLBM_OK;
}

int check_k(const amlbm_batch* b, int k) {
  if (!b) return fail(AMLBM_EINVAL, "NULL batch");
  if (k < 0 || k >= b->n) return fail(AMLBM_EINVAL, "instance index out of range");
  return AMLBM_OK;
}

// f = f^eq(rho, u) for instance k from device arrays (uz, ur nullable).
int init_device(amlbm_batch* b, int k, const double* rho, const double* uz, const double* ur) {
  const InstDesc& d = b->desc[k];
  const cudaError_t e = amlbm::launch_init(b->storage, b->d_desc, k, d.Nz, d.Nr, rho, uz, ur,
                                           b->parity, b->stream);
  if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("init kernel: ") + cudaGetErrorString(e));
  b->steps[k] = 0;
  return AMLBM_OK;
}

int init_host(amlbm_batch* b, int k, const double* rho, const double* uz, const double* ur) {
  int rc = check_k(b, k);
  if (rc) return rc;
  if (!rho) return fail(AMLBM_EINVAL, "rho is NULL");
  const InstDesc& d = b->desc[k];
  const size_t N = (size_t)d.Nz * d.Nr;
  double* st = reinterpret_cast<double*>(b->arena + b->L.upload);
  for (size_t n = 0; n < N; ++n)
    if (!(rho[n] > 0) || !std::isfinite(rho[n]))
      return fail(AMLBM_EINVAL, "rho must be positive and finite at every site");
  AMLBM_CK(cudaMemcpyAsync(st, rho, N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  if (uz) AMLBM_CK(cudaMemcpyAsync(st + N, uz, N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  if (ur) AMLBM_CK(cudaMemcpyAsync(st + 2 * N, ur, N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  rc = init_device(b, k, st, uz ? st + N : nullptr, ur ? st + 2 * N : nullptr);
  if (rc) return rc;
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  return AMLBM_OK;
}

int set_inlet(amlbm_batch* b, int k, const double* uz, const double* ur) {
  int rc = check_k(b, k);
  if (rc) return rc;
  const InstDesc& d = b->desc[k];
  if (d.rlo != AMLBM_RLO_INLET) return fail(AMLBM_EINVAL, "the lattice has no inlet row");
  if (!uz || !ur) return fail(AMLBM_EINVAL, "uz and ur must not be NULL");
  for (int q = 0; q < d.Nz; ++q)
    if (!std::isfinite(uz[q]) || !std::isfinite(ur[q]))
      return fail(AMLBM_EINVAL, "inlet velocities must be finite");
  double* dst = const_cast<double*>(d.inlet);
  AMLBM_CK(cudaMemcpyAsync(dst, uz, d.Nz * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  AMLBM_CK(cudaMemcpyAsync(dst + d.Nz, ur, d.Nz * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  // the host arrays are the caller's again when the call returns
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  return AMLBM_OK;
}

// rho and u of nt tiles of the read-back list from toff into the read-back planes
cudaError_t launch_readback(amlbm_batch* b, int nt, int toff) {
  if (b->sched == amlbm::SCHED_PAIR)
    return amlbm::launch_readback_pair(b->storage, b->tz, b->tr, b->d_desc, b->d_rb_tiles, nt, toff, b->parity,
                                       b->stream);
  int rz, rr;
  amlbm::rb_tile(b->storage, &rz, &rr);
  return amlbm::launch_macro(b->storage, rz, rr, b->d_desc, b->d_rb_tiles, nt, toff, b->parity, b->stream);
}

int macro_for(amlbm_batch* b, int k) {
  const InstDesc& d = b->desc[k];
  const int nt = d.rb_tiles_z * d.rb_tiles_r;
  const cudaError_t e = launch_readback(b, nt, d.rb_tile_base);
  if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("macro kernel: ") + cudaGetErrorString(e));
  return AMLBM_OK;
}

int read_host(amlbm_batch* b, int k, double* rho, double* uz, double* ur, double* f) {
  int rc = check_k(b, k);
  if (rc) return rc;
  const InstDesc& d = b->desc[k];
  const size_t N = (size_t)d.Nz * d.Nr;
  // the read-back holds the compute type: FP64 copies straight into the caller's
  // arrays, FP32 through host staging, widened after the copy
  double* dst[3] = {rho, uz, ur};
  void* srcs[3] = {d.rho_out, d.uz_out, d.ur_out};
  const bool wide = compute_bytes(b->storage) == 8;
  std::vector<float> stage[3];
  if (rho || uz || ur) {
    rc = macro_for(b, k);
    if (rc) return rc;
    for (int q = 0; q < 3; ++q) {
      if (!dst[q]) continue;
      if (wide) {
        AMLBM_CK(cudaMemcpyAsync(dst[q], srcs[q], N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
      } else {
        stage[q].resize(N);
        AMLBM_CK(cudaMemcpyAsync(stage[q].data(), srcs[q], N * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
      }
    }
  }
  if (f) {
    double* un = reinterpret_cast<double*>(b->arena + b->L.unpack);
    const cudaError_t e = amlbm::launch_unpack(b->storage, b->d_desc, k, d.Nz, d.Nr, b->parity, un, b->stream);
    if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("unpack kernel: ") + cudaGetErrorString(e));
    AMLBM_CK(cudaMemcpyAsync(f, un, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  for (int q = 0; q < 3; ++q)
    if (dst[q] && !wide)
      for (size_t n = 0; n < N; ++n) dst[q][n] = double(stage[q][n]);
  return AMLBM_OK;
}

// Every instance from host arrays holding them back to back.  The new state is
// written into the buffers of the other parity, and becomes current only when
// the device check finds every rho positive and finite.
// Device address of a host array the GPU can read in place (page-locked memory,
// mapped into the unified address space), or nullptr.
template <class In>
const In* device_view(const In* h) {
  if (!h) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<const In*>(a.devicePointer) : nullptr;
}

template <class In>
int init_all_host(amlbm_batch* b, const In* rho, const In* uz, const In* ur) {
  if (!b) return fail(AMLBM_EINVAL, "NULL batch");
  if (!rho) return fail(AMLBM_EINVAL, "rho is NULL");
  const long long T = b->sites;
  In* st = reinterpret_cast<In*>(b->arena + b->L.upload);  // room for three FP64 arrays
  const long long* off = reinterpret_cast<const long long*>(b->arena + b->L.site_off);
  int* bad = b->d_ctr + 4;
  // Page-locked host arrays are read by the init kernel in place (over the
  // CPU-GPU link, without a separate copy); others are copied to the device first.
  const In* src[3] = {rho, uz, ur};
  const In* dev[3] = {nullptr, nullptr, nullptr};
  for (int q = 0; q < 3; ++q) {
    if (!src[q]) continue;
    dev[q] = device_view(src[q]);
    if (!dev[q]) {
      AMLBM_CK(cudaMemcpyAsync(st + q * T, src[q], T * sizeof(In), cudaMemcpyHostToDevice, b->stream));
      dev[q] = st + q * T;
    }
  }
  AMLBM_CK(cudaMemsetAsync(bad, 0, sizeof(int), b->stream));
  const cudaError_t e = amlbm::launch_init_all(b->storage, b->d_desc, b->n, off, T, dev[0], dev[1], dev[2],
                                               b->parity ^ 1, bad, b->stream);
  if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("init kernel: ") + cudaGetErrorString(e));
  int nbad = 0;
  AMLBM_CK(cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  if (nbad)
    return fail(AMLBM_EINVAL, "rho must be positive and finite at every site (" + std::to_string(nbad) +
                                  " sites are not); the state is unchanged");
  b->parity ^= 1;
  // tile counters and step numbers (the stochastic-rounding stream) restart
  // from zero, as in a new batch
  AMLBM_CK(cudaMemsetAsync(b->d_ctr, 0, 4 * sizeof(int), b->stream));
  for (auto& s : b->steps) s = 0;
  return AMLBM_OK;
}

// Every instance in one read-back launch, one partial-sum launch and one final
// launch; out[k] for instance k.  Unstable instances are reported after every
// output is filled.
int diag_all_host(amlbm_batch* b, const amlbm_diag_params* dp, amlbm_diag* out) {
  if (!b) return fail(AMLBM_EINVAL, "NULL batch");
  if (!out) return fail(AMLBM_EINVAL, "out is NULL");
  std::vector<amlbm::DiagJob> jobs(b->n);
  int blk = 0, col = 0;
  for (int k = 0; k < b->n; ++k) {
    const InstDesc& d = b->desc[k];
    const amlbm_diag_params p = dp ? dp[k] : diag_defaults(d);
    if (!(p.R > 0) || !(p.rho_l != p.rho_v))
      return fail(AMLBM_EINVAL, "diag params of instance " + std::to_string(k) + ": need R > 0, rho_l != rho_v");
    amlbm::DiagJob& J = jobs[k];
    J.zc = p.zc; J.R = p.R; J.rho_l = p.rho_l; J.rho_v = p.rho_v;
    amlbm::diag_job_constants(J);
    J.inst = k;
    J.blk0 = blk;
    J.nblk = amlbm::diag_blocks(d.Nz, d.Nr);
    J.col0 = col;
    blk += J.nblk;
    col += d.Nz;
  }
  amlbm::DiagJob* d_jobs = reinterpret_cast<amlbm::DiagJob*>(b->arena + b->L.diag_jobs);
  const size_t jbytes = jobs.size() * sizeof(jobs[0]), rbytes = (size_t)16 * b->n * sizeof(double);
  if (!b->pin && cudaMallocHost(reinterpret_cast<void**>(&b->pin), jbytes + rbytes) != cudaSuccess) {
    b->pin = nullptr;  // pageable copies below
    cudaGetLastError();
  }
  // a time-stepping loop asks for the same parameters every time: upload once
  if (b->last_jobs.size() != jobs.size() || std::memcmp(b->last_jobs.data(), jobs.data(), jbytes) != 0) {
    const void* src = jobs.data();
    if (b->pin) {
      std::memcpy(b->pin, jobs.data(), jbytes);
      src = b->pin;
    }
    AMLBM_CK(cudaMemcpyAsync(d_jobs, src, jbytes, cudaMemcpyHostToDevice, b->stream));
    if (!b->pin) AMLBM_CK(cudaStreamSynchronize(b->stream));  // the pageable source goes out of scope
    b->last_jobs = jobs;
  }
  cudaError_t e = launch_readback(b, b->L.rb_ntiles, 0);
  if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("macro kernel: ") + cudaGetErrorString(e));
  double* part = reinterpret_cast<double*>(b->arena + b->L.diag_part);
  double* cols = reinterpret_cast<double*>(b->arena + b->L.diag_cols);
  double* res = reinterpret_cast<double*>(b->arena + b->L.diag_out);
  const int* blkjob = reinterpret_cast<const int*>(b->arena + b->L.diag_blkjob);
  e = amlbm::launch_diag_all(b->storage, b->d_desc, d_jobs, blkjob, b->n, blk, b->parity, part, cols, res,
                             b->stream);
  if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("diag kernels: ") + cudaGetErrorString(e));
  std::vector<double> hv;
  double* h = b->pin ? reinterpret_cast<double*>(b->pin + jbytes) : nullptr;
  if (!h) {
    hv.resize((size_t)16 * b->n);
    h = hv.data();
  }
  AMLBM_CK(cudaMemcpyAsync(h, res, rbytes, cudaMemcpyDeviceToHost, b->stream));
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  int first_bad = -1;
  for (int k = 0; k < b->n; ++k) {
    fill_diag(&h[(size_t)16 * k], b->steps[k], &out[k]);
    if (out[k].bad > 0 && first_bad < 0) first_bad = k;
  }
  if (first_bad >= 0)
    return fail(AMLBM_EUNSTABLE, "non-finite or non-positive density in instance " + std::to_string(first_bad) +
                                     " (" + std::to_string((long long)out[first_bad].bad) + " sites)");
  return AMLBM_OK;
}

int diag_host(amlbm_batch* b, int k, const amlbm_diag_params* dp, amlbm_diag* out) {
  int rc = check_k(b, k);
  if (rc) return rc;
  if (!out) return fail(AMLBM_EINVAL, "out is NULL");
  const InstDesc& d = b->desc[k];
  const amlbm_diag_params p = dp ? *dp : diag_defaults(d);
  if (!(p.R > 0) || !(p.rho_l != p.rho_v)) return fail(AMLBM_EINVAL, "diag params: need R > 0, rho_l != rho_v");
  rc = macro_for(b, k);
  if (rc) return rc;
  double* part = reinterpret_cast<double*>(b->arena + b->L.diag_part);
  double* cols = reinterpret_cast<double*>(b->arena + b->L.diag_cols);
  double* res = reinterpret_cast<double*>(b->arena + b->L.diag_out);
  const int nblk = amlbm::diag_blocks(d.Nz, d.Nr);
  const cudaError_t e = amlbm::launch_diag(b->storage, b->d_desc, k, d.Nz, d.Nr, b->parity, p.zc, p.R,
                                           p.rho_l, p.rho_v, part, nblk, cols, res, b->stream);
  if (e != cudaSuccess) return fail(AMLBM_ECUDA, std::string("diag kernels: ") + cudaGetErrorString(e));
  double h[16];
  AMLBM_CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  fill_diag(h, b->steps[k], out);
  if (out->bad > 0) return fail(AMLBM_EUNSTABLE, amlbm::unstable_message(out->bad));
  return AMLBM_OK;
}

}  // namespace

extern "C" {

const char* amlbm_last_error(void) { return g_err.c_str(); }
const char* amlbm_version(void) { return "amlbm 0.2 (sm_103a)"; }

int amlbm_tiles(int storage, int schedule, int* tz, int* tr, int cap) {
  return amlbm::tile_list(storage, schedule, tz, tr, cap);
}

size_t amlbm_batch_workspace_bytes(int n, const amlbm_instance* inst) {
  if (n < 1 || !inst) return 0;
  std::vector<amlbm_instance> v(inst, inst + n);
  for (int i = 0; i < n; ++i)
    if (validate(v[i], i)) return 0;
  // room for whichever compiled tile the tune picks (the tile list grows with
  // the number of tiles)
  size_t need = 0;
  for (int sc = amlbm::SCHED_FUSED; sc <= amlbm::SCHED_PAIR; ++sc) {
    int tz[32], tr[32];
    const int nt = std::min(32, amlbm::tile_list(v[0].bc.storage, sc, tz, tr, 32));
    for (int c = 0; c < nt; ++c)
      need = std::max(need, make_layout(v, v[0].bc.storage, tz[c], tr[c], sc).total);
  }
  return need;
}

int amlbm_batch_create(int n, const amlbm_instance* inst, const amlbm_tune* tune, void* stream,
                       void* workspace, size_t workspace_bytes, amlbm_batch** out) {
  if (n < 1 || !inst) return fail(AMLBM_EINVAL, "need n >= 1 instances");
  std::vector<amlbm_instance> v(inst, inst + n);
  return batch_build(v, tune, stream, workspace, workspace_bytes, out);
}

int amlbm_batch_init_fields(amlbm_batch* b, int k, const double* rho, const double* uz, const double* ur) {
  return init_host(b, k, rho, uz, ur);
}

int amlbm_batch_set_inlet(amlbm_batch* b, int k, const double* uz, const double* ur) {
  return set_inlet(b, k, uz, ur);
}

int amlbm_batch_step(amlbm_batch* b, int n) {
  if (!b) return fail(AMLBM_EINVAL, "NULL batch");
  if (n < 0) return fail(AMLBM_EINVAL, "n must be >= 0");
  int left = n;
  if (b->graph_chunk > 0) {
    while (left >= b->graph_chunk) {
      int rc = ensure_graph(b, b->parity);
      if (rc) return rc;
      AMLBM_CK(cudaGraphLaunch(b->graph[b->parity], b->stream));
      left -= b->graph_chunk;  // an even chunk leaves the parity unchanged
    }
  }
  const int rc = launch_steps_direct(b, left);
  if (rc) return rc;
  for (auto& s : b->steps) s += n;
  return AMLBM_OK;
}

int amlbm_batch_read(amlbm_batch* b, int k, double* rho, double* uz, double* ur, double* f) {
  return read_host(b, k, rho, uz, ur, f);
}

int amlbm_batch_diagnostics(amlbm_batch* b, int k, const amlbm_diag_params* dp, amlbm_diag* out) {
  return diag_host(b, k, dp, out);
}

int amlbm_batch_init_all(amlbm_batch* b, const double* rho, const double* uz, const double* ur) {
  return init_all_host<double>(b, rho, uz, ur);
}

int amlbm_batch_init_all_f32(amlbm_batch* b, const float* rho, const float* uz, const float* ur) {
  return init_all_host<float>(b, rho, uz, ur);
}

int amlbm_batch_diagnostics_all(amlbm_batch* b, const amlbm_diag_params* dp, amlbm_diag* out) {
  return diag_all_host(b, dp, out);
}

long long amlbm_batch_sites(const amlbm_batch* b) { return b ? b->sites : 0; }

int amlbm_batch_config(const amlbm_batch* b, int* schedule, int* tile_z, int* tile_r, int* launches_per_step) {
  if (!b) return fail(AMLBM_EINVAL, "NULL batch");
  if (schedule) *schedule = b->sched;
  if (tile_z) *tile_z = b->tz;
  if (tile_r) *tile_r = b->tr;
  if (launches_per_step) *launches_per_step = b->sched == amlbm::SCHED_SPLIT ? 2 : 1;
  return AMLBM_OK;
}

void amlbm_batch_destroy(amlbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (auto& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  if (b->pin) cudaFreeHost(b->pin);
  if (b->owns && b->arena) cudaFree(b->arena);
  delete b;
}

// ------------------------------------------------------------- one lattice --

static amlbm_instance one(int Nz, int Nr, double tau, double G, double rho0, const amlbm_bc* bc) {
  amlbm_instance I;
  I.Nz = Nz; I.Nr = Nr; I.tau = tau; I.G = G; I.rho0 = rho0;
  I.bc = bc ? *bc : default_bc();
  return I;
}

size_t amlbm_workspace_bytes(int Nz, int Nr, int storage) {
  amlbm_bc bc = default_bc();
  bc.storage = storage;
  // room for every shift mode of this storage (the equilibrium shift keeps the
  // velocity beside psi)
  if (storage != AMLBM_STORE_F64) bc.shift = AMLBM_SHIFT_EQUILIBRIUM;
  amlbm_instance I = one(Nz, Nr, 1.0, -5.0, 1.0, &bc);
  return amlbm_batch_workspace_bytes(1, &I);
}

int amlbm_create(int Nz, int Nr, double tau, double G, double rho0, const amlbm_bc* bc,
                 void* cuda_stream, void* workspace, size_t workspace_bytes, amlbm_ctx** out) {
  if (!out) return fail(AMLBM_EINVAL, "out is NULL");
  *out = nullptr;
  std::vector<amlbm_instance> v{one(Nz, Nr, tau, G, rho0, bc)};
  amlbm_batch* b = nullptr;
  const int rc = batch_build(v, nullptr, cuda_stream, workspace, workspace_bytes, &b);
  if (rc) return rc;
  amlbm_ctx* c = new (std::nothrow) amlbm_ctx{b};
  if (!c) { amlbm_batch_destroy(b); return fail(AMLBM_ENOMEM, "host allocation failed"); }
  *out = c;
  return AMLBM_OK;
}

int amlbm_init_fields(amlbm_ctx* c, const double* rho, const double* uz, const double* ur) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  return init_host(c->b, 0, rho, uz, ur);
}

int amlbm_init_fields_device(amlbm_ctx* c, const double* rho, const double* uz, const double* ur) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  if (!rho) return fail(AMLBM_EINVAL, "rho is NULL");
  return init_device(c->b, 0, rho, uz, ur);
}

int amlbm_set_inlet(amlbm_ctx* c, const double* uz, const double* ur) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  return set_inlet(c->b, 0, uz, ur);
}

int amlbm_step(amlbm_ctx* c, int n) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  return amlbm_batch_step(c->b, n);
}

int amlbm_read_fields(amlbm_ctx* c, double* rho, double* uz, double* ur, double* f) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  return read_host(c->b, 0, rho, uz, ur, f);
}

int amlbm_diagnostics(amlbm_ctx* c, const amlbm_diag_params* dp, amlbm_diag* out) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  return diag_host(c->b, 0, dp, out);
}

namespace {
struct StateHeader {
  char magic[8];
  int Nz, Nr, storage;
  int rstep;  // step number of the stochastic-rounding stream at the saved state
  long long steps;
  size_t fbytes, pbytes;
};
}  // namespace

int amlbm_save_state(amlbm_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return fail(AMLBM_EINVAL, "NULL argument");
  amlbm_batch* b = c->b;
  const InstDesc& d = b->desc[0];
  const size_t plane = (size_t)d.P * d.Nr;
  const size_t fb = 9 * plane * elem_bytes(b->storage),
               pb = plane * compute_bytes(b->storage) * psi_planes(d.shift);
  const size_t need = sizeof(StateHeader) + fb + pb;
  if (!buf) { *len = need; return AMLBM_OK; }
  if (*len < need) return fail(AMLBM_EINVAL, "buffer too small: need " + std::to_string(need));
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "AMLBMST1", 8);
  h.Nz = d.Nz; h.Nr = d.Nr; h.storage = b->storage; h.steps = b->steps[0]; h.fbytes = fb; h.pbytes = pb;
  AMLBM_CK(cudaMemcpyAsync(&h.rstep, b->d_ctr + 2 + b->parity, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof(h));
  AMLBM_CK(cudaMemcpyAsync(p + sizeof(h), d.f[b->parity], fb, cudaMemcpyDeviceToHost, b->stream));
  AMLBM_CK(cudaMemcpyAsync(p + sizeof(h) + fb, d.psi[b->parity], pb, cudaMemcpyDeviceToHost, b->stream));
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  *len = need;
  return AMLBM_OK;
}

int amlbm_load_state(amlbm_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) return fail(AMLBM_EINVAL, "NULL argument");
  amlbm_batch* b = c->b;
  const InstDesc& d = b->desc[0];
  StateHeader h;
  if (len < sizeof(h)) return fail(AMLBM_EINVAL, "buffer too small");
  std::memcpy(&h, buf, sizeof(h));
  const size_t plane = (size_t)d.P * d.Nr;
  const size_t fb = 9 * plane * elem_bytes(b->storage),
               pb = plane * compute_bytes(b->storage) * psi_planes(d.shift);
  if (std::memcmp(h.magic, "AMLBMST1", 8) || h.Nz != d.Nz || h.Nr != d.Nr || h.storage != b->storage ||
      h.fbytes != fb || h.pbytes != pb || len < sizeof(h) + fb + pb)
    return fail(AMLBM_EINVAL, "state does not match this context");
  const char* p = static_cast<const char*>(buf);
  AMLBM_CK(cudaMemcpyAsync(d.f[b->parity], p + sizeof(h), fb, cudaMemcpyHostToDevice, b->stream));
  AMLBM_CK(cudaMemcpyAsync(d.psi[b->parity], p + sizeof(h) + fb, pb, cudaMemcpyHostToDevice, b->stream));
  AMLBM_CK(cudaMemcpyAsync(b->d_ctr + 2 + b->parity, &h.rstep, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  AMLBM_CK(cudaStreamSynchronize(b->stream));
  b->steps[0] = h.steps;
  return AMLBM_OK;
}

int amlbm_device_state(amlbm_ctx* c, void** f, void** psi, int* pitch) {
  if (!c) return fail(AMLBM_EINVAL, "NULL context");
  const InstDesc& d = c->b->desc[0];
  if (f) *f = d.f[c->b->parity];
  if (psi) *psi = d.psi[c->b->parity];
  if (pitch) *pitch = d.P;
  return AMLBM_OK;
}

void amlbm_destroy(amlbm_ctx* c) {
  if (!c) return;
  amlbm_batch_destroy(c->b);
  delete c;
}

}  // extern "C"

// ------------------------------------------- helpers for other entry points --
namespace amlbm {

int ctx_info(amlbm_ctx* c, CtxInfo* out) {
  if (!c || !c->b || !out) return fail(AMLBM_EINVAL, "NULL context");
  const amlbm_batch* b = c->b;
  out->d_desc = b->d_desc;
  out->host = b->desc[0];
  out->Nz = b->desc[0].Nz;
  out->Nr = b->desc[0].Nr;
  out->storage = b->storage;
  out->parity = b->parity;
  out->steps = b->steps[0];
  out->stream = b->stream;
  return AMLBM_OK;
}

int ctx_readback(amlbm_ctx* c) {
  if (!c || !c->b) return fail(AMLBM_EINVAL, "NULL context");
  return macro_for(c->b, 0);
}

int set_error(int code, const std::string& msg) { return fail(code, msg); }

}  // namespace amlbm
