// Autotuner of the step launch: times every compiled (schedule, tile) pair of a
// batch's storage form on a synthetic state of the batch's own lattice shapes
// and returns the fastest.  Built on the public entry points only: each
// candidate is a temporary batch (its own device memory), stepped on the
// caller's stream and timed with CUDA events on that stream.
//
// The paper runs one lattice at a time and has no launch configuration to
// tune; the candidates differ only in how the same update is tiled, and every
// candidate gives the same state (the split and fused schedules are
// bit-identical, and so are all tilings).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "amlbm.h"
#include "amlbm_internal.cuh"

namespace {

// A resting drop of radius min(Nz, 2 Nr) / 4 on the axis (tanh interface of
// width 2 between densities 1.9 and 0.16): every code path of the step (bulk,
// interface, axis and wall rows) runs as it does on the workloads.
void synthetic_rho(int Nz, int Nr, std::vector<double>& rho) {
  rho.resize((size_t)Nz * Nr);
  const double R = std::max(2.0, std::min(Nz, 2 * Nr) / 4.0), zc = Nz / 2.0;
  for (int j = 0; j < Nr; ++j)
    for (int k = 0; k < Nz; ++k) {
      const double r = j + 0.5, dz = k - zc, d = std::sqrt(dz * dz + r * r);
      rho[(size_t)j * Nz + k] = 0.16 + (1.9 - 0.16) * 0.5 * (1.0 - std::tanh((d - R) / 2.0));
    }
}

constexpr double kTie = 0.005;

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" int amlbm_autotune(int n, const amlbm_instance* inst, int steps, void* stream,
                              amlbm_tune* best, amlbm_tune_result* results, int cap) {
  using amlbm::set_error;
  if (n < 1 || !inst || !best) return set_error(AMLBM_EINVAL, "autotune: need n >= 1 instances and best");
  if (steps < 1) return set_error(AMLBM_EINVAL, "autotune: steps must be >= 1");
  const int storage = inst[0].bc.storage;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Events ev;
  if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess)
    return set_error(AMLBM_ECUDA, "autotune: cudaEventCreate failed");
  std::vector<std::vector<double>> rho(n);
  for (int i = 0; i < n; ++i) synthetic_rho(inst[i].Nz, inst[i].Nr, rho[i]);
  long long sites = 0;
  for (int i = 0; i < n; ++i) sites += (long long)inst[i].Nz * inst[i].Nr;

  // lattices with walls in z, an inlet, an outlet or the Guo forcing run on the
  // fused schedule only
  bool fused_only = false, pair = true;
  for (int i = 0; i < n; ++i) {
    fused_only = fused_only || inst[i].bc.z_bc != AMLBM_Z_PERIODIC ||
                 inst[i].bc.r_lo != AMLBM_RLO_AXIS || inst[i].bc.wall_r == AMLBM_WALL_OUTLET ||
                 inst[i].bc.forcing != AMLBM_FORCE_SHIFT;
    // the pair schedule's conditions (amlbm_batch_create checks the rest)
    pair = pair && inst[i].bc.z_bc == AMLBM_Z_PERIODIC && inst[i].bc.r_lo == AMLBM_RLO_AXIS &&
           inst[i].bc.wall_r != AMLBM_WALL_OUTLET && inst[i].bc.src_mode == AMLBM_SRC_LOCAL &&
           inst[i].Nz % 2 == 0;
  }
  int timed = 0;
  double best_ms = 1e300;
  for (int sched = AMLBM_SCHED_FUSED; sched <= AMLBM_SCHED_PAIR; ++sched) {
    if (sched == AMLBM_SCHED_SPLIT && fused_only) continue;
    if (sched == AMLBM_SCHED_PAIR && !pair) continue;
    int tz[64], tr[64];
    const int nt = std::min(64, amlbm_tiles(storage, sched, tz, tr, 64));
    for (int c = 0; c < nt; ++c) {
      amlbm_tune t;
      t.tile_z = tz[c];
      t.tile_r = tr[c];
      t.graph_chunk = 0;
      t.schedule = sched;
      amlbm_batch* b = nullptr;
      int rc = amlbm_batch_create(n, inst, &t, stream, nullptr, 0, &b);
      if (rc == AMLBM_ENOMEM) continue;  // a tile whose workspace does not fit is no candidate
      if (rc == AMLBM_EINVAL && sched == AMLBM_SCHED_PAIR) continue;  // lattices too large for it
      if (rc) return rc;
      for (int i = 0; i < n && !rc; ++i) rc = amlbm_batch_init_fields(b, i, rho[i].data(), nullptr, nullptr);
      if (!rc) rc = amlbm_batch_step(b, 3);  // warm-up: kernel attributes, first-touch
      // three timed repeats of `steps` timesteps; the fastest counts
      float ms = 1e30f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(ev.a, s);
        rc = amlbm_batch_step(b, steps);
        cudaEventRecord(ev.b, s);
        if (rc) break;
        if (cudaEventSynchronize(ev.b) != cudaSuccess) {
          rc = set_error(AMLBM_ECUDA, "autotune: event synchronisation failed");
          break;
        }
        float m = 0.f;
        cudaEventElapsedTime(&m, ev.a, ev.b);
        ms = std::min(ms, m);
      }
      amlbm_batch_destroy(b);
      if (rc) return rc;
      const double per_step = ms / steps;
      if (results && timed < cap) {
        results[timed].tune = t;
        results[timed].ms_per_step = per_step;
        results[timed].mlups = sites / (per_step * 1e-3) / 1e6;
      }
      ++timed;
      // a later candidate replaces the best only when it is faster by more than
      // the repeats' timing noise (0.5 %), so near-ties go to the earlier one in
      // amlbm_tiles order
      if (per_step < best_ms * (1.0 - kTie)) {
        best_ms = per_step;
        *best = t;
      }
    }
  }
  if (!timed) return set_error(AMLBM_ENOMEM, "autotune: no candidate fits in device memory");
  return timed;
}
