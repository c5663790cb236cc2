// Fused axisymmetric Shan-Chen LBM step for sm_103a (arXiv:1310.1871, Sec. II).
//
// One CTA updates one tile of BZ x BR sites of one lattice of a batch.  The
// whole per-site chain of the paper's update runs inside the CTA:
//   psi tile + halo 7 (from the previous step's psi, staged in shared memory)
//   -> isotropic d_r psi and 1D d_r psi (Sec. II.D), halo 5
//   -> moments, Shan-Chen force (Eq. scforce), axisymmetric force
//      (Eq. scAxisExtra), u and u^eq (Eqs. uhydro, ueq), halo 3
//   -> velocity gradients and the sources S, H_z, H_r (Eq. condition_h), halo 1
//   -> pull streaming of the BGK-collided populations (Eq. lbm2d_mod_new) with
//      the axis / wall / periodic maps of Sec. II.E, and psi of the new state.
// Global traffic per site and step: 9 populations read (halo re-reads hit L2),
// 9 written, psi written once and read once (halo re-reads hit L2).
// No tensor cores: the update is a stencil, not a contraction.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <stdint.h>

#include <type_traits>

#include "amlbm.h"
#include "amlbm_internal.cuh"

namespace amlbm {
namespace {

// D2Q9 velocities (c_z, c_r), weights, specular (r-flipped) and reversed directions.
__host__ __device__ constexpr int cz_(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int cr_(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr double w_(int i) {
  return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int mirror_(int i) {
  return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i;
}
__host__ __device__ constexpr int opp_(int i) {
  return i == 0 ? 0 : i == 1 ? 3 : i == 3 ? 1 : i == 2 ? 4 : i == 4 ? 2
       : i == 5 ? 7 : i == 7 ? 5 : i == 6 ? 8 : 6;
}

// Storage codecs: conversion between the stored element and the arithmetic
// type.  The shift W_i s of the FP32 / 16-bit forms is applied by the callers
// (decode: f = q + W_i s; encode: q = f - W_i s).  IEEE half holds q * 2^10 so
// that the shifted populations (down to ~1e-7) stay in its normal range; the
// power-of-two scale is exact.  from_sr rounds stochastically with the random
// bits r: the bits below the stored precision are added to r and truncated, so
// a value rounds up with probability equal to its distance from the lower
// neighbour (unbiased in expectation).
template <class S> struct Store;
template <> struct Store<double> {
  using C = double;
  static __device__ __forceinline__ C to(double v) { return v; }
  static __device__ __forceinline__ double from(C v) { return v; }
  static __device__ __forceinline__ double from_sr(C v, uint32_t) { return v; }
};
template <> struct Store<float> {
  using C = float;
  static __device__ __forceinline__ C to(float v) { return v; }
  static __device__ __forceinline__ float from(C v) { return v; }
  static __device__ __forceinline__ float from_sr(C v, uint32_t) { return v; }
};
template <> struct Store<__half> {
  using C = float;
  static __device__ __forceinline__ C to(__half v) { return __half2float(v) * (1.0f / 1024.0f); }
  static __device__ __forceinline__ __half from(C v) { return __float2half_rn(v * 1024.0f); }
  static __device__ __forceinline__ __half from_sr(C v, uint32_t r) {
    // FP32 keeps 13 more mantissa bits than FP16 (for FP16-normal values)
    const uint32_t b = __float_as_uint(v * 1024.0f) + (r & 0x1FFFu);
    return __float2half_rz(__uint_as_float(b));
  }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ C to(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 from(C v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ __nv_bfloat16 from_sr(C v, uint32_t r) {
    // bfloat16 is the upper half of the FP32 bit pattern
    const uint32_t b = __float_as_uint(v) + (r & 0xFFFFu);
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
  }
};

// Integer hash for the stochastic-rounding bits (a xorshift-multiply mixer).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// Store the nine new populations of a site with the shift W_i sb, rounding to
// nearest or (rounding != 0) stochastically with bits drawn from (site, step).
template <class S>
__device__ __forceinline__ void store_site(S* o, size_t plane, const typename Store<S>::C* fn,
                                           typename Store<S>::C sb, int rounding, uint32_t site,
                                           uint32_t step) {
  using C = typename Store<S>::C;
  if (sizeof(S) == 2 && rounding) {
    const uint32_t h = mix32(site ^ mix32(step + 0x9E3779B9u));
#pragma unroll
    for (int i = 0; i < 9; ++i)
      o[i * plane] = Store<S>::from_sr(fn[i] - C(w_(i)) * sb, mix32(h + 0x632BE5ABu * (uint32_t)(i + 1)));
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i * plane] = Store<S>::from(fn[i] - C(w_(i)) * sb);
  }
}

// exp / log / reciprocal of the arithmetic type.  The FP32 forms use the SFU
// approximations (relative error ~1e-7, far below the storage rounding).
__device__ __forceinline__ double exp_c(double x) { return exp(x); }
__device__ __forceinline__ float exp_c(float x) { return __expf(x); }
__device__ __forceinline__ double rcp_c(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_c(float x) { return __frcp_rn(x); }

// Shift s of a site from its stored psi: 0 (none), rho_ref (global), or the
// density recovered from psi, -rho0 ln(1 - psi/rho0) (local).  Writer and
// reader evaluate it from the same stored psi with the same non-contracted
// operations, so both see the same s bit for bit.
__device__ __forceinline__ double shift_base(int mode, double psi, double inv_rho0, double rho0,
                                             double rref) {
  (void)psi; (void)inv_rho0; (void)rho0;
  return mode == 1 ? rref : 0.0;  // FP64 storage is never shifted locally
}
__device__ __forceinline__ float shift_base(int mode, float psi, float inv_rho0, float rho0,
                                            float rref) {
  if (mode == 2) {
    const float q = __fsub_rn(1.0f, __fmul_rn(psi, inv_rho0));
    return __fmul_rn(-rho0, __logf(q));
  }
  return mode == 1 ? rref : 0.0f;
}

__device__ __forceinline__ int wrapz(int k, int Nz) {
  k %= Nz;
  return k < 0 ? k + Nz : k;
}
// Row whose value a ghost row mirrors (about r = 0 and r = Nr), clamped so that
// rows deeper than any stencil reaches still address real memory.
__device__ __forceinline__ int reflect_row(int j, int Nr) {
  if (j < 0) j = -1 - j;
  if (j >= Nr) j = 2 * Nr - 1 - j;
  return j < 0 ? 0 : (j >= Nr ? Nr - 1 : j);
}

// Isotropic 4th-order first derivatives, Sec. II.D Eq. forthorder_firstderivativex:
//   d_a phi(x) = (1/36) sum_i c_ia (8 phi(x + c_i) - phi(x + 2 c_i)).
// p points at x in a row-major tile whose rows (r) are `st` apart.  The terms
// are added in z-mirror pairs (c_1, c_3), (c_5, c_6), (c_8, c_7) so that a
// field mirrored in z gives an exactly mirrored derivative: without this, the
// rounding of the FP32 forms carries a net axial bias every step and a drop
// drifts along the axis.
template <class C>
__device__ __forceinline__ C link8(const C* p, int dz, int dr, int st) {
  return C(8) * p[dr * st + dz] - p[2 * dr * st + 2 * dz];
}
template <class C>
__device__ __forceinline__ C iso_r(const C* p, int st) {
  const C a = link8(p, 0, 1, st) - link8(p, 0, -1, st);
  const C b = (link8(p, 1, 1, st) + link8(p, -1, 1, st)) - (link8(p, 1, -1, st) + link8(p, -1, -1, st));
  return (a + b) * C(1.0 / 36.0);
}
template <class C>
__device__ __forceinline__ C iso_z(const C* p, int st) {
  const C a = link8(p, 1, 0, st) - link8(p, -1, 0, st);
  const C b = (link8(p, 1, 1, st) - link8(p, -1, 1, st)) + (link8(p, 1, -1, st) - link8(p, -1, -1, st));
  return (a + b) * C(1.0 / 36.0);
}
// 1D 4th-order central difference with element step `step` (Sec. II.D).
template <class C>
__device__ __forceinline__ C d1(const C* p, int step) {
  return (C(8) * (p[step] - p[-step]) - (p[2 * step] - p[-2 * step])) * C(1.0 / 12.0);
}

template <class C>
__device__ __forceinline__ C feq(int i, C rho, C vz, C vr) {
  const C cv = C(cz_(i)) * vz + C(cr_(i)) * vr;
  const C vv = vz * vz + vr * vr;
  return C(w_(i)) * rho * (C(1) + C(3) * cv + C(4.5) * cv * cv - C(1.5) * vv);
}
// rho = sum_i f_i, added in z-mirror pairs.
template <class C>
__device__ __forceinline__ C moment0(const C* f) {
  return (f[0] + (f[2] + f[4])) + ((f[1] + f[3]) + ((f[5] + f[6]) + (f[7] + f[8])));
}
// h_i = W_i (S + (c_iz H_z + c_ir H_r) / c_s^2), Eq. condition_h.
template <class C>
__device__ __forceinline__ C source(int i, C S_, C Hz, C Hr) {
  return C(w_(i)) * (S_ + C(3) * (C(cz_(i)) * Hz + C(cr_(i)) * Hr));
}

// The nine equilibria with f^eq_0 = rho - sum_{i>0} f^eq_i: the same value as
// W_0 rho (1 - 1.5 u^2) in exact arithmetic, but the collision then conserves
// mass to rounding.  With the directly evaluated f^eq_0 the FP32-rounded
// weights do not sum to 1 and the FP32 forms gain mass every step (a 1.5e-5
// drift over 1000 steps of the static drop, and a 1e-4 density error at the
// interface).
template <class C>
__device__ __forceinline__ void equilibrium(C rho, C vz, C vr, C* fe) {
#pragma unroll
  for (int i = 1; i < 9; ++i) fe[i] = feq(i, rho, vz, vr);
  fe[0] = rho - ((fe[2] + fe[4]) + ((fe[1] + fe[3]) + ((fe[5] + fe[6]) + (fe[7] + fe[8]))));
}
// The nine sources with h_0 = S - sum_{i>0} h_i, so that sum_i h_i = S to
// rounding (the App. A zeroth moment) in every precision.
template <class C>
__device__ __forceinline__ void sources(C S_, C Hz, C Hr, C* h) {
#pragma unroll
  for (int i = 1; i < 9; ++i) h[i] = source(i, S_, Hz, Hr);
  h[0] = S_ - ((h[2] + h[4]) + ((h[1] + h[3]) + ((h[5] + h[6]) + (h[7] + h[8]))));
}

// 256 threads per CTA.  A 2D region of a tile whose width is a multiple of 32
// is walked as warp tasks: a task is a 32-wide segment of one row, so each warp
// reads and writes one contiguous run of a row and branches that depend on the
// row never diverge.
constexpr int NT = 256, NWARP = NT / 32;

//
// A region whose width is not a multiple of 32 would leave lanes idle in its
// last segment of every row (a 36-wide row costs 64 lanes), so such regions
// are walked with a flat index instead (the division is by a compile-time
// constant); a warp may then span two rows.
template <int ROWS, int W, class F>
__device__ __forceinline__ void for_tile(F&& body) {
  if constexpr (W % 32 == 0) {
    constexpr int SEGS = W / 32;
    const int lane = threadIdx.x & 31;
    for (int t = threadIdx.x >> 5; t < ROWS * SEGS; t += NWARP) {
      const int lr = t / SEGS, lc = (t - lr * SEGS) * 32 + lane;
      body(lr, lc);
    }
  } else {
    for (int t = threadIdx.x; t < ROWS * W; t += NT) {
      const int lr = t / W, lc = t - lr * W;
      body(lr, lc);
    }
  }
}

// Tile geometry.  Halos: psi 7, isotropic d_r psi 5, 1D d_r psi (z 5, r 3),
// rho and u 3, collided populations and sources 1.
template <class C, int BZ, int BR>
struct Geo {
  static constexpr int HP = 7, HD = 5, HF = 3;
  static constexpr int PZ = BZ + 2 * HP, PR = BR + 2 * HP;
  static constexpr int DZ = BZ + 2 * HD, DR = BR + 2 * HD;
  static constexpr int EZ = BZ + 2 * HD, ER = BR + 2 * HF;
  static constexpr int FZ = BZ + 2 * HF, FR = BR + 2 * HF;
  static constexpr int SZ = BZ + 2, SR = BR + 2;
  static constexpr int nP = PZ * PR, nD = DZ * DR, nE = EZ * ER, nF = FZ * FR, nS = SZ * SR;
  // region A holds psi and its derivatives, later the sources S, H_z, H_r
  static constexpr int nA = (nP + nD + nE) > 3 * nS ? (nP + nD + nE) : 3 * nS;
  static constexpr int int_bytes = ((PZ + PR) * 4 + 15) / 16 * 16;
  static constexpr size_t bytes = int_bytes + sizeof(C) * (size_t)(nA + 3 * nF + 9 * nS);
};

struct Tile {
  int inst, k0, j0;
};

__device__ __forceinline__ Tile tile_of(const InstDesc* descs, const int* tile_inst, int b, int BZ,
                                        int BR, bool readback = false) {
  Tile t;
  t.inst = tile_inst[b];
  const int tb = readback ? descs[t.inst].rb_tile_base : descs[t.inst].tile_base;
  const int tz = readback ? descs[t.inst].rb_tiles_z : descs[t.inst].tiles_z;
  const int l = b - tb;
  t.k0 = (l % tz) * BZ;
  t.j0 = (l / tz) * BR;
  return t;
}

// The fused update of one tile.  MODE 0: the timestep; MODE 1 (read-back):
// only rho and u of the tile; MODE 2: the forward intermediates of the tile for
// the adjoint (into `inter`, I_COUNT planes of `iplane` elements).
// Resident CTAs per SM the register allocation must allow: five for the FP32
// arithmetic forms (their tiles use at most ~40 KB of shared memory).
template <class S>
struct MinBlocks { static constexpr int value = std::is_same<S, double>::value ? 1 : 5; };

template <class S, int BZ, int BR, int MODE>
__device__ __forceinline__ void lbm_tile(const InstDesc* __restrict__ descs,
                                         const int* __restrict__ tile_inst, int tile, int parity,
                                         typename Store<S>::C* __restrict__ inter, size_t iplane,
                                         uint32_t step = 0) {
  constexpr bool READBACK = MODE == 1;
  using C = typename Store<S>::C;
  using G = Geo<C, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* colmap = reinterpret_cast<int*>(smem_raw);
  int* rowmap = colmap + G::PZ;
  C* base = reinterpret_cast<C*>(smem_raw + G::int_bytes);
  C* sPsi = base;
  C* sDr = sPsi + G::nP;
  C* sD1 = sDr + G::nD;
  C* sS = base;  // after stage 2
  C* sHz = sS + G::nS;
  C* sHr = sHz + G::nS;
  C* sRho = base + G::nA;
  C* sUz = sRho + G::nF;
  C* sUr = sUz + G::nF;
  C* sFs = sUr + G::nF;

  const Tile T = tile_of(descs, tile_inst, tile, BZ, BR, READBACK);
  const InstDesc& D = descs[T.inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P, k0 = T.k0, j0 = T.j0;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const C tau = C(D.tau), omega = C(1) / tau, Gc = C(D.G), gz = C(D.gz), rho0 = C(D.rho0),
          rref = C(D.rho_ref), gfac = -(Gc / C(2)) * C(1.0 / 9.0), inv_rho0 = rcp_c(rho0);

  for (int i = threadIdx.x; i < G::PZ; i += NT) colmap[i] = wrapz(k0 - G::HP + i, Nz);
  for (int i = threadIdx.x; i < G::PR; i += NT) rowmap[i] = reflect_row(j0 - G::HP + i, Nr);
  __syncthreads();

  // Stage 0: psi with ghost cells (periodic z, even mirror in r).
  for_tile<G::PR, G::PZ>([&](int lr, int lc) {
    sPsi[lr * G::PZ + lc] = psin[(size_t)rowmap[lr] * P + colmap[lc]];
  });
  __syncthreads();

  // Stage 1: isotropic d_r psi (tile + 5) and 1D d_r psi (z: tile + 5, r: tile + 3).
  if (ax) {
    for_tile<G::DR, G::DZ>([&](int lr, int lc) {
      sDr[lr * G::DZ + lc] = iso_r(sPsi + (lr + G::HP - G::HD) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    });
    for_tile<G::ER, G::EZ>([&](int lr, int lc) {
      sD1[lr * G::EZ + lc] = d1(sPsi + (lr + G::HP - G::HF) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    });
    __syncthreads();
  }

  // Stage 2 (tile + 3): moments, Shan-Chen force (Eq. scforce), axisymmetric
  // force (Eq. scAxisExtra, c_s^4 = 1/9), body force, u (Eq. uhydro); on the
  // tile + 1 also u^eq (Eq. ueq) and the BGK collision of all nine populations,
  // kept in shared memory for the streaming stage.
  for_tile<G::FR, G::FZ>([&](int lr, int lc) {
    const int j = j0 - G::HF + lr;
    if (j < 0 || j >= Nr) return;
    const C r = C(j) + C(0.5), inv_r = rcp_c(r);
    const bool srow = lr >= 2 && lr < G::FR - 2;
    {
      const C* p = sPsi + (lr + G::HP - G::HF) * G::PZ + (lc + G::HP - G::HF);
      const C psi = p[0];
      const C sb = shift_base(shift, psi, inv_rho0, rho0, rref);
      const S* fp = fin + (size_t)j * P + colmap[lc + G::HP - G::HF];
      C f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = Store<S>::to(fp[i * plane]) + C(w_(i)) * sb;
      // moments and the Shan-Chen neighbour sums in z-mirror pairs (see iso_r)
      const C rho = moment0(f);
      const C jz = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
      const C jr = (f[2] - f[4]) + ((f[5] - f[8]) + (f[6] - f[7]));
      const int Z = G::PZ;
      const C sz = C(1.0 / 9.0) * (p[1] - p[-1]) +
                   C(1.0 / 36.0) * ((p[Z + 1] - p[Z - 1]) + (p[-Z + 1] - p[-Z - 1]));
      const C sr = C(1.0 / 9.0) * (p[Z] - p[-Z]) +
                   C(1.0 / 36.0) * ((p[Z + 1] - p[-Z + 1]) + (p[Z - 1] - p[-Z - 1]));
      C Fz = -Gc * psi * sz, Fr = -Gc * psi * sr;
      if (ax) {
        const C* dr = sDr + (lr + G::HD - G::HF) * G::DZ + (lc + G::HD - G::HF);
        const C Drr = iso_r(dr, G::DZ);
        const C Dzr = d1(sD1 + lr * G::EZ + (lc + G::HD - G::HF), 1);
        const C g = gfac * psi * inv_r;
        Fz += g * Dzr;
        Fr += g * (Drr - dr[0] * inv_r);
      }
      Fz += rho * gz;
      const C inv_rho = rcp_c(rho);
      const int fi = lr * G::FZ + lc;
      sRho[fi] = rho;
      sUz[fi] = (jz + C(0.5) * Fz) * inv_rho;
      sUr[fi] = (jr + C(0.5) * Fr) * inv_rho;
      if (MODE == 2 && lr >= G::HF && lr < G::HF + BR && lc >= G::HF && lc < G::HF + BZ &&
          k0 + lc - G::HF < Nz) {
        C* o = inter + (size_t)j * P + (k0 + lc - G::HF);
        o[I_RHO * iplane] = rho;
        o[I_UZ * iplane] = sUz[fi];
        o[I_UR * iplane] = sUr[fi];
        o[I_VZ * iplane] = (jz + tau * Fz) * inv_rho;
        o[I_VR * iplane] = (jr + tau * Fr) * inv_rho;
        o[I_FZ * iplane] = Fz;
        o[I_FR * iplane] = Fr;
        o[I_PSI * iplane] = psi;
        o[I_SZ * iplane] = sz;
        o[I_SR * iplane] = sr;
        if (ax) {
          const C* dr = sDr + (lr + G::HD - G::HF) * G::DZ + (lc + G::HD - G::HF);
          o[I_DR * iplane] = dr[0];
          o[I_DRR * iplane] = iso_r(dr, G::DZ);
          o[I_DZR * iplane] = d1(sD1 + lr * G::EZ + (lc + G::HD - G::HF), 1);
        } else {
          o[I_DR * iplane] = C(0);
          o[I_DRR * iplane] = C(0);
          o[I_DZR * iplane] = C(0);
        }
      }
      if (MODE == 0 && srow && lc >= 2 && lc < G::FZ - 2) {
        const C vz = (jz + tau * Fz) * inv_rho, vr = (jr + tau * Fr) * inv_rho;
        C fe[9];
        equilibrium(rho, vz, vr, fe);
        C* out = sFs + (lr - 2) * G::SZ + (lc - 2);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i * G::nS] = f[i] + (fe[i] - f[i]) * omega;
      }
    }
  });
  __syncthreads();

  if (READBACK) {
    for_tile<BR, BZ>([&](int lr, int lc) {
      const int j = j0 + lr, k = k0 + lc;
      if (j >= Nr || k >= Nz) return;
      const int fi = (lr + G::HF) * G::FZ + (lc + G::HF);
      const size_t o = (size_t)j * Nz + k;
      D.rho_out[o] = double(sRho[fi]);
      D.uz_out[o] = double(sUz[fi]);
      D.ur_out[o] = double(sUr[fi]);
    });
    return;
  }

  // Ghost rows of u (depth 2) on tiles that touch the axis or the wall: u_z even
  // and u_r odd about the axis; about the outer wall u_r odd and u_z even
  // (free-slip) or odd (no-slip).
  if (ax && (j0 < G::HF || j0 + BR + G::HF > Nr)) {
    for_tile<G::FR, G::FZ>([&](int lr, int lc) {
      const int j = j0 - G::HF + lr;
      int m;
      C sgz;
      if (j == -1 || j == -2) {
        m = -1 - j;
        sgz = C(1);
      } else if (j == Nr || j == Nr + 1) {
        m = 2 * Nr - 1 - j;
        sgz = D.wall == AMLBM_WALL_NOSLIP ? C(-1) : C(1);
      } else {
        return;
      }
      const int src = (m - (j0 - G::HF)) * G::FZ + lc;
      sUz[lr * G::FZ + lc] = sgz * sUz[src];
      sUr[lr * G::FZ + lc] = -sUr[src];
    });
    __syncthreads();
  }

  // Stage 3 (tile + 1): velocity gradients and the sources of App. A,
  // S = -rho u_r / r, H_z, H_r with mu = rho c_s^2 (tau - 1/2), added to the
  // collided populations (the whole h_i, or half of it for the link average).
  const bool link = D.src == AMLBM_SRC_LINK;
  for_tile<G::SR, G::SZ>([&](int lr, int lc) {
    const int j = j0 - 1 + lr;
    if (j < 0 || j >= Nr) return;
    const C r = C(j) + C(0.5), inv_r = rcp_c(r);
    {
      const int si = lr * G::SZ + lc;
      C S_ = C(0), Hz = C(0), Hr = C(0);
      if (ax) {
        const int fi = (lr + 2) * G::FZ + (lc + 2);
        const C druz = iso_r(sUz + fi, G::FZ);
        const C dzur = iso_z(sUr + fi, G::FZ);
        const C drur = iso_r(sUr + fi, G::FZ);
        if (MODE == 2) {
          if (lr >= 1 && lr <= BR && lc >= 1 && lc <= BZ && k0 + lc - 1 < Nz) {
            C* o = inter + (size_t)j * P + (k0 + lc - 1);
            o[I_G1 * iplane] = druz;
            o[I_G2 * iplane] = dzur;
            o[I_G3 * iplane] = drur;
          }
          return;
        }
        const C rho = sRho[fi], uz = sUz[fi], ur = sUr[fi];
        const C mu = rho * (tau - C(0.5)) * C(1.0 / 3.0);
        S_ = -rho * ur * inv_r;
        Hz = (mu * (druz + dzur) - rho * ur * uz) * inv_r;
        Hr = (C(2) * mu * (drur - ur * inv_r) - rho * ur * ur) * inv_r;
        const C hw = link ? C(0.5) : C(1);
        C h[9];
        sources(S_, Hz, Hr, h);
#pragma unroll
        for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] += hw * h[i];
      }
      if (MODE == 2) {
        if (!ax && lr >= 1 && lr <= BR && lc >= 1 && lc <= BZ && k0 + lc - 1 < Nz) {
          C* o = inter + (size_t)j * P + (k0 + lc - 1);
          o[I_G1 * iplane] = C(0);
          o[I_G2 * iplane] = C(0);
          o[I_G3 * iplane] = C(0);
        }
        return;
      }
      sS[si] = S_;
      sHz[si] = Hz;
      sHr[si] = Hr;
    }
  });
  if (MODE == 2) return;
  __syncthreads();

  // Stage 4 (tile): pull streaming.  Away from the axis and the wall every
  // population comes from x - c_i in the same direction; rows 0 and Nr-1 apply
  // the reflection maps (a warp covers one row, so the paths never diverge).
  // Then psi of the new state and the shifted store.
  S* __restrict__ fout = static_cast<S*>(D.f[parity ^ 1]);
  C* __restrict__ psout = static_cast<C*>(D.psi[parity ^ 1]);
  const bool noslip = D.wall == AMLBM_WALL_NOSLIP;
  for_tile<BR, BZ>([&](int lr, int lc) {
    const int j = j0 + lr, k = k0 + lc;
    if (j >= Nr || k >= Nz) return;
    const bool edge = (j == 0) || (j == Nr - 1);
    {
      C fn[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        int sl = lr + 1 - cr_(i), sc = lc + 1 - cz_(i), ii = i;
        if (edge) {
          if (cr_(i) > 0 && j == 0) {  // through the axis: specular reflection
            sl = lr + 1; ii = mirror_(i);
          } else if (cr_(i) < 0 && j == Nr - 1) {  // through the outer wall
            sl = lr + 1;
            if (noslip) { sc = lc + 1; ii = opp_(i); }
            else { ii = mirror_(i); }
          }
        }
        fn[i] = sFs[ii * G::nS + sl * G::SZ + sc];
      }
      if (link) {
        const int di = (lr + 1) * G::SZ + (lc + 1);
        C h[9];
        sources(sS[di], sHz[di], sHr[di], h);
#pragma unroll
        for (int i = 0; i < 9; ++i) fn[i] += C(0.5) * h[i];
      }
      const C rho = moment0(fn);
      const C psi = rho0 * (C(1) - exp_c(-rho / rho0));
      const C sb = shift_base(shift, psi, inv_rho0, rho0, rref);
      store_site<S>(fout + (size_t)j * P + k, plane, fn, sb, D.rounding, (uint32_t)(j * Nz + k), step);
      psout[(size_t)j * P + k] = psi;
    }
  });
}


template <class S, int BZ, int BR, int MODE>
__global__ void __launch_bounds__(NT, MinBlocks<S>::value) lbm_kernel(const InstDesc* __restrict__ descs,
                                                 const int* __restrict__ tile_inst, int toff,
                                                 int parity, typename Store<S>::C* __restrict__ inter,
                                                 size_t iplane) {
  lbm_tile<S, BZ, BR, MODE>(descs, tile_inst, blockIdx.x + toff, parity, inter, iplane);
}

// The timestep as a persistent grid (as many CTAs as fit on the GPU at once):
// CTAs take tiles from a counter in the order of the tile list until none is
// left, so uneven lattices and ragged tiles leave no partial last wave.
// ctr[parity] counts this step's tiles; ctr[parity ^ 1], last used by the
// previous step (which the stream has completed), is reset for the next one.
// No CTA waits on another.  ctr[2], ctr[3] carry the step number the same way.
template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT, MinBlocks<S>::value) lbm_persistent(
    const InstDesc* __restrict__ descs, const int* __restrict__ tile_inst, int ntiles, int parity,
    int* __restrict__ ctr) {
  __shared__ int s_tile;
  // ctr[2 + parity] is this step's number (for the stochastic rounding); the
  // next step reads ctr[2 + (parity ^ 1)].
  const uint32_t step = (uint32_t)ctr[2 + parity];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr[parity ^ 1] = 0;
    ctr[2 + (parity ^ 1)] = (int)(step + 1);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctr[parity], 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) return;
    lbm_tile<S, BZ, BR, 0>(descs, tile_inst, t, parity, nullptr, 0, step);
    __syncthreads();
  }
}

// ------------------------------------------------------------ split schedule --
// The same update as lbm_kernel MODE 0 in two kernels, so that the heavy
// per-site chain runs once per site instead of on a halo of 3:
//   force_kernel  : psi tile + 4, d_r psi on tile + 2, 1D d_r psi on tile
//                   (z + 2); per site of the tile the moments, forces, u and u^eq,
//                   written to four planes;
//   stream_kernel : u with a halo of 3 (ghost rows mirrored), populations on the
//                   tile + 1, collision, gradients and sources, gather-stream.
// The arithmetic is the fused kernel's, operation for operation, so the two
// schedules give bit-identical states.
template <class C, int BZ, int BR>
struct GeoA {
  static constexpr int HP = 4, HD = 2;
  static constexpr int PZ = BZ + 2 * HP, PR = BR + 2 * HP;
  static constexpr int DZ = BZ + 2 * HD, DR = BR + 2 * HD;
  static constexpr int EZ = BZ + 2 * HD, ER = BR;
  static constexpr int nP = PZ * PR, nD = DZ * DR, nE = EZ * ER;
  static constexpr int int_bytes = ((PZ + PR) * 4 + 15) / 16 * 16;
  static constexpr size_t bytes = int_bytes + sizeof(C) * (size_t)(nP + nD + nE);
};

template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT) force_kernel(const InstDesc* __restrict__ descs,
                                                   const int* __restrict__ tile_inst, int toff,
                                                   int parity) {
  using C = typename Store<S>::C;
  using G = GeoA<C, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* colmap = reinterpret_cast<int*>(smem_raw);
  int* rowmap = colmap + G::PZ;
  C* sPsi = reinterpret_cast<C*>(smem_raw + G::int_bytes);
  C* sDr = sPsi + G::nP;
  C* sD1 = sDr + G::nD;
  const Tile T = tile_of(descs, tile_inst, blockIdx.x + toff, BZ, BR);
  const InstDesc& D = descs[T.inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P, k0 = T.k0, j0 = T.j0;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  C* __restrict__ uv = static_cast<C*>(D.uv);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const C tau = C(D.tau), Gc = C(D.G), gz = C(D.gz), rho0 = C(D.rho0), rref = C(D.rho_ref),
          gfac = -(Gc / C(2)) * C(1.0 / 9.0), inv_rho0 = rcp_c(rho0);

  for (int i = threadIdx.x; i < G::PZ; i += NT) colmap[i] = wrapz(k0 - G::HP + i, Nz);
  for (int i = threadIdx.x; i < G::PR; i += NT) rowmap[i] = reflect_row(j0 - G::HP + i, Nr);
  __syncthreads();
  for_tile<G::PR, G::PZ>([&](int lr, int lc) {
    sPsi[lr * G::PZ + lc] = psin[(size_t)rowmap[lr] * P + colmap[lc]];
  });
  __syncthreads();
  if (ax) {
    for_tile<G::DR, G::DZ>([&](int lr, int lc) {
      sDr[lr * G::DZ + lc] = iso_r(sPsi + (lr + G::HP - G::HD) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    });
    for_tile<G::ER, G::EZ>([&](int lr, int lc) {
      sD1[lr * G::EZ + lc] = d1(sPsi + (lr + G::HP) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    });
    __syncthreads();
  }
  for_tile<BR, BZ>([&](int lr, int lc) {
    const int j = j0 + lr, k = k0 + lc;
    if (j >= Nr || k >= Nz) return;
    const C r = C(j) + C(0.5), inv_r = rcp_c(r);
    const C* p = sPsi + (lr + G::HP) * G::PZ + (lc + G::HP);
    const C psi = p[0];
    const C sb = shift_base(shift, psi, inv_rho0, rho0, rref);
    const S* fp = fin + (size_t)j * P + k;
    C f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Store<S>::to(fp[i * plane]) + C(w_(i)) * sb;
    const C rho = moment0(f);
    const C jz = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    const C jr = (f[2] - f[4]) + ((f[5] - f[8]) + (f[6] - f[7]));
    const int Z = G::PZ;
    const C sz = C(1.0 / 9.0) * (p[1] - p[-1]) +
                 C(1.0 / 36.0) * ((p[Z + 1] - p[Z - 1]) + (p[-Z + 1] - p[-Z - 1]));
    const C sr = C(1.0 / 9.0) * (p[Z] - p[-Z]) +
                 C(1.0 / 36.0) * ((p[Z + 1] - p[-Z + 1]) + (p[Z - 1] - p[-Z - 1]));
    C Fz = -Gc * psi * sz, Fr = -Gc * psi * sr;
    if (ax) {
      const C* dr = sDr + (lr + G::HD) * G::DZ + (lc + G::HD);
      const C Drr = iso_r(dr, G::DZ);
      const C Dzr = d1(sD1 + lr * G::EZ + (lc + G::HD), 1);
      const C g = gfac * psi * inv_r;
      Fz += g * Dzr;
      Fr += g * (Drr - dr[0] * inv_r);
    }
    Fz += rho * gz;
    const C inv_rho = rcp_c(rho);
    C* o = uv + (size_t)j * P + k;
    o[0] = (jz + C(0.5) * Fz) * inv_rho;
    o[plane] = (jr + C(0.5) * Fr) * inv_rho;
    o[2 * plane] = (jz + tau * Fz) * inv_rho;
    o[3 * plane] = (jr + tau * Fr) * inv_rho;
  });
}

template <class C, int BZ, int BR>
struct GeoB {
  static constexpr int HF = 3;
  static constexpr int FZ = BZ + 2 * HF, FR = BR + 2 * HF;
  static constexpr int SZ = BZ + 2, SR = BR + 2;
  static constexpr int nF = FZ * FR, nS = SZ * SR;
  static constexpr int int_bytes = (FZ * 4 + 15) / 16 * 16;
  static constexpr size_t bytes = int_bytes + sizeof(C) * (size_t)(2 * nF + 13 * nS);
};

template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT) stream_kernel(const InstDesc* __restrict__ descs,
                                                    const int* __restrict__ tile_inst, int toff,
                                                    int parity, int* __restrict__ ctr) {
  const uint32_t step = ctr ? (uint32_t)ctr[2 + parity] : 0u;
  if (ctr && blockIdx.x == 0 && threadIdx.x == 0) ctr[2 + (parity ^ 1)] = (int)(step + 1);
  using C = typename Store<S>::C;
  using G = GeoB<C, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* colmap = reinterpret_cast<int*>(smem_raw);
  C* sUz = reinterpret_cast<C*>(smem_raw + G::int_bytes);
  C* sUr = sUz + G::nF;
  C* sRho = sUr + G::nF;
  C* sS = sRho + G::nS;
  C* sHz = sS + G::nS;
  C* sHr = sHz + G::nS;
  C* sFs = sHr + G::nS;
  const Tile T = tile_of(descs, tile_inst, blockIdx.x + toff, BZ, BR);
  const InstDesc& D = descs[T.inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P, k0 = T.k0, j0 = T.j0;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  const C* __restrict__ uv = static_cast<const C*>(D.uv);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const C tau = C(D.tau), omega = C(1) / tau, rho0 = C(D.rho0), rref = C(D.rho_ref),
          inv_rho0 = rcp_c(rho0);
  const bool noslip = D.wall == AMLBM_WALL_NOSLIP;

  for (int i = threadIdx.x; i < G::FZ; i += NT) colmap[i] = wrapz(k0 - G::HF + i, Nz);
  __syncthreads();
  // u on the tile + 3; ghost rows (depth 2) by the mirror rules of the fused kernel
  if (ax) {
    for_tile<G::FR, G::FZ>([&](int lr, int lc) {
      const int j = j0 - G::HF + lr;
      int m = j;
      C sgz = C(1), sgr = C(1);
      if (j == -1 || j == -2) {
        m = -1 - j;
        sgr = C(-1);
      } else if (j == Nr || j == Nr + 1) {
        m = 2 * Nr - 1 - j;
        sgr = C(-1);
        sgz = noslip ? C(-1) : C(1);
      } else if (j < 0 || j >= Nr) {
        return;  // never read
      }
      const size_t o = (size_t)m * P + colmap[lc];
      sUz[lr * G::FZ + lc] = sgz * uv[o];
      sUr[lr * G::FZ + lc] = sgr * uv[plane + o];
    });
  }
  // populations on the tile + 1: rho and the collision towards f^eq(rho, u^eq)
  for_tile<G::SR, G::SZ>([&](int lr, int lc) {
    const int j = j0 - 1 + lr;
    if (j < 0 || j >= Nr) return;
    const size_t o = (size_t)j * P + colmap[lc + G::HF - 1];
    const C sb = shift_base(shift, psin[o], inv_rho0, rho0, rref);
    C f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Store<S>::to(fin[i * plane + o]) + C(w_(i)) * sb;
    const C rho = moment0(f);
    const C vz = uv[2 * plane + o], vr = uv[3 * plane + o];
    C fe[9];
    equilibrium(rho, vz, vr, fe);
    const int si = lr * G::SZ + lc;
    sRho[si] = rho;
#pragma unroll
    for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = f[i] + (fe[i] - f[i]) * omega;
  });
  __syncthreads();
  // gradients and sources on the tile + 1
  const bool link = D.src == AMLBM_SRC_LINK;
  for_tile<G::SR, G::SZ>([&](int lr, int lc) {
    const int j = j0 - 1 + lr;
    if (j < 0 || j >= Nr) return;
    const int si = lr * G::SZ + lc;
    C S_ = C(0), Hz = C(0), Hr = C(0);
    if (ax) {
      const C r = C(j) + C(0.5), inv_r = rcp_c(r);
      const int fi = (lr + 2) * G::FZ + (lc + 2);
      const C druz = iso_r(sUz + fi, G::FZ);
      const C dzur = iso_z(sUr + fi, G::FZ);
      const C drur = iso_r(sUr + fi, G::FZ);
      const C rho = sRho[si], uz = sUz[fi], ur = sUr[fi];
      const C mu = rho * (tau - C(0.5)) * C(1.0 / 3.0);
      S_ = -rho * ur * inv_r;
      Hz = (mu * (druz + dzur) - rho * ur * uz) * inv_r;
      Hr = (C(2) * mu * (drur - ur * inv_r) - rho * ur * ur) * inv_r;
      const C hw = link ? C(0.5) : C(1);
      C h[9];
      sources(S_, Hz, Hr, h);
#pragma unroll
      for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] += hw * h[i];
    }
    sS[si] = S_;
    sHz[si] = Hz;
    sHr[si] = Hr;
  });
  __syncthreads();
  S* __restrict__ fout = static_cast<S*>(D.f[parity ^ 1]);
  C* __restrict__ psout = static_cast<C*>(D.psi[parity ^ 1]);
  for_tile<BR, BZ>([&](int lr, int lc) {
    const int j = j0 + lr, k = k0 + lc;
    if (j >= Nr || k >= Nz) return;
    const bool edge = (j == 0) || (j == Nr - 1);
    C fn[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      int sl = lr + 1 - cr_(i), sc = lc + 1 - cz_(i), ii = i;
      if (edge) {
        if (cr_(i) > 0 && j == 0) {
          sl = lr + 1; ii = mirror_(i);
        } else if (cr_(i) < 0 && j == Nr - 1) {
          sl = lr + 1;
          if (noslip) { sc = lc + 1; ii = opp_(i); }
          else { ii = mirror_(i); }
        }
      }
      fn[i] = sFs[ii * G::nS + sl * G::SZ + sc];
    }
    if (link) {
      const int di = (lr + 1) * G::SZ + (lc + 1);
      C h[9];
      sources(sS[di], sHz[di], sHr[di], h);
#pragma unroll
      for (int i = 0; i < 9; ++i) fn[i] += C(0.5) * h[i];
    }
    const C rho = moment0(fn);
    const C psi = rho0 * (C(1) - exp_c(-rho / rho0));
    const C sb = shift_base(shift, psi, inv_rho0, rho0, rref);
    store_site<S>(fout + (size_t)j * P + k, plane, fn, sb, D.rounding, (uint32_t)(j * Nz + k), step);
    psout[(size_t)j * P + k] = psi;
  });
}

// f = f^eq(rho, u) (no force shift) and psi of the new state.
// Site n = j*Nz + k of instance D: f = f^eq(rho, u) with u^eq = u (the
// initial state of the scheme), stored in the instance's storage form, and psi.
template <class S>
__device__ __forceinline__ void init_site(const InstDesc& D, int n, double rho_d, double uz_d,
                                          double ur_d, int parity) {
  using C = typename Store<S>::C;
  const int j = n / D.Nz, k = n - j * D.Nz;
  const size_t plane = (size_t)D.P * D.Nr, o = (size_t)j * D.P + k;
  S* f = static_cast<S*>(D.f[parity]);
  C* psi_out = static_cast<C*>(D.psi[parity]);
  const C rho0 = C(D.rho0), rref = C(D.rho_ref);
  C fe[9];
  equilibrium(C(rho_d), C(uz_d), C(ur_d), fe);
  const C rho = moment0(fe);
  const C psi = rho0 * (C(1) - exp_c(-rho / rho0));
  const C sb = shift_base(D.shift, psi, rcp_c(rho0), rho0, rref);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i * plane + o] = Store<S>::from(fe[i] - C(w_(i)) * sb);
  psi_out[o] = psi;
}

template <class S>
__global__ void init_kernel(const InstDesc* __restrict__ descs, int inst, const double* rho_in,
                            const double* uz_in, const double* ur_in, int parity) {
  const InstDesc& D = descs[inst];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= D.Nz * D.Nr) return;
  init_site<S>(D, n, rho_in[n], uz_in ? uz_in[n] : 0.0, ur_in ? ur_in[n] : 0.0, parity);
}

// Every instance of a batch from arrays holding them back to back: global site
// g belongs to the instance m with site_off[m] <= g < site_off[m + 1].  Sites
// whose rho is not positive and finite are counted into *bad and the state is
// written all the same (the caller writes into the buffers of the other parity
// and discards them when *bad is non-zero).
template <class S>
__global__ void init_all_kernel(const InstDesc* __restrict__ descs, int n_inst,
                                const long long* __restrict__ site_off, long long total,
                                const double* rho_in, const double* uz_in, const double* ur_in,
                                int parity, int* bad) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (site_off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  const double rho = rho_in[g];
  const bool ok = rho > 0 && isfinite(rho);
  if (!ok) atomicAdd(bad, 1);
  init_site<S>(descs[lo], (int)(g - site_off[lo]), ok ? rho : 1.0, uz_in ? uz_in[g] : 0.0,
               ur_in ? ur_in[g] : 0.0, parity);
}

template <class S>
__global__ void unpack_kernel(const InstDesc* __restrict__ descs, int inst, int parity,
                              double* out) {
  using C = typename Store<S>::C;
  const InstDesc& D = descs[inst];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = D.Nz * D.Nr;
  if (n >= N) return;
  const int j = n / D.Nz, k = n - j * D.Nz;
  const size_t plane = (size_t)D.P * D.Nr, o = (size_t)j * D.P + k;
  const S* f = static_cast<const S*>(D.f[parity]);
  const C psi = static_cast<const C*>(D.psi[parity])[o];
  const C sb = shift_base(D.shift, psi, rcp_c(C(D.rho0)), C(D.rho0), C(D.rho_ref));
#pragma unroll
  for (int i = 0; i < 9; ++i) out[(size_t)i * N + n] = double(Store<S>::to(f[i * plane + o]) + C(w_(i)) * sb);
}

template <class S, int BZ, int BR, int MODE>
cudaError_t launch_t(const InstDesc* d, const int* ti, int ntiles, int toff, int parity,
                     cudaStream_t s, void* inter = nullptr, size_t iplane = 0, int* ctr = nullptr) {
  using C = typename Store<S>::C;
  constexpr size_t smem = Geo<C, BZ, BR>::bytes;
  static bool attr = false;
  static int grid_cap = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(lbm_kernel<S, BZ, BR, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && MODE == 0)
      e = cudaFuncSetAttribute(lbm_persistent<S, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e != cudaSuccess) return e;
    if (MODE == 0) {
      int dev = 0, sms = 0, per_sm = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm_persistent<S, BZ, BR>, NT, smem);
      if (e != cudaSuccess) return e;
      grid_cap = sms * (per_sm > 0 ? per_sm : 1);
    }
    attr = true;
  }
  if (MODE == 0 && ctr && toff == 0) {
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    lbm_persistent<S, BZ, BR><<<grid, NT, smem, s>>>(d, ti, ntiles, parity, ctr);
  } else {
    lbm_kernel<S, BZ, BR, MODE><<<ntiles, NT, smem, s>>>(d, ti, toff, parity, static_cast<C*>(inter),
                                                         iplane);
  }
  return cudaGetLastError();
}

template <class S, int BZ, int BR>
cudaError_t launch_split_t(const InstDesc* d, const int* ti, int ntiles, int toff, int parity,
                           cudaStream_t s, int* ctr) {
  using C = typename Store<S>::C;
  constexpr size_t sa = GeoA<C, BZ, BR>::bytes, sbb = GeoB<C, BZ, BR>::bytes;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(force_kernel<S, BZ, BR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(stream_kernel<S, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sbb);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  force_kernel<S, BZ, BR><<<ntiles, NT, sa, s>>>(d, ti, toff, parity);
  stream_kernel<S, BZ, BR><<<ntiles, NT, sbb, s>>>(d, ti, toff, parity, ctr);
  return cudaGetLastError();
}

// Tile shapes compiled for each storage form.
struct TileEntry { int storage, sched, tz, tr; };
#define AMLBM_TILES_16(ST)                                                                    \
  {ST, SCHED_FUSED, 32, 8}, {ST, SCHED_FUSED, 64, 8}, {ST, SCHED_FUSED, 58, 8},               \
  {ST, SCHED_FUSED, 58, 16}, {ST, SCHED_FUSED, 26, 16}, {ST, SCHED_FUSED, 32, 16},            \
  {ST, SCHED_FUSED, 122, 8}, {ST, SCHED_SPLIT, 32, 8}, {ST, SCHED_SPLIT, 64, 8},              \
  {ST, SCHED_SPLIT, 32, 16}, {ST, SCHED_SPLIT, 64, 16}, {ST, SCHED_SPLIT, 128, 8},            \
  {ST, SCHED_SPLIT, 64, 4}, {ST, SCHED_FUSED, 32, 32}, {ST, SCHED_FUSED, 64, 16}
constexpr TileEntry kTiles[] = {
    {AMLBM_STORE_F64, SCHED_FUSED, 32, 8}, {AMLBM_STORE_F64, SCHED_FUSED, 64, 8},
    {AMLBM_STORE_F64, SCHED_FUSED, 58, 8}, {AMLBM_STORE_F64, SCHED_FUSED, 26, 8},
    {AMLBM_STORE_F64, SCHED_SPLIT, 32, 8}, {AMLBM_STORE_F64, SCHED_SPLIT, 64, 8},
    {AMLBM_STORE_F64, SCHED_SPLIT, 32, 16},
    AMLBM_TILES_16(AMLBM_STORE_F32), AMLBM_TILES_16(AMLBM_STORE_F16), AMLBM_TILES_16(AMLBM_STORE_BF16),
};
#undef AMLBM_TILES_16

template <class S>
cudaError_t dispatch(bool macro, int sched, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                     int toff, int par, cudaStream_t s, int* ctr) {
  if (nt <= 0) return cudaSuccess;
  if (sched == SCHED_SPLIT && !macro) {
#define AMLBM_SPLIT(TZ, TR) \
  if (tz == TZ && tr == TR) return launch_split_t<S, TZ, TR>(d, ti, nt, toff, par, s, ctr);
    AMLBM_SPLIT(32, 8)
    AMLBM_SPLIT(64, 8)
    AMLBM_SPLIT(32, 16)
    if constexpr (!std::is_same<S, double>::value) {
      AMLBM_SPLIT(64, 16)
      AMLBM_SPLIT(128, 8)
      AMLBM_SPLIT(64, 4)
    }
#undef AMLBM_SPLIT
    return cudaErrorInvalidValue;
  }
#define AMLBM_TILE(TZ, TR)                                                \
  if (tz == TZ && tr == TR)                                               \
    return macro ? launch_t<S, TZ, TR, 1>(d, ti, nt, toff, par, s)        \
                 : launch_t<S, TZ, TR, 0>(d, ti, nt, toff, par, s, nullptr, 0, ctr);
  if (macro) {  // read-back always uses a fused tile compiled for every storage
    AMLBM_TILE(32, 8)
    return cudaErrorInvalidValue;
  }
  AMLBM_TILE(32, 8)
  AMLBM_TILE(64, 8)
  AMLBM_TILE(58, 8)
  if constexpr (std::is_same<S, double>::value) {
    AMLBM_TILE(26, 8)
  } else {
    AMLBM_TILE(58, 16)
    AMLBM_TILE(26, 16)
    AMLBM_TILE(32, 16)
    AMLBM_TILE(122, 8)
    AMLBM_TILE(32, 32)
    AMLBM_TILE(64, 16)
  }
#undef AMLBM_TILE
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_storage(int storage, bool macro, int sched, int tz, int tr, const InstDesc* d,
                             const int* ti, int nt, int toff, int par, cudaStream_t s, int* ctr) {
  switch (storage) {
    case AMLBM_STORE_F64: return dispatch<double>(macro, sched, tz, tr, d, ti, nt, toff, par, s, ctr);
    case AMLBM_STORE_F32: return dispatch<float>(macro, sched, tz, tr, d, ti, nt, toff, par, s, ctr);
    case AMLBM_STORE_F16: return dispatch<__half>(macro, sched, tz, tr, d, ti, nt, toff, par, s, ctr);
    case AMLBM_STORE_BF16:
      return dispatch<__nv_bfloat16>(macro, sched, tz, tr, d, ti, nt, toff, par, s, ctr);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool tile_supported(int storage, int sched, int tz, int tr) {
  for (const auto& e : kTiles)
    if (e.storage == storage && e.sched == sched && e.tz == tz && e.tr == tr) return true;
  return false;
}

int tile_list(int storage, int sched, int* tz, int* tr, int cap) {
  int n = 0;
  for (const auto& e : kTiles)
    if (e.storage == storage && e.sched == sched) {
      if (n < cap && tz && tr) { tz[n] = e.tz; tr[n] = e.tr; }
      ++n;
    }
  return n;
}

size_t step_smem_bytes(int storage, int tz, int tr) {
  const size_t c = storage == AMLBM_STORE_F64 ? 8 : 4;
  const int nP = (tz + 14) * (tr + 14), nD = (tz + 10) * (tr + 10), nE = (tz + 10) * (tr + 6);
  const int nF = (tz + 6) * (tr + 6), nS = (tz + 2) * (tr + 2);
  const int nA = (nP + nD + nE) > 3 * nS ? (nP + nD + nE) : 3 * nS;
  const size_t ib = ((size_t)(tz + 14 + tr + 14) * 4 + 15) / 16 * 16;
  return ib + c * (size_t)(nA + 3 * nF + 9 * nS);
}

cudaError_t launch_step(int storage, int sched, int tz, int tr, const InstDesc* d, const int* ti,
                        int nt, int toff, int parity, cudaStream_t s, int* ctr) {
  return dispatch_storage(storage, false, sched, tz, tr, d, ti, nt, toff, parity, s, ctr);
}
cudaError_t launch_macro(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                         int toff, int parity, cudaStream_t s) {
  return dispatch_storage(storage, true, SCHED_FUSED, tz, tr, d, ti, nt, toff, parity, s, nullptr);
}

cudaError_t launch_inter(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                         void* inter, size_t plane, cudaStream_t s) {
  if (storage == AMLBM_STORE_F64) {
    if (tz == 32 && tr == 8) return launch_t<double, 32, 8, 2>(d, ti, nt, 0, 0, s, inter, plane);
  } else if (storage == AMLBM_STORE_F32) {
    if (tz == 32 && tr == 8) return launch_t<float, 32, 8, 2>(d, ti, nt, 0, 0, s, inter, plane);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_init(int storage, const InstDesc* d, int inst, int Nz, int Nr, const double* rho,
                        const double* uz, const double* ur, int parity, cudaStream_t s) {
  const int N = Nz * Nr, nb = (N + 255) / 256;
  switch (storage) {
    case AMLBM_STORE_F64: init_kernel<double><<<nb, 256, 0, s>>>(d, inst, rho, uz, ur, parity); break;
    case AMLBM_STORE_F32: init_kernel<float><<<nb, 256, 0, s>>>(d, inst, rho, uz, ur, parity); break;
    case AMLBM_STORE_F16: init_kernel<__half><<<nb, 256, 0, s>>>(d, inst, rho, uz, ur, parity); break;
    case AMLBM_STORE_BF16: init_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>(d, inst, rho, uz, ur, parity); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init_all(int storage, const InstDesc* d, int n, const long long* site_off,
                            long long total, const double* rho, const double* uz, const double* ur,
                            int parity, int* bad, cudaStream_t s) {
  if (total < 1) return cudaErrorInvalidValue;
  const unsigned nb = (unsigned)((total + 255) / 256);
  switch (storage) {
    case AMLBM_STORE_F64:
      init_all_kernel<double><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad); break;
    case AMLBM_STORE_F32:
      init_all_kernel<float><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad); break;
    case AMLBM_STORE_F16:
      init_all_kernel<__half><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad); break;
    case AMLBM_STORE_BF16:
      init_all_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack(int storage, const InstDesc* d, int inst, int Nz, int Nr, int parity,
                          double* out, cudaStream_t s) {
  const int N = Nz * Nr, nb = (N + 255) / 256;
  switch (storage) {
    case AMLBM_STORE_F64: unpack_kernel<double><<<nb, 256, 0, s>>>(d, inst, parity, out); break;
    case AMLBM_STORE_F32: unpack_kernel<float><<<nb, 256, 0, s>>>(d, inst, parity, out); break;
    case AMLBM_STORE_F16: unpack_kernel<__half><<<nb, 256, 0, s>>>(d, inst, parity, out); break;
    case AMLBM_STORE_BF16: unpack_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>(d, inst, parity, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace amlbm
