// Fused axisymmetric Shan-Chen LBM step for sm_103a (arXiv:1310.1871, Sec. II).
//
// One CTA updates one tile of lattice sites of one lattice of a batch.  The
// whole per-site chain of the paper's update runs inside the CTA:
//   psi tile + halo 7 (from the previous step's psi, staged in shared memory)
//   -> isotropic d_r psi and 1D d_r psi (Sec. II.D), halo 5
//   -> moments, Shan-Chen force (Eq. scforce), axisymmetric force
//      (Eq. scAxisExtra), u and u^eq (Eqs. uhydro, ueq), halo 3
//   -> velocity gradients (1D 4th-order differences of Sec. II.D) and the
//      sources S, H_z, H_r (Eq. condition_h), halo 1
//   -> pull streaming of the BGK-collided populations (Eq. lbm2d_mod_new) with
//      the axis / wall / periodic maps of Sec. II.E, and psi of the new state.
// Global traffic per site and step: 9 populations read (halo re-reads hit L2),
// 9 written, psi written once and read once (halo re-reads hit L2).
// No tensor cores: the update is a stencil, not a contraction.
//
// The arithmetic is written once on "lane" types, F1 (FP32) and D1 (FP64),
// whose every operation is an explicitly rounded intrinsic: each fused
// multiply-add is written out and nothing else is left to the compiler's
// contraction, so every schedule and tiling computes a site with the same
// operations and gets the same bits.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <stdint.h>

#include <mutex>
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

// ---------------------------------------------------------------- lanes --
struct F1 { float v; };
struct D1 { double v; };

__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return {__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return {__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return {__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator-(F1 a) { return {-a.v}; }
__device__ __forceinline__ F1 fma(F1 a, F1 b, F1 c) { return {__fmaf_rn(a.v, b.v, c.v)}; }

__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return {__dadd_rn(a.v, b.v)}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return {__dsub_rn(a.v, b.v)}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return {__dmul_rn(a.v, b.v)}; }
__device__ __forceinline__ D1 operator-(D1 a) { return {-a.v}; }
__device__ __forceinline__ D1 fma(D1 a, D1 b, D1 c) { return {__fma_rn(a.v, b.v, c.v)}; }

template <class T> struct Lane;
template <> struct Lane<F1> { using C = float; static constexpr int N = 1; };
template <> struct Lane<D1> { using C = double; static constexpr int N = 1; };

template <class T> __device__ __forceinline__ T lit(double c);
template <> __device__ __forceinline__ F1 lit<F1>(double c) { return {float(c)}; }
template <> __device__ __forceinline__ D1 lit<D1>(double c) { return {c}; }

// Reciprocal and exponential.  FP32 uses the correctly rounded
// reciprocal and the SFU exponential (relative error ~1e-7, far below the
// storage rounding); FP64 the correctly rounded reciprocal and exp.
__device__ __forceinline__ F1 rcp(F1 a) { return {__frcp_rn(a.v)}; }
__device__ __forceinline__ D1 rcp(D1 a) { return {__drcp_rn(a.v)}; }
__device__ __forceinline__ F1 expl(F1 a) { return {__expf(a.v)}; }
__device__ __forceinline__ D1 expl(D1 a) { return {exp(a.v)}; }

// ------------------------------------------------------------- storage --
// Storage codecs: conversion between the stored element and the arithmetic
// type.  The shift W_i s of the FP32 / 16-bit forms is applied by the callers
// (decode: f = q + W_i s; encode: q = f - W_i s).  IEEE half holds q * 2^10 so
// that the shifted populations (down to ~1e-7) stay in its normal range; the
// power-of-two scale is exact.  from_sr rounds stochastically with the random
// word x: its top bits are added to the bits below the stored precision and the
// sum is truncated, so a value rounds up with probability equal to its distance
// from the lower neighbour (unbiased in expectation).
template <class S> struct Store;
template <> struct Store<double> {
  using C = double;
  using T = D1;
  static __device__ __forceinline__ C to(double v) { return v; }
  static __device__ __forceinline__ double from(C v) { return v; }
  static __device__ __forceinline__ double from_sr(C v, uint32_t) { return v; }
};
template <> struct Store<float> {
  using C = float;
  using T = F1;
  static __device__ __forceinline__ C to(float v) { return v; }
  static __device__ __forceinline__ float from(C v) { return v; }
  static __device__ __forceinline__ float from_sr(C v, uint32_t) { return v; }
};
template <> struct Store<__half> {
  using C = float;
  using T = F1;
  static __device__ __forceinline__ C to(__half v) { return __half2float(v) * (1.0f / 1024.0f); }
  static __device__ __forceinline__ __half from(C v) { return __float2half_rn(v * 1024.0f); }
  static __device__ __forceinline__ __half from_sr(C v, uint32_t x) {
    // FP32 keeps 13 more mantissa bits than FP16 (for FP16-normal values)
    const uint32_t b = __float_as_uint(v * 1024.0f) + (x >> 19);
    return __float2half_rz(__uint_as_float(b));
  }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  using T = F1;
  static __device__ __forceinline__ C to(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 from(C v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ __nv_bfloat16 from_sr(C v, uint32_t x) {
    // bfloat16 is the upper half of the FP32 bit pattern
    const uint32_t b = __float_as_uint(v) + (x >> 16);
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
  }
};

__device__ __forceinline__ float fma_c(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_c(double a, double b, double c) { return __fma_rn(a, b, c); }

// Random words of the stochastic rounding.  Each site seeds its own stream with
// an integer hash (a xorshift-multiply mixer) of (site, step); the nine
// populations then take successive states of the linear congruential generator
// x <- 1664525 x + 1013904223 (mod 2^32) (Knuth / Numerical Recipes constants),
// whose top bits are the ones the codecs use.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ uint32_t lcg_next(uint32_t x) { return x * 1664525u + 1013904223u; }

// Store the nine new populations fn[i] of one site with the shift W_i sb,
// rounding to nearest or (rounding != 0) stochastically with words drawn from
// (site, step).
template <class S>
__device__ __forceinline__ void store_site(S* o, size_t plane, const typename Store<S>::C* fn,
                                           typename Store<S>::C sb, int rounding, uint32_t site,
                                           uint32_t step) {
  using C = typename Store<S>::C;
  if (sizeof(S) == 2 && rounding) {
    uint32_t x = mix32(site ^ mix32(step + 0x9E3779B9u));
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      x = lcg_next(x);
      o[i * plane] = Store<S>::from_sr(fma_c(C(-w_(i)), sb, fn[i]), x);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i * plane] = Store<S>::from(fma_c(C(-w_(i)), sb, fn[i]));
  }
}

// Store q_i = fn[i] - base[i] (the equilibrium shift), rounding as store_site.
template <class S>
__device__ __forceinline__ void store_site_base(S* o, size_t plane, const typename Store<S>::C* fn,
                                                const typename Store<S>::C* base, int rounding,
                                                uint32_t site, uint32_t step) {
  if (sizeof(S) == 2 && rounding) {
    uint32_t x = mix32(site ^ mix32(step + 0x9E3779B9u));
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      x = lcg_next(x);
      o[i * plane] = Store<S>::from_sr(fn[i] - base[i], x);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i * plane] = Store<S>::from(fn[i] - base[i]);
  }
}

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
  if (mode >= 2) {
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
// The same with inlet and outlet rows, whose ghosts mirror about the boundary
// row itself (zero normal derivative of psi there).
__device__ __forceinline__ int ghost_row(int j, int Nr, bool inlet, bool outlet) {
  if (j < 0) j = inlet ? -j : -1 - j;
  if (j >= Nr) j = outlet ? 2 * (Nr - 1) - j : 2 * Nr - 1 - j;
  return j < 0 ? 0 : (j >= Nr ? Nr - 1 : j);
}
// Column of a ghost column: periodic wrap, or the mirror about the walls at
// z = -1/2 and z = Nz - 1/2 (clamped like the rows).
__device__ __forceinline__ int ghost_col(int k, int Nz, bool walls) {
  if (!walls) return wrapz(k, Nz);
  if (k < 0) k = -1 - k;
  if (k >= Nz) k = 2 * Nz - 1 - k;
  return k < 0 ? 0 : (k >= Nz ? Nz - 1 : k);
}

// ------------------------------------------------------------- physics --
// Isotropic 4th-order first derivative along r, Sec. II.D Eq. forthorder_firstderivativex:
//   d_r phi(x) = (1/36) sum_i c_ir (8 phi(x + c_i) - phi(x + 2 c_i)).
// p points at x in a row-major tile whose rows (r) are `st` apart.  The terms
// are added in z-mirror pairs (c_5, c_6), (c_8, c_7) so that a field mirrored
// in z gives an exactly mirrored derivative: without this, the rounding of the
// FP32 forms carries a net axial bias every step and a drop drifts along the
// axis.
template <class T>
__device__ __forceinline__ T link8(const T* p, int dz, int dr, int st) {
  return fma(lit<T>(8.0), p[dr * st + dz], -p[2 * dr * st + 2 * dz]);
}
template <class T>
__device__ __forceinline__ T iso_r(const T* p, int st) {
  const T a = link8(p, 0, 1, st) - link8(p, 0, -1, st);
  const T b = (link8(p, 1, 1, st) + link8(p, -1, 1, st)) - (link8(p, 1, -1, st) + link8(p, -1, -1, st));
  return (a + b) * lit<T>(1.0 / 36.0);
}
// 1D 4th-order central difference with element step `step` (Sec. II.D): the
// inner and outer operators of d_zr psi, and the velocity gradients of the
// sources.  (The velocity gradients do not take the isotropic stencil: its
// diagonal taps reverse the sign of d_r u_z on a mode alternating in z, and
// mu d_r u_z / r then amplifies that mode next to a no-slip wall.)
template <class T>
__device__ __forceinline__ T d1(const T* p, int step) {
  return fma(lit<T>(8.0), p[step] - p[-step], -(p[2 * step] - p[-2 * step])) * lit<T>(1.0 / 12.0);
}

// c_i . v of direction i
template <class T>
__device__ __forceinline__ T cdot(int i, T vz, T vr) {
  switch (i) {
    case 1: return vz;
    case 2: return vr;
    case 3: return -vz;
    case 4: return -vr;
    case 5: return vz + vr;
    case 6: return vr - vz;
    case 7: return -(vz + vr);
    default: return vz - vr;
  }
}
// rho = sum_i f_i and j = sum_i c_i f_i, added in z-mirror pairs.
template <class T>
__device__ __forceinline__ T moment0(const T* f) {
  return (f[0] + (f[2] + f[4])) + ((f[1] + f[3]) + ((f[5] + f[6]) + (f[7] + f[8])));
}
template <class T>
__device__ __forceinline__ T moment_z(const T* f) {
  return (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
}
template <class T>
__device__ __forceinline__ T moment_r(const T* f) {
  return (f[2] - f[4]) + ((f[5] - f[8]) + (f[6] - f[7]));
}
// The nine equilibria (Eq. feq; W_i rho (1 + 3 c.v + 4.5 (c.v)^2 - 1.5 v^2))
// with f^eq_0 = rho - sum_{i>0} f^eq_i: the same value in exact arithmetic, but
// the collision then conserves mass to rounding.  With the directly evaluated
// f^eq_0 the FP32-rounded weights do not sum to 1 and the FP32 forms gain mass
// every step (a 1.5e-5 drift over 1000 steps of the static drop, and a 1e-4
// density error at the interface).
template <class T>
__device__ __forceinline__ void equilibrium(T rho, T vz, T vr, T* fe) {
  const T A = fma(fma(vz, vz, vr * vr), lit<T>(-1.5), lit<T>(1.0));
  const T r9 = rho * lit<T>(1.0 / 9.0), r36 = rho * lit<T>(1.0 / 36.0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const T cv = cdot(i, vz, vr);
    fe[i] = (i < 5 ? r9 : r36) * fma(fma(cv, lit<T>(4.5), lit<T>(3.0)), cv, A);
  }
  fe[0] = rho - ((fe[2] + fe[4]) + ((fe[1] + fe[3]) + ((fe[5] + fe[6]) + (fe[7] + fe[8]))));
}
// h_i = W_i (S + (c_iz H_z + c_ir H_r) / c_s^2), Eq. condition_h, with
// h_0 = S - sum_{i>0} h_i, so that sum_i h_i = S to rounding (the App. A
// zeroth moment) in every precision.
template <class T>
__device__ __forceinline__ void sources(T S_, T Hz, T Hr, T* h) {
  const T z3 = Hz * lit<T>(3.0), r3 = Hr * lit<T>(3.0);
#pragma unroll
  for (int i = 1; i < 9; ++i) h[i] = lit<T>(w_(i)) * (S_ + cdot(i, z3, r3));
  h[0] = S_ - ((h[2] + h[4]) + ((h[1] + h[3]) + ((h[5] + h[6]) + (h[7] + h[8]))));
}
// Discrete force of the Guo forcing (Guo, Zheng & Shi 2002):
//   s_i = W_i (3 (c_i . F - u . F) + 9 (c_i . u)(c_i . F)),
// with s_0 = -sum_{i>0} s_i (zeroth moment 0 to rounding; first moment F).
template <class T>
__device__ __forceinline__ void guo_force(T uz, T ur, T Fz, T Fr, T* s) {
  const T uF = fma(uz, Fz, ur * Fr);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const T cF = cdot(i, Fz, Fr), cu = cdot(i, uz, ur);
    s[i] = lit<T>(w_(i)) * fma(cu * lit<T>(9.0), cF, (cF - uF) * lit<T>(3.0));
  }
  s[0] = -((s[2] + s[4]) + ((s[1] + s[3]) + ((s[5] + s[6]) + (s[7] + s[8]))));
}
// Shan-Chen neighbour sums sum_i W_i psi(x + c_i) c_i (Eq. scforce) around p.
template <class T>
__device__ __forceinline__ void sc_sums(const T* p, int Z, T& sz, T& sr) {
  sz = fma(p[1] - p[-1], lit<T>(1.0 / 9.0),
           ((p[Z + 1] - p[Z - 1]) + (p[-Z + 1] - p[-Z - 1])) * lit<T>(1.0 / 36.0));
  sr = fma(p[Z] - p[-Z], lit<T>(1.0 / 9.0),
           ((p[Z + 1] - p[-Z + 1]) + (p[Z - 1] - p[-Z - 1])) * lit<T>(1.0 / 36.0));
}
// The instance constants of the step in the lane type.
template <class T>
struct Par {
  T tau, omega, negG, gfac, gz, rho0, inv_rho0, cmu;
};
__device__ __forceinline__ float kc(const InstDesc& D, int c, float) { return D.k32[c]; }
__device__ __forceinline__ double kc(const InstDesc& D, int c, double) { return D.k64[c]; }
template <class T>
__device__ __forceinline__ T splat(typename Lane<T>::C c);
template <> __device__ __forceinline__ F1 splat<F1>(float c) { return {c}; }
template <> __device__ __forceinline__ D1 splat<D1>(double c) { return {c}; }
// q.gfac = -(G / 2) c_s^4 with c_s^4 = 1/9; q.cmu = mu / rho = c_s^2 (tau - 1/2)
template <class T>
__device__ __forceinline__ Par<T> par_of(const InstDesc& D) {
  using C = typename Lane<T>::C;
  Par<T> q;
  q.tau = splat<T>(kc(D, K_TAU, C()));
  q.omega = splat<T>(kc(D, K_OMEGA, C()));
  q.negG = splat<T>(kc(D, K_NEGG, C()));
  q.gfac = splat<T>(kc(D, K_GFAC, C()));
  q.gz = splat<T>(kc(D, K_GZ, C()));
  q.rho0 = splat<T>(kc(D, K_RHO0, C()));
  q.inv_rho0 = splat<T>(kc(D, K_INVRHO0, C()));
  q.cmu = splat<T>(kc(D, K_CMU, C()));
  return q;
}
// 1 / r of row j, r = j + r0 with r0 = r_off + 1/2 the radius of row 0 (the sum
// is exact in either precision for the half-integer radii of the workloads)
__device__ __forceinline__ F1 inv_r_of(F1, int j, float r0) { return rcp(F1{__int2float_rn(j) + r0}); }
__device__ __forceinline__ D1 inv_r_of(D1, int j, double r0) { return rcp(D1{__int2double_rn(j) + r0}); }

// Total force on a site (Eq. scforce, Eq. scAxisExtra, body force rho g_z).
template <class T>
__device__ __forceinline__ void forces(const Par<T>& q, T rho, T psi, T sz, T sr, bool ax, T dr0, T Drr,
                                       T Dzr, T inv_r, T& Fz, T& Fr) {
  const T gpsi = psi * q.negG;
  Fz = gpsi * sz;
  Fr = gpsi * sr;
  if (ax) {
    const T g = (psi * q.gfac) * inv_r;
    Fz = fma(g, Dzr, Fz);
    Fr = fma(g, fma(-dr0, inv_r, Drr), Fr);
  }
  Fz = fma(rho, q.gz, Fz);
}
// Axisymmetric sources of App. A at a site: S = -rho u_r / r,
// H_z = (mu (d_r u_z + d_z u_r) - rho u_r u_z) / r,
// H_r = (2 mu (d_r u_r - u_r / r) - rho u_r^2) / r.
template <class T>
__device__ __forceinline__ void site_sources(const Par<T>& q, T rho, T uz, T ur, T druz, T dzur, T drur,
                                             T inv_r, T& S_, T& Hz, T& Hr) {
  const T mu = rho * q.cmu, rur = rho * ur;
  S_ = -(rur * inv_r);
  Hz = fma(mu, druz + dzur, -(rur * uz)) * inv_r;
  Hr = fma(mu * lit<T>(2.0), fma(-ur, inv_r, drur), -(rur * ur)) * inv_r;
}
// psi = rho0 (1 - exp(-rho / rho0)), Eq. psi.
template <class T>
__device__ __forceinline__ T psi_of(const Par<T>& q, T rho) {
  return (lit<T>(1.0) - expl(-rho * q.inv_rho0)) * q.rho0;
}

// Decode the nine populations of a site from their stored values q[i * plane]:
// f_i = q_i + W_i s (shift modes 0-2, one fused multiply-add) or, in the
// equilibrium mode (3), f_i = q_i + f^eq_i(s, v) with the velocity v stored in
// the two planes that follow psi (pv points at the site's psi).
template <class S, class T>
__device__ __forceinline__ void decode_site(int mode, const S* q, size_t plane, typename Store<S>::C psi,
                                            const typename Store<S>::C* pv, typename Store<S>::C inv_rho0,
                                            typename Store<S>::C rho0, typename Store<S>::C rref, T* f) {
  const T sbt{shift_base(mode, psi, inv_rho0, rho0, rref)};
  if (mode == 3) {
    T fe[9];
    equilibrium(sbt, T{pv[plane]}, T{pv[2 * plane]}, fe);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = T{Store<S>::to(q[i * plane])} + fe[i];
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fma(lit<T>(w_(i)), sbt, T{Store<S>::to(q[i * plane])});
  }
}

// Store the new populations fn of a site and its psi (at *pso); in the
// equilibrium mode also the bare velocity v = sum_i c_i fn_i / rho of the new
// state (after psi) and q_i = fn_i - f^eq_i(s, v).
template <class S, class T>
__device__ __forceinline__ void encode_site(int mode, S* o, typename Store<S>::C* pso, size_t plane,
                                            const T* fn, T rho, typename Store<S>::C psi,
                                            typename Store<S>::C inv_rho0, typename Store<S>::C rho0,
                                            typename Store<S>::C rref, int rounding, uint32_t site,
                                            uint32_t step) {
  using C = typename Store<S>::C;
  const C sb = shift_base(mode, psi, inv_rho0, rho0, rref);
  C fv[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fv[i] = fn[i].v;
  if (mode == 3) {
    const T ir = rcp(rho), vz = moment_z(fn) * ir, vr = moment_r(fn) * ir;
    T fe[9];
    equilibrium(T{sb}, vz, vr, fe);
    C base[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) base[i] = fe[i].v;
    store_site_base<S>(o, plane, fv, base, rounding, site, step);
    pso[plane] = vz.v;
    pso[2 * plane] = vr.v;
  } else {
    store_site<S>(o, plane, fv, sb, rounding, site, step);
  }
  pso[0] = psi;
}

// ---------------------------------------------------------------- tiles --
// 256 threads per CTA.  A 2D region of a tile whose width is a multiple of 32
// is walked as warp tasks: a task is a 32-wide segment of one row, so each warp
// reads and writes one contiguous run of a row and branches that depend on the
// row never diverge.  A region whose width is not a multiple of 32 would leave
// lanes idle in its last segment of every row (a 36-wide row costs 64 lanes),
// so such regions are walked with a flat index instead (the division is by a
// compile-time constant); a warp may then span two rows.
constexpr int NT = 256, NWARP = NT / 32;

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

// Tile geometry (BZ x BR sites).  Halos: psi 7, isotropic d_r psi 5, rho and u
// 3, collided populations and sources 1.  The integer maps hold the wrapped
// column and the mirrored row of the psi region.
template <class T, int BZ, int BR>
struct Geo {
  static constexpr int HP = 7, HD = 5, HF = 3;
  static constexpr int PZ = BZ + 2 * HP, PR = BR + 2 * HP;
  static constexpr int DZ = BZ + 2 * HD, DR = BR + 2 * HD;
  static constexpr int FZ = BZ + 2 * HF, FR = BR + 2 * HF;
  static constexpr int SZ = BZ + 2, SR = BR + 2;
  static constexpr int nP = PZ * PR, nD = DZ * DR, nF = FZ * FR, nS = SZ * SR;
  // region A holds psi and d_r psi, later the sources S, H_z, H_r
  static constexpr int nA = (nP + nD) > 3 * nS ? (nP + nD) : 3 * nS;
  static constexpr int int_bytes = ((PZ + PR) * 4 + 15) / 16 * 16;
  static constexpr size_t bytes = int_bytes + sizeof(T) * (size_t)(nA + 3 * nF + 9 * nS);
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

// Resident CTAs per SM the register allocation must allow: for the FP32
// arithmetic forms as many as the tile's shared memory lets fit in the 228 KB of
// an SM (1 KB of it reserved per CTA), at most five (48 registers a thread:
// at six the 40-register budget spills and the step is slower).
template <class S, class T, int BZ, int BR>
struct MinBlocks {
  static constexpr int fit = int((228u * 1024u) / (Geo<T, BZ, BR>::bytes + 1024u));
  static constexpr int value =
      std::is_same<S, double>::value ? 1 : (fit > 5 ? 5 : (fit < 1 ? 1 : fit));
};

// The fused update of one BZ x BR tile in the lane type T of the storage form.
// MODE 0: the timestep; MODE 1 (read-back): only rho and u of the tile; MODE 3:
// the timestep and the forward intermediates of the state it starts from, for
// the adjoint (into `inter`, I_COUNT planes of `iplane` elements).
template <class S, class T, int BZ, int BR, int MODE>
__device__ __forceinline__ void lbm_tile(const InstDesc* __restrict__ descs,
                                         const int* __restrict__ tile_inst, int tile, int parity,
                                         typename Store<S>::C* __restrict__ inter, size_t iplane,
                                         uint32_t step = 0) {
  constexpr bool READBACK = MODE == 1;
  using C = typename Store<S>::C;
  using G = Geo<T, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* colmap = reinterpret_cast<int*>(smem_raw);
  int* rowmap = colmap + G::PZ;
  T* base = reinterpret_cast<T*>(smem_raw + G::int_bytes);
  T* sPsi = base;
  T* sDr = sPsi + G::nP;
  T* sS = base;  // after stage 2
  T* sHz = sS + G::nS;
  T* sHr = sHz + G::nS;
  T* sRho = base + G::nA;
  T* sUz = sRho + G::nF;
  T* sUr = sUz + G::nF;
  T* sFs = sUr + G::nF;

  const Tile Tl = tile_of(descs, tile_inst, tile, BZ, BR, READBACK);
  const InstDesc& D = descs[Tl.inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P, k0 = Tl.k0, j0 = Tl.j0;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const Par<T> q = par_of<T>(D);
  const C rho0c = kc(D, K_RHO0, C()), rrefc = kc(D, K_RREF, C()), inv_rho0c = kc(D, K_INVRHO0, C());
  // bounded domains (Sec. II.E, Sec. III.2): walls at both ends in z, an inlet
  // row at row 0, an outlet row at row Nr - 1
  const bool zw = D.zbc == AMLBM_Z_NOSLIP;
  const bool inl = D.rlo == AMLBM_RLO_INLET, outl = D.wall == AMLBM_WALL_OUTLET;
  const bool guo = D.forcing == AMLBM_FORCE_GUO;

  for (int i = threadIdx.x; i < G::PZ; i += NT) colmap[i] = ghost_col(k0 - G::HP + i, Nz, zw);
  for (int i = threadIdx.x; i < G::PR; i += NT) rowmap[i] = ghost_row(j0 - G::HP + i, Nr, inl, outl);
  __syncthreads();

  // Stage 0: psi with ghost cells (periodic z or mirrored about the z walls,
  // even mirror in r).
  for_tile<G::PR, G::PZ>([&](int lr, int lc) {
    sPsi[lr * G::PZ + lc] = T{psin[(size_t)rowmap[lr] * P + colmap[lc]]};
  });
  __syncthreads();

  // Stage 1: isotropic d_r psi (tile + 5).
  if (ax) {
    for_tile<G::DR, G::DZ>([&](int lr, int lc) {
      sDr[lr * G::DZ + lc] = iso_r(sPsi + (lr + G::HP - G::HD) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    });
    __syncthreads();
  }

  // Stage 2 (tile + 3): moments, forces, u (Eq. uhydro); on the tile + 1 also
  // u^eq (Eq. ueq) and the BGK collision of all nine populations, kept in
  // shared memory for the streaming stage.
  for_tile<G::FR, G::FZ>([&](int lr, int lc) {
    const int j = j0 - G::HF + lr;
    if (j < 0 || j >= Nr) return;
    const T inv_r = inv_r_of(T(), j, kc(D, K_R0, C()));
    const bool srow = lr >= 2 && lr < G::FR - 2;
    const T* p = sPsi + (lr + G::HP - G::HF) * G::PZ + (lc + G::HP - G::HF);
    const T psi = p[0];
    T f[9];
    {
      const size_t so = (size_t)j * P + colmap[lc + G::HP - G::HF];
      decode_site<S>(shift, fin + so, plane, psi.v, psin + so, inv_rho0c, rho0c, rrefc, f);
    }
    const T rho = moment0(f), jz = moment_z(f), jr = moment_r(f);
    T sz, sr;
    sc_sums(p, G::PZ, sz, sr);
    T dr0 = lit<T>(0.0), Drr = lit<T>(0.0), Dzr = lit<T>(0.0);
    if (ax) {
      const T* dr = sDr + (lr + G::HD - G::HF) * G::DZ + (lc + G::HD - G::HF);
      dr0 = dr[0];
      Drr = iso_r(dr, G::DZ);
      // d_zr psi = 1D d_z of the 1D d_r psi of the four z-neighbours (Sec. II.D)
      T e[5];
#pragma unroll
      for (int m = -2; m <= 2; ++m) e[m + 2] = m ? d1(p + m, G::PZ) : lit<T>(0.0);
      Dzr = d1(e + 2, 1);
    }
    T Fz, Fr;
    forces(q, rho, psi, sz, sr, ax, dr0, Drr, Dzr, inv_r, Fz, Fr);
    const T inv_rho = rcp(rho);
    const int fi = lr * G::FZ + lc;
    const T uz = fma(Fz, lit<T>(0.5), jz) * inv_rho, ur = fma(Fr, lit<T>(0.5), jr) * inv_rho;
    sRho[fi] = rho;
    sUz[fi] = uz;
    sUr[fi] = ur;
    if constexpr (MODE == 3) {
      if (lr >= G::HF && lr < G::HF + BR && lc >= G::HF && lc < G::HF + BZ && k0 + lc - G::HF < Nz) {
        C* o = inter + (size_t)j * P + (k0 + lc - G::HF);
        o[I_RHO * iplane] = (rho).v;
        o[I_UZ * iplane] = (uz).v;
        o[I_UR * iplane] = (ur).v;
        o[I_VZ * iplane] = (fma(Fz, q.tau, jz) * inv_rho).v;
        o[I_VR * iplane] = (fma(Fr, q.tau, jr) * inv_rho).v;
        o[I_FZ * iplane] = (Fz).v;
        o[I_FR * iplane] = (Fr).v;
        o[I_PSI * iplane] = (psi).v;
        o[I_SZ * iplane] = (sz).v;
        o[I_SR * iplane] = (sr).v;
        o[I_DR * iplane] = (dr0).v;
        o[I_DRR * iplane] = (Drr).v;
        o[I_DZR * iplane] = (Dzr).v;
      }
    }
    if ((MODE == 0 || MODE == 3) && srow && lc >= 2 && lc < G::FZ - 2) {
      T* out = sFs + (lr - 2) * G::SZ + (lc - 2);
      T fe[9];
      if (guo) {  // f^eq at u, plus (1 - 1/(2 tau)) times the discrete force
        equilibrium(rho, uz, ur, fe);
        T s[9];
        guo_force(uz, ur, Fz, Fr, s);
        const T gk = splat<T>(kc(D, K_GUO, C()));
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i * G::nS] = fma(s[i], gk, fma(fe[i] - f[i], q.omega, f[i]));
      } else {    // the velocity shift: f^eq at u^eq
        const T vz = fma(Fz, q.tau, jz) * inv_rho, vr = fma(Fr, q.tau, jr) * inv_rho;
        equilibrium(rho, vz, vr, fe);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i * G::nS] = fma(fe[i] - f[i], q.omega, f[i]);
      }
    }
  });
  __syncthreads();

  if constexpr (READBACK) {
    for_tile<BR, BZ>([&](int lr, int lc) {
      const int j = j0 + lr, k = k0 + lc;
      if (j >= Nr || k >= Nz) return;
      const int fi = (lr + G::HF) * G::FZ + (lc + G::HF);
      const size_t o = (size_t)j * Nz + k;
      static_cast<C*>(D.rho_out)[o] = (sRho[fi]).v;
      static_cast<C*>(D.uz_out)[o] = (sUz[fi]).v;
      static_cast<C*>(D.ur_out)[o] = (sUr[fi]).v;
    });
    return;
  }

  // Ghost columns of u (depth 2) at the z walls: u_z and u_r odd (no-slip) about
  // the wall half a spacing beyond the first and last columns.
  if (ax && zw && (k0 < G::HF || k0 + BZ + G::HF > Nz)) {
    for_tile<G::FR, G::FZ>([&](int lr, int lc) {
      const int j = j0 - G::HF + lr, k = k0 - G::HF + lc;
      if (j < 0 || j >= Nr) return;
      int m;
      if (k == -1 || k == -2) m = -1 - k;
      else if (k == Nz || k == Nz + 1) m = 2 * Nz - 1 - k;
      else return;
      const int src = lr * G::FZ + (m - (k0 - G::HF));
      sUz[lr * G::FZ + lc] = -sUz[src];
      sUr[lr * G::FZ + lc] = -sUr[src];
    });
    __syncthreads();
  }

  // Ghost rows of u (depth 2) on tiles that touch row 0 or row Nr - 1: u_z even
  // and u_r odd about the axis; about the outer wall u_r odd and u_z even
  // (free-slip) or odd (no-slip); beyond an inlet or outlet row b the linear
  // continuation u(b - m) = 2 u(b) - u(b + m).  Ghost columns were filled first.
  if (ax && (j0 < G::HF || j0 + BR + G::HF > Nr)) {
    for_tile<G::FR, G::FZ>([&](int lr, int lc) {
      const int j = j0 - G::HF + lr;
      int m, b = -1;
      bool flip_z;
      if (j == -1 || j == -2) {
        if (inl) { b = 0; m = -j; } else { m = -1 - j; }
        flip_z = false;
      } else if (j == Nr || j == Nr + 1) {
        if (outl) { b = Nr - 1; m = 2 * (Nr - 1) - j; } else { m = 2 * Nr - 1 - j; }
        flip_z = D.wall == AMLBM_WALL_NOSLIP;
      } else {
        return;
      }
      const int src = (m - (j0 - G::HF)) * G::FZ + lc;
      if (b >= 0) {
        const int bi = (b - (j0 - G::HF)) * G::FZ + lc;
        sUz[lr * G::FZ + lc] = fma(lit<T>(2.0), sUz[bi], -sUz[src]);
        sUr[lr * G::FZ + lc] = fma(lit<T>(2.0), sUr[bi], -sUr[src]);
      } else {
        sUz[lr * G::FZ + lc] = flip_z ? -sUz[src] : sUz[src];
        sUr[lr * G::FZ + lc] = -sUr[src];
      }
    });
    __syncthreads();
  }

  // Inlet and outlet rows (Sec. II.E, imposed before streaming): what leaves
  // them is the equilibrium of the imposed velocity and the density of row 1
  // (inlet), or of the imposed density and the velocity of row Nr - 2
  // (outlet), without source; it is also their state after the step.
  if ((inl && j0 == 0) || (outl && j0 + BR >= Nr - 1)) {
    for_tile<G::SR, G::SZ>([&](int lr, int lc) {
      const int j = j0 - 1 + lr, k = k0 - 1 + lc;
      const bool bin = inl && j == 0, bout = outl && j == Nr - 1;
      // the ghost columns of a periodic lattice too: column 0 pulls from column -1
      if (!(bin || bout) || (zw && (k < 0 || k >= Nz))) return;
      const int kk = wrapz(k, Nz);
      const int nb = (lr + (bin ? 3 : 1)) * G::FZ + (lc + 2);  // row 1 or Nr - 2, tile + 3 indexing
      T rho, uz, ur;
      if (bin) {
        rho = sRho[nb];
        uz = splat<T>(C(D.inlet[kk]));
        ur = splat<T>(C(D.inlet[Nz + kk]));
      } else {
        rho = splat<T>(kc(D, K_RHOOUT, C()));
        uz = sUz[nb];
        ur = sUr[nb];
      }
      T fe[9];
      equilibrium(rho, uz, ur, fe);
      const int si = lr * G::SZ + lc;
#pragma unroll
      for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = fe[i];
    });
    __syncthreads();
  }

  // Stage 3 (tile + 1): velocity gradients and the sources of App. A, added to
  // the collided populations (the whole h_i, or half of it for the link average).
  const bool link = D.src == AMLBM_SRC_LINK;
  for_tile<G::SR, G::SZ>([&](int lr, int lc) {
    const int j = j0 - 1 + lr;
    if (j < 0 || j >= Nr) return;
    const int si = lr * G::SZ + lc;
    T S_ = lit<T>(0.0), Hz = lit<T>(0.0), Hr = lit<T>(0.0);
    const bool brow = (inl && j == 0) || (outl && j == Nr - 1);  // no source on boundary rows
    if (ax && !brow) {
      const T inv_r = inv_r_of(T(), j, kc(D, K_R0, C()));
      const int fi = (lr + 2) * G::FZ + (lc + 2);
      const T druz = d1(sUz + fi, G::FZ);
      const T dzur = d1(sUr + fi, 1);
      const T drur = d1(sUr + fi, G::FZ);
      if constexpr (MODE == 3) {
        if (lr >= 1 && lr <= BR && lc >= 1 && lc <= BZ && k0 + lc - 1 < Nz) {
          C* o = inter + (size_t)j * P + (k0 + lc - 1);
          o[I_G1 * iplane] = (druz).v;
          o[I_G2 * iplane] = (dzur).v;
          o[I_G3 * iplane] = (drur).v;
        }
      }
      site_sources(q, sRho[fi], sUz[fi], sUr[fi], druz, dzur, drur, inv_r, S_, Hz, Hr);
      T h[9];
      sources(S_, Hz, Hr, h);
      if (link) {
#pragma unroll
        for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = fma(h[i], lit<T>(0.5), sFs[i * G::nS + si]);
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = sFs[i * G::nS + si] + h[i];
      }
    }
    if constexpr (MODE == 3) {
      if (!ax && lr >= 1 && lr <= BR && lc >= 1 && lc <= BZ && k0 + lc - 1 < Nz) {
        C* o = inter + (size_t)j * P + (k0 + lc - 1);
        o[I_G1 * iplane] = C(0);
        o[I_G2 * iplane] = C(0);
        o[I_G3 * iplane] = C(0);
      }
    }
    sS[si] = S_;
    sHz[si] = Hz;
    sHr[si] = Hr;
  });
  __syncthreads();

  // Stage 4 (tile): pull streaming.  Away from the boundaries every population
  // comes from x - c_i in the same direction; rows 0 and Nr-1 apply the
  // reflection maps, the first and last columns the bounce-back of the z walls
  // (which takes precedence at the corners); inlet and outlet rows keep their
  // own boundary populations.  Then psi of the new state and the shifted store.
  S* __restrict__ fout = static_cast<S*>(D.f[parity ^ 1]);
  C* __restrict__ psout = static_cast<C*>(D.psi[parity ^ 1]);
  const bool noslip = D.wall == AMLBM_WALL_NOSLIP;
  for_tile<BR, BZ>([&](int lr, int lc) {
    const int j = j0 + lr, k = k0 + lc;
    if (j >= Nr || k >= Nz) return;
    const bool brow = (inl && j == 0) || (outl && j == Nr - 1);
    const bool edge = (j == 0) || (j == Nr - 1) || (zw && (k == 0 || k == Nz - 1));
    T fn[9];
    if (!edge) {  // interior site: constant offsets, no per-population branch
#pragma unroll
      for (int i = 0; i < 9; ++i) fn[i] = sFs[i * G::nS + (lr + 1 - cr_(i)) * G::SZ + (lc + 1 - cz_(i))];
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        int sl = lr + 1 - cr_(i), sc = lc + 1 - cz_(i), ii = i;
        const int ks = k - cz_(i);
        if (brow) {  // inlet / outlet row: its own boundary populations
          sl = lr + 1; sc = lc + 1;
        } else if (zw && (ks < 0 || ks >= Nz)) {  // through a z wall: bounce-back
          sl = lr + 1; sc = lc + 1; ii = opp_(i);
        } else if (cr_(i) > 0 && j == 0) {  // through the axis: specular reflection
          sl = lr + 1; ii = mirror_(i);
        } else if (cr_(i) < 0 && j == Nr - 1) {  // through the outer wall
          sl = lr + 1;
          if (noslip) { sc = lc + 1; ii = opp_(i); }
          else { ii = mirror_(i); }
        }
        fn[i] = sFs[ii * G::nS + sl * G::SZ + sc];
      }
    }
    if (link && !brow) {
      const int di = (lr + 1) * G::SZ + (lc + 1);
      T h[9];
      sources(sS[di], sHz[di], sHr[di], h);
#pragma unroll
      for (int i = 0; i < 9; ++i) fn[i] = fma(h[i], lit<T>(0.5), fn[i]);
    }
    const T rho = moment0(fn);
    encode_site<S>(shift, fout + (size_t)j * P + k, psout + (size_t)j * P + k, plane, fn, rho,
                   psi_of(q, rho).v, inv_rho0c, rho0c, rrefc, D.rounding, (uint32_t)(j * Nz + k), step);
  });
}

template <class S, int BZ, int BR, int MODE>
__global__ void __launch_bounds__(NT, (MinBlocks<S, typename Store<S>::T, BZ, BR>::value)) lbm_kernel(
    const InstDesc* __restrict__ descs, const int* __restrict__ tile_inst, int toff, int parity,
    typename Store<S>::C* __restrict__ inter, size_t iplane) {
  lbm_tile<S, typename Store<S>::T, BZ, BR, MODE>(descs, tile_inst, blockIdx.x + toff, parity, inter,
                                                  iplane);
}

// The timestep as a persistent grid (as many CTAs as fit on the GPU at once):
// CTAs take tiles from a counter in the order of the tile list until none is
// left, so uneven lattices and ragged tiles leave no partial last wave.
// ctr[parity] counts this step's tiles; ctr[parity ^ 1], last used by the
// previous step (which the stream has completed), is reset for the next one.
// No CTA waits on another.  ctr[2], ctr[3] carry the step number the same way.
template <class S, class T, int BZ, int BR>
__global__ void __launch_bounds__(NT, (MinBlocks<S, T, BZ, BR>::value)) lbm_persistent(
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
    lbm_tile<S, T, BZ, BR, 0>(descs, tile_inst, t, parity, nullptr, 0, step);
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
template <class T, int BZ, int BR>
struct GeoA {
  static constexpr int HP = 4, HD = 2;
  static constexpr int PZ = BZ + 2 * HP, PR = BR + 2 * HP;
  static constexpr int DZ = BZ + 2 * HD, DR = BR + 2 * HD;
  static constexpr int EZ = BZ + 2 * HD, ER = BR;
  static constexpr int nP = PZ * PR, nD = DZ * DR, nE = EZ * ER;
  static constexpr int int_bytes = ((PZ + PR) * 4 + 15) / 16 * 16;
  static constexpr size_t bytes = int_bytes + sizeof(T) * (size_t)(nP + nD + nE);
};

template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT) force_kernel(const InstDesc* __restrict__ descs,
                                                   const int* __restrict__ tile_inst, int toff,
                                                   int parity) {
  using C = typename Store<S>::C;
  using T = typename Store<S>::T;
  using G = GeoA<T, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* colmap = reinterpret_cast<int*>(smem_raw);
  int* rowmap = colmap + G::PZ;
  T* sPsi = reinterpret_cast<T*>(smem_raw + G::int_bytes);
  T* sDr = sPsi + G::nP;
  T* sD1 = sDr + G::nD;
  const Tile Tl = tile_of(descs, tile_inst, blockIdx.x + toff, BZ, BR);
  const InstDesc& D = descs[Tl.inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P, k0 = Tl.k0, j0 = Tl.j0;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  C* __restrict__ uv = static_cast<C*>(D.uv);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const Par<T> q = par_of<T>(D);
  const C rho0c = kc(D, K_RHO0, C()), rrefc = kc(D, K_RREF, C()), inv_rho0c = kc(D, K_INVRHO0, C());

  for (int i = threadIdx.x; i < G::PZ; i += NT) colmap[i] = wrapz(k0 - G::HP + i, Nz);
  for (int i = threadIdx.x; i < G::PR; i += NT) rowmap[i] = reflect_row(j0 - G::HP + i, Nr);
  __syncthreads();
  for_tile<G::PR, G::PZ>([&](int lr, int lc) {
    sPsi[lr * G::PZ + lc] = T{psin[(size_t)rowmap[lr] * P + colmap[lc]]};
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
    const T inv_r = inv_r_of(T(), j, kc(D, K_R0, C()));
    const T* p = sPsi + (lr + G::HP) * G::PZ + (lc + G::HP);
    const T psi = p[0];
    T f[9];
    decode_site<S>(shift, fin + (size_t)j * P + k, plane, psi.v, psin + (size_t)j * P + k, inv_rho0c, rho0c,
                   rrefc, f);
    const T rho = moment0(f), jz = moment_z(f), jr = moment_r(f);
    T sz, sr;
    sc_sums(p, G::PZ, sz, sr);
    T dr0 = lit<T>(0.0), Drr = lit<T>(0.0), Dzr = lit<T>(0.0);
    if (ax) {
      const T* dr = sDr + (lr + G::HD) * G::DZ + (lc + G::HD);
      dr0 = dr[0];
      Drr = iso_r(dr, G::DZ);
      Dzr = d1(sD1 + lr * G::EZ + (lc + G::HD), 1);
    }
    T Fz, Fr;
    forces(q, rho, psi, sz, sr, ax, dr0, Drr, Dzr, inv_r, Fz, Fr);
    const T inv_rho = rcp(rho);
    C* o = uv + (size_t)j * P + k;
    o[0] = (fma(Fz, lit<T>(0.5), jz) * inv_rho).v;
    o[plane] = (fma(Fr, lit<T>(0.5), jr) * inv_rho).v;
    o[2 * plane] = (fma(Fz, q.tau, jz) * inv_rho).v;
    o[3 * plane] = (fma(Fr, q.tau, jr) * inv_rho).v;
  });
}

template <class T, int BZ, int BR>
struct GeoB {
  static constexpr int HF = 3;
  static constexpr int FZ = BZ + 2 * HF, FR = BR + 2 * HF;
  static constexpr int SZ = BZ + 2, SR = BR + 2;
  static constexpr int nF = FZ * FR, nS = SZ * SR;
  static constexpr int int_bytes = (FZ * 4 + 15) / 16 * 16;
  static constexpr size_t bytes = int_bytes + sizeof(T) * (size_t)(2 * nF + 13 * nS);
};

template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT) stream_kernel(const InstDesc* __restrict__ descs,
                                                    const int* __restrict__ tile_inst, int toff,
                                                    int parity, int* __restrict__ ctr) {
  const uint32_t step = ctr ? (uint32_t)ctr[2 + parity] : 0u;
  if (ctr && blockIdx.x == 0 && threadIdx.x == 0) ctr[2 + (parity ^ 1)] = (int)(step + 1);
  using C = typename Store<S>::C;
  using T = typename Store<S>::T;
  using G = GeoB<T, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* colmap = reinterpret_cast<int*>(smem_raw);
  T* sUz = reinterpret_cast<T*>(smem_raw + G::int_bytes);
  T* sUr = sUz + G::nF;
  T* sRho = sUr + G::nF;
  T* sS = sRho + G::nS;
  T* sHz = sS + G::nS;
  T* sHr = sHz + G::nS;
  T* sFs = sHr + G::nS;
  const Tile Tl = tile_of(descs, tile_inst, blockIdx.x + toff, BZ, BR);
  const InstDesc& D = descs[Tl.inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P, k0 = Tl.k0, j0 = Tl.j0;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  const C* __restrict__ uv = static_cast<const C*>(D.uv);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const Par<T> q = par_of<T>(D);
  const C rho0c = kc(D, K_RHO0, C()), rrefc = kc(D, K_RREF, C()), inv_rho0c = kc(D, K_INVRHO0, C());
  const bool noslip = D.wall == AMLBM_WALL_NOSLIP;

  for (int i = threadIdx.x; i < G::FZ; i += NT) colmap[i] = wrapz(k0 - G::HF + i, Nz);
  __syncthreads();
  // u on the tile + 3; ghost rows (depth 2) by the mirror rules of the fused kernel
  if (ax) {
    for_tile<G::FR, G::FZ>([&](int lr, int lc) {
      const int j = j0 - G::HF + lr;
      int m = j;
      bool flip_z = false, flip_r = false;
      if (j == -1 || j == -2) {
        m = -1 - j;
        flip_r = true;
      } else if (j == Nr || j == Nr + 1) {
        m = 2 * Nr - 1 - j;
        flip_r = true;
        flip_z = noslip;
      } else if (j < 0 || j >= Nr) {
        return;  // never read
      }
      const size_t o = (size_t)m * P + colmap[lc];
      sUz[lr * G::FZ + lc] = T{flip_z ? -uv[o] : uv[o]};
      sUr[lr * G::FZ + lc] = T{flip_r ? -uv[plane + o] : uv[plane + o]};
    });
  }
  // populations on the tile + 1: rho and the collision towards f^eq(rho, u^eq)
  for_tile<G::SR, G::SZ>([&](int lr, int lc) {
    const int j = j0 - 1 + lr;
    if (j < 0 || j >= Nr) return;
    const size_t o = (size_t)j * P + colmap[lc + G::HF - 1];
    T f[9];
    decode_site<S>(shift, fin + o, plane, psin[o], psin + o, inv_rho0c, rho0c, rrefc, f);
    const T rho = moment0(f);
    const T vz{uv[2 * plane + o]}, vr{uv[3 * plane + o]};
    T fe[9];
    equilibrium(rho, vz, vr, fe);
    const int si = lr * G::SZ + lc;
    sRho[si] = rho;
#pragma unroll
    for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = fma(fe[i] - f[i], q.omega, f[i]);
  });
  __syncthreads();
  // gradients and sources on the tile + 1
  const bool link = D.src == AMLBM_SRC_LINK;
  for_tile<G::SR, G::SZ>([&](int lr, int lc) {
    const int j = j0 - 1 + lr;
    if (j < 0 || j >= Nr) return;
    const int si = lr * G::SZ + lc;
    T S_ = lit<T>(0.0), Hz = lit<T>(0.0), Hr = lit<T>(0.0);
    if (ax) {
      const T inv_r = inv_r_of(T(), j, kc(D, K_R0, C()));
      const int fi = (lr + 2) * G::FZ + (lc + 2);
      const T druz = d1(sUz + fi, G::FZ);
      const T dzur = d1(sUr + fi, 1);
      const T drur = d1(sUr + fi, G::FZ);
      site_sources(q, sRho[si], sUz[fi], sUr[fi], druz, dzur, drur, inv_r, S_, Hz, Hr);
      T h[9];
      sources(S_, Hz, Hr, h);
      if (link) {
#pragma unroll
        for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = fma(h[i], lit<T>(0.5), sFs[i * G::nS + si]);
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) sFs[i * G::nS + si] = sFs[i * G::nS + si] + h[i];
      }
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
    T fn[9];
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
      T h[9];
      sources(sS[di], sHz[di], sHr[di], h);
#pragma unroll
      for (int i = 0; i < 9; ++i) fn[i] = fma(h[i], lit<T>(0.5), fn[i]);
    }
    const T rho = moment0(fn);
    encode_site<S>(shift, fout + (size_t)j * P + k, psout + (size_t)j * P + k, plane, fn, rho,
                   psi_of(q, rho).v, inv_rho0c, rho0c, rrefc, D.rounding, (uint32_t)(j * Nz + k), step);
  });
}

// Site n = j*Nz + k of instance D: f = f^eq(rho, u) with u^eq = u (the
// initial state of the scheme), stored in the instance's storage form, and psi.
template <class S>
__device__ __forceinline__ void init_site(const InstDesc& D, int n, double rho_d, double uz_d,
                                          double ur_d, int parity) {
  using C = typename Store<S>::C;
  using T = typename Store<S>::T;
  const int j = n / D.Nz, k = n - j * D.Nz;
  const size_t plane = (size_t)D.P * D.Nr, o = (size_t)j * D.P + k;
  S* f = static_cast<S*>(D.f[parity]);
  C* psi_out = static_cast<C*>(D.psi[parity]);
  const Par<T> q = par_of<T>(D);
  T fe[9];
  equilibrium(T{C(rho_d)}, T{C(uz_d)}, T{C(ur_d)}, fe);
  const T rho = moment0(fe);
  encode_site<S>(D.shift, f + o, psi_out + o, plane, fe, rho, psi_of(q, rho).v, kc(D, K_INVRHO0, C()),
                 kc(D, K_RHO0, C()), kc(D, K_RREF, C()), 0, 0u, 0u);
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
  // the inputs first (they may be host memory read over the CPU-GPU link): their
  // latency overlaps the search for the instance
  const double rho = rho_in[g];
  const double uz = uz_in ? uz_in[g] : 0.0, ur = ur_in ? ur_in[g] : 0.0;
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (site_off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  const bool ok = rho > 0 && isfinite(rho);
  if (!ok) atomicAdd(bad, 1);
  init_site<S>(descs[lo], (int)(g - site_off[lo]), ok ? rho : 1.0, uz, ur, parity);
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
  const C* ps = static_cast<const C*>(D.psi[parity]) + o;
  using T = typename Store<S>::T;
  T fv[9];
  decode_site<S>(D.shift, f + o, plane, ps[0], ps, kc(D, K_INVRHO0, C()), kc(D, K_RHO0, C()),
                 kc(D, K_RREF, C()), fv);
#pragma unroll
  for (int i = 0; i < 9; ++i) out[(size_t)i * N + n] = double(fv[i].v);
}

// ------------------------------------------------------------- launchers --
// One-time set-up of a kernel family on each device (function attributes are
// per device), safe when several host threads launch at once.
constexpr int kMaxDevices = 64;
struct DeviceOnce {
  std::once_flag once[kMaxDevices];
  cudaError_t err[kMaxDevices] = {};
  int grid_cap[kMaxDevices] = {};
};

template <class F>
cudaError_t once_per_device(DeviceOnce& st, F&& init, int* grid_cap = nullptr) {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::call_once(st.once[dev], [&] { st.err[dev] = init(dev, &st.grid_cap[dev]); });
  if (grid_cap) *grid_cap = st.grid_cap[dev];
  return st.err[dev];
}

template <class S, class T, int BZ, int BR, int MODE>
cudaError_t launch_t(const InstDesc* d, const int* ti, int ntiles, int toff, int parity,
                     cudaStream_t s, void* inter = nullptr, size_t iplane = 0, int* ctr = nullptr) {
  using C = typename Store<S>::C;
  constexpr size_t smem = Geo<T, BZ, BR>::bytes;
  static DeviceOnce st;
  int grid_cap = 0;
  const cudaError_t ie = once_per_device(st, [](int dev, int* cap) {
    cudaError_t e = cudaFuncSetAttribute(lbm_kernel<S, BZ, BR, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && MODE == 0)
      e = cudaFuncSetAttribute(lbm_persistent<S, T, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e == cudaSuccess && MODE == 0) {
      int sms = 0, per_sm = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm_persistent<S, T, BZ, BR>, NT, smem);
      *cap = sms * (per_sm > 0 ? per_sm : 1);
    }
    return e;
  }, &grid_cap);
  if (ie != cudaSuccess) return ie;
  if (MODE == 0 && ctr && toff == 0) {
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    lbm_persistent<S, T, BZ, BR><<<grid, NT, smem, s>>>(d, ti, ntiles, parity, ctr);
  } else {
    lbm_kernel<S, BZ, BR, MODE><<<ntiles, NT, smem, s>>>(d, ti, toff, parity, static_cast<C*>(inter), iplane);
  }
  return cudaGetLastError();
}

template <class S, int BZ, int BR>
cudaError_t launch_split_t(const InstDesc* d, const int* ti, int ntiles, int toff, int parity,
                           cudaStream_t s, int* ctr) {
  using T = typename Store<S>::T;
  constexpr size_t sa = GeoA<T, BZ, BR>::bytes, sbb = GeoB<T, BZ, BR>::bytes;
  static DeviceOnce st;
  const cudaError_t ie = once_per_device(st, [](int, int*) {
    cudaError_t e = cudaFuncSetAttribute(force_kernel<S, BZ, BR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(stream_kernel<S, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sbb);
    return e;
  });
  if (ie != cudaSuccess) return ie;
  force_kernel<S, BZ, BR><<<ntiles, NT, sa, s>>>(d, ti, toff, parity);
  stream_kernel<S, BZ, BR><<<ntiles, NT, sbb, s>>>(d, ti, toff, parity, ctr);
  return cudaGetLastError();
}

// Tile shapes compiled for each storage form.
struct TileEntry { int storage, sched, tz, tr; };
#define AMLBM_TILES_16(ST)                                                                    \
  {ST, SCHED_FUSED, 26, 16}, {ST, SCHED_FUSED, 32, 16}, {ST, SCHED_FUSED, 64, 8},             \
  {ST, SCHED_FUSED, 58, 8}, {ST, SCHED_FUSED, 32, 8}, {ST, SCHED_FUSED, 32, 32},              \
  {ST, SCHED_FUSED, 64, 16}, {ST, SCHED_SPLIT, 32, 16}, {ST, SCHED_SPLIT, 64, 8},             \
  {ST, SCHED_SPLIT, 64, 16}, {ST, SCHED_SPLIT, 32, 8}
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
  using T = typename Store<S>::T;
  if (nt <= 0) return cudaSuccess;
  if (sched == SCHED_SPLIT && !macro) {
#define AMLBM_SPLIT(TZ, TR) \
  if (tz == TZ && tr == TR) return launch_split_t<S, TZ, TR>(d, ti, nt, toff, par, s, ctr);
    AMLBM_SPLIT(32, 8)
    AMLBM_SPLIT(64, 8)
    AMLBM_SPLIT(32, 16)
    if constexpr (!std::is_same<S, double>::value) {
      AMLBM_SPLIT(64, 16)
    }
#undef AMLBM_SPLIT
    return cudaErrorInvalidValue;
  }
#define AMLBM_TILE(TZ, TR)                                                   \
  if (tz == TZ && tr == TR)                                                  \
    return macro ? launch_t<S, T, TZ, TR, 1>(d, ti, nt, toff, par, s)        \
                 : launch_t<S, T, TZ, TR, 0>(d, ti, nt, toff, par, s, nullptr, 0, ctr);
  if (macro) {  // read-back: 32 x 8 for every storage, 26 x 16 for the FP32-arithmetic forms
    AMLBM_TILE(32, 8)
    if constexpr (!std::is_same<S, double>::value) {
      AMLBM_TILE(26, 16)
    }
    return cudaErrorInvalidValue;
  }
  AMLBM_TILE(32, 8)
  AMLBM_TILE(64, 8)
  AMLBM_TILE(58, 8)
  if constexpr (std::is_same<S, double>::value) {
    AMLBM_TILE(26, 8)
  } else {
    AMLBM_TILE(26, 16)
    AMLBM_TILE(32, 16)
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

cudaError_t launch_step(int storage, int sched, int tz, int tr, const InstDesc* d, const int* ti,
                        int nt, int toff, int parity, cudaStream_t s, int* ctr) {
  return dispatch_storage(storage, false, sched, tz, tr, d, ti, nt, toff, parity, s, ctr);
}
cudaError_t launch_macro(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                         int toff, int parity, cudaStream_t s) {
  return dispatch_storage(storage, true, SCHED_FUSED, tz, tr, d, ti, nt, toff, parity, s, nullptr);
}

cudaError_t launch_step_inter(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                              void* inter, size_t plane, cudaStream_t s) {
  if (storage == AMLBM_STORE_F64) {
    if (tz == 32 && tr == 8) return launch_t<double, D1, 32, 8, 3>(d, ti, nt, 0, 0, s, inter, plane);
  } else if (storage == AMLBM_STORE_F32) {
    if (tz == 32 && tr == 8) return launch_t<float, F1, 32, 8, 3>(d, ti, nt, 0, 0, s, inter, plane);
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
