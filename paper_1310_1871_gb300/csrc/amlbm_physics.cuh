// Per-site arithmetic of the axisymmetric Shan-Chen LBM step (arXiv:1310.1871,
// Sec. II and App. A) on explicitly rounded lane types, shared by the step
// kernels of every schedule.  Every kernel that includes this header is compiled
// with -fmad=false and states each fused multiply-add itself, so that every
// schedule computes a site with the same operations and gets the same bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

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
// an integer hash of (site, step): the xorshift-multiply mixer with shifts
// 16, 15, 16 and multipliers 0x7feb352d, 0x846ca68b published by C. Wellons
// ("lowbias32", hash-prospector, 2018); the nine
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

// Decode the nine populations of a site from their stored values q[i]:
// f_i = q_i + W_i s (shift modes 0-2, one fused multiply-add) or, in the
// equilibrium mode (3), f_i = q_i + f^eq_i(s, v) with the stored velocity
// v = (vz, vr).
template <class S, class T>
__device__ __forceinline__ void decode_values(int mode, const S* q, typename Store<S>::C psi,
                                              typename Store<S>::C vz, typename Store<S>::C vr,
                                              typename Store<S>::C inv_rho0, typename Store<S>::C rho0,
                                              typename Store<S>::C rref, T* f) {
  const T sbt{shift_base(mode, psi, inv_rho0, rho0, rref)};
  if (mode == 3) {
    T fe[9];
    equilibrium(sbt, T{vz}, T{vr}, fe);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = T{Store<S>::to(q[i])} + fe[i];
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fma(lit<T>(w_(i)), sbt, T{Store<S>::to(q[i])});
  }
}

// The same from global memory: q[i * plane], and in the equilibrium mode the
// velocity in the two planes that follow psi (pv points at the site's psi).
template <class S, class T>
__device__ __forceinline__ void decode_site(int mode, const S* q, size_t plane, typename Store<S>::C psi,
                                            const typename Store<S>::C* pv, typename Store<S>::C inv_rho0,
                                            typename Store<S>::C rho0, typename Store<S>::C rref, T* f) {
  using C = typename Store<S>::C;
  S qv[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) qv[i] = q[i * plane];
  const C vz = mode == 3 ? pv[plane] : C(0), vr = mode == 3 ? pv[2 * plane] : C(0);
  decode_values<S>(mode, qv, psi, vz, vr, inv_rho0, rho0, rref, f);
}

// The stored values of the new populations fn of a site: q_i = fn_i - W_i s
// (shift modes 0-2) or, in the equilibrium mode, q_i = fn_i - f^eq_i(s, v) with
// the bare velocity v = sum_i c_i fn_i / rho of the new state (returned in
// vz, vr); 16-bit stores round to nearest or (rounding != 0) stochastically
// with words drawn from (site, step).
template <class S, class T>
__device__ __forceinline__ void encode_values(int mode, const T* fn, T rho, typename Store<S>::C psi,
                                              typename Store<S>::C inv_rho0, typename Store<S>::C rho0,
                                              typename Store<S>::C rref, int rounding, uint32_t site,
                                              uint32_t step, S* q, typename Store<S>::C& vz_out,
                                              typename Store<S>::C& vr_out) {
  using C = typename Store<S>::C;
  const C sb = shift_base(mode, psi, inv_rho0, rho0, rref);
  C fv[9], base[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fv[i] = fn[i].v;
  if (mode == 3) {
    const T ir = rcp(rho), vz = moment_z(fn) * ir, vr = moment_r(fn) * ir;
    T fe[9];
    equilibrium(T{sb}, vz, vr, fe);
#pragma unroll
    for (int i = 0; i < 9; ++i) base[i] = fv[i] - fe[i].v;
    vz_out = vz.v;
    vr_out = vr.v;
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) base[i] = fma_c(C(-w_(i)), sb, fv[i]);
    vz_out = C(0);
    vr_out = C(0);
  }
  if (sizeof(S) == 2 && rounding) {
    uint32_t x = mix32(site ^ mix32(step + 0x9E3779B9u));
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      x = lcg_next(x);
      q[i] = Store<S>::from_sr(base[i], x);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i] = Store<S>::from(base[i]);
  }
}

// Store the new populations fn of a site and its psi (at *pso); in the
// equilibrium mode also the bare velocity v of the new state (after psi).
template <class S, class T>
__device__ __forceinline__ void encode_site(int mode, S* o, typename Store<S>::C* pso, size_t plane,
                                            const T* fn, T rho, typename Store<S>::C psi,
                                            typename Store<S>::C inv_rho0, typename Store<S>::C rho0,
                                            typename Store<S>::C rref, int rounding, uint32_t site,
                                            uint32_t step) {
  using C = typename Store<S>::C;
  S q[9];
  C vz, vr;
  encode_values<S>(mode, fn, rho, psi, inv_rho0, rho0, rref, rounding, site, step, q, vz, vr);
#pragma unroll
  for (int i = 0; i < 9; ++i) o[i * plane] = q[i];
  if (mode == 3) {
    pso[plane] = vz;
    pso[2 * plane] = vr;
  }
  pso[0] = psi;
}

}  // namespace
}  // namespace amlbm
