// Two-element vector accesses and the helpers that the pair and strip
// schedules of the step share (a pair is two adjacent z-sites of one row).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "amlbm_physics.cuh"

namespace amlbm {
namespace {

// Two adjacent elements of a storage or compute type as one vector access.
template <class S> struct Vec2;
template <> struct Vec2<double> { using V = double2; };
template <> struct Vec2<float> { using V = float2; };
template <> struct Vec2<__half> { using V = __half2; };
template <> struct Vec2<__nv_bfloat16> { using V = __nv_bfloat162; };

template <class S>
__device__ __forceinline__ void ld2(const S* p, S& a, S& b) {
  const typename Vec2<S>::V v = *reinterpret_cast<const typename Vec2<S>::V*>(p);
  a = v.x;
  b = v.y;
}
template <class S>
__device__ __forceinline__ void st2(S* p, S a, S b) {
  typename Vec2<S>::V v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<typename Vec2<S>::V*>(p) = v;
}
// Lane-typed shared-memory pairs (the lane types are one scalar wide).
template <class T>
__device__ __forceinline__ void lds2(const T* p, T& a, T& b) {
  using C = typename Lane<T>::C;
  C x, y;
  ld2<C>(reinterpret_cast<const C*>(p), x, y);
  a = T{x};
  b = T{y};
}
template <class T>
__device__ __forceinline__ void sts2(T* p, T a, T b) {
  using C = typename Lane<T>::C;
  st2<C>(reinterpret_cast<C*>(p), a.v, b.v);
}
// N pairs of a shared-memory row from p into w[0 .. 2N).
template <class T, int N>
__device__ __forceinline__ void load_row(const T* p, T* w) {
#pragma unroll
  for (int m = 0; m < N; ++m) lds2(p + 2 * m, w[2 * m], w[2 * m + 1]);
}

// Column of the periodic lattice for a region column k in [-16, Nz + BZ + 16)
// (tiny: the lattice is narrower than a region, which may wrap more than once).
__device__ __forceinline__ int wrap_col(int k, int Nz, bool tiny) {
  if (tiny) return wrapz(k, Nz);
  return k < 0 ? k + Nz : (k >= Nz ? k - Nz : k);
}

// The force of Eq. scforce and Eq. scAxisExtra without the body force rho g_z
// (forces() of the fused schedule, operation for operation, up to its last
// fused multiply-add, which the caller applies once rho is known).
template <class T>
__device__ __forceinline__ void forces_partial(const Par<T>& q, T psi, T sz, T sr, bool ax, T dr0, T Drr, T Dzr,
                                               T inv_r, T& Fz, T& Fr) {
  const T gpsi = psi * q.negG;
  Fz = gpsi * sz;
  Fr = gpsi * sr;
  if (ax) {
    const T g = (psi * q.gfac) * inv_r;
    Fz = fma(g, Dzr, Fz);
    Fr = fma(g, fma(-dr0, inv_r, Drr), Fr);
  }
}

}  // namespace
}  // namespace amlbm
