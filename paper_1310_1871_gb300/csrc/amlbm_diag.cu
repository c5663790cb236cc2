// Diagnostics of a lattice state: FP64 sums over the meridional sites and the
// interface radius of every column, for one instance or for every instance of
// a batch in the same three launches.
//
// Quantities (r = j + 1/2 + r_off is the node radius, sums over real sites):
//   mass2d = sum rho, mass3d = sum 2 pi r rho (the volume integral of the
//   axisymmetric density, Sec. II.A), momz3d = sum 2 pi r rho u_z,
//   E_ke = pi sum r rho |u|^2 (the kinetic energy whose constancy marks the
//   steady pipe flow, Sec. III.A), max |u|, the l = 2 moment a_2 of the liquid
//   fraction about the drop centre (Sec. III.C), the r-intercept of the
//   interface on the centre column and its minimum over z (the neck of a thread,
//   Sec. III.D), and the Shan-Chen pressure p = rho/3 + G psi^2/6 (the equation
//   of state of Sec. II.B with c_s^2 = 1/3) inside and outside the drop.
//
// The read-back kernel must have written rho, u_z, u_r of the state into the
// instance's rho_out / uz_out / ur_out arrays first (in the compute type C).

#include <cuda_runtime.h>

#include "amlbm.h"
#include "amlbm_internal.cuh"

namespace amlbm {
namespace {

constexpr int DIAG_NT = 256;
constexpr int DIAG_WARPS = DIAG_NT / 32;
constexpr int NSUM = 8;  // mass2d mass3d momz3d Eke q2 sumS bad | max |u|^2 (max-reduced)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <class C>
__device__ __forceinline__ C warp_sum_t(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class C>
__device__ __forceinline__ C warp_max_t(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Interface radius of column k, one warp: the first row (from row 0) whose
// density is below mid, interpolated linearly against the row before it; r0 - 1/2
// (the axis, or the lattice's inner edge) when row 0 is already below, Nr + r0 - 1/2
// when no row is.  r0 is the radius of row 0.  Rows are scanned 32 at a time.
template <class C>
__device__ double col_radius_warp(const C* __restrict__ rho, int Nz, int Nr, int k, double mid, double r0) {
  const C midc = C(mid);
  const int lane = threadIdx.x & 31;
  for (int j0 = 0; j0 < Nr; j0 += 32) {
    const int j = j0 + lane;
    const bool below = j < Nr && rho[(size_t)j * Nz + k] < midc;
    const unsigned m = __ballot_sync(0xffffffffu, below);
    if (m) {  // one lane interpolates (an FP64 division), the others take its value
      const int jf = j0 + __ffs(m) - 1;
      double res = r0 - 0.5;
      if (lane == 0 && jf > 0) {  // the fraction in C (an FP64 division is slow here)
        const C v0 = rho[(size_t)(jf - 1) * Nz + k], v = rho[(size_t)jf * Nz + k];
        res = (jf - 1 + r0) + double((v0 - midc) / (v0 - v));
      }
      return __shfl_sync(0xffffffffu, res, 0);
    }
  }
  return Nr + r0 - 0.5;
}

__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_t(double x) { return __drcp_rn(x); }

// Block blk of the nblk blocks of job J: partial sums over the sites
// blk*NT + tid + m*nblk*NT into partials[(J.blk0 + blk) * NSUM + q], and the
// radii of the columns blk*WARPS + warp + m*nblk*WARPS into cols[J.col0 + k].
// The per-site terms are formed in the arithmetic type C of the storage form
// (its values are no more precise than that) and summed per thread and per warp
// in C, then across warps and blocks in FP64; FP64 runs at a small fraction of
// the FP32 rate on GB300, so there is no FP64 operation, division or square root
// per site or lane (|u|^2 is max-reduced, its root taken once at the end).  The
// FP64 form (C = double) is FP64 throughout.
template <class C>
__device__ void partial_block(const InstDesc& D, const DiagJob& J, int blk, double* partials,
                              double* cols) {
  const int Nz = D.Nz, Nr = D.Nr, N = Nz * Nr;
  const C two_pi = C(2.0 * 3.14159265358979323846);
  const C inv_dl = C(J.inv_dl), rho_v = C(J.rho_v), zc = C(J.zc);
  const C r0 = sizeof(C) == 8 ? C(D.k64[K_R0]) : C(D.k32[K_R0]);
  const C* __restrict__ rho_o = static_cast<const C*>(D.rho_out);
  const C* __restrict__ uz_o = static_cast<const C*>(D.uz_out);
  const C* __restrict__ ur_o = static_cast<const C*>(D.ur_out);
  // Each thread first adds its own few sites (about four) in C, then the block
  // and the final pass reduce those per-thread sums in FP64: the FP32 forms then
  // need one FP64 conversion and addition per sum and thread, not per site.
  C tacc[NSUM] = {C(0), C(0), C(0), C(0), C(0), C(0), C(0), C(0)};
  // sites n = blk * NT + tid + m * S, S = nblk * NT; (j, k) advanced without a
  // division per site
  const int S = J.nblk * DIAG_NT, sj = S / Nz, sk = S - sj * Nz;
  const int n0 = blk * DIAG_NT + threadIdx.x;
  int j = n0 / Nz, k = n0 - (n0 / Nz) * Nz;
  for (int n = n0; n < N; n += S) {
    const C r = C(j) + r0, rho = rho_o[n], uz = uz_o[n], ur = ur_o[n];
    const C u2 = uz * uz + ur * ur, w = two_pi * r * rho;
    tacc[0] += rho;
    tacc[1] += w;
    tacc[2] += w * uz;
    tacc[3] += C(0.5) * w * u2;
    const C dz = C(k) - zc;
    tacc[4] += two_pi * r * ((rho - rho_v) * inv_dl) * (dz * dz - C(0.5) * r * r);
    tacc[5] += -rho * ur * rcp_t(r);
    const bool bad = !(rho > C(0)) || !isfinite(rho) || !isfinite(u2);
    tacc[6] += bad ? C(1) : C(0);
    tacc[7] = fmax(tacc[7], bad ? C(0) : u2);
    k += sk;
    j += sj;
    if (k >= Nz) {
      k -= Nz;
      ++j;
    }
  }
  // The warp's sums (128 sites) pairwise in C too, then FP64 across warps and
  // blocks: the FP32 forms convert 8 values per warp instead of per thread.
#pragma unroll
  for (int q = 0; q < NSUM - 1; ++q) tacc[q] = warp_sum_t(tacc[q]);
  tacc[NSUM - 1] = warp_max_t(tacc[NSUM - 1]);
  double acc[NSUM];
#pragma unroll
  for (int q = 0; q < NSUM; ++q) acc[q] = double(tacc[q]);
  __shared__ double red[DIAG_WARPS][NSUM];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NSUM; ++q) red[warp][q] = acc[q];
  }
  __syncthreads();
  if (threadIdx.x < NSUM) {
    const int q = threadIdx.x;
    double v = red[0][q];
    for (int w = 1; w < DIAG_WARPS; ++w) v = q == NSUM - 1 ? fmax(v, red[w][q]) : v + red[w][q];
    partials[(size_t)(J.blk0 + blk) * NSUM + q] = v;
  }
  const double mid = 0.5 * (J.rho_l + J.rho_v);
  for (int k = blk * DIAG_WARPS + warp; k < Nz; k += J.nblk * DIAG_WARPS) {
    const double rad = col_radius_warp<C>(rho_o, Nz, Nr, k, mid, D.k64[K_R0]);
    if (lane == 0) cols[J.col0 + k] = rad;
  }
}

// One warp: the job's partial sums and column radii reduced into out[16].  Lane
// q + 8 s (q < 8, s < 4) folds quantity q of the blocks b = s (mod 4) in FP64,
// two shuffles join the four, and every lane takes the minimum over a share of
// the columns: short FP64 chains and no block barrier (GB300's FP64 operations
// are slow, so the pass is bound by their latency).
constexpr int FINAL_NT = 32;

template <class C>
__device__ void final_warp(const InstDesc& D, const DiagJob& J, int parity, const double* partials,
                           const double* cols, double* out) {
  const int Nz = D.Nz, Nr = D.Nr;
  const int lane = threadIdx.x & 31, q = lane & (NSUM - 1), sub = lane >> 3;
  double acc = 0.0;
  for (int b = sub; b < J.nblk; b += 4) {
    const double v = partials[(size_t)(J.blk0 + b) * NSUM + q];
    acc = q == NSUM - 1 ? fmax(acc, v) : acc + v;
  }
#pragma unroll
  for (int o = 8; o < 32; o <<= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, acc, o);
    acc = q == NSUM - 1 ? fmax(acc, v) : acc + v;
  }
  double cmin = 1e300;
  for (int k = lane; k < Nz; k += 32) cmin = fmin(cmin, cols[J.col0 + k]);
  cmin = warp_min(cmin);
  double t[NSUM];
#pragma unroll
  for (int i = 0; i < NSUM; ++i) t[i] = __shfl_sync(0xffffffffu, acc, i);
  if (lane == 0) {
    out[0] = t[0];
    out[1] = t[1];
    out[2] = t[2];
    out[3] = t[3];
    out[4] = sqrt(t[7]);
    out[5] = t[4] * J.a2norm;
    int kc = (int)llround(J.zc);
    kc %= Nz;
    if (kc < 0) kc += Nz;
    out[6] = cols[J.col0 + kc];
    out[7] = cmin;
    const C* psi = static_cast<const C*>(D.psi[parity]);
    const double G = D.G;
    auto pres = [&](int k, int j) {
      const double rho = double(static_cast<const C*>(D.rho_out)[(size_t)j * Nz + k]);
      const double ps = double(psi[(size_t)j * D.P + k]);
      return rho / 3.0 + G * ps * ps / 6.0;
    };
    const int ko = (kc + Nz / 2) % Nz;
    out[8] = pres(kc, 0);
    out[9] = pres(ko, Nr - 1);
    out[10] = out[8] - out[9];
    out[11] = t[6];
    out[12] = t[5];
    out[13] = out[14] = out[15] = 0.0;
  }
}

template <class C>
__global__ void __launch_bounds__(DIAG_NT) diag_partial_one(const InstDesc* __restrict__ descs, DiagJob J,
                                                            double* partials, double* cols) {
  partial_block<C>(descs[J.inst], J, blockIdx.x, partials, cols);
}

template <class C>
__global__ void __launch_bounds__(FINAL_NT) diag_final_one(const InstDesc* __restrict__ descs, DiagJob J,
                                                           int parity, const double* partials,
                                                           const double* cols, double* out) {
  final_warp<C>(descs[J.inst], J, parity, partials, cols, out);
}

// Every job of a batch: block b belongs to job blkjob[b] (the host's table of
// the jobs' block ranges [blk0, blk0 + nblk)).
template <class C>
__global__ void __launch_bounds__(DIAG_NT) diag_partial_all(const InstDesc* __restrict__ descs,
                                                            const DiagJob* __restrict__ jobs,
                                                            const int* __restrict__ blkjob,
                                                            double* partials, double* cols) {
  const DiagJob J = jobs[blkjob[blockIdx.x]];
  partial_block<C>(descs[J.inst], J, blockIdx.x - J.blk0, partials, cols);
}

template <class C>
__global__ void __launch_bounds__(FINAL_NT) diag_final_all(const InstDesc* __restrict__ descs,
                                                           const DiagJob* __restrict__ jobs, int parity,
                                                           const double* partials, const double* cols,
                                                           double* out) {
  const DiagJob J = jobs[blockIdx.x];
  final_warp<C>(descs[J.inst], J, parity, partials, cols, out + (size_t)16 * blockIdx.x);
}

}  // namespace

double a2_norm(double R) { return 5.0 / (4.0 * 3.14159265358979323846 * std::pow(R, 5.0)); }

void diag_job_constants(DiagJob& J) {
  J.a2norm = a2_norm(J.R);
  J.inv_dl = 1.0 / (J.rho_l - J.rho_v);
}

int diag_blocks(int Nz, int Nr) {
  const int N = Nz * Nr;
  int nb = (N + DIAG_NT * 4 - 1) / (DIAG_NT * 4);
  const int nbz = (Nz + DIAG_NT - 1) / DIAG_NT;
  if (nb < nbz) nb = nbz;
  if (nb > 1024) nb = 1024;
  return nb < 1 ? 1 : nb;
}

cudaError_t launch_diag(int storage, const InstDesc* d, int inst, int Nz, int Nr, int parity,
                        double zc, double R, double rho_l, double rho_v, double* partials,
                        int nblk, double* cols, double* out, cudaStream_t s) {
  (void)Nz;
  (void)Nr;
  DiagJob J;
  J.zc = zc;
  J.R = R;
  J.rho_l = rho_l;
  J.rho_v = rho_v;
  diag_job_constants(J);
  J.inst = inst;
  J.blk0 = 0;
  J.nblk = nblk;
  J.col0 = 0;
  if (storage == AMLBM_STORE_F64) {
    diag_partial_one<double><<<nblk, DIAG_NT, 0, s>>>(d, J, partials, cols);
    diag_final_one<double><<<1, FINAL_NT, 0, s>>>(d, J, parity, partials, cols, out);
  } else {
    diag_partial_one<float><<<nblk, DIAG_NT, 0, s>>>(d, J, partials, cols);
    diag_final_one<float><<<1, FINAL_NT, 0, s>>>(d, J, parity, partials, cols, out);
  }
  return cudaGetLastError();
}

cudaError_t diag_preload() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, diag_partial_one<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, diag_final_one<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, diag_partial_one<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, diag_final_one<float>);
  return e;
}

cudaError_t launch_diag_all(int storage, const InstDesc* d, const DiagJob* d_jobs, const int* d_blkjob,
                            int njobs, int total_blocks, int parity, double* partials, double* cols,
                            double* out, cudaStream_t s) {
  if (njobs < 1 || total_blocks < 1) return cudaErrorInvalidValue;
  if (storage == AMLBM_STORE_F64) {
    diag_partial_all<double><<<total_blocks, DIAG_NT, 0, s>>>(d, d_jobs, d_blkjob, partials, cols);
    diag_final_all<double><<<njobs, FINAL_NT, 0, s>>>(d, d_jobs, parity, partials, cols, out);
  } else {
    diag_partial_all<float><<<total_blocks, DIAG_NT, 0, s>>>(d, d_jobs, d_blkjob, partials, cols);
    diag_final_all<float><<<njobs, FINAL_NT, 0, s>>>(d, d_jobs, parity, partials, cols, out);
  }
  return cudaGetLastError();
}

}  // namespace amlbm
