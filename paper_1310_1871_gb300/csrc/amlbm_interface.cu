// Flat liquid-vapour interface: the coexistence densities and the surface
// tension of the Shan-Chen model for given G, tau, rho0 (the measurement of
// Table I, Sec. IV.1).  A lattice of 1 x n sites starts from a tanh slab
// (liquid below r = n/2, vapour above), runs `steps` timesteps of the library's
// own step kernel, then takes one more step that also writes the forward
// intermediates of the equilibrated state (d_r psi, the total force, rho, u),
// from which one block integrates
//   gamma       = -(G c_s^4 / 2) sum_j (d_r psi)^2                 (Eq. st)
//   gamma_tilde = gamma + (tau - 1/2)^2 sum_j F_r^2 / rho           (Eq. stc)
// with c_s^4 = 1/9 and the isotropic d_r psi of Sec. II.D.  Eq. st is the
// tension of the Guo forcing (no tau-correction), Eq. stc that of the Shan-Chen
// velocity shift (Sec. II.B); Table I lists both.

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "amlbm.h"
#include "amlbm_internal.cuh"

namespace {

using amlbm::InstDesc;

constexpr int RED_NT = 256;

// psi of row j of column 0 with the even mirror ghosts about r = 0 and the outer wall.
template <class C>
__device__ __forceinline__ double psi_row(const C* psi, int P, int Nr, int j) {
  if (j < 0) j = -1 - j;
  if (j >= Nr) j = 2 * Nr - 1 - j;
  return double(psi[(size_t)j * P]);
}

// One block: the sums over the rows of column 0, then the bulk densities (rows 0
// and n - 1) and the row position where rho crosses their mean.  out: gamma,
// gamma_tilde, rho_l, rho_v, position, umax.  d_r psi is taken from psi itself:
// on a lattice uniform in z the isotropic stencil of Sec. II.D reduces exactly to
// the 1D fourth-order difference (8 (psi_{j+1} - psi_{j-1}) - (psi_{j+2} - psi_{j-2}))/12,
// and the step kernel computes d_r psi only when the axisymmetric terms are on.
template <class C>
__global__ void __launch_bounds__(RED_NT) interface_reduce(const C* __restrict__ inter, size_t plane, int P,
                                                           int Nr, double G, double tau, double r0,
                                                           double* out) {
  __shared__ double sa[RED_NT], sb[RED_NT], su[RED_NT];
  double a = 0.0, b = 0.0, u = 0.0;
  const C* psi = inter + amlbm::I_PSI * plane;
  for (int j = threadIdx.x; j < Nr; j += RED_NT) {
    const size_t o = (size_t)j * P;
    const double dr = (8.0 * (psi_row(psi, P, Nr, j + 1) - psi_row(psi, P, Nr, j - 1)) -
                       (psi_row(psi, P, Nr, j + 2) - psi_row(psi, P, Nr, j - 2))) / 12.0;
    const double fr = double(inter[amlbm::I_FR * plane + o]);
    const double rho = double(inter[amlbm::I_RHO * plane + o]);
    const double uz = double(inter[amlbm::I_UZ * plane + o]), ur = double(inter[amlbm::I_UR * plane + o]);
    a += dr * dr;
    b += fr * fr / rho;
    u = fmax(u, uz * uz + ur * ur);
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  su[threadIdx.x] = u;
  __syncthreads();
  for (int w = RED_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
      su[threadIdx.x] = fmax(su[threadIdx.x], su[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double gam = -(G / 18.0) * sa[0];
    out[0] = gam;
    out[1] = gam + (tau - 0.5) * (tau - 0.5) * sb[0];
    const double rl = double(inter[amlbm::I_RHO * plane]);
    const double rv = double(inter[amlbm::I_RHO * plane + (size_t)(Nr - 1) * P]);
    out[2] = rl;
    out[3] = rv;
    const double mid = 0.5 * (rl + rv);
    double pos = -1.0;
    for (int j = 1; j < Nr && pos < 0.0; ++j) {
      const double v0 = double(inter[amlbm::I_RHO * plane + (size_t)(j - 1) * P]);
      const double v1 = double(inter[amlbm::I_RHO * plane + (size_t)j * P]);
      if ((v0 - mid) * (v1 - mid) <= 0.0 && v0 != v1) pos = (j - 1 + r0) + (v0 - mid) / (v0 - v1);
    }
    out[4] = pos;
    out[5] = sqrt(su[0]);
  }
}

struct DevBufs {
  void* p[4] = {nullptr, nullptr, nullptr, nullptr};
  ~DevBufs() {
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

}  // namespace

extern "C" int amlbm_flat_interface(double G, double tau, double rho0, int axisym, int forcing, int storage,
                                    int n, int steps, double rho_l0, double rho_v0, void* stream,
                                    amlbm_interface* out) {
  using amlbm::set_error;
  if (!out) return set_error(AMLBM_EINVAL, "flat interface: out is NULL");
  if (storage != AMLBM_STORE_F64 && storage != AMLBM_STORE_F32)
    return set_error(AMLBM_EINVAL, "flat interface: FP64 or FP32 storage");
  if (n < 8 || n > (1 << 20) || steps < 0) return set_error(AMLBM_EINVAL, "flat interface: need 8 <= n <= 2^20, steps >= 0");
  if (!(rho_l0 > rho_v0) || !(rho_v0 > 0) || !std::isfinite(rho_l0))
    return set_error(AMLBM_EINVAL, "flat interface: need rho_l0 > rho_v0 > 0");
  if (axisym != 0 && axisym != 1) return set_error(AMLBM_EINVAL, "flat interface: axisym must be 0 or 1");
  if (forcing != AMLBM_FORCE_SHIFT && forcing != AMLBM_FORCE_GUO)
    return set_error(AMLBM_EINVAL, "flat interface: bad forcing");
  amlbm_bc bc = {};
  bc.wall_r = AMLBM_WALL_FREESLIP;
  bc.axisym = axisym;
  bc.src_mode = AMLBM_SRC_LOCAL;
  bc.storage = storage;
  bc.shift = AMLBM_SHIFT_NONE;
  bc.rounding = AMLBM_ROUND_DEFAULT;
  bc.rho_ref = 1.0;
  bc.rho_out = 1.0;
  bc.forcing = forcing;
  amlbm_ctx* ctx = nullptr;
  int rc = amlbm_create(1, n, tau, G, rho0, &bc, stream, nullptr, 0, &ctx);
  if (rc) return rc;
  // the slab rho = rho_v + (rho_l - rho_v)/2 (1 - tanh((r - n/2)/2)), r = j + 1/2
  std::vector<double> rho(n);
  for (int j = 0; j < n; ++j)
    rho[j] = rho_v0 + 0.5 * (rho_l0 - rho_v0) * (1.0 - std::tanh((j + 0.5 - 0.5 * n) / 2.0));
  rc = amlbm_init_fields(ctx, rho.data(), nullptr, nullptr);
  if (!rc) rc = amlbm_step(ctx, steps);
  amlbm::CtxInfo ci;
  if (!rc) rc = amlbm::ctx_info(ctx, &ci);
  if (rc) {
    amlbm_destroy(ctx);
    return rc;
  }
  // one more step from the current state, writing the intermediates of that state
  InstDesc d = ci.host;
  d.f[0] = ci.host.f[ci.parity];
  d.psi[0] = ci.host.psi[ci.parity];
  d.f[1] = ci.host.f[ci.parity ^ 1];
  d.psi[1] = ci.host.psi[ci.parity ^ 1];
  d.tiles_z = 1;
  d.tiles_r = (n + 7) / 8;
  d.tile_base = 0;
  const int ntiles = d.tiles_r;
  const size_t cb = storage == AMLBM_STORE_F64 ? 8 : 4;
  const size_t plane = (size_t)d.P * n;
  DevBufs B;
  double res[6] = {0, 0, 0, 0, 0, 0};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMalloc(&B.p[0], sizeof(InstDesc));
  if (e == cudaSuccess) e = cudaMalloc(&B.p[1], ntiles * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B.p[2], amlbm::I_COUNT * plane * cb);
  if (e == cudaSuccess) e = cudaMalloc(&B.p[3], 8 * sizeof(double));
  if (e != cudaSuccess) {
    amlbm_destroy(ctx);
    return set_error(AMLBM_ENOMEM, std::string("flat interface: cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(B.p[0], &d, sizeof(InstDesc), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.p[1], 0, ntiles * sizeof(int), s);
  if (e == cudaSuccess)
    e = amlbm::launch_step_inter(storage, 32, 8, static_cast<const InstDesc*>(B.p[0]),
                                 static_cast<const int*>(B.p[1]), ntiles, B.p[2], plane, s);
  if (e == cudaSuccess) {
    const double r0 = 0.5;
    if (storage == AMLBM_STORE_F64)
      interface_reduce<double><<<1, RED_NT, 0, s>>>(static_cast<const double*>(B.p[2]), plane, d.P, n, G, tau,
                                                    r0, static_cast<double*>(B.p[3]));
    else
      interface_reduce<float><<<1, RED_NT, 0, s>>>(static_cast<const float*>(B.p[2]), plane, d.P, n, G, tau,
                                                   r0, static_cast<double*>(B.p[3]));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, B.p[3], sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  amlbm_destroy(ctx);
  if (e != cudaSuccess) return set_error(AMLBM_ECUDA, std::string("flat interface: ") + cudaGetErrorString(e));
  out->gamma = res[0];
  out->gamma_tilde = res[1];
  out->rho_l = res[2];
  out->rho_v = res[3];
  out->position = res[4];
  out->umax = res[5];
  return AMLBM_OK;
}
