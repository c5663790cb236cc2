// amlbm_diagnostics_noalloc: the diagnostics of amlbm_diagnostics computed
// without any device allocation.
//
// Some callers cannot allocate device memory at the moment they want a
// diagnostic: for example a monitoring hook called from inside a host
// application whose caching allocator already owns the device memory (a raw
// cudaMalloc can then fail, and cudaMalloc / cudaFree synchronise the whole
// device, stalling the application's other streams).  This entry point
// therefore takes its reduction scratch (per-block partial sums, per-column
// interface radii and the 16-double result) from a fixed array in the
// library's own device memory, held from the moment the library's code is
// loaded on a device until the process exits.  The CUDA runtime loads that
// code lazily; the first lattice created on a device looks up the array's
// address there and loads the code of the diagnostics kernels (noalloc_prepare),
// so that code is on the device before this entry point can be called and the
// entry point itself never triggers the loading.  The lattice context supplies the input (its current state); the
// caller supplies the output struct.
//
// The array is shared by every call on a device: a call overwrites every
// entry it reads before reading it, so nothing has to be cleared between
// calls, but calls whose work overlaps on the GPU (from several host threads,
// or on several streams of one device) race on it and must be serialised by
// the caller.

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "amlbm.h"
#include "amlbm_internal.cuh"

namespace {

// Reduction blocks of the diagnostics kernel (its grid never exceeds this) and
// the largest Nz whose column radii fit.
constexpr int kMaxBlocks = 1024;
constexpr int kResult = 16;
constexpr size_t kScratchDoubles = (size_t)kMaxBlocks * 8 + AMLBM_NOALLOC_MAX_NZ + kResult;

// 131,200 bytes of device memory per device that loads the library.
static __device__ __align__(256) double g_diag_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

thread_local std::string g_err_local;

// Device address of the scratch array on the current device, looked up once
// per device with that device current (by the first lattice created there, or
// else by the first call).
int scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_err_local = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return AMLBM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    g_err_local = "device index out of range for the static diagnostics scratch";
    return AMLBM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_diag_scratch);
    if (e != cudaSuccess || !p) {
      g_err_local = std::string("cudaGetSymbolAddress(g_diag_scratch): ") +
                    cudaGetErrorString(e);
      return AMLBM_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return AMLBM_OK;
}

}  // namespace

namespace amlbm {
int noalloc_prepare(int storage) {
  double* p = nullptr;
  const int rc = scratch_for_current_device(&p);
  if (rc) return rc;
  // the code of the kernels it launches (read-back, diagnostics), so that its
  // first call loads nothing
  if (macro_preload(storage) != cudaSuccess || diag_preload() != cudaSuccess) return AMLBM_ECUDA;
  return AMLBM_OK;
}
}  // namespace amlbm

extern "C" int amlbm_diagnostics_noalloc(amlbm_ctx* ctx, const amlbm_diag_params* dp,
                                         amlbm_diag* out) {
  using amlbm::set_error;
  if (!ctx || !out) return set_error(AMLBM_EINVAL, "NULL context or output");
  amlbm::CtxInfo ci;
  int rc = amlbm::ctx_info(ctx, &ci);
  if (rc) return rc;
  const int Nz = ci.Nz, Nr = ci.Nr;
  if (Nz > AMLBM_NOALLOC_MAX_NZ)
    return set_error(AMLBM_EINVAL, "amlbm_diagnostics_noalloc: Nz = " + std::to_string(Nz) +
                                        " exceeds the static scratch limit AMLBM_NOALLOC_MAX_NZ = " +
                                        std::to_string(AMLBM_NOALLOC_MAX_NZ));
  const int nblk = amlbm::diag_blocks(Nz, Nr);
  if (nblk > kMaxBlocks)
    return set_error(AMLBM_EINVAL, "amlbm_diagnostics_noalloc: lattice too large");
  double* scratch = nullptr;
  rc = scratch_for_current_device(&scratch);
  if (rc) return set_error(rc, g_err_local);
  const amlbm_diag_params p = dp ? *dp : amlbm::diag_defaults(ci.host);
  if (!(p.R > 0) || !(p.rho_l != p.rho_v))
    return set_error(AMLBM_EINVAL, "diag params: need R > 0, rho_l != rho_v");
  rc = amlbm::ctx_readback(ctx);  // rho and u of the current state into the context's buffers
  if (rc) return rc;
  cudaStream_t s = ci.stream;
  double* part = scratch;
  double* cols = scratch + (size_t)kMaxBlocks * 8;
  double* res = cols + AMLBM_NOALLOC_MAX_NZ;
  cudaError_t e = amlbm::launch_diag(ci.storage, ci.d_desc, 0, Nz, Nr, ci.parity, p.zc, p.R,
                                     p.rho_l, p.rho_v, part, nblk, cols, res, s);
  if (e != cudaSuccess) return set_error(AMLBM_ECUDA, std::string("diag kernels: ") + cudaGetErrorString(e));
  double h[kResult];
  e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(AMLBM_ECUDA, std::string("diag read-back: ") + cudaGetErrorString(e));
  amlbm::fill_diag(h, ci.steps, out);
  if (out->bad > 0) return set_error(AMLBM_EUNSTABLE, amlbm::unstable_message(out->bad));
  return AMLBM_OK;
}
