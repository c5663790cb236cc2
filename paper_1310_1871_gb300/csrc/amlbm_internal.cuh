// Internal declarations shared by the kernels and the C-ABI host code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "amlbm.h"

namespace amlbm {

// One lattice of a batch as the kernels see it.  Populations are stored as
// [9][Nr][P] (z contiguous, row pitch P elements) and psi as [Nr][P]; both come
// in two copies (ping-pong) selected by the batch-wide parity.
struct InstDesc {
  int Nz, Nr, P;
  int wall, axisym, src;
  int tiles_z, tiles_r, tile_base;     // tiling of the step kernels
  int rb_tiles_z, rb_tiles_r, rb_tile_base;  // tiling of the read-back kernel (rb_tile())
  int shift;     // 0 none, 1 global (rho_ref), 2 local (rho recovered from psi)
  int rounding;  // 16-bit storage: 0 to nearest, 1 stochastic
  int zbc;       // AMLBM_Z_*: periodic, or no-slip walls at both ends in z
  int rlo;       // AMLBM_RLO_*: the axis, or an inlet row at row 0
  int forcing;   // AMLBM_FORCE_*: Shan-Chen velocity shift or Guo forcing
  double tau, G, rho0, gz, rho_ref;
  // the constants of the step, computed on the host in FP64 and also held
  // rounded to FP32 (kernels read them without conversion or division):
  // tau, 1/tau, -G, -G/18, g_z, rho0, 1/rho0, (tau - 1/2)/3, rho_ref,
  // the radius of row 0 (r_off + 1/2), the outlet density and 1 - 1/(2 tau)
  double k64[12];
  float k32[12];
  const double* inlet;  // inlet row velocity, u_z[Nz] then u_r[Nz] (zero until set)
  void* f[2];
  void* psi[2];
  void* uv;         // split schedule: u_z, u_r, u^eq_z, u^eq_r, 4 planes [Nr][P] of the compute type
  // [Nr][Nz] read-back of rho, u_z, u_r for the diagnostics and the host, in the
  // compute type (FP64 for FP64 storage, else FP32: GB300's FP64 path is slow, and
  // the FP32 forms' values are FP32 numbers anyway); room for FP64 either way
  void* rho_out;
  void* uz_out;
  void* ur_out;
};

// Slots of InstDesc::k64 / k32.
enum { K_TAU, K_OMEGA, K_NEGG, K_GFAC, K_GZ, K_RHO0, K_INVRHO0, K_CMU, K_RREF, K_R0, K_RHOOUT, K_GUO };

// Kernel launchers (defined in amlbm_step.cu).  storage = AMLBM_STORE_*.
// Every launcher returns the cudaGetLastError() of its launch.
// The step and macro kernels run CTAs for the flattened tiles
// [toff, toff + ntiles) of the batch.  schedule: 1 fused (one kernel), 2 split
// (force kernel, then collide-stream kernel), 3 pair (the fused update with two
// adjacent z-sites per thread; amlbm_step_pair.cu).
enum { SCHED_FUSED = 1, SCHED_SPLIT = 2, SCHED_PAIR = 3 };
// ctr (four ints, zero at creation): tile counters of the persistent fused
// grid and the step numbers for stochastic rounding, one per parity; nullptr
// launches one CTA per tile.
cudaError_t launch_step(int storage, int schedule, int tz, int tr, const InstDesc* d_desc,
                        const int* d_tile_inst, int ntiles, int toff, int parity, cudaStream_t s,
                        int* ctr);
cudaError_t launch_macro(int storage, int tz, int tr, const InstDesc* d_desc,
                         const int* d_tile_inst, int ntiles, int toff, int parity, cudaStream_t s);
// Loads the code of the read-back kernel of a storage form on the current
// device (the CUDA runtime otherwise loads it at its first launch).
cudaError_t macro_preload(int storage);
// Tile of the read-back kernel: 26 x 16 for the FP32-arithmetic forms (less halo
// work per site than 32 x 8), 32 x 8 for FP64.
inline void rb_tile(int storage, int* tz, int* tr) {
  const bool f64 = storage == 0;  // AMLBM_STORE_F64
  *tz = f64 ? 32 : 26;
  *tr = f64 ? 8 : 16;
}
cudaError_t launch_init(int storage, const InstDesc* d_desc, int inst, int Nz, int Nr,
                        const double* rho, const double* uz, const double* ur, int parity,
                        cudaStream_t s);
cudaError_t launch_unpack(int storage, const InstDesc* d_desc, int inst, int Nz, int Nr,
                          int parity, double* f_out, cudaStream_t s);
// Forward intermediates of one step, per site, [Nr][P] arrays of the compute
// type, for the adjoint: rho, u, u^eq, total force, psi, the Shan-Chen
// neighbour sums, d_r psi, d_rr psi, d_zr psi and the velocity gradients
// d_r u_z, d_z u_r, d_r u_r.
enum InterField {
  I_RHO, I_UZ, I_UR, I_VZ, I_VR, I_FZ, I_FR, I_PSI, I_SZ, I_SR, I_DR, I_DRR, I_DZR,
  I_G1, I_G2, I_G3, I_COUNT
};
// The timestep of instance 0 of d_desc from f[0] / psi[0] into f[1] / psi[1]
// (FP64 / FP32 storage, no shift) together with the intermediates of the state
// it starts from (I_COUNT planes of `plane` elements of the compute type).
cudaError_t launch_step_inter(int storage, int tz, int tr, const InstDesc* d_desc,
                              const int* d_tile_inst, int ntiles, void* inter, size_t plane,
                              cudaStream_t s);
// Diagnostics (amlbm_diag.cu) of the state whose rho / u the read-back kernel
// has written: partial sums into `partials` (nblk x 8 doubles) and the Nz column
// radii into `cols`, then a single-block pass into out[16].
cudaError_t launch_diag(int storage, const InstDesc* d_desc, int inst, int Nz, int Nr,
                        int parity, double zc, double R, double rho_l, double rho_v,
                        double* partials, int nblk, double* cols, double* out, cudaStream_t s);
int diag_blocks(int Nz, int Nr);
// Loads the code of the single-lattice diagnostics kernels on the current device
// (the CUDA runtime otherwise loads it at their first launch).
cudaError_t diag_preload();
// One instance's share of a batched diagnostics pass: its parameters, its
// blocks [blk0, blk0 + nblk) of the partial-sum grid (nblk = diag_blocks) and
// its columns [col0, col0 + Nz) of the radius array.
struct DiagJob {
  double zc, R, rho_l, rho_v;
  double a2norm;  // 5 / (4 pi R^5), the normalisation of a2 (computed on the host)
  double inv_dl;  // 1 / (rho_l - rho_v) (computed on the host)
  int inst, blk0, nblk, col0;
};
// The job's constants that need a division or a power (a2norm, inv_dl), from R,
// rho_l and rho_v, on the host: GB300's FP64 division is slow.
void diag_job_constants(DiagJob& J);
// Every job in one partial launch (total_blocks = sum of nblk; d_blkjob[b] is
// the job of partial block b) and one final launch (one block per job,
// out[16 * job]).
cudaError_t launch_diag_all(int storage, const InstDesc* d_desc, const DiagJob* d_jobs, const int* d_blkjob,
                            int njobs, int total_blocks, int parity, double* partials, double* cols,
                            double* out, cudaStream_t s);
double a2_norm(double R);
// f = f^eq(rho, u) for every instance from device arrays holding all
// instances back to back (site_off: n + 1 prefix offsets); counts the sites
// whose rho is not positive and finite into *bad (which must start at zero).
// FP64 or FP32 inputs.
cudaError_t launch_init_all(int storage, const InstDesc* d_desc, int n, const long long* d_site_off,
                            long long total, const double* rho, const double* uz, const double* ur,
                            int parity, int* bad, cudaStream_t s);
cudaError_t launch_init_all(int storage, const InstDesc* d_desc, int n, const long long* d_site_off,
                            long long total, const float* rho, const float* uz, const float* ur,
                            int parity, int* bad, cudaStream_t s);
bool tile_supported(int storage, int schedule, int tz, int tr);
int tile_list(int storage, int schedule, int* tz, int* tr, int cap);
// The pair schedule (amlbm_step_pair.cu): its compiled tiles and its persistent
// launch over all tiles (ctr as for the fused persistent launch).
bool pair_tile_supported(int storage, int tz, int tr);
int pair_tile_list(int storage, int* tz, int* tr, int cap);
cudaError_t launch_step_pair(int storage, int tz, int tr, const InstDesc* d_desc, const int* d_tile_inst,
                             int ntiles, int parity, cudaStream_t s, int* ctr);
// The read-back (rho, u into the read-back planes) of a pair batch, whose
// read-back list is tiled like its step: nt tiles from toff.  And the loading of
// that kernel's code on the current device (launches nothing).
cudaError_t launch_readback_pair(int storage, int tz, int tr, const InstDesc* d_desc, const int* d_tile_inst,
                                 int nt, int toff, int parity, cudaStream_t s);
cudaError_t readback_pair_preload(int storage, int tz, int tr);

// Access to a lattice context for entry points defined outside the ABI file
// (amlbm_abi.cu implements these).
struct CtxInfo {
  const InstDesc* d_desc;  // device descriptor array (one instance)
  InstDesc host;           // host copy of that descriptor
  int Nz, Nr, storage, parity;
  long long steps;
  cudaStream_t stream;
};
}  // namespace amlbm
struct amlbm_ctx;
namespace amlbm {
int ctx_info(amlbm_ctx* ctx, CtxInfo* out);
// Enqueue the read-back kernel (rho and u of the current state into the
// context's own buffers).
int ctx_readback(amlbm_ctx* ctx);
// Record a message for amlbm_last_error() and return code.
int set_error(int code, const std::string& msg);
// Shared by the diagnostics entry points (amlbm_abi.cu): the amlbm_diag of a
// result out[16] after `steps` steps, the parameters used when the caller
// passes none, and the message of AMLBM_EUNSTABLE.
void fill_diag(const double* h, long long steps, amlbm_diag* out);
amlbm_diag_params diag_defaults(const InstDesc& d);
std::string unstable_message(double bad);
// Looks up, once per device and with that device current, the device address of
// the allocation-free diagnostics' scratch array (amlbm_noalloc.cu), and loads
// the code of the kernels that entry point launches for this storage form.
// Lattice creation calls it, so that the lookup and the loading (which the CUDA
// runtime otherwise does lazily) happen in a call that allocates anyway.
int noalloc_prepare(int storage);

}  // namespace amlbm
