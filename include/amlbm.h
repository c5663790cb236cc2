/*
 * amlbm.h -- C ABI of the GB300 (sm_103a) axisymmetric multiphase lattice
 * Boltzmann library (Srivastava, Perlekar, ten Thije Boonkkamp, Verma, Toschi,
 * "Axisymmetric Multiphase Lattice Boltzmann Method", arXiv:1310.1871).
 *
 * What the library computes (one timestep of every site of the D2Q9 meridional
 * (z, r) lattice, Sec. II):
 *   rho = sum_i f_i, rho u = sum_i c_i f_i                        (App. A, Eq. hydro_var)
 *   psi = rho0 (1 - exp(-rho / rho0))                             (Sec. II.A)
 *   F   = F_SC (Eq. scforce) + F^{gamma,sym} (Eq. scAxisExtra, with the
 *         isotropic stencils of Sec. II.D) + rho g_z e_z          (Sec. III.1)
 *   u   = (rho u + F/2)/rho,  u^eq = (rho u + tau F)/rho          (Eqs. uhydro, ueq)
 *   h_i = W_i (S + 3 (c_iz H_z + c_ir H_r)), S = -rho u_r / r     (Eq. condition_h, App. A)
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f^eq_i(rho, u^eq))/tau + h_i   (Eq. lbm2d_mod_new)
 * with mid-grid specular reflection on the axis, mid-grid specular (free-slip)
 * or bounce-back (no-slip) at the outer radial wall, and periodic z (Sec. II.E).
 * Bounded domains (the flow between two discs, Sec. III.2): no-slip walls at the
 * ends in z, an inlet row and an outlet row that hold the equilibrium of an
 * imposed velocity or density (Sec. II.E), and rows that start off the axis.
 *
 * Lattice conventions
 *   Sites (k, j), k = 0..Nz-1 along z (z_k = k), j = 0..Nr-1 along r
 *   (r_j = j + 1/2 + r_off; with the axis r_off = 0 and the axis lies half a
 *   spacing below row 0).
 *   Velocities (c_z, c_r): c_0 = (0,0), c_1 = (1,0), c_2 = (0,1), c_3 = (-1,0),
 *   c_4 = (0,-1), c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1), c_8 = (1,-1).
 *   Host field arrays are float64, row-major [Nr][Nz] (a[j * Nz + k]);
 *   populations on the host are float64 [9][Nr][Nz].
 *
 * Memory and ownership
 *   A context owns one device arena.  The caller either passes device memory
 *   (workspace != NULL, at least amlbm_*_workspace_bytes() bytes, 256-byte
 *   aligned, kept alive until destroy) or lets the library cudaMalloc it.
 *   Host arrays passed to any call are read or written during the call only.
 *   All work is enqueued on the stream given at creation (a cudaStream_t;
 *   NULL = legacy default stream).  Calls that return host data synchronise
 *   that stream; amlbm_step and amlbm_batch_step do not.
 *
 * Errors
 *   Every int-returning call returns AMLBM_OK (0) or a negative AMLBM_E* code
 *   and never throws.  amlbm_last_error() returns a thread-local message for
 *   the last failing call on the calling thread.  A CUDA error from an
 *   asynchronous launch may surface at a later call that synchronises.
 */
#ifndef AMLBM_H
#define AMLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMLBM_OK 0
#define AMLBM_EINVAL (-1)    /* bad argument (sizes, tau <= 1/2, rho0 <= 0, G < -6.5, ...) */
#define AMLBM_ENOMEM (-2)    /* device allocation failed or workspace too small */
#define AMLBM_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define AMLBM_EUNSTABLE (-5) /* diagnostics found a non-finite or non-positive density */

/* Outer radial boundary (Sec. II.E). */
#define AMLBM_WALL_FREESLIP 0 /* mid-grid specular reflection */
#define AMLBM_WALL_NOSLIP 1   /* mid-grid bounce-back */
#define AMLBM_WALL_OUTLET 2   /* outlet row: row Nr-1 holds f^eq(rho_out, u of row Nr-2) */

/* Ends of the lattice in z. */
#define AMLBM_Z_PERIODIC 0 /* periodic */
#define AMLBM_Z_NOSLIP 1   /* mid-grid bounce-back walls at z = -1/2 and z = Nz - 1/2 */

/* How the force F enters the collision (Sec. II.B; Sec. IV.1 compares the two). */
#define AMLBM_FORCE_SHIFT 0 /* Shan-Chen velocity shift: f^eq at u^eq = (rho u + tau F)/rho */
#define AMLBM_FORCE_GUO 1   /* Guo, Zheng & Shi (2002): f^eq at u, plus (1 - 1/(2 tau)) times
                               W_i [3 (c_i - u) + 9 (c_i . u) c_i] . F; fused schedule only, no adjoint */

/* Lower radial boundary. */
#define AMLBM_RLO_AXIS 0  /* the axis r = 0, half a spacing below row 0 (r_off = 0) */
#define AMLBM_RLO_INLET 1 /* inlet row: row 0 holds f^eq(rho of row 1, u_in(z)), u_in set by
                             amlbm_set_inlet (zero until set) */

/* Discretisation of h_i(x + c_i/2, t + 1/2) in Eq. lbm2d_mod_new. */
#define AMLBM_SRC_LOCAL 0 /* h at the departure site, time t (default) */
#define AMLBM_SRC_LINK 1  /* average of h at both ends of the link, time t */

/* Storage of the populations; arithmetic is FP64 for F64 and FP32 otherwise. */
#define AMLBM_STORE_F64 0
#define AMLBM_STORE_F32 1
#define AMLBM_STORE_F16 2  /* IEEE half of (f_i - W_i s) 2^10 (s: see AMLBM_SHIFT_*) */
#define AMLBM_STORE_BF16 3 /* bfloat16 of f_i - W_i s */

/* What the FP32 and 16-bit forms store: f_i - W_i s (or f_i - f^eq_i, EQUILIBRIUM).
 * FP64 storage is never shifted. */
#define AMLBM_SHIFT_DEFAULT 0 /* NONE for FP32, LOCAL for FP16 / BF16 */
#define AMLBM_SHIFT_NONE 1    /* s = 0 */
#define AMLBM_SHIFT_GLOBAL 2  /* s = rho_ref, one constant per lattice */
#define AMLBM_SHIFT_LOCAL 3   /* s = -rho0 ln(1 - psi/rho0) of the site's stored psi: the
                                 site's own density recovered from psi, no extra bytes */
#define AMLBM_SHIFT_EQUILIBRIUM 4 /* store f_i - f^eq_i(s, v) with s as LOCAL and v the bare
                                     velocity sum_i c_i f_i / rho of the stored state, kept in
                                     two FP32 planes beside psi (8 more bytes per site): the
                                     16-bit value then carries only the non-equilibrium part */

/* Rounding of the 16-bit stores.  Stochastic rounding draws its bits from a hash
 * of (site, population, step number), so a run is reproducible and unbiased in
 * expectation; round-to-nearest repeats the same error at every step of a
 * slowly varying state, and those errors add up. */
#define AMLBM_ROUND_DEFAULT 0 /* stochastic for BF16 with the W_i s shifts, else to nearest */
#define AMLBM_ROUND_NEAREST 1
#define AMLBM_ROUND_STOCHASTIC 2

/* Boundary and model options of one lattice. */
typedef struct amlbm_bc {
  int wall_r;     /* AMLBM_WALL_* */
  int axisym;     /* 1: axisymmetric sources and force (default); 0: planar 2D Shan-Chen */
  int src_mode;   /* AMLBM_SRC_* */
  int storage;    /* AMLBM_STORE_* (a batch uses the storage of its first instance) */
  int shift;      /* AMLBM_SHIFT_* */
  int rounding;   /* AMLBM_ROUND_* (16-bit storage) */
  double g_z;     /* body acceleration along +z (force rho g_z), Sec. III.1 */
  double rho_ref; /* constant of AMLBM_SHIFT_GLOBAL */
  /* Bounded domains; all zero gives the periodic lattice on the axis above. */
  int z_bc;       /* AMLBM_Z_* */
  int r_lo;       /* AMLBM_RLO_* */
  double r_off;   /* r_j = j + 1/2 + r_off, r_off >= 0; must be 0 with the axis */
  double rho_out; /* density of the outlet row (AMLBM_WALL_OUTLET), > 0 */
  int forcing;    /* AMLBM_FORCE_* (0: the paper's velocity shift) */
} amlbm_bc;

/* Parameters of the diagnostics (where to measure the drop or thread). */
typedef struct amlbm_diag_params {
  double zc;    /* axial position of the drop centre / probe column */
  double R;     /* radius used to normalise the quadrupole amplitude a2 */
  double rho_l; /* liquid density of the indicator phi = (rho - rho_v)/(rho_l - rho_v) */
  double rho_v; /* vapour density of the indicator */
} amlbm_diag_params;

/* Diagnostics of the current state, all accumulated in FP64 (deterministic order). */
typedef struct amlbm_diag {
  double mass2d; /* sum rho */
  double mass3d; /* sum 2 pi r rho */
  double momz3d; /* sum 2 pi r rho u_z (hydrodynamic u) */
  double Eke;    /* pi sum r rho |u|^2 (Sec. III) */
  double umax;   /* max |u| */
  double a2;     /* 5/(4 pi R^5) sum 2 pi r phi ((z - zc)^2 - r^2/2) */
  double A;      /* interface radius on column round(zc): first row where rho < (rho_l+rho_v)/2, interpolated */
  double neck;   /* minimum over columns of the interface radius */
  double p_in;   /* p = c_s^2 rho + c_s^2 G psi^2 / 2 (Eq. pressure) at (round(zc), row 0) */
  double p_out;  /* the same at (round(zc) + Nz/2, row Nr-1) */
  double dp;     /* p_in - p_out */
  double bad;    /* number of sites with non-finite or non-positive rho */
  double sumS;   /* sum over sites of the mass source -rho u_r / r */
  double steps;  /* timesteps taken since the fields were set */
  double reserved[2];
} amlbm_diag;

/* ---------------------------------------------------------------- one lattice */

typedef struct amlbm_ctx amlbm_ctx;

/* Device bytes a context of this size and storage needs. */
size_t amlbm_workspace_bytes(int Nz, int Nr, int storage);

/* Create a lattice of Nz x Nr sites with relaxation time tau (nu = (tau - 1/2)/3),
 * Shan-Chen coupling G and pseudopotential scale rho0.  bc may be NULL (defaults:
 * free-slip, axisymmetric, departure-site source, FP64 storage, default
 * shift, g_z = 0, rho_ref = 1, periodic z on the axis).  Requires Nz >= 1, Nr >= 4,
 * tau > 1/2, rho0 > 0, G >= -6.5 (the paper's stability limit is G >= -6,
 * Sec. II.D); z walls need Nz >= 4, inlet or outlet rows Nr >= 6.  A bounded
 * domain (z walls, inlet or outlet) runs on the fused schedule only and has no
 * adjoint (AMLBM_EINVAL).  cuda_stream is a cudaStream_t.  workspace: see
 * "Memory and ownership". */
int amlbm_create(int Nz, int Nr, double tau, double G, double rho0, const amlbm_bc* bc,
                 void* cuda_stream, void* workspace, size_t workspace_bytes, amlbm_ctx** out);

/* f = f^eq(rho, u) from host arrays [Nr][Nz] (uz, ur may be NULL for rest). */
int amlbm_init_fields(amlbm_ctx* ctx, const double* rho, const double* uz, const double* ur);

/* The same from device float64 arrays [Nr][Nz] (uz, ur may be NULL). */
int amlbm_init_fields_device(amlbm_ctx* ctx, const double* rho, const double* uz,
                             const double* ur);

/* Velocity of the inlet row (AMLBM_RLO_INLET): host arrays of Nz values, the
 * hydrodynamic u_z and u_r imposed at column k (Sec. II.E; for the flow between
 * discs, Middleman's profile at r = R_i, Sec. III.2).  Copied on the context's
 * stream; takes effect from the next step.  AMLBM_EINVAL if the lattice has no
 * inlet. */
int amlbm_set_inlet(amlbm_ctx* ctx, const double* uz, const double* ur);

/* Enqueue n timesteps (n >= 0) on the context's stream. */
int amlbm_step(amlbm_ctx* ctx, int n);

/* Density and hydrodynamic velocity (Eq. uhydro) of the current state into host
 * arrays [Nr][Nz]; any pointer may be NULL.  f (nullable) receives the decoded
 * populations [9][Nr][Nz].  Synchronises. */
int amlbm_read_fields(amlbm_ctx* ctx, double* rho, double* uz, double* ur, double* f);

/* Diagnostics of the current state; dp may be NULL (zc = Nz/2, R = 1, rho_l = 2,
 * rho_v = 0.1).  Returns AMLBM_EUNSTABLE (after filling *out) when bad > 0.
 * Synchronises. */
int amlbm_diagnostics(amlbm_ctx* ctx, const amlbm_diag_params* dp, amlbm_diag* out);

/* Copy the full state (populations, psi, the stored velocity of the equilibrium
 * shift, the step count and the position of the stochastic-rounding stream) to /
 * from a host buffer, so that a restarted run continues bit for bit.  The inlet
 * velocity of amlbm_set_inlet is configuration, not state: the context that
 * loads needs the same call.
 * amlbm_save_state with buf == NULL stores the needed size in *len. */
int amlbm_save_state(amlbm_ctx* ctx, void* buf, size_t* len);
int amlbm_load_state(amlbm_ctx* ctx, const void* buf, size_t len);

/* Device pointers of the current populations ([9][Nr][pitch], element type of
 * the storage) and psi ([Nr][pitch], FP64 for F64 storage, else FP32), and the
 * row pitch in elements.  Valid until the next step. */
int amlbm_device_state(amlbm_ctx* ctx, void** f, void** psi, int* pitch);

void amlbm_destroy(amlbm_ctx* ctx);

/* amlbm_diagnostics without any device allocation (the paper has no
 * counterpart: this is a library facility).  For callers that must not
 * allocate device memory when they ask for diagnostics, e.g. a monitoring hook
 * inside an application whose caching allocator owns the device memory (a raw
 * cudaMalloc may then fail, and cudaMalloc / cudaFree synchronise the whole
 * device).  Same arguments, result and errors as amlbm_diagnostics; the
 * context is the input and *out the output.  The reduction scratch is a fixed
 * array of the library's own device memory (131,200 bytes on every device
 * where the library's code is loaded, held until the process exits).  The
 * CUDA runtime loads that code lazily; amlbm_create (which allocates anyway)
 * loads it, and the code of the diagnostics kernels, on its device and looks up
 * the array's address there, so this call triggers no loading and no
 * allocation.  So:
 *   - lattices with Nz > AMLBM_NOALLOC_MAX_NZ are rejected with AMLBM_EINVAL;
 *   - call it with the context's device current;
 *   - every call shares the array: each call writes every entry it reads, so
 *     nothing needs clearing, but calls that overlap on the GPU (several host
 *     threads or streams of one device) race and must be serialised.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
#define AMLBM_NOALLOC_MAX_NZ 8192
int amlbm_diagnostics_noalloc(amlbm_ctx* ctx, const amlbm_diag_params* dp, amlbm_diag* out);

/* ------------------------------------------------------- flat interface tool */

/* Equilibrium of a flat liquid-vapour interface, the measurement of Table I
 * (Sec. IV.1): a lattice of 1 x n sites (free-slip outer wall) starts from the
 * slab rho = rho_v0 + (rho_l0 - rho_v0)/2 (1 - tanh((r - n/2)/2)), r = j + 1/2
 * (liquid below r = n/2), runs `steps` timesteps of the step kernel, then
 *   gamma       = -(G c_s^4 / 2) sum_j (d_r psi)^2             (Eq. st)
 *   gamma_tilde = gamma + (tau - 1/2)^2 sum_j F_r^2 / rho       (Eq. stc)
 * over the rows, with the isotropic d_r psi (Sec. II.D) and the total force F of
 * the equilibrated state.  gamma_tilde is the tension of the Shan-Chen velocity
 * shift the library uses; gamma that of a scheme without the tau-correction.
 * rho_l, rho_v are the densities on row 0 and row n-1: the coexistence densities
 * once the slab has relaxed (they do not depend on rho_l0, rho_v0, which only
 * need to lie on either side of the coexistence pair).  axisym = 0 is the planar
 * model (Table I, "2D"), 1 the axisymmetric one (a liquid cylinder of radius
 * ~n/2; Table I, "axis").  forcing: AMLBM_FORCE_* (Table I's "SC" columns are
 * gamma_tilde of the shift, its "Guo" columns gamma of the Guo forcing).
 * storage: AMLBM_STORE_F64 or AMLBM_STORE_F32.
 * Allocates and frees its own device memory on cuda_stream and synchronises it;
 * AMLBM_EINVAL for bad arguments (as amlbm_create, and n < 8, steps < 0,
 * rho_l0 <= rho_v0 or rho_v0 <= 0). */
typedef struct amlbm_interface {
  double gamma;       /* Eq. st */
  double gamma_tilde; /* Eq. stc */
  double rho_l;       /* density on row 0 */
  double rho_v;       /* density on row n-1 */
  double position;    /* radius where rho crosses (rho_l + rho_v)/2 */
  double umax;        /* max |u| of the equilibrated state (spurious current) */
} amlbm_interface;

int amlbm_flat_interface(double G, double tau, double rho0, int axisym, int forcing, int storage, int n,
                         int steps, double rho_l0, double rho_v0, void* cuda_stream, amlbm_interface* out);

/* ---------------------------------------------------------- differentiation */

/* Objectives of the differentiable runs (both linear in rho inside J). */
#define AMLBM_OBJ_A2SQ 0 /* J = a2(T)^2, a2 = 5/(4 pi R^5) sum 2 pi r phi ((z - zc)^2 - r^2/2) */
#define AMLBM_OBJ_NECK 1 /* J = sqrt(2 sum_j r_j phi(kstar, j)): the radius of column kstar */

/* A differentiable run: the initial density is a shape-perturbed drop
 *   rho = rho_v + (rho_l - rho_v)/2 (1 - tanh((d - R_s)/w)),
 *   R_s(theta) = R (1 + sum_m amps[m] P_{l0+m}(cos theta)),
 * d and theta measured from (zc, 0); f = f^eq(rho, 0); T timesteps; then J.
 * phi = (rho - rho_v)/(rho_l - rho_v). */
typedef struct amlbm_adjoint_problem {
  int T;           /* timesteps (>= 1) */
  int ckpt_every;  /* steps between stored states (>= 1); device memory ~ T/ckpt_every
                      states + ckpt_every states and their intermediates (26 planes each),
                      twice when T > ckpt_every (the recompute of one segment overlaps the
                      backward sweep of the next) */
  int objective;   /* AMLBM_OBJ_* */
  int l0;          /* Legendre degree of amps[0] */
  int n_amps;      /* 0..32 */
  int kstar;       /* column of AMLBM_OBJ_NECK */
  double zc, R, w, rho_l, rho_v;
  double obj_R;    /* R of the a2 normalisation */
  const double* amps; /* host array of n_amps amplitudes */
} amlbm_adjoint_problem;

/* Device bytes amlbm_adjoint needs for this context and problem (0 if invalid). */
size_t amlbm_adjoint_workspace_bytes(amlbm_ctx* ctx, const amlbm_adjoint_problem* p);

/* Hand-written discrete adjoint of the run above (the paper differentiates
 * nothing): J and dJ/dG, dJ/dtau, dJ/d(amps) (n_amps values).
 * The forward run stores the state every ckpt_every steps; the backward sweep
 * recomputes each segment (keeping every state of it and the forward
 * intermediates of each; on a second stream of its own, overlapping the backward
 * sweep of the segment after it) and applies the transposed step (inverse streaming,
 * adjoint collision and sources, transposed gradient and force stencils with the
 * mirror ghosts folded back) from the last step to the first.  Parameter
 * gradients accumulate in FP64.  Needs FP64 or FP32 storage without shift and the
 * departure-site source (AMLBM_SRC_LOCAL).  Overwrites the context's state.
 * workspace: device memory of amlbm_adjoint_workspace_bytes() bytes, or NULL
 * (then the library allocates and frees it).  Synchronises. */
int amlbm_adjoint(amlbm_ctx* ctx, const amlbm_adjoint_problem* p, void* workspace,
                  size_t workspace_bytes, double* J, double* dJ_dG, double* dJ_dtau,
                  double* dJ_damps);

/* J of the same run without the adjoint (for finite differences).  Overwrites the
 * context's state.  Synchronises. */
int amlbm_objective(amlbm_ctx* ctx, const amlbm_adjoint_problem* p, double* J);

/* ---------------------------------------------------------------- batches */

/* One independent lattice of a batch. */
typedef struct amlbm_instance {
  int Nz, Nr;
  double tau, G, rho0;
  amlbm_bc bc;
} amlbm_instance;

/* How a timestep is launched.  FUSED: one kernel per tile computes the whole
 * update, recomputing forces and velocities on a 3-site halo.  SPLIT: a force
 * kernel writes u and u^eq per site, then a collide-stream kernel reads them with
 * a halo (less recomputation, 16 or 32 more bytes per site through L2).  PAIR:
 * the fused update with two adjacent z-sites per thread (vector loads and
 * stores, stencil taps shared by the pair); it takes periodic lattices on the
 * axis with an even Nz, a free-slip or no-slip outer wall, the source at the
 * departure site (AMLBM_SRC_LOCAL) and either forcing, and 9 x pitch x Nr below
 * 2^31 elements.  All three give bit-identical states. */
#define AMLBM_SCHED_AUTO 0
#define AMLBM_SCHED_FUSED 1
#define AMLBM_SCHED_SPLIT 2
#define AMLBM_SCHED_PAIR 3

/* Schedule and tile shape (sites along z x sites along r) of the step kernels;
 * all zero lets the library choose.  A tile given with AMLBM_SCHED_AUTO runs on
 * the split schedule, or on the fused one if any instance is a bounded domain. */
typedef struct amlbm_tune {
  int tile_z, tile_r;
  int graph_chunk; /* steps per captured CUDA graph in amlbm_batch_step (0 = no graph) */
  int schedule;    /* AMLBM_SCHED_* */
} amlbm_tune;

typedef struct amlbm_batch amlbm_batch;

/* Tiles compiled for a storage form and schedule, as pairs (tile_z, tile_r);
 * returns the count (tz, tr may be NULL to query it). */
int amlbm_tiles(int storage, int schedule, int* tz, int* tr, int cap);

/* One candidate of the autotuner and its measured step time. */
typedef struct amlbm_tune_result {
  amlbm_tune tune;
  double ms_per_step; /* fastest of three timed repeats, CUDA events on the stream */
  double mlups;       /* sites of all instances / ms_per_step */
} amlbm_tune_result;

/* Autotuner (no counterpart in the paper, which fixes no launch shape): for the
 * n instances (all with inst[0].bc.storage) it creates a temporary batch for
 * every compiled (schedule, tile) pair, sets a resting drop on every lattice,
 * runs 3 warm-up and 3 x `steps` timed timesteps on cuda_stream, and writes the
 * fastest pair to *best (graph_chunk 0; a candidate within 0.5 % of an earlier
 * one, in schedule and amlbm_tiles order, does not replace it) and, when results
 * is not NULL, up to cap candidates with their timings.  Every candidate computes the same state.
 * Allocates and frees device memory for each candidate (it is not capturable)
 * and synchronises the stream.  Returns the number of candidates timed (> 0)
 * or a negative status. */
int amlbm_autotune(int n, const amlbm_instance* inst, int steps, void* cuda_stream,
                   amlbm_tune* best, amlbm_tune_result* results, int cap);

size_t amlbm_batch_workspace_bytes(int n, const amlbm_instance* inst);

/* n independent lattices stepped together: one kernel launch per timestep covers
 * every tile of every instance.  All instances use inst[0].bc.storage. */
int amlbm_batch_create(int n, const amlbm_instance* inst, const amlbm_tune* tune,
                       void* cuda_stream, void* workspace, size_t workspace_bytes,
                       amlbm_batch** out);
int amlbm_batch_init_fields(amlbm_batch* b, int k, const double* rho, const double* uz,
                            const double* ur);
/* amlbm_set_inlet for instance k. */
int amlbm_batch_set_inlet(amlbm_batch* b, int k, const double* uz, const double* ur);
int amlbm_batch_step(amlbm_batch* b, int n);
int amlbm_batch_read(amlbm_batch* b, int k, double* rho, double* uz, double* ur, double* f);
int amlbm_batch_diagnostics(amlbm_batch* b, int k, const amlbm_diag_params* dp, amlbm_diag* out);
/* Every instance at once, f = f^eq(rho, u) as amlbm_batch_init_fields does per
 * instance (the initial state of Sec. II), from caller-owned host arrays that
 * hold all instances back to back in instance order: instance k's [Nr][Nz]
 * block starts at the sum of Nz*Nr over the instances before it, and the total
 * length is amlbm_batch_sites().  uz and ur may be NULL (zero velocity).  One
 * kernel launch; it reads page-locked (pinned) host arrays in place over the
 * CPU-GPU link, and any other array is first copied to the device (one
 * host-to-device copy per array).  The arrays are read during the call only.  rho is checked on the
 * device and the call returns AMLBM_EINVAL, with every instance's state
 * unchanged, if any value is not positive and finite.  Resets every instance's
 * step count and restarts the stochastic-rounding stream, so that the steps
 * that follow equal those of a newly created batch.  Synchronises the batch
 * stream. */
int amlbm_batch_init_all(amlbm_batch* b, const double* rho, const double* uz, const double* ur);
/* amlbm_batch_init_all from FP32 host arrays (same layout, ownership, checks
 * and errors), half the bytes over the CPU-GPU link.  Each value is widened
 * exactly to FP64, so the state equals that of amlbm_batch_init_all given the
 * same values in FP64; the FP32-arithmetic forms (FP32, FP16 and BF16 storage)
 * round their FP64 inputs to FP32 first, so for them it equals
 * amlbm_batch_init_all of any FP64 arrays that round to these values. */
int amlbm_batch_init_all_f32(amlbm_batch* b, const float* rho, const float* uz, const float* ur);
/* The diagnostics of every instance in one pass (one read-back launch, one
 * partial-sum launch, one final launch, one device-to-host copy): dp holds n
 * parameter sets (NULL: the defaults of amlbm_batch_diagnostics), out receives
 * n results, each equal to what amlbm_batch_diagnostics gives for that
 * instance.  Returns AMLBM_EUNSTABLE, after filling every output, if any
 * instance has a non-finite or non-positive density (the message names the
 * first).  Synchronises the batch stream. */
int amlbm_batch_diagnostics_all(amlbm_batch* b, const amlbm_diag_params* dp, amlbm_diag* out);
/* Sites of all instances (the work of one batch timestep). */
long long amlbm_batch_sites(const amlbm_batch* b);
/* The schedule and tile the batch runs with, and kernel launches per timestep. */
int amlbm_batch_config(const amlbm_batch* b, int* schedule, int* tile_z, int* tile_r,
                       int* launches_per_step);
void amlbm_batch_destroy(amlbm_batch* b);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* amlbm_last_error(void);

/* Library version string. */
const char* amlbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AMLBM_H */
