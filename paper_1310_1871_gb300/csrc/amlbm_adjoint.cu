// Discrete adjoint of the axisymmetric Shan-Chen LBM step (the reverse sweep of
// the update of Sec. II, transposed operation by operation), the device map from
// Legendre shape amplitudes to the initial drop, the objectives, and the
// checkpointed driver behind amlbm_adjoint / amlbm_objective.
//
// The forward intermediates of every state of a checkpoint segment are written
// while the segment is recomputed (lbm_kernel MODE 3: the step and the
// intermediates of the state it starts from in one pass).  One adjoint step
// (lambda^{n+1} -> lambda^n, state f^n) then runs as:
//   post   : mu = transpose of the streaming map (a gather), then the adjoint of
//            the BGK collision and of the sources S, H_z, H_r  -> rho, u, u^eq,
//            velocity-gradient adjoints, tau part
//   vel    : transposed gradient stencils with the u ghosts folded back, the
//            adjoint of u = (j + F/2)/rho and u^eq = (j + tau F)/rho, and at the
//            same site the adjoint of F_SC (Eq. scforce) and F^gamma (Eq.
//            scAxisExtra) (local psi factor, d_zr, d_rr, d_r parts), G part
//   deriv  : transposed 1D d_z (of d_zr) and isotropic d_r (of d_rr)
//   final  : transposed Shan-Chen neighbour sum, 1D d_r and isotropic d_r on psi,
//            psi ghosts folded onto their mirrors, d psi/d rho, and
//            lambda^n_i = (1 - omega) mu_i + rho_bar + c_i . j_bar.
// All kernels are gathers (no atomics), so the sweep is deterministic.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "amlbm.h"
#include "amlbm_internal.cuh"

namespace amlbm {
namespace {

__host__ __device__ constexpr int acz(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int acr(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr double aw(int i) {
  return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int amirror(int i) {
  return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i;
}
__host__ __device__ constexpr int aopp(int i) {
  return i == 0 ? 0 : i == 1 ? 3 : i == 3 ? 1 : i == 2 ? 4 : i == 4 ? 2
       : i == 5 ? 7 : i == 7 ? 5 : i == 6 ? 8 : 6;
}

// Periodic wrap of a column that lies a few sites outside [0, Nz) (no
// division: stencil offsets are at most 4, so one or two corrections suffice
// unless Nz is smaller than that).
__device__ __forceinline__ int wz(int k, int Nz) {
  while (k < 0) k += Nz;
  while (k >= Nz) k -= Nz;
  return k;
}

template <class C>
struct Adj {
  int Nz, Nr, P, wall, axisym;
  size_t plane;
  C tau, omega, G, rho0, gz, inv_rho0;
  const C* lam_in;
  C* lam_out;
  const C* f;      // state f^n, 9 planes
  const C* inter;  // I_COUNT planes
  C* mu;           // 9 planes
  C *rhob, *uzb, *urb, *vzb, *vrb, *g1b, *g2b, *g3b, *jzb, *jrb, *Fzb, *Frb;
  C *psib, *qz, *qr, *dzrb, *drrb, *drdb, *eb;
  C* drpb;  // d_r psi adjoint on rows -2 .. Nr+1 (row offset 2)
  double *accG, *accT;
};

// value of a [Nr][P] field at (k, j), zero outside the real rows
template <class C>
__device__ __forceinline__ C at(const C* a, int k, int j, const Adj<C>& A) {
  if (j < 0 || j >= A.Nr) return C(0);
  return a[(size_t)j * A.P + wz(k, A.Nz)];
}
// d_r psi adjoint on the padded rows -2 .. Nr+1, zero outside
template <class C>
__device__ __forceinline__ C atpad(const C* a, int k, int j, const Adj<C>& A) {
  if (j < -2 || j > A.Nr + 1) return C(0);
  return a[(size_t)(j + 2) * A.P + wz(k, A.Nz)];
}

template <class C>
__device__ __forceinline__ C feq_std(int i, C rho, C vz, C vr) {
  const C cv = C(acz(i)) * vz + C(acr(i)) * vr;
  return C(aw(i)) * rho * (C(1) + C(3) * cv + C(4.5) * cv * cv - C(1.5) * (vz * vz + vr * vr));
}

// ---- shared-memory windows of the tiled transposed kernels
// A block of ATZ x ATR threads handles the ATZ x ATR sites (k0 + tx, j0 + ty).  A
// window holds a [Nr][P] field on rows j0 - HR .. j0 + ATR - 1 + HR and columns
// k0 - 2 .. k0 + ATZ + 1 (wrapped in z), with the value the global accessors give
// outside the stored rows (zero), so the transposed stencils read it exactly as
// they would read global memory.  Blocks away from the axis and the wall load only
// the rows their own sites' stencils reach (radius 2).
constexpr int ATZ = 32, ATR = 8, ANT = ATZ * ATR;

template <class C, int HR>
struct Win {
  static constexpr int W = ATZ + 4, H = ATR + 2 * HR;
  C v[H * W];
};

template <bool PAD, class C, int HR>
__device__ __forceinline__ void load_win(Win<C, HR>& w, const C* g, int k0, int j0, bool near_edge,
                                         const Adj<C>& A) {
  constexpr int W = Win<C, HR>::W;
  const int r_lo = near_edge ? 0 : HR - 2, r_hi = near_edge ? Win<C, HR>::H : HR + ATR + 2;
  for (int i = r_lo * W + threadIdx.x; i < r_hi * W; i += ANT) {
    const int rr = i / W, cc = i - rr * W;
    const int y = j0 - HR + rr, k = k0 - 2 + cc;
    w.v[i] = PAD ? atpad(g, k, y, A) : at(g, k, y, A);
  }
}

template <class C, int HR>
__device__ __forceinline__ C wat(const Win<C, HR>& w, int k, int y, int k0, int j0) {
  return w.v[(y - j0 + HR) * Win<C, HR>::W + (k - k0 + 2)];
}

// Transpose of the isotropic derivative along r (AX = 1) or z (AX = 0) at the
// (possibly ghost) position (k, j), on a window:
//   sum_i c_i,AX (8 g(y - c_i) - g(y - 2 c_i)) / 36.
template <int AX, class C, int HR>
__device__ __forceinline__ C iso_tw(const Win<C, HR>& g, int k, int j, int k0, int j0) {
  C s = C(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = AX ? acr(i) : acz(i);
    if (c == 0) continue;
    const C a = wat(g, k - acz(i), j - acr(i), k0, j0);
    const C b = wat(g, k - 2 * acz(i), j - 2 * acr(i), k0, j0);
    s += C(c) * (C(8) * a - b);
  }
  return s * C(1.0 / 36.0);
}

// Transpose of the 1D 4th-order difference along r (AX = 1) or z (AX = 0) at the
// (possibly ghost) position (k, j), on a window.  The forward operator
// (8 (g(y + e) - g(y - e)) - (g(y + 2e) - g(y - 2e))) / 12 is antisymmetric, so
// its transpose is its negative.
template <int AX, class C, int HR>
__device__ __forceinline__ C d1_tw(const Win<C, HR>& g, int k, int j, int k0, int j0) {
  const int ez = AX ? 0 : 1, er = AX ? 1 : 0;
  const C a = wat(g, k + ez, j + er, k0, j0) - wat(g, k - ez, j - er, k0, j0);
  const C b = wat(g, k + 2 * ez, j + 2 * er, k0, j0) - wat(g, k - 2 * ez, j - 2 * er, k0, j0);
  return -(C(8) * a - b) * C(1.0 / 12.0);
}

// ---- post: inverse streaming, collision and source adjoints (per real site)
template <class C>
__global__ void __launch_bounds__(ANT) adj_post(Adj<C> A) {
  // lambda^{n+1} on the tile + 1 (9 planes), the rows and columns every arrival
  // site of the tile's populations lies in
  constexpr int W = ATZ + 2, H = ATR + 2;
  __shared__ C wl[9][H * W];
  const int k0 = blockIdx.x * ATZ, j0 = blockIdx.y * ATR;
  for (int i = threadIdx.x; i < H * W; i += ANT) {
    const int rr = i / W, cc = i - rr * W;
    const int y = j0 - 1 + rr, x = k0 - 1 + cc;
    const bool in = y >= 0 && y < A.Nr;
    const size_t g = in ? (size_t)y * A.P + wz(x, A.Nz) : 0;
#pragma unroll
    for (int d = 0; d < 9; ++d) wl[d][i] = in ? A.lam_in[d * A.plane + g] : C(0);
  }
  __syncthreads();
  const int k = k0 + (int)threadIdx.x % ATZ, j = j0 + (int)threadIdx.x / ATZ;
  if (k >= A.Nz || j >= A.Nr) return;
  const size_t o = (size_t)j * A.P + k;
  const bool noslip = A.wall == AMLBM_WALL_NOSLIP;
  C mu[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    // where population q leaving (k, j) arrives after streaming (Sec. II.E maps)
    int yk = k + acz(q), yj = j + acr(q), d = q;
    if (yj < 0) {
      yj = 0; d = amirror(q);
    } else if (yj >= A.Nr) {
      if (noslip) { yk = k; yj = A.Nr - 1; d = aopp(q); }
      else { yj = A.Nr - 1; d = amirror(q); }
    }
    mu[q] = wl[d][(yj - j0 + 1) * W + (yk - k0 + 1)];
    A.mu[q * A.plane + o] = mu[q];
  }
  const C* I = A.inter + o;
  const C rho = I[I_RHO * A.plane], vz = I[I_VZ * A.plane], vr = I[I_VR * A.plane];
  const C uz = I[I_UZ * A.plane], ur = I[I_UR * A.plane];
  C rb = C(0), vzb = C(0), vrb = C(0), tb = C(0);
  const C irho = C(1) / rho;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const C fe = feq_std(q, rho, vz, vr);
    const C cv = C(acz(q)) * vz + C(acr(q)) * vr;
    const C m = A.omega * mu[q];
    rb += m * fe * irho;
    const C com = m * C(aw(q)) * rho;
    vzb += com * (C(3) * C(acz(q)) + C(9) * cv * C(acz(q)) - C(3) * vz);
    vrb += com * (C(3) * C(acr(q)) + C(9) * cv * C(acr(q)) - C(3) * vr);
    tb += -A.omega * A.omega * mu[q] * (fe - A.f[q * A.plane + o]);
  }
  C uzb = C(0), urb = C(0), g1b = C(0), g2b = C(0), g3b = C(0);
  if (A.axisym) {
    C Sb = C(0), Hzb = C(0), Hrb = C(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Sb += mu[q] * C(aw(q));
      Hzb += C(3) * mu[q] * C(aw(q)) * C(acz(q));
      Hrb += C(3) * mu[q] * C(aw(q)) * C(acr(q));
    }
    const C r = C(j) + C(0.5), ir = C(1) / r;
    const C g1 = I[I_G1 * A.plane], g2 = I[I_G2 * A.plane], g3 = I[I_G3 * A.plane];
    const C cmu = (A.tau - C(0.5)) * C(1.0 / 3.0);
    const C muv = rho * cmu;
    // S = -rho u_r / r
    rb += -Sb * ur * ir;
    urb += -Sb * rho * ir;
    // H_z = (mu (g1 + g2) - rho u_r u_z) / r
    C mvb = Hzb * (g1 + g2) * ir;
    g1b = Hzb * muv * ir;
    g2b = Hzb * muv * ir;
    rb += -Hzb * ur * uz * ir;
    urb += -Hzb * rho * uz * ir;
    uzb += -Hzb * rho * ur * ir;
    // H_r = (2 mu (g3 - u_r / r) - rho u_r^2) / r
    mvb += Hrb * C(2) * (g3 - ur * ir) * ir;
    g3b = Hrb * C(2) * muv * ir;
    urb += Hrb * (-C(2) * muv * ir - C(2) * rho * ur) * ir;
    rb += -Hrb * ur * ur * ir;
    // mu = rho (tau - 1/2) / 3
    rb += mvb * cmu;
    tb += mvb * rho * C(1.0 / 3.0);
  }
  A.rhob[o] = rb;
  A.uzb[o] = uzb;
  A.urb[o] = urb;
  A.vzb[o] = vzb;
  A.vrb[o] = vrb;
  A.g1b[o] = g1b;
  A.g2b[o] = g2b;
  A.g3b[o] = g3b;
  A.accT[o] += double(tb);
}

// ---- vel: transposed gradient stencils (u ghosts folded), adjoint of u and u^eq;
// then (same site, no neighbours) the local adjoint of F_SC and F^gamma
template <class C>
__global__ void __launch_bounds__(ANT) adj_vel(Adj<C> A) {
  constexpr int HR = 5;  // ghost rows -2, -1 and Nr, Nr + 1 reach two rows further
  __shared__ Win<C, HR> w1, w2, w3;
  const int k0 = blockIdx.x * ATZ, j0 = blockIdx.y * ATR;
  const int k = k0 + (int)threadIdx.x % ATZ, j = j0 + (int)threadIdx.x / ATZ;
  if (A.axisym) {
    const bool near_edge = j0 < 2 || j0 + ATR > A.Nr - 2;
    load_win<false>(w1, A.g1b, k0, j0, near_edge, A);
    load_win<false>(w2, A.g2b, k0, j0, near_edge, A);
    load_win<false>(w3, A.g3b, k0, j0, near_edge, A);
    __syncthreads();
  }
  if (k >= A.Nz || j >= A.Nr) return;
  const size_t o = (size_t)j * A.P + k;
  C uzb = A.uzb[o], urb = A.urb[o];
  if (A.axisym) {
    const C szw = A.wall == AMLBM_WALL_NOSLIP ? C(-1) : C(1);
    uzb += d1_tw<1>(w1, k, j, k0, j0);
    urb += d1_tw<0>(w2, k, j, k0, j0) + d1_tw<1>(w3, k, j, k0, j0);
    // ghost rows (depth 2) that mirror this row: u_z even / u_r odd at the axis;
    // at the wall u_r odd and u_z even (free-slip) or odd (no-slip)
    const int ga = -1 - j;
    if (ga >= -2) {
      uzb += d1_tw<1>(w1, k, ga, k0, j0);
      urb -= d1_tw<0>(w2, k, ga, k0, j0) + d1_tw<1>(w3, k, ga, k0, j0);
    }
    const int gw = 2 * A.Nr - 1 - j;
    if (gw <= A.Nr + 1) {
      uzb += szw * d1_tw<1>(w1, k, gw, k0, j0);
      urb -= d1_tw<0>(w2, k, gw, k0, j0) + d1_tw<1>(w3, k, gw, k0, j0);
    }
  }
  const C* I = A.inter + o;
  const C rho = I[I_RHO * A.plane], ir = C(1) / rho;
  const C uz = I[I_UZ * A.plane], ur = I[I_UR * A.plane], vz = I[I_VZ * A.plane],
          vr = I[I_VR * A.plane], Fz = I[I_FZ * A.plane], Fr = I[I_FR * A.plane];
  const C vzb = A.vzb[o], vrb = A.vrb[o];
  A.jzb[o] = (uzb + vzb) * ir;
  A.jrb[o] = (urb + vrb) * ir;
  const C Fzb = (C(0.5) * uzb + A.tau * vzb) * ir, Frb = (C(0.5) * urb + A.tau * vrb) * ir;
  A.Fzb[o] = Fzb;
  A.Frb[o] = Frb;
  A.rhob[o] += -(uzb * uz + urb * ur + vzb * vz + vrb * vr) * ir + Fzb * A.gz;
  double tacc = double((vzb * Fz + vrb * Fr) * ir);
  // F_SC = -G psi s
  const C psi = I[I_PSI * A.plane], sz = I[I_SZ * A.plane], sr = I[I_SR * A.plane];
  C pb = -A.G * (Fzb * sz + Frb * sr);
  double gb = double(-psi * (Fzb * sz + Frb * sr));
  A.qz[o] = -A.G * psi * Fzb;
  A.qr[o] = -A.G * psi * Frb;
  C dzrb = C(0), drrb = C(0), drdb = C(0);
  if (A.axisym) {
    const C irr = C(1) / (C(j) + C(0.5));
    const C Dr = I[I_DR * A.plane], Drr = I[I_DRR * A.plane], Dzr = I[I_DZR * A.plane];
    const C gf = -A.G * C(1.0 / 18.0);
    const C t = Fzb * Dzr * irr + Frb * (Drr * irr - Dr * irr * irr);
    pb += gf * t;
    gb += double(-psi * t * C(1.0 / 18.0));
    dzrb = gf * psi * Fzb * irr;
    drrb = gf * psi * Frb * irr;
    drdb = -gf * psi * Frb * irr * irr;
  }
  A.psib[o] = pb;
  A.dzrb[o] = dzrb;
  A.drrb[o] = drrb;
  A.drdb[o] = drdb;
  A.accG[o] += gb;
  A.accT[o] += tacc;
}


// ---- deriv: transposed 1D d_z (into the 1D d_r field) and isotropic d_r (into
// the padded d_r psi field, rows -2 .. Nr+1); tiles of the padded rows
template <class C>
__global__ void __launch_bounds__(ANT) adj_deriv(Adj<C> A) {
  __shared__ Win<C, 2> wr;             // d_rr psi adjoint, padded rows jp0 - 2 .. jp0 + ATR + 1
  __shared__ C wd[ATR * (ATZ + 4)];    // d_zr psi adjoint, rows jp0 .. jp0 + ATR - 1
  const int k0 = blockIdx.x * ATZ, jp0 = -2 + (int)blockIdx.y * ATR;
  load_win<false>(wr, A.drrb, k0, jp0, true, A);
  for (int i = threadIdx.x; i < ATR * (ATZ + 4); i += ANT) {
    const int rr = i / (ATZ + 4), cc = i - rr * (ATZ + 4);
    const int y = jp0 + rr;
    wd[i] = (y >= 0 && y < A.Nr) ? A.dzrb[(size_t)y * A.P + wz(k0 - 2 + cc, A.Nz)] : C(0);
  }
  __syncthreads();
  const int tx = (int)threadIdx.x % ATZ, ty = (int)threadIdx.x / ATZ;
  const int k = k0 + tx, jp = jp0 + ty;
  if (k >= A.Nz || jp > A.Nr + 1) return;
  if (jp >= 0 && jp < A.Nr) {
    const C* d = wd + ty * (ATZ + 4) + tx + 2;  // column k
    const C e = (C(8) * (d[-1] - d[1]) - (d[-2] - d[2])) * C(1.0 / 12.0);
    A.eb[(size_t)jp * A.P + k] = e;
  }
  C v = iso_tw<1>(wr, k, jp, k0, jp0);
  if (jp >= 0 && jp < A.Nr) v += A.drdb[(size_t)jp * A.P + k];
  A.drpb[(size_t)(jp + 2) * A.P + k] = v;
}

// psi adjoint at the (possibly ghost) position (k, y): transposed Shan-Chen
// neighbour sum, 1D d_r and isotropic d_r, from the windows of q_z, q_r, the 1D
// d_r adjoint e and the padded d_r psi adjoint.
template <class C, int HR>
__device__ __forceinline__ C psi_pad_adj(int k, int y, int k0, int j0, const Win<C, HR>& qz,
                                         const Win<C, HR>& qr, const Win<C, HR>& eb,
                                         const Win<C, HR>& dp, bool axisym) {
  C s = C(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const C w = C(aw(i));
    if (acz(i)) s += w * C(acz(i)) * wat(qz, k - acz(i), y - acr(i), k0, j0);
    if (acr(i)) s += w * C(acr(i)) * wat(qr, k - acz(i), y - acr(i), k0, j0);
  }
  if (axisym) {
    s += (C(8) * (wat(eb, k, y - 1, k0, j0) - wat(eb, k, y + 1, k0, j0)) -
          (wat(eb, k, y - 2, k0, j0) - wat(eb, k, y + 2, k0, j0))) * C(1.0 / 12.0);
    s += iso_tw<1>(dp, k, y, k0, j0);
  }
  return s;
}

// ---- final: psi ghosts folded (even mirrors, depth 4), d psi / d rho, lambda^n
template <class C>
__global__ void __launch_bounds__(ANT) adj_final(Adj<C> A) {
  constexpr int HR = 9;  // ghost rows down to -4 and up to Nr + 3, read at distance 2
  __shared__ Win<C, HR> wqz, wqr, web, wdp;
  const int k0 = blockIdx.x * ATZ, j0 = blockIdx.y * ATR;
  const int k = k0 + (int)threadIdx.x % ATZ, j = j0 + (int)threadIdx.x / ATZ;
  const bool near_edge = j0 < 4 || j0 + ATR > A.Nr - 4;
  load_win<false>(wqz, A.qz, k0, j0, near_edge, A);
  load_win<false>(wqr, A.qr, k0, j0, near_edge, A);
  if (A.axisym) {
    load_win<false>(web, A.eb, k0, j0, near_edge, A);
    load_win<true>(wdp, A.drpb, k0, j0, near_edge, A);
  }
  __syncthreads();
  if (k >= A.Nz || j >= A.Nr) return;
  const size_t o = (size_t)j * A.P + k;
  const bool ax = A.axisym != 0;
  C pb = A.psib[o] + psi_pad_adj(k, j, k0, j0, wqz, wqr, web, wdp, ax);
  const int ga = -1 - j;
  if (ga >= -4) pb += psi_pad_adj(k, ga, k0, j0, wqz, wqr, web, wdp, ax);
  const int gw = 2 * A.Nr - 1 - j;
  if (gw <= A.Nr + 3) pb += psi_pad_adj(k, gw, k0, j0, wqz, wqr, web, wdp, ax);
  const C rho = A.inter[I_RHO * A.plane + o];
  const C rb = A.rhob[o] + pb * exp(-rho * A.inv_rho0);
  const C jzb = A.jzb[o], jrb = A.jrb[o];
#pragma unroll
  for (int q = 0; q < 9; ++q)
    A.lam_out[q * A.plane + o] =
        (C(1) - A.omega) * A.mu[q * A.plane + o] + rb + C(acz(q)) * jzb + C(acr(q)) * jrb;
}

// ---- the differentiable initial drop and its adjoint
struct DropMap {
  int Nz, Nr, l0, namp;
  double zc, R, w, rho_l, rho_v;
  double amp[32];
};

__device__ double legendre_d(int l, double x) {
  double p0 = 1.0, p1 = x;
  if (l == 0) return p0;
  for (int m = 1; m < l; ++m) {
    const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

__global__ void drop_kernel(DropMap M, double* rho) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M.Nz * M.Nr) return;
  const int j = n / M.Nz, k = n - j * M.Nz;
  const double dz = k - M.zc, r = j + 0.5, d = sqrt(dz * dz + r * r), ct = dz / d;
  double s = 0.0;
  for (int m = 0; m < M.namp; ++m) s += M.amp[m] * legendre_d(M.l0 + m, ct);
  const double Rs = M.R * (1.0 + s);
  rho[n] = M.rho_v + 0.5 * (M.rho_l - M.rho_v) * (1.0 - tanh((d - Rs) / M.w));
}

constexpr int RED_NT = 256;
// per-block sums of sum_x rho_bar(x) d rho(x) / d a_m, rho_bar = sum_i W_i lambda^0_i
template <class C>
__global__ void __launch_bounds__(RED_NT) drop_adj_kernel(DropMap M, const C* lam, size_t plane,
                                                          int P, double* partials) {
  __shared__ double red[RED_NT];
  double acc[32];
  for (int m = 0; m < M.namp; ++m) acc[m] = 0.0;
  for (int n = blockIdx.x * RED_NT + threadIdx.x; n < M.Nz * M.Nr; n += gridDim.x * RED_NT) {
    const int j = n / M.Nz, k = n - j * M.Nz;
    const size_t o = (size_t)j * P + k;
    double rb = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) rb += aw(q) * double(lam[q * plane + o]);
    const double dz = k - M.zc, r = j + 0.5, d = sqrt(dz * dz + r * r), ct = dz / d;
    double s = 0.0;
    for (int m = 0; m < M.namp; ++m) s += M.amp[m] * legendre_d(M.l0 + m, ct);
    const double X = (d - M.R * (1.0 + s)) / M.w, sh = 1.0 / cosh(X);
    const double dr_dRs = 0.5 * (M.rho_l - M.rho_v) * sh * sh / M.w;
    for (int m = 0; m < M.namp; ++m) acc[m] += rb * dr_dRs * M.R * legendre_d(M.l0 + m, ct);
  }
  for (int m = 0; m < M.namp; ++m) {
    red[threadIdx.x] = acc[m];
    __syncthreads();
    for (int s = RED_NT / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x * 32 + m] = red[0];
    __syncthreads();
  }
}

// per-block sums of two per-site FP64 arrays ([Nr][P]) -> partials[b * 2 + {0, 1}]
__global__ void __launch_bounds__(RED_NT) sum2_kernel(const double* a, const double* b, int Nz, int Nr,
                                                      int P, double* partials) {
  __shared__ double ra[RED_NT], rb[RED_NT];
  double sa = 0.0, sb = 0.0;
  for (int n = blockIdx.x * RED_NT + threadIdx.x; n < Nz * Nr; n += gridDim.x * RED_NT) {
    const int j = n / Nz, k = n - j * Nz;
    sa += a[(size_t)j * P + k];
    sb += b[(size_t)j * P + k];
  }
  ra[threadIdx.x] = sa;
  rb[threadIdx.x] = sb;
  __syncthreads();
  for (int s = RED_NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      ra[threadIdx.x] += ra[threadIdx.x + s];
      rb[threadIdx.x] += rb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2] = ra[0];
    partials[blockIdx.x * 2 + 1] = rb[0];
  }
}

// lambda^T = dJ/df_i(x) = dJ/drho(x) for every i
template <class C>
__global__ void seed_kernel(int kind, int Nz, int Nr, int P, size_t plane, double zc, double objR,
                            double rho_l, double rho_v, int kstar, double a2_or_J, C* lam) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= Nz * Nr) return;
  const int j = n / Nz, k = n - j * Nz;
  const double pi = 3.14159265358979323846, r = j + 0.5, dz = k - zc;
  double s;
  if (kind == AMLBM_OBJ_A2SQ)
    s = 2.0 * a2_or_J * 5.0 / (4.0 * pi * pow(objR, 5.0)) * 2.0 * pi * r * (dz * dz - 0.5 * r * r) /
        (rho_l - rho_v);
  else
    s = k == kstar ? r / ((rho_l - rho_v) * a2_or_J) : 0.0;
#pragma unroll
  for (int q = 0; q < 9; ++q) lam[q * plane + (size_t)j * P + k] = C(s);
}

// J of the neck objective from the read-back density (one thread)
template <class C>
__global__ void neck_kernel(const C* rho, int Nz, int Nr, int kstar, double rho_l, double rho_v, double* J) {
  double s = 0.0;
  for (int j = 0; j < Nr; ++j) s += (j + 0.5) * (double(rho[(size_t)j * Nz + kstar]) - rho_v) / (rho_l - rho_v);
  *J = sqrt(2.0 * s);
}

}  // namespace
}  // namespace amlbm

// ------------------------------------------------------------------ driver --
using amlbm::InstDesc;

namespace {

struct AdjLayout {
  size_t total = 0;
  size_t ckpt = 0, seg = 0, lam = 0, inter = 0, mu = 0, arr = 0, drp = 0, acc = 0, rho0 = 0,
         red = 0, descs = 0, tiles = 0;
  int nck = 0, nseg = 0, ntiles = 0, nred = 0;
  int nbuf = 1;            // segment buffers: two when there are several segments
  size_t state_elems = 0;  // 10 planes (f and psi)
};

constexpr int kAdjArrays = 19;

size_t al(size_t x) { return (x + 255) / 256 * 256; }

AdjLayout adj_layout(const amlbm::CtxInfo& ci, const amlbm_adjoint_problem& p) {
  AdjLayout L;
  const size_t cb = ci.storage == AMLBM_STORE_F64 ? 8 : 4;
  const size_t plane = (size_t)ci.host.P * ci.Nr;
  L.nck = (p.T + p.ckpt_every - 1) / p.ckpt_every;
  L.nseg = std::min(p.ckpt_every, p.T);
  L.nbuf = L.nck > 1 ? 2 : 1;
  L.state_elems = 10 * plane;
  L.ntiles = ((ci.Nz + 31) / 32) * ((ci.Nr + 7) / 8);
  L.nred = std::min(1024, (ci.Nz * ci.Nr + 255) / 256);
  size_t o = 0;
  auto take = [&](size_t b) { const size_t a = o; o = al(o + b); return a; };
  L.ckpt = take((size_t)L.nck * L.state_elems * cb);
  // per segment buffer: the segment's states and their intermediates
  L.seg = take((size_t)L.nbuf * (L.nseg + 1) * L.state_elems * cb);
  L.lam = take(2 * 9 * plane * cb);
  L.inter = take((size_t)L.nbuf * L.nseg * amlbm::I_COUNT * plane * cb);
  L.mu = take(9 * plane * cb);
  L.arr = take((size_t)kAdjArrays * plane * cb);
  L.drp = take((size_t)(ci.Nr + 4) * ci.host.P * cb);
  L.acc = take(2 * plane * sizeof(double));
  L.rho0 = take((size_t)ci.Nz * ci.Nr * sizeof(double));
  const int nblk = amlbm::diag_blocks(ci.Nz, ci.Nr);
  L.red = take((size_t)(std::max(L.nred * 34, 8 * nblk + ci.Nz + 16) + 64) * sizeof(double));
  L.descs = take((size_t)L.nbuf * L.nseg * sizeof(InstDesc));
  L.tiles = take((size_t)L.ntiles * sizeof(int));
  L.total = o;
  return L;
}

int check_problem(const amlbm::CtxInfo& ci, const amlbm_adjoint_problem* p) {
  using amlbm::set_error;
  if (!p) return set_error(AMLBM_EINVAL, "NULL problem");
  if (ci.storage != AMLBM_STORE_F64 && ci.storage != AMLBM_STORE_F32)
    return set_error(AMLBM_EINVAL, "the adjoint needs FP64 or FP32 storage");
  if (ci.host.shift != 0) return set_error(AMLBM_EINVAL, "the adjoint needs unshifted storage");
  if (ci.host.zbc != AMLBM_Z_PERIODIC || ci.host.rlo != AMLBM_RLO_AXIS || ci.host.wall == AMLBM_WALL_OUTLET)
    return set_error(AMLBM_EINVAL, "the adjoint takes periodic lattices on the axis only");
  if (ci.host.forcing != AMLBM_FORCE_SHIFT)
    return set_error(AMLBM_EINVAL, "the adjoint implements the velocity-shift forcing only");
  if (ci.host.src != AMLBM_SRC_LOCAL)
    return set_error(AMLBM_EINVAL, "the adjoint implements the departure-site source only");
  if (p->T < 1 || p->ckpt_every < 1) return set_error(AMLBM_EINVAL, "need T >= 1, ckpt_every >= 1");
  if (p->n_amps < 0 || p->n_amps > 32 || (p->n_amps > 0 && !p->amps) || p->l0 < 0)
    return set_error(AMLBM_EINVAL, "need 0 <= n_amps <= 32, amps, l0 >= 0");
  if (p->objective != AMLBM_OBJ_A2SQ && p->objective != AMLBM_OBJ_NECK)
    return set_error(AMLBM_EINVAL, "bad objective");
  if (p->objective == AMLBM_OBJ_NECK && (p->kstar < 0 || p->kstar >= ci.Nz))
    return set_error(AMLBM_EINVAL, "kstar outside the lattice");
  if (!(p->w > 0) || !(p->R > 0) || !(p->obj_R > 0) || !(p->rho_l != p->rho_v))
    return set_error(AMLBM_EINVAL, "need w > 0, R > 0, obj_R > 0, rho_l != rho_v");
  return AMLBM_OK;
}

#define ADJ_CK(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      rc = amlbm::set_error(AMLBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
      goto done;                                                                       \
    }                                                                                  \
  } while (0)

template <class C>
int run(amlbm_ctx* ctx, const amlbm_adjoint_problem* p, void* ws, size_t ws_bytes, bool adjoint,
        double* J, double* dG, double* dT, double* dA) {
  using namespace amlbm;
  CtxInfo ci;
  int rc = ctx_info(ctx, &ci);
  if (rc) return rc;
  if ((rc = check_problem(ci, p))) return rc;
  const AdjLayout L = adj_layout(ci, *p);
  const cudaStream_t s = ci.stream;
  const int Nz = ci.Nz, Nr = ci.Nr, P = ci.host.P, N = Nz * Nr;
  const size_t plane = (size_t)P * Nr;
  const int nb = (N + 255) / 256;
  char* base = static_cast<char*>(ws);
  bool owns = false;
  std::vector<double> red;
  double Jv = 0.0;
  if (!base) {
    const cudaError_t e = cudaMalloc(&base, L.total);
    if (e != cudaSuccess) return set_error(AMLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    owns = true;
  } else if (ws_bytes < L.total || reinterpret_cast<uintptr_t>(ws) % 256) {
    return set_error(AMLBM_ENOMEM, "adjoint workspace too small or not 256-byte aligned: need " +
                                       std::to_string(L.total) + " bytes");
  }
  {
    C* ckpt = reinterpret_cast<C*>(base + L.ckpt);
    C* seg = reinterpret_cast<C*>(base + L.seg);
    C* lam[2] = {reinterpret_cast<C*>(base + L.lam), reinterpret_cast<C*>(base + L.lam) + 9 * plane};
    double* rho_init = reinterpret_cast<double*>(base + L.rho0);
    double* redbuf = reinterpret_cast<double*>(base + L.red);
    const size_t SB = L.state_elems * sizeof(C), FB = 9 * plane * sizeof(C), PB = plane * sizeof(C);
    void* fcur;
    void* pcur;
    int pitch;

    DropMap M;
    std::memset(&M, 0, sizeof(M));
    M.Nz = Nz; M.Nr = Nr; M.l0 = p->l0; M.namp = p->n_amps;
    M.zc = p->zc; M.R = p->R; M.w = p->w; M.rho_l = p->rho_l; M.rho_v = p->rho_v;
    for (int m = 0; m < p->n_amps; ++m) M.amp[m] = p->amps[m];

    // forward: initial drop, T steps, states every ckpt_every steps
    drop_kernel<<<nb, 256, 0, s>>>(M, rho_init);
    ADJ_CK(cudaGetLastError());
    ADJ_CK(launch_init(ci.storage, ci.d_desc, 0, Nz, Nr, rho_init, nullptr, nullptr, ci.parity, s));
    for (int n = 0; n < p->T; ++n) {
      if (adjoint && n % p->ckpt_every == 0) {
        amlbm_device_state(ctx, &fcur, &pcur, &pitch);
        C* dst = ckpt + (size_t)(n / p->ckpt_every) * L.state_elems;
        ADJ_CK(cudaMemcpyAsync(dst, fcur, FB, cudaMemcpyDeviceToDevice, s));
        ADJ_CK(cudaMemcpyAsync(dst + 9 * plane, pcur, PB, cudaMemcpyDeviceToDevice, s));
      }
      if ((rc = amlbm_step(ctx, 1))) goto done;
    }
    // objective of the final state
    if ((rc = ctx_readback(ctx))) goto done;
    {
      double a2 = 0.0;
      if (p->objective == AMLBM_OBJ_A2SQ) {
        const int nblk = diag_blocks(Nz, Nr);
        ADJ_CK(launch_diag(ci.storage, ci.d_desc, 0, Nz, Nr, ci.parity ^ (p->T & 1), p->zc, p->obj_R,
                           p->rho_l, p->rho_v, redbuf, nblk, redbuf + 8 * nblk, redbuf + 8 * nblk + Nz, s));
        ADJ_CK(cudaMemcpyAsync(&a2, redbuf + 8 * nblk + Nz + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
        ADJ_CK(cudaStreamSynchronize(s));
        Jv = a2 * a2;
      } else {
        neck_kernel<C><<<1, 1, 0, s>>>(static_cast<const C*>(ci.host.rho_out), Nz, Nr, p->kstar, p->rho_l,
                                       p->rho_v, redbuf);
        ADJ_CK(cudaGetLastError());
        ADJ_CK(cudaMemcpyAsync(&Jv, redbuf, sizeof(double), cudaMemcpyDeviceToHost, s));
        ADJ_CK(cudaStreamSynchronize(s));
      }
      if (J) *J = Jv;
      if (!adjoint) goto done;
      seed_kernel<C><<<nb, 256, 0, s>>>(p->objective, Nz, Nr, P, plane, p->zc, p->obj_R, p->rho_l,
                                        p->rho_v, p->kstar, p->objective == AMLBM_OBJ_A2SQ ? a2 : Jv,
                                        lam[0]);
      ADJ_CK(cudaGetLastError());
    }
    // descriptors of the segment slots (tile 32 x 8): descriptor q of buffer b
    // steps slot q of that buffer into slot q + 1
    {
      std::vector<InstDesc> d((size_t)L.nbuf * L.nseg, ci.host);
      for (int b = 0; b < L.nbuf; ++b)
        for (int q = 0; q < L.nseg; ++q) {
          InstDesc& x = d[(size_t)b * L.nseg + q];
          x.tiles_z = (Nz + 31) / 32;
          x.tiles_r = (Nr + 7) / 8;
          x.tile_base = 0;
          C* sb = seg + (size_t)b * (L.nseg + 1) * L.state_elems;
          for (int h = 0; h < 2; ++h) {
            x.f[h] = sb + (size_t)(q + h) * L.state_elems;
            x.psi[h] = sb + (size_t)(q + h) * L.state_elems + 9 * plane;
          }
        }
      std::vector<int> tiles(L.ntiles, 0);
      ADJ_CK(cudaMemcpyAsync(base + L.descs, d.data(), d.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, s));
      ADJ_CK(cudaMemcpyAsync(base + L.tiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      ADJ_CK(cudaMemsetAsync(base + L.acc, 0, 2 * plane * sizeof(double), s));
      ADJ_CK(cudaStreamSynchronize(s));  // host vectors above go out of scope
    }
    {
      Adj<C> A;
      A.Nz = Nz; A.Nr = Nr; A.P = P; A.wall = ci.host.wall; A.axisym = ci.host.axisym;
      A.plane = plane;
      A.tau = C(ci.host.tau); A.omega = C(1) / A.tau; A.G = C(ci.host.G); A.rho0 = C(ci.host.rho0);
      A.gz = C(ci.host.gz);
      A.inv_rho0 = C(1.0 / ci.host.rho0);
      A.mu = reinterpret_cast<C*>(base + L.mu);
      C* arr = reinterpret_cast<C*>(base + L.arr);
      C** fields[kAdjArrays] = {&A.rhob, &A.uzb, &A.urb, &A.vzb, &A.vrb, &A.g1b, &A.g2b, &A.g3b, &A.jzb,
                                &A.jrb, &A.Fzb, &A.Frb, &A.psib, &A.qz, &A.qr, &A.dzrb, &A.drrb, &A.drdb,
                                &A.eb};
      for (int q = 0; q < kAdjArrays; ++q) *fields[q] = arr + (size_t)q * plane;
      A.drpb = reinterpret_cast<C*>(base + L.drp);
      A.accG = reinterpret_cast<double*>(base + L.acc);
      A.accT = A.accG + plane;
      const InstDesc* d_seg = reinterpret_cast<const InstDesc*>(base + L.descs);
      const int* d_tiles = reinterpret_cast<const int*>(base + L.tiles);
      const dim3 tgrid((Nz + ATZ - 1) / ATZ, (Nr + ATR - 1) / ATR);
      const dim3 dgrid((Nz + ATZ - 1) / ATZ, (Nr + 4 + ATR - 1) / ATR);  // padded rows -2 .. Nr + 1
      C* inter_seg = reinterpret_cast<C*>(base + L.inter);
      const size_t iseg = (size_t)I_COUNT * plane;
      // Segment buffer b: states, intermediates and step descriptors.
      auto seg_of = [&](int b) { return seg + (size_t)b * (L.nseg + 1) * L.state_elems; };
      auto inter_of = [&](int b) { return inter_seg + (size_t)b * L.nseg * iseg; };
      // The recompute of a segment of `len` steps into buffer b (each step writes
      // the next state and the intermediates of the state it starts from).
      auto recompute = [&](int len, int b, cudaStream_t st) -> cudaError_t {
        for (int q = 0; q < len; ++q) {
          const cudaError_t e = launch_step_inter(ci.storage, 32, 8, d_seg + (size_t)b * L.nseg + q, d_tiles,
                                                  L.ntiles, inter_of(b) + q * iseg, plane, st);
          if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
      };
      // The transposed steps of a segment in buffer b, from the last to the first,
      // starting with lambda in lam[c0].
      auto backward = [&](int len, int b, int c0, cudaStream_t st) -> cudaError_t {
        Adj<C> B = A;
        int c = c0;
        for (int q = len - 1; q >= 0; --q) {
          B.inter = inter_of(b) + q * iseg;
          B.f = seg_of(b) + (size_t)q * L.state_elems;
          B.lam_in = lam[c];
          B.lam_out = lam[c ^ 1];
          adj_post<C><<<tgrid, ANT, 0, st>>>(B);
          adj_vel<C><<<tgrid, ANT, 0, st>>>(B);
          adj_deriv<C><<<dgrid, ANT, 0, st>>>(B);
          adj_final<C><<<tgrid, ANT, 0, st>>>(B);
          c ^= 1;
        }
        return cudaGetLastError();
      };
      // Segments run from the last to the first.  The recompute of segment m - 1
      // (on stream rs, into the other buffer) does not depend on the backward
      // sweep of segment m (on s), so the two overlap: each is a few hundred CTAs
      // and leaves most of the GPU idle.  Events order each recompute after the
      // backward sweep that last read its buffer, and each backward sweep after
      // its recompute.  Full segments issue the same launches every time, so after
      // one direct run each part is replayed from a captured CUDA graph (keyed by
      // buffer, and by the starting lambda buffer for the backward part).  Any
      // failure of the graph machinery falls back to direct launches.
      cudaStream_t rs = nullptr, gs = nullptr;
      cudaEvent_t ev0 = nullptr, evR[2] = {nullptr, nullptr}, evB[2] = {nullptr, nullptr};
      cudaGraphExec_t gR[2] = {nullptr, nullptr}, gB[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
      bool usedB[2] = {false, false};
      bool streams_ok = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking) == cudaSuccess &&
                        cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming) == cudaSuccess;
      for (int b = 0; b < 2 && streams_ok; ++b)
        streams_ok = cudaEventCreateWithFlags(&evR[b], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&evB[b], cudaEventDisableTiming) == cudaSuccess;
      bool use_graph = streams_ok && cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) == cudaSuccess;
      bool r_direct = false, b_direct = false;  // a full segment has run directly
      // capture `fn` (which launches on its stream argument) into *gx
      auto capture = [&](cudaGraphExec_t* gx, auto fn) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal);
        const cudaError_t e1 = e == cudaSuccess ? fn(gs) : e;
        if (e == cudaSuccess) e = cudaStreamEndCapture(gs, &g);
        if (e == cudaSuccess && e1 == cudaSuccess) e = cudaGraphInstantiate(gx, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || e1 != cudaSuccess) {
          use_graph = false;
          *gx = nullptr;
          cudaGetLastError();  // the direct path reports real errors
        }
      };
      cudaStream_t rstream = streams_ok ? rs : s;  // without a second stream, no overlap
#define SEG_CK(call)                                                                          \
  {                                                                                           \
    const cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                                  \
      rc = amlbm::set_error(AMLBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
      break;                                                                                  \
    }                                                                                         \
  }
      // issue the checkpoint copy and the recompute of segment m into buffer b on rstream
      auto issue_recompute = [&](int m, int b) -> cudaError_t {
        const int n0 = m * p->ckpt_every, len = std::min(p->T, n0 + p->ckpt_every) - n0;
        if (streams_ok && usedB[b]) {  // the backward sweep that last read buffer b
          const cudaError_t e = cudaStreamWaitEvent(rstream, evB[b], 0);
          if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaMemcpyAsync(seg_of(b), ckpt + (size_t)m * L.state_elems, SB,
                                        cudaMemcpyDeviceToDevice, rstream);
        if (e != cudaSuccess) return e;
        const bool full = len == p->ckpt_every;
        if (use_graph && r_direct && full) {
          if (!gR[b]) capture(&gR[b], [&](cudaStream_t st) { return recompute(len, b, st); });
          if (use_graph) e = cudaGraphLaunch(gR[b], rstream);
          else e = recompute(len, b, rstream);
        } else {
          e = recompute(len, b, rstream);
          if (full) r_direct = true;
        }
        if (e == cudaSuccess && streams_ok) e = cudaEventRecord(evR[b], rstream);
        return e;
      };
      int cur = 0;
      do {
        if (streams_ok) {  // the recompute stream starts after the forward run and the seed
          SEG_CK(cudaEventRecord(ev0, s));
          SEG_CK(cudaStreamWaitEvent(rs, ev0, 0));
        }
        SEG_CK(issue_recompute(L.nck - 1, (L.nck - 1) % L.nbuf));
        for (int m = L.nck - 1; m >= 0 && rc == AMLBM_OK; --m) {
          const int b = m % L.nbuf;
          const int n0 = m * p->ckpt_every, len = std::min(p->T, n0 + p->ckpt_every) - n0;
          // the next segment's recompute goes ahead on the other buffer; with one
          // stream it would have to wait for this backward sweep, so it is issued after it
          if (m >= 1 && streams_ok) SEG_CK(issue_recompute(m - 1, (m - 1) % L.nbuf));
          if (streams_ok) SEG_CK(cudaStreamWaitEvent(s, evR[b], 0));
          const bool full = len == p->ckpt_every;
          if (use_graph && b_direct && full) {
            if (!gB[b][cur]) capture(&gB[b][cur], [&](cudaStream_t st) { return backward(len, b, cur, st); });
            if (use_graph) SEG_CK(cudaGraphLaunch(gB[b][cur], s))
            else SEG_CK(backward(len, b, cur, s))
          } else {
            SEG_CK(backward(len, b, cur, s));
            if (full) b_direct = true;
          }
          if (streams_ok) {
            SEG_CK(cudaEventRecord(evB[b], s));
            usedB[b] = true;
          }
          if (m >= 1 && !streams_ok) SEG_CK(issue_recompute(m - 1, (m - 1) % L.nbuf));
          if (len & 1) cur ^= 1;
        }
      } while (false);
      // graphs run on s and rs: let them finish before their executables go
      if (rs) cudaStreamSynchronize(rs);
      if (gs) cudaStreamSynchronize(gs);
      cudaStreamSynchronize(s);
      for (auto& g : gR)
        if (g) cudaGraphExecDestroy(g);
      for (auto& row : gB)
        for (auto& g : row)
          if (g) cudaGraphExecDestroy(g);
      for (auto* ev : {ev0, evR[0], evR[1], evB[0], evB[1]})
        if (ev) cudaEventDestroy(ev);
      if (rs) cudaStreamDestroy(rs);
      if (gs) cudaStreamDestroy(gs);
#undef SEG_CK
      if (rc) goto done;
      // parameter gradients (FP64, fixed order)
      sum2_kernel<<<L.nred, RED_NT, 0, s>>>(A.accG, A.accT, Nz, Nr, P, redbuf);
      ADJ_CK(cudaGetLastError());
      if (p->n_amps > 0) {
        drop_adj_kernel<C><<<L.nred, RED_NT, 0, s>>>(M, lam[cur], plane, P, redbuf + 2 * L.nred);
        ADJ_CK(cudaGetLastError());
      }
      red.resize((size_t)L.nred * 34);
      ADJ_CK(cudaMemcpyAsync(red.data(), redbuf, red.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      ADJ_CK(cudaStreamSynchronize(s));
      double g = 0.0, t = 0.0;
      for (int b = 0; b < L.nred; ++b) { g += red[2 * b]; t += red[2 * b + 1]; }
      if (dG) *dG = g;
      if (dT) *dT = t;
      for (int m = 0; m < p->n_amps; ++m) {
        double a = 0.0;
        for (int b = 0; b < L.nred; ++b) a += red[2 * L.nred + (size_t)b * 32 + m];
        if (dA) dA[m] = a;
      }
    }
  }
done:
  if (owns) {
    cudaStreamSynchronize(s);
    cudaFree(base);
  }
  return rc;
}

}  // namespace

extern "C" {

size_t amlbm_adjoint_workspace_bytes(amlbm_ctx* ctx, const amlbm_adjoint_problem* p) {
  amlbm::CtxInfo ci;
  if (!ctx || amlbm::ctx_info(ctx, &ci) || check_problem(ci, p)) return 0;
  return adj_layout(ci, *p).total;
}

int amlbm_adjoint(amlbm_ctx* ctx, const amlbm_adjoint_problem* p, void* workspace, size_t bytes,
                  double* J, double* dJ_dG, double* dJ_dtau, double* dJ_damps) {
  amlbm::CtxInfo ci;
  if (!ctx) return amlbm::set_error(AMLBM_EINVAL, "NULL context");
  const int rc = amlbm::ctx_info(ctx, &ci);
  if (rc) return rc;
  if (ci.storage == AMLBM_STORE_F64)
    return run<double>(ctx, p, workspace, bytes, true, J, dJ_dG, dJ_dtau, dJ_damps);
  return run<float>(ctx, p, workspace, bytes, true, J, dJ_dG, dJ_dtau, dJ_damps);
}

int amlbm_objective(amlbm_ctx* ctx, const amlbm_adjoint_problem* p, double* J) {
  amlbm::CtxInfo ci;
  if (!ctx) return amlbm::set_error(AMLBM_EINVAL, "NULL context");
  const int rc = amlbm::ctx_info(ctx, &ci);
  if (rc) return rc;
  if (ci.storage == AMLBM_STORE_F64) return run<double>(ctx, p, nullptr, 0, false, J, nullptr, nullptr, nullptr);
  return run<float>(ctx, p, nullptr, 0, false, J, nullptr, nullptr, nullptr);
}

}  // extern "C"
