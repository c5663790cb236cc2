// Fused axisymmetric Shan-Chen LBM step with two adjacent z-sites per thread
// (the "pair" schedule) for sm_103a (arXiv:1310.1871, Sec. II).
//
// The per-site chain is the fused schedule's, stage for stage:
//   psi, tile + (8 in z, 7 in r), from the previous step's psi
//   -> isotropic d_r psi and the 1D d_r psi (Sec. II.D), tile + (6, 5)
//   -> moments, Shan-Chen force (Eq. scforce), axisymmetric force
//      (Eq. scAxisExtra), u and u^eq (Eqs. uhydro, ueq), tile + (4, 3); the BGK
//      collision (Eq. lbm2d) on tile + (2, 1)
//   -> velocity gradients (1D 4th-order differences, Sec. II.D) and the sources
//      S, H_z, H_r, h_i (Eq. condition_h, App. A) on tile + (2, 1)
//   -> pull streaming with the axis / wall / periodic maps of Sec. II.E, psi of
//      the new state, store.
// Every task of every stage is a pair of adjacent sites (z = 2m, 2m + 1 of the
// region): populations, psi and the stored velocity move as 2-element vectors
// between HBM and registers, and each stencil reads its taps as 2-element
// vectors from shared memory into a small register window that both sites of
// the pair share.  The arithmetic is the same functions on the same values as
// the fused schedule, so the two give identical bits.
//
// Lattices this schedule takes: z periodic with Nz even, the axis below row 0,
// an outer wall that reflects (free-slip) or bounces back (no-slip), the source
// at the departure site, either forcing.  Pairs never straddle the periodic
// seam because Nz and every tile origin are even.
//
// The file also holds the schedule's read-back (rho and u of the current state,
// the input of the diagnostics): stages 0 and 1 as above, then the force,
// moments and u at the tile's own sites.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <stdint.h>

#include <mutex>
#include <type_traits>

#include "amlbm.h"
#include "amlbm_internal.cuh"
#include "amlbm_physics.cuh"
#include "amlbm_vec2.cuh"

namespace amlbm {
namespace {

// Tile geometry (BZ x BR sites, BZ even).  Halos in (z, r): psi (8, 7),
// d_r psi (6, 5), rho and u (4, 3), collided populations (2, 1); the z halos
// are the fused schedule's rounded up to whole pairs.  Region A holds psi, d_r psi
// and 1D d_r psi until the forces are known, then the nine collided populations.
// Region B holds three planes of the force region: between the two halves of
// stage 2 psi and the force without the body force, then rho, u_z and u_r, each
// written over the value the same thread read from it.
template <class T, int BZ, int BR>
struct PGeo {
  static_assert(BZ % 2 == 0, "pair tiles are an even number of sites wide");
  static constexpr int PZ = BZ + 16, PR = BR + 14;
  static constexpr int DZ = BZ + 12, DR = BR + 10;
  static constexpr int FZ = BZ + 8, FR = BR + 6;
  static constexpr int SZ = BZ + 4, SR = BR + 2;
  static constexpr int nP = PZ * PR, nD = DZ * DR, nF = FZ * FR, nS = SZ * SR;
  static constexpr int nA = (nP + 2 * nD) > 9 * nS ? (nP + 2 * nD) : 9 * nS;
  static constexpr size_t elems = (size_t)nA + 3 * nF;
  static constexpr size_t bytes = sizeof(T) * elems;
};

// Threads per CTA and the resident CTAs per SM the register budget must allow.
// FP32 arithmetic: as many CTAs per SM as the tile's shared memory fits in the
// SM's 228 KB (1 KB reserved per CTA), at most four: four of 256 threads at 64
// registers, three of 256 at 80, and two of 384 at 80 (a tile that fits only
// two keeps 24 warps per SM that way).  FP64: 256 threads, one CTA.
template <class T, int BZ, int BR>
struct Threads {
  static constexpr int fit = (int)(233472 / (PGeo<T, BZ, BR>::bytes + 1024 + 16));
  static constexpr int min_blocks = fit >= 4 ? 4 : (fit >= 1 ? fit : 1);
  static constexpr int value = min_blocks == 2 ? 384 : 256;
};
template <int BZ, int BR>
struct Threads<D1, BZ, BR> {
  static constexpr int value = 256, min_blocks = 1;
};

// Flat walk over the pair tasks of a ROWS x PAIRS region.
template <int NTH, int ROWS, int PAIRS, class F>
__device__ __forceinline__ void for_pairs(F&& body) {
  for (int t = threadIdx.x; t < ROWS * PAIRS; t += NTH) {
    const int lr = t / PAIRS, cp = t - lr * PAIRS;
    body(lr, cp);
  }
}

// Stage 0 of a tile: psi on tile + (8, 7); rows mirrored about the axis and the
// wall.  All of a thread's loads are issued before its first store, so that
// their latencies overlap.
template <class C, class T, int BZ, int BR, int NTH>
__device__ __forceinline__ void stage_psi(T* sPsi, const C* __restrict__ psin, int j0, int k0, int Nz, int Nr,
                                          int P, bool tiny) {
  using G = PGeo<T, BZ, BR>;
  constexpr int PP = G::PZ / 2, TOT = G::PR * PP, NB = (TOT + NTH - 1) / NTH;
  C va[NB], vb[NB];
#pragma unroll
  for (int n = 0; n < NB; ++n) {
    const int t = threadIdx.x + n * NTH;
    if (t < TOT) {
      const int lr = t / PP, cp = t - lr * PP;
      const int jj = reflect_row(j0 - 7 + lr, Nr);
      const int kk = wrap_col(k0 - 8 + 2 * cp, Nz, tiny);
      ld2<C>(psin + jj * P + kk, va[n], vb[n]);
    }
  }
#pragma unroll
  for (int n = 0; n < NB; ++n) {
    const int t = threadIdx.x + n * NTH;
    if (t < TOT) sts2(sPsi + 2 * t, T{va[n]}, T{vb[n]});  // PZ = 2 PP: row-major pairs
  }
}

// Stage 1 of a tile: isotropic d_r psi and 1D d_r psi on tile + (6, 5).
template <class T, int BZ, int BR, int NTH>
__device__ __forceinline__ void stage_dr(const T* sPsi, T* sDr, T* sD1) {
  using G = PGeo<T, BZ, BR>;
  for_pairs<NTH, G::DR, G::DZ / 2>([&](int lr, int cp) {
    // psi rows -2..2 around the pair, columns -2..3 (row 0 is not a tap)
    T w[5 * 6];
    const T* p = sPsi + (lr + 2) * G::PZ + 2 * cp;  // column -2 of the window at row 0
#pragma unroll
    for (int r = 0; r < 5; ++r)
      if (r != 2) load_row<T, 3>(p + (r - 2) * G::PZ, w + 6 * r);
    T dr[2], d1r[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      dr[s] = iso_r(w + 12 + 2 + s, 6);
      d1r[s] = d1(w + 12 + 2 + s, 6);
    }
    sts2(sDr + lr * G::DZ + 2 * cp, dr[0], dr[1]);
    sts2(sD1 + lr * G::DZ + 2 * cp, d1r[0], d1r[1]);
  });
}

// The force without its body-force term (Shan-Chen sums, d_rr psi, d_zr psi) of
// the pair at (lr, cp) of the force region (tile + (4, 3)), row j of the
// lattice; psi of the two sites in ps.
template <class T, int BZ, int BR>
__device__ __forceinline__ void force_pair(const T* sPsi, const T* sDr, const T* sD1, const Par<T>& q, bool ax,
                                           T inv_r, int lr, int cp, T* Fz2, T* Fr2, T* ps) {
  using G = PGeo<T, BZ, BR>;
  // psi rows -1..1, columns -2..3 around the pair
  T wp[3 * 6];
  const T* p = sPsi + (lr + 4) * G::PZ + 2 * cp + 2;
#pragma unroll
  for (int r = 0; r < 3; ++r) load_row<T, 3>(p + (r - 1) * G::PZ, wp + 6 * r);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T psi = wp[6 + 2 + s];
    T sz, sr;
    sc_sums(wp + 6 + 2 + s, 6, sz, sr);
    T dr0 = lit<T>(0.0), Drr = lit<T>(0.0), Dzr = lit<T>(0.0);
    if (ax) {
      // d_r psi rows -2..2 (columns -1..2 on rows -1, 1; -2..3 on rows -2, 2; 0..1
      // on row 0) and 1D d_r psi row 0 (columns -2..3)
      const T* pd = sDr + (lr + 2) * G::DZ + 2 * cp + 2 + s;
      T w[5 * 5];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const bool tap = (r == 2 && c == 2) || ((r == 1 || r == 3) && c >= 1 && c <= 3) ||
                           ((r == 0 || r == 4) && (c == 0 || c == 2 || c == 4));
          if (tap) w[5 * r + c] = pd[(r - 2) * G::DZ + (c - 2)];
        }
      dr0 = w[12];
      Drr = iso_r(w + 12, 5);
      const T* pe = sD1 + (lr + 2) * G::DZ + 2 * cp + 2 + s;
      T e[5];
#pragma unroll
      for (int m = -2; m <= 2; ++m) e[m + 2] = m ? pe[m] : lit<T>(0.0);
      Dzr = d1(e + 2, 1);
    }
    forces_partial(q, psi, sz, sr, ax, dr0, Drr, Dzr, inv_r, Fz2[s], Fr2[s]);
  }
  ps[0] = wp[8];
  ps[1] = wp[9];
}

template <class S, class T, int BZ, int BR>
__device__ __forceinline__ void pair_tile(const InstDesc* __restrict__ descs, const int* __restrict__ tile_inst,
                                          int tile, int parity, uint32_t step) {
  using C = typename Store<S>::C;
  using G = PGeo<T, BZ, BR>;
  constexpr int NTH = Threads<T, BZ, BR>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sPsi = reinterpret_cast<T*>(smem_raw);  // region A, stages 0-2a
  T* sDr = sPsi + G::nP;
  T* sD1 = sDr + G::nD;
  T* sFs = sPsi;  // region A, stages 2b-4
  T* sRho = sPsi + G::nA;  // region B
  T* sUz = sRho + G::nF;
  T* sUr = sUz + G::nF;
  T* sFz = sUz;  // stage 2a writes, stage 2b reads and overwrites (same task, same thread)
  T* sFr = sUr;
  T* sPs = sRho;

  const int inst = tile_inst[tile];
  const InstDesc& D = descs[inst];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P;
  const int l = tile - D.tile_base;
  const int k0 = (l % D.tiles_z) * BZ, j0 = (l / D.tiles_z) * BR;
  const int plane = P * Nr;  // < 2^31 / 9 (the batch checks it)
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const Par<T> q = par_of<T>(D);
  const C rho0c = kc(D, K_RHO0, C()), rrefc = kc(D, K_RREF, C()), inv_rho0c = kc(D, K_INVRHO0, C());
  const C r0c = kc(D, K_R0, C());
  const bool guo = D.forcing == AMLBM_FORCE_GUO;
  const bool tiny = Nz < BZ + 16;  // region columns may wrap more than once

  // Stage 0: psi on tile + (8, 7)
  stage_psi<C, T, BZ, BR, NTH>(sPsi, psin, j0, k0, Nz, Nr, P, tiny);
  __syncthreads();

  // Stage 1: isotropic d_r psi and 1D d_r psi on tile + (6, 5)
  if (ax) {
    stage_dr<T, BZ, BR, NTH>(sPsi, sDr, sD1);
    __syncthreads();
  }

  // Stage 2a (tile + (4, 3)): Shan-Chen sums, d_rr psi, d_zr psi and the force
  // without its body-force term; psi copied beside it (region A is reused next).
  for_pairs<NTH, G::FR, G::FZ / 2>([&](int lr, int cp) {
    const int j = j0 - 3 + lr;
    if (j < 0 || j >= Nr) return;
    T Fz2[2], Fr2[2], ps[2];
    force_pair<T, BZ, BR>(sPsi, sDr, sD1, q, ax, inv_r_of(T(), j, r0c), lr, cp, Fz2, Fr2, ps);
    const int fi = lr * G::FZ + 2 * cp;
    sts2(sFz + fi, Fz2[0], Fz2[1]);
    sts2(sFr + fi, Fr2[0], Fr2[1]);
    sts2(sPs + fi, ps[0], ps[1]);
  });
  __syncthreads();

  // Stage 2b (tile + (4, 3)): populations from global memory, moments, the body
  // force, u (Eq. uhydro); on tile + (2, 1) also u^eq (Eq. ueq) and the BGK
  // collision of all nine populations into region A.
  for_pairs<NTH, G::FR, G::FZ / 2>([&](int lr, int cp) {
    const int j = j0 - 3 + lr;
    if (j < 0 || j >= Nr) return;
    const int so = j * P + wrap_col(k0 - 4 + 2 * cp, Nz, tiny);
    S qa[9], qb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) ld2<S>(fin + i * plane + so, qa[i], qb[i]);
    C va = C(0), vb = C(0), wa = C(0), wb = C(0);
    if (shift == 3) {
      ld2<C>(psin + plane + so, va, vb);
      ld2<C>(psin + 2 * plane + so, wa, wb);
    }
    const int fi = lr * G::FZ + 2 * cp;
    T ps[2], fz[2], fr[2];
    lds2(sPs + fi, ps[0], ps[1]);
    lds2(sFz + fi, fz[0], fz[1]);
    lds2(sFr + fi, fr[0], fr[1]);
    const bool coll = lr >= 2 && lr < G::FR - 2 && cp >= 1 && cp < G::FZ / 2 - 1;
    T rho2[2], uz2[2], ur2[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      T f[9];
      decode_values<S>(shift, s ? qb : qa, ps[s].v, s ? vb : va, s ? wb : wa, inv_rho0c, rho0c, rrefc, f);
      const T rho = moment0(f), jz = moment_z(f), jr = moment_r(f);
      const T Fz = fma(rho, q.gz, fz[s]), Fr = fr[s];
      const T inv_rho = rcp(rho);
      const T uz = fma(Fz, lit<T>(0.5), jz) * inv_rho, ur = fma(Fr, lit<T>(0.5), jr) * inv_rho;
      rho2[s] = rho;
      uz2[s] = uz;
      ur2[s] = ur;
      if (coll) {
        T* out = sFs + (lr - 2) * G::SZ + (2 * cp - 2) + s;
        T fe[9];
        if (guo) {
          equilibrium(rho, uz, ur, fe);
          T sg[9];
          guo_force(uz, ur, Fz, Fr, sg);
          const T gk = splat<T>(kc(D, K_GUO, C()));
#pragma unroll
          for (int i = 0; i < 9; ++i) out[i * G::nS] = fma(sg[i], gk, fma(fe[i] - f[i], q.omega, f[i]));
        } else {
          const T vz = fma(Fz, q.tau, jz) * inv_rho, vr = fma(Fr, q.tau, jr) * inv_rho;
          equilibrium(rho, vz, vr, fe);
#pragma unroll
          for (int i = 0; i < 9; ++i) out[i * G::nS] = fma(fe[i] - f[i], q.omega, f[i]);
        }
      }
    }
    sts2(sRho + fi, rho2[0], rho2[1]);
    sts2(sUz + fi, uz2[0], uz2[1]);
    sts2(sUr + fi, ur2[0], ur2[1]);
    // Ghost rows of u (depth 2) for the sources' gradients, written by the thread
    // that computed the row they mirror: rows -1, -2 mirror rows 0, 1 about the
    // axis (u_z even, u_r odd); rows Nr, Nr + 1 mirror rows Nr - 1, Nr - 2 about
    // the outer wall (u_r odd, u_z even for free-slip and odd for no-slip).
    if (ax) {
      if (j <= 1) {
        const int lg = (-1 - j) - (j0 - 3);
        if (lg >= 0) {
          sts2(sUz + lg * G::FZ + 2 * cp, uz2[0], uz2[1]);
          sts2(sUr + lg * G::FZ + 2 * cp, -ur2[0], -ur2[1]);
        }
      }
      if (j >= Nr - 2) {
        const int lg = (2 * Nr - 1 - j) - (j0 - 3);
        if (lg < G::FR) {
          const bool flip_z = D.wall == AMLBM_WALL_NOSLIP;
          sts2(sUz + lg * G::FZ + 2 * cp, flip_z ? -uz2[0] : uz2[0], flip_z ? -uz2[1] : uz2[1]);
          sts2(sUr + lg * G::FZ + 2 * cp, -ur2[0], -ur2[1]);
        }
      }
    }
  });
  __syncthreads();

  // Stage 3 (tile + (2, 1)): velocity gradients and the sources of App. A,
  // added to the collided populations.
  if (ax) {
    for_pairs<NTH, G::SR, G::SZ / 2>([&](int lr, int cp) {
      const int j = j0 - 1 + lr;
      if (j < 0 || j >= Nr) return;
      const int fi = (lr + 2) * G::FZ + 2 * cp + 2;  // u at the pair's first site
      // u_z rows -2..2 and u_r rows -2..2 at the pair; u_r row 0 columns -2..3
      T wz[5 * 2], wr[5 * 2], wr0[6];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        lds2(sUz + fi + (r - 2) * G::FZ, wz[2 * r], wz[2 * r + 1]);
        if (r != 2) lds2(sUr + fi + (r - 2) * G::FZ, wr[2 * r], wr[2 * r + 1]);
      }
      load_row<T, 3>(sUr + fi - 2, wr0);
      wr[4] = wr0[2];
      wr[5] = wr0[3];
      T rr[2];
      lds2(sRho + fi, rr[0], rr[1]);
      const T inv_r = inv_r_of(T(), j, r0c);
      T* o = sFs + lr * G::SZ + 2 * cp;
      T h[2][9];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T druz = d1(wz + 4 + s, 2);
        const T dzur = d1(wr0 + 2 + s, 1);
        const T drur = d1(wr + 4 + s, 2);
        T S_, Hz, Hr;
        site_sources(q, rr[s], wz[4 + s], wr[4 + s], druz, dzur, drur, inv_r, S_, Hz, Hr);
        sources(S_, Hz, Hr, h[s]);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) {  // both sites' populations of direction i as one pair
        T a, b;
        lds2(o + i * G::nS, a, b);
        sts2(o + i * G::nS, a + h[0][i], b + h[1][i]);
      }
    });
    __syncthreads();
  }

  // Stage 4 (tile): pull streaming.  Away from rows 0 and Nr - 1 every
  // population comes from x - c_i in the same direction; those two rows apply
  // the axis and wall maps.  Then psi of the new state and the store.
  S* __restrict__ fout = static_cast<S*>(D.f[parity ^ 1]);
  C* __restrict__ psout = static_cast<C*>(D.psi[parity ^ 1]);
  const bool noslip = D.wall == AMLBM_WALL_NOSLIP;
  for_pairs<NTH, BR, BZ / 2>([&](int lr, int cp) {
    const int j = j0 + lr, k = k0 + 2 * cp;
    if (j >= Nr || k >= Nz) return;
    const bool edge = (j == 0) || (j == Nr - 1);
    const T* c0 = sFs + (lr + 1) * G::SZ + 2 * cp + 2;  // the pair's first site
    const int o = j * P + k;
    S qv[2][9];
    C ps[2], vz[2], vr[2];
    T fn2[2][9];
    if (!edge) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const T* src = c0 + i * G::nS - cr_(i) * G::SZ - cz_(i);
        if (cz_(i) == 0) {  // the two sources are an aligned pair
          lds2(src, fn2[0][i], fn2[1][i]);
        } else {
          fn2[0][i] = src[0];
          fn2[1][i] = src[1];
        }
      }
    } else {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          int dl = -cr_(i), dc = -cz_(i), ii = i;
          if (cr_(i) > 0 && j == 0) {  // through the axis: specular reflection
            dl = 0;
            ii = mirror_(i);
          } else if (cr_(i) < 0 && j == Nr - 1) {  // through the outer wall
            dl = 0;
            if (noslip) { dc = 0; ii = opp_(i); }
            else { ii = mirror_(i); }
          }
          fn2[s][i] = c0[ii * G::nS + dl * G::SZ + dc + s];
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T* fn = fn2[s];
      const T rho = moment0(fn);
      ps[s] = psi_of(q, rho).v;
      encode_values<S>(shift, fn, rho, ps[s], inv_rho0c, rho0c, rrefc, D.rounding, (uint32_t)(j * Nz + k + s),
                       step, qv[s], vz[s], vr[s]);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) st2<S>(fout + i * plane + o, qv[0][i], qv[1][i]);
    st2<C>(psout + o, ps[0], ps[1]);
    if (shift == 3) {
      st2<C>(psout + plane + o, vz[0], vz[1]);
      st2<C>(psout + 2 * plane + o, vr[0], vr[1]);
    }
  });
}

// The read-back of the pair schedule: rho, u_z and u_r of the current state on
// every site of a tile, in the compute type, into the instance's [Nr][Nz]
// read-back planes.  Stages 0 and 1 of the step, then the force, moments and
// velocity of stage 2 at the tile's own sites only (nothing downstream needs
// them on the halo): the step's operations on the step's values, so the
// results equal those of the fused schedule's read-back bit for bit.  One CTA
// per tile of the read-back list (which, for a pair batch, is tiled like the step).
template <class T, int BZ, int BR>
struct RGeo {
  using G = PGeo<T, BZ, BR>;
  static constexpr size_t bytes = sizeof(T) * ((size_t)G::nP + 2 * (size_t)G::nD);
};

template <class S, class T, int BZ, int BR>
__global__ void __launch_bounds__(Threads<T, BZ, BR>::value, Threads<T, BZ, BR>::min_blocks) pair_readback(
    const InstDesc* __restrict__ descs, const int* __restrict__ tile_inst, int toff, int parity) {
  using C = typename Store<S>::C;
  using G = PGeo<T, BZ, BR>;
  constexpr int NTH = Threads<T, BZ, BR>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sPsi = reinterpret_cast<T*>(smem_raw);
  T* sDr = sPsi + G::nP;
  T* sD1 = sDr + G::nD;

  const int tile = blockIdx.x + toff;
  const InstDesc& D = descs[tile_inst[tile]];
  const int Nz = D.Nz, Nr = D.Nr, P = D.P;
  const int l = tile - D.rb_tile_base;
  const int k0 = (l % D.rb_tiles_z) * BZ, j0 = (l / D.rb_tiles_z) * BR;
  const int plane = P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  const bool ax = D.axisym != 0;
  const int shift = D.shift;
  const Par<T> q = par_of<T>(D);
  const C rho0c = kc(D, K_RHO0, C()), rrefc = kc(D, K_RREF, C()), inv_rho0c = kc(D, K_INVRHO0, C());
  const C r0c = kc(D, K_R0, C());
  const bool tiny = Nz < BZ + 16;

  stage_psi<C, T, BZ, BR, NTH>(sPsi, psin, j0, k0, Nz, Nr, P, tiny);
  __syncthreads();
  if (ax) {
    stage_dr<T, BZ, BR, NTH>(sPsi, sDr, sD1);
    __syncthreads();
  }
  C* rho_out = static_cast<C*>(D.rho_out);
  C* uz_out = static_cast<C*>(D.uz_out);
  C* ur_out = static_cast<C*>(D.ur_out);
  for_pairs<NTH, BR, BZ / 2>([&](int lr, int cp) {
    const int j = j0 + lr, k = k0 + 2 * cp;
    if (j >= Nr || k >= Nz) return;
    const int so = j * P + k;
    S qa[9], qb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) ld2<S>(fin + i * plane + so, qa[i], qb[i]);
    C va = C(0), vb = C(0), wa = C(0), wb = C(0);
    if (shift == 3) {
      ld2<C>(psin + plane + so, va, vb);
      ld2<C>(psin + 2 * plane + so, wa, wb);
    }
    T fz[2], fr[2], ps[2];
    force_pair<T, BZ, BR>(sPsi, sDr, sD1, q, ax, inv_r_of(T(), j, r0c), lr + 3, cp + 2, fz, fr, ps);
    C rho2[2], uz2[2], ur2[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      T f[9];
      decode_values<S>(shift, s ? qb : qa, ps[s].v, s ? vb : va, s ? wb : wa, inv_rho0c, rho0c, rrefc, f);
      const T rho = moment0(f), jz = moment_z(f), jr = moment_r(f);
      const T Fz = fma(rho, q.gz, fz[s]), Fr = fr[s];
      const T inv_rho = rcp(rho);
      rho2[s] = rho.v;
      uz2[s] = (fma(Fz, lit<T>(0.5), jz) * inv_rho).v;
      ur2[s] = (fma(Fr, lit<T>(0.5), jr) * inv_rho).v;
    }
    const int o = j * Nz + k;  // Nz and k are even: an aligned pair
    st2<C>(rho_out + o, rho2[0], rho2[1]);
    st2<C>(uz_out + o, uz2[0], uz2[1]);
    st2<C>(ur_out + o, ur2[0], ur2[1]);
  });
}

// The timestep as a persistent grid: CTAs take tiles from a counter until none
// is left (ctr as for the fused schedule: this step's tile counter and step
// number at [parity] and [2 + parity], the next step's reset here).
template <class S, class T, int BZ, int BR>
__global__ void __launch_bounds__(Threads<T, BZ, BR>::value, Threads<T, BZ, BR>::min_blocks) pair_persistent(
    const InstDesc* __restrict__ descs, const int* __restrict__ tile_inst, int ntiles, int parity,
    int* __restrict__ ctr) {
  __shared__ int s_tile;
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
    pair_tile<S, T, BZ, BR>(descs, tile_inst, t, parity, step);
    __syncthreads();
  }
}

constexpr int kMaxDev = 64;
struct PairOnce {
  std::once_flag once[kMaxDev];
  cudaError_t err[kMaxDev] = {};
  int grid_cap[kMaxDev] = {};
};

template <class S, int BZ, int BR>
cudaError_t launch_pair_t(const InstDesc* d, const int* ti, int ntiles, int parity, cudaStream_t s, int* ctr) {
  using T = typename Store<S>::T;
  constexpr size_t smem = PGeo<T, BZ, BR>::bytes;
  static PairOnce st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::call_once(st.once[dev], [&] {
    cudaError_t r = cudaFuncSetAttribute(pair_persistent<S, T, BZ, BR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int sms = 0, per_sm = 0;
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (r == cudaSuccess)
      r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_persistent<S, T, BZ, BR>,
                                                        Threads<T, BZ, BR>::value, smem);
    st.grid_cap[dev] = sms * (per_sm > 0 ? per_sm : 1);
    st.err[dev] = r;
  });
  if (st.err[dev] != cudaSuccess) return st.err[dev];
  if (!ctr) return cudaErrorInvalidValue;
  const int grid = ntiles < st.grid_cap[dev] ? ntiles : st.grid_cap[dev];
  pair_persistent<S, T, BZ, BR><<<grid, Threads<T, BZ, BR>::value, smem, s>>>(d, ti, ntiles, parity, ctr);
  return cudaGetLastError();
}

template <class S, int BZ, int BR>
cudaError_t launch_readback_t(const InstDesc* d, const int* ti, int nt, int toff, int parity, cudaStream_t s) {
  using T = typename Store<S>::T;
  constexpr size_t smem = RGeo<T, BZ, BR>::bytes;
  static_assert(smem <= 48 * 1024, "read-back tiles fit the default shared-memory limit");
  pair_readback<S, T, BZ, BR><<<nt, Threads<T, BZ, BR>::value, smem, s>>>(d, ti, toff, parity);
  return cudaGetLastError();
}

struct PairTile { int storage, tz, tr; };
#define AMLBM_PAIR_TILES(ST) {ST, 40, 24}, {ST, 48, 20}, {ST, 64, 24}, {ST, 32, 16}, {ST, 48, 16}, \
                             {ST, 24, 16}, {ST, 64, 16}, {ST, 32, 32}
constexpr PairTile kPairTiles[] = {
    {AMLBM_STORE_F64, 32, 8}, {AMLBM_STORE_F64, 28, 8},
    AMLBM_PAIR_TILES(AMLBM_STORE_F32), AMLBM_PAIR_TILES(AMLBM_STORE_F16), AMLBM_PAIR_TILES(AMLBM_STORE_BF16),
};
#undef AMLBM_PAIR_TILES

// kind 0: the timestep (ctr: its counters); 1: the read-back of nt tiles from
// toff; 2: load the read-back kernel's code (nothing is launched)
template <class S>
cudaError_t pair_dispatch(int kind, int tz, int tr, const InstDesc* d, const int* ti, int nt, int toff, int par,
                          cudaStream_t s, int* ctr) {
  using T = typename Store<S>::T;
  if (kind != 2 && nt <= 0) return cudaSuccess;
#define AMLBM_PT(TZ, TR)                                                             \
  if (tz == TZ && tr == TR) {                                                        \
    if (kind == 0) return launch_pair_t<S, TZ, TR>(d, ti, nt, par, s, ctr);          \
    if (kind == 1) return launch_readback_t<S, TZ, TR>(d, ti, nt, toff, par, s);     \
    cudaFuncAttributes a;                                                            \
    return cudaFuncGetAttributes(&a, pair_readback<S, T, TZ, TR>);                   \
  }
  if constexpr (std::is_same<S, double>::value) {
    AMLBM_PT(32, 8)
    AMLBM_PT(28, 8)
  } else {
    AMLBM_PT(40, 24)
    AMLBM_PT(48, 20)
    AMLBM_PT(64, 24)
    AMLBM_PT(32, 16)
    AMLBM_PT(48, 16)
    AMLBM_PT(24, 16)
    AMLBM_PT(64, 16)
    AMLBM_PT(32, 32)
  }
#undef AMLBM_PT
  return cudaErrorInvalidValue;
}

}  // namespace

bool pair_tile_supported(int storage, int tz, int tr) {
  for (const auto& e : kPairTiles)
    if (e.storage == storage && e.tz == tz && e.tr == tr) return true;
  return false;
}

int pair_tile_list(int storage, int* tz, int* tr, int cap) {
  int n = 0;
  for (const auto& e : kPairTiles)
    if (e.storage == storage) {
      if (n < cap && tz && tr) { tz[n] = e.tz; tr[n] = e.tr; }
      ++n;
    }
  return n;
}

static cudaError_t pair_kind(int kind, int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                             int toff, int parity, cudaStream_t s, int* ctr) {
  switch (storage) {
    case AMLBM_STORE_F64: return pair_dispatch<double>(kind, tz, tr, d, ti, nt, toff, parity, s, ctr);
    case AMLBM_STORE_F32: return pair_dispatch<float>(kind, tz, tr, d, ti, nt, toff, parity, s, ctr);
    case AMLBM_STORE_F16: return pair_dispatch<__half>(kind, tz, tr, d, ti, nt, toff, parity, s, ctr);
    case AMLBM_STORE_BF16: return pair_dispatch<__nv_bfloat16>(kind, tz, tr, d, ti, nt, toff, parity, s, ctr);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_pair(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt, int parity,
                             cudaStream_t s, int* ctr) {
  return pair_kind(0, storage, tz, tr, d, ti, nt, 0, parity, s, ctr);
}

cudaError_t launch_readback_pair(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt, int toff,
                                 int parity, cudaStream_t s) {
  return pair_kind(1, storage, tz, tr, d, ti, nt, toff, parity, s, nullptr);
}

cudaError_t readback_pair_preload(int storage, int tz, int tr) {
  return pair_kind(2, storage, tz, tr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr);
}

}  // namespace amlbm
