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
#include "amlbm_physics.cuh"

namespace amlbm {
namespace {

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
// and discards them when *bad is non-zero).  The inputs are FP64 or FP32 (In);
// FP32 inputs are widened exactly, so they give the state of the same values in FP64.
template <class S, class In>
__global__ void init_all_kernel(const InstDesc* __restrict__ descs, int n_inst,
                                const long long* __restrict__ site_off, long long total,
                                const In* rho_in, const In* uz_in, const In* ur_in,
                                int parity, int* bad) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  // the inputs first (they may be host memory read over the CPU-GPU link): their
  // latency overlaps the search for the instance
  const double rho = rho_in[g];
  const double uz = uz_in ? (double)uz_in[g] : 0.0, ur = ur_in ? (double)ur_in[g] : 0.0;
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
  if (sched == SCHED_PAIR) return pair_tile_supported(storage, tz, tr);
  for (const auto& e : kTiles)
    if (e.storage == storage && e.sched == sched && e.tz == tz && e.tr == tr) return true;
  return false;
}

int tile_list(int storage, int sched, int* tz, int* tr, int cap) {
  if (sched == SCHED_PAIR) return pair_tile_list(storage, tz, tr, cap);
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
  if (sched == SCHED_PAIR) {
    if (toff != 0) return cudaErrorInvalidValue;
    return launch_step_pair(storage, tz, tr, d, ti, nt, parity, s, ctr);
  }
  return dispatch_storage(storage, false, sched, tz, tr, d, ti, nt, toff, parity, s, ctr);
}
cudaError_t launch_macro(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                         int toff, int parity, cudaStream_t s) {
  return dispatch_storage(storage, true, SCHED_FUSED, tz, tr, d, ti, nt, toff, parity, s, nullptr);
}

cudaError_t macro_preload(int storage) {
  cudaFuncAttributes a;
  switch (storage) {  // the read-back tiles of rb_tile()
    case AMLBM_STORE_F64: return cudaFuncGetAttributes(&a, lbm_kernel<double, 32, 8, 1>);
    case AMLBM_STORE_F32: return cudaFuncGetAttributes(&a, lbm_kernel<float, 26, 16, 1>);
    case AMLBM_STORE_F16: return cudaFuncGetAttributes(&a, lbm_kernel<__half, 26, 16, 1>);
    case AMLBM_STORE_BF16: return cudaFuncGetAttributes(&a, lbm_kernel<__nv_bfloat16, 26, 16, 1>);
    default: return cudaErrorInvalidValue;
  }
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

template <class In>
static cudaError_t launch_init_all_t(int storage, const InstDesc* d, int n, const long long* site_off,
                                    long long total, const In* rho, const In* uz, const In* ur, int parity,
                                    int* bad, cudaStream_t s) {
  if (total < 1) return cudaErrorInvalidValue;
  const unsigned nb = (unsigned)((total + 255) / 256);
  switch (storage) {
    case AMLBM_STORE_F64:
      init_all_kernel<double, In><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad); break;
    case AMLBM_STORE_F32:
      init_all_kernel<float, In><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad); break;
    case AMLBM_STORE_F16:
      init_all_kernel<__half, In><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad); break;
    case AMLBM_STORE_BF16:
      init_all_kernel<__nv_bfloat16, In><<<nb, 256, 0, s>>>(d, n, site_off, total, rho, uz, ur, parity, bad);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init_all(int storage, const InstDesc* d, int n, const long long* site_off,
                            long long total, const double* rho, const double* uz, const double* ur,
                            int parity, int* bad, cudaStream_t s) {
  return launch_init_all_t<double>(storage, d, n, site_off, total, rho, uz, ur, parity, bad, s);
}

cudaError_t launch_init_all(int storage, const InstDesc* d, int n, const long long* site_off,
                            long long total, const float* rho, const float* uz, const float* ur,
                            int parity, int* bad, cudaStream_t s) {
  return launch_init_all_t<float>(storage, d, n, site_off, total, rho, uz, ur, parity, bad, s);
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
