// Fused axisymmetric Shan-Chen LBM step for sm_103a (arXiv:1310.1871, Sec. II).
//
// One CTA updates one tile of BZ x BR sites of one lattice of a batch.  The
// whole per-site chain of the paper's update runs inside the CTA:
//   psi tile + halo 7 (from the previous step's psi, staged in shared memory)
//   -> isotropic d_r psi and 1D d_r psi (Sec. II.D), halo 5
//   -> moments, Shan-Chen force (Eq. scforce), axisymmetric force
//      (Eq. scAxisExtra), u and u^eq (Eqs. uhydro, ueq), halo 3
//   -> velocity gradients and the sources S, H_z, H_r (Eq. condition_h), halo 1
//   -> pull streaming of the BGK-collided populations (Eq. lbm2d_mod_new) with
//      the axis / wall / periodic maps of Sec. II.E, and psi of the new state.
// Global traffic per site and step: 9 populations read (halo re-reads hit L2),
// 9 written, psi written once and read once (halo re-reads hit L2).
// No tensor cores: the update is a stencil, not a contraction.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

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

// Storage codecs.  The 16-bit forms hold f_i - W_i rho_ref.
template <class S> struct Store;
template <> struct Store<double> {
  using C = double;
  static __device__ __forceinline__ C load(const double* p, C) { return *p; }
  static __device__ __forceinline__ void store(double* p, C v, C) { *p = v; }
  static __device__ __forceinline__ C round(C v, C) { return v; }
};
template <> struct Store<float> {
  using C = float;
  static __device__ __forceinline__ C load(const float* p, C) { return *p; }
  static __device__ __forceinline__ void store(float* p, C v, C) { *p = v; }
  static __device__ __forceinline__ C round(C v, C) { return v; }
};
template <> struct Store<__half> {
  using C = float;
  static __device__ __forceinline__ C load(const __half* p, C s) { return __half2float(*p) + s; }
  static __device__ __forceinline__ void store(__half* p, C v, C s) { *p = __float2half_rn(v - s); }
  static __device__ __forceinline__ C round(C v, C s) { return __half2float(__float2half_rn(v - s)) + s; }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ C load(const __nv_bfloat16* p, C s) {
    return __bfloat162float(*p) + s;
  }
  static __device__ __forceinline__ void store(__nv_bfloat16* p, C v, C s) {
    *p = __float2bfloat16_rn(v - s);
  }
  static __device__ __forceinline__ C round(C v, C s) {
    return __bfloat162float(__float2bfloat16_rn(v - s)) + s;
  }
};

__device__ __forceinline__ double exp_c(double x) { return exp(x); }
__device__ __forceinline__ float exp_c(float x) { return expf(x); }

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

// Isotropic 4th-order first derivative, Sec. II.D Eq. forthorder_firstderivativex:
// (1/36) sum_i c_i,AX (8 phi(x + c_i) - phi(x + 2 c_i)); AX = 1 along r, 0 along z.
// p points at x in a row-major tile whose rows (r) are `stride` apart.
template <int AX, class C>
__device__ __forceinline__ C iso(const C* p, int stride) {
  C s = C(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = AX ? cr_(i) : cz_(i);
    if (c != 0) {
      const C a = p[cr_(i) * stride + cz_(i)];
      const C b = p[2 * cr_(i) * stride + 2 * cz_(i)];
      s += c > 0 ? (C(8) * a - b) : -(C(8) * a - b);
    }
  }
  return s * C(1.0 / 36.0);
}
// 1D 4th-order central difference with element step `step` (Sec. II.D).
template <class C>
__device__ __forceinline__ C d1(const C* p, int step) {
  return (-p[2 * step] + C(8) * p[step] - C(8) * p[-step] + p[-2 * step]) * C(1.0 / 12.0);
}

template <class C>
__device__ __forceinline__ C feq(int i, C rho, C vz, C vr) {
  const C cv = C(cz_(i)) * vz + C(cr_(i)) * vr;
  const C vv = vz * vz + vr * vr;
  return C(w_(i)) * rho * (C(1) + C(3) * cv + C(4.5) * cv * cv - C(1.5) * vv);
}

// BGK collision of population i loaded from p, towards f^eq(rho, u^eq) (Eq. lbm2d).
template <class S>
__device__ __forceinline__ typename Store<S>::C collide(int i, const S* p, typename Store<S>::C rho,
                                                        typename Store<S>::C vz, typename Store<S>::C vr,
                                                        typename Store<S>::C omega,
                                                        typename Store<S>::C rref) {
  using C = typename Store<S>::C;
  const C f = Store<S>::load(p, C(w_(i)) * rref);
  return f + (feq(i, rho, vz, vr) - f) * omega;
}
// h_i = W_i (S + (c_iz H_z + c_ir H_r) / c_s^2), Eq. condition_h.
template <class C>
__device__ __forceinline__ C source(int i, C S_, C Hz, C Hr) {
  return C(w_(i)) * (S_ + C(3) * (C(cz_(i)) * Hz + C(cr_(i)) * Hr));
}

// Tile geometry: halos of psi (7), d_r psi (5), 1D d_r psi (z 5, r 3),
// macroscopic fields (3) and sources (1).
template <class C, int BZ, int BR>
struct Geo {
  static constexpr int HP = 7, HD = 5, HF = 3;
  static constexpr int PZ = BZ + 2 * HP, PR = BR + 2 * HP;
  static constexpr int DZ = BZ + 2 * HD, DR = BR + 2 * HD;
  static constexpr int EZ = BZ + 2 * HD, ER = BR + 2 * HF;
  static constexpr int FZ = BZ + 2 * HF, FR = BR + 2 * HF;
  static constexpr int SZ = BZ + 2, SR = BR + 2;
  static constexpr int nP = PZ * PR, nD = DZ * DR, nE = EZ * ER, nF = FZ * FR, nS = SZ * SR;
  // S, H_z, H_r reuse the psi / derivative region, which is dead by then.
  static_assert(nP + nD + nE >= 3 * nS, "source tiles must fit in the stencil region");
  static constexpr size_t bytes = sizeof(C) * (size_t)(nP + nD + nE + 5 * nF);
};

constexpr int NT = 256;

// Stages 0-2: psi tile, derivative tiles, and rho, u, u^eq on the tile plus 3.
template <class S, int BZ, int BR>
__device__ void macro_tile(const InstDesc& D, int k0, int j0, const S* __restrict__ fin,
                           const typename Store<S>::C* __restrict__ psin,
                           typename Store<S>::C* sm) {
  using C = typename Store<S>::C;
  using G = Geo<C, BZ, BR>;
  const int Nz = D.Nz, Nr = D.Nr, P = D.P;
  const size_t plane = (size_t)P * Nr;
  C* sPsi = sm;
  C* sDr = sPsi + G::nP;
  C* sD1 = sDr + G::nD;
  C* sRho = sD1 + G::nE;
  C* sUz = sRho + G::nF;
  C* sUr = sUz + G::nF;
  C* sVz = sUr + G::nF;
  C* sVr = sVz + G::nF;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < G::nP; idx += NT) {
    const int lr = idx / G::PZ, lc = idx - lr * G::PZ;
    const int j = reflect_row(j0 - G::HP + lr, Nr);
    const int k = wrapz(k0 - G::HP + lc, Nz);
    sPsi[idx] = psin[(size_t)j * P + k];
  }
  __syncthreads();
  const bool ax = D.axisym != 0;
  if (ax) {
    for (int idx = tid; idx < G::nD; idx += NT) {
      const int lr = idx / G::DZ, lc = idx - lr * G::DZ;
      sDr[idx] = iso<1>(sPsi + (lr + G::HP - G::HD) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    }
    for (int idx = tid; idx < G::nE; idx += NT) {
      const int lr = idx / G::EZ, lc = idx - lr * G::EZ;
      sD1[idx] = d1(sPsi + (lr + G::HP - G::HF) * G::PZ + (lc + G::HP - G::HD), G::PZ);
    }
    __syncthreads();
  }

  const C tau = C(D.tau), Gc = C(D.G), gz = C(D.gz), rref = C(D.rho_ref);
  for (int idx = tid; idx < G::nF; idx += NT) {
    const int lr = idx / G::FZ, lc = idx - lr * G::FZ;
    const int j = j0 - G::HF + lr;
    if (j < 0 || j >= Nr) continue;
    const int k = wrapz(k0 - G::HF + lc, Nz);
    const S* fp = fin + (size_t)j * P + k;
    C rho = C(0), jz = C(0), jr = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const C fi = Store<S>::load(fp + i * plane, C(w_(i)) * rref);
      rho += fi;
      if (cz_(i) > 0) jz += fi;
      if (cz_(i) < 0) jz -= fi;
      if (cr_(i) > 0) jr += fi;
      if (cr_(i) < 0) jr -= fi;
    }
    const C* p = sPsi + (lr + G::HP - G::HF) * G::PZ + (lc + G::HP - G::HF);
    const C psi = p[0];
    // Shan-Chen force, Eq. scforce: -G psi sum_i W_i psi(x + c_i) c_i.
    C sz = C(0), sr = C(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const C q = C(w_(i)) * p[cr_(i) * G::PZ + cz_(i)];
      if (cz_(i) > 0) sz += q;
      if (cz_(i) < 0) sz -= q;
      if (cr_(i) > 0) sr += q;
      if (cr_(i) < 0) sr -= q;
    }
    C Fz = -Gc * psi * sz, Fr = -Gc * psi * sr;
    if (ax) {
      // Eq. scAxisExtra with c_s^4 = 1/9: d_rr psi = iso d_r of iso d_r psi,
      // d_zr psi = 1D d_z of 1D d_r psi.
      const C r = C(j) + C(0.5);
      const C* dr = sDr + (lr + G::HD - G::HF) * G::DZ + (lc + G::HD - G::HF);
      const C Dr = dr[0];
      const C Drr = iso<1>(dr, G::DZ);
      const C Dzr = d1(sD1 + lr * G::EZ + (lc + G::HD - G::HF), 1);
      const C g = -(Gc / C(2)) * C(1.0 / 9.0) * psi;
      Fz += g * Dzr / r;
      Fr += g * (Drr / r - Dr / (r * r));
    }
    Fz += rho * gz;
    sRho[idx] = rho;
    sUz[idx] = (jz + Fz / C(2)) / rho;
    sUr[idx] = (jr + Fr / C(2)) / rho;
    sVz[idx] = (jz + tau * Fz) / rho;
    sVr[idx] = (jr + tau * Fr) / rho;
  }
  __syncthreads();
  if (ax) {
    // Ghost rows of u (depth 2): u_z even and u_r odd about the axis; about the
    // outer wall u_r odd and u_z even (free-slip) or odd (no-slip).
    for (int idx = tid; idx < G::nF; idx += NT) {
      const int lr = idx / G::FZ, lc = idx - lr * G::FZ;
      const int j = j0 - G::HF + lr;
      int m;
      C sgz;
      if (j == -1 || j == -2) {
        m = -1 - j;
        sgz = C(1);
      } else if (j == Nr || j == Nr + 1) {
        m = 2 * Nr - 1 - j;
        sgz = D.wall == AMLBM_WALL_NOSLIP ? C(-1) : C(1);
      } else {
        continue;
      }
      const int src = (m - (j0 - G::HF)) * G::FZ + lc;
      sUz[idx] = sgz * sUz[src];
      sUr[idx] = -sUr[src];
    }
    __syncthreads();
  }
}

template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT) step_kernel(const InstDesc* __restrict__ descs,
                                                  const int* __restrict__ tile_inst, int toff,
                                                  int parity) {
  using C = typename Store<S>::C;
  using G = Geo<C, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int b = blockIdx.x + toff;
  const int inst = tile_inst[b];
  const InstDesc& D = descs[inst];
  const int t = b - D.tile_base;
  const int tzi = t % D.tiles_z, tri = t / D.tiles_z;
  const int k0 = tzi * BZ, j0 = tri * BR;
  const int Nz = D.Nz, Nr = D.Nr, P = D.P;
  const size_t plane = (size_t)P * Nr;
  const S* __restrict__ fin = static_cast<const S*>(D.f[parity]);
  S* __restrict__ fout = static_cast<S*>(D.f[parity ^ 1]);
  const C* __restrict__ psin = static_cast<const C*>(D.psi[parity]);
  C* __restrict__ psout = static_cast<C*>(D.psi[parity ^ 1]);

  macro_tile<S, BZ, BR>(D, k0, j0, fin, psin, sm);

  C* sRho = sm + G::nP + G::nD + G::nE;
  C* sUz = sRho + G::nF;
  C* sUr = sUz + G::nF;
  C* sVz = sUr + G::nF;
  C* sVr = sVz + G::nF;
  C* sS = sm;
  C* sHz = sS + G::nS;
  C* sHr = sHz + G::nS;
  const bool ax = D.axisym != 0;
  const C tau = C(D.tau), omega = C(1) / tau, rho0 = C(D.rho0), rref = C(D.rho_ref);
  const int tid = threadIdx.x;

  // Stage 3: velocity gradients and axisymmetric sources on the tile plus 1
  // (App. A: S = -rho u_r / r, H_z, H_r of Eqs. corr_z_ns_eqn, corr_r_ns_eqn,
  // mu = rho c_s^2 (tau - 1/2)).
  for (int idx = tid; idx < G::nS; idx += NT) {
    const int lr = idx / G::SZ, lc = idx - lr * G::SZ;
    const int j = j0 - 1 + lr;
    C S_ = C(0), Hz = C(0), Hr = C(0);
    if (ax && j >= 0 && j < Nr) {
      const int fi = (lr + 2) * G::FZ + (lc + 2);
      const C druz = iso<1>(sUz + fi, G::FZ);
      const C dzur = iso<0>(sUr + fi, G::FZ);
      const C drur = iso<1>(sUr + fi, G::FZ);
      const C rho = sRho[fi], uz = sUz[fi], ur = sUr[fi];
      const C r = C(j) + C(0.5);
      const C mu = rho * (tau - C(0.5)) / C(3);
      S_ = -rho * ur / r;
      Hz = (mu * (druz + dzur) - rho * ur * uz) / r;
      Hr = (C(2) * mu * (drur - ur / r) - rho * ur * ur) / r;
    }
    sS[idx] = S_;
    sHz[idx] = Hz;
    sHr[idx] = Hr;
  }
  __syncthreads();

  // Stage 4: pull streaming of the collided populations with the boundary maps.
  // Rows away from the axis and the wall take every population from x - c_i in
  // the same direction (compile-time indices); rows 0 and Nr-1 apply the
  // reflection maps.  A warp covers one row, so the two paths never diverge.
  const bool link = D.src == AMLBM_SRC_LINK;
  const bool noslip = D.wall == AMLBM_WALL_NOSLIP;
  for (int idx = tid; idx < BZ * BR; idx += NT) {
    const int lr = idx / BZ, lc = idx - lr * BZ;
    const int j = j0 + lr, k = k0 + lc;
    if (j >= Nr || k >= Nz) continue;
    const bool edge = (j == 0) || (j == Nr - 1);
    const int di = (lr + 1) * G::SZ + (lc + 1);
    C rho_new = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      int sl = lr - cr_(i), sc = lc - cz_(i), sj = j - cr_(i), sk = k - cz_(i), ii = i;
      if (edge) {
        if (cr_(i) > 0 && j == 0) {  // arrives through the axis: specular reflection
          sl = lr; sj = 0; ii = mirror_(i);
        } else if (cr_(i) < 0 && j == Nr - 1) {  // arrives through the outer wall
          sl = lr; sj = Nr - 1;
          if (noslip) { sc = lc; sk = k; ii = opp_(i); }
          else { ii = mirror_(i); }
        }
      }
      if (sk < 0) sk += Nz; else if (sk >= Nz) sk -= Nz;
      const int fi = (sl + G::HF) * G::FZ + (sc + G::HF);
      const int si = (sl + 1) * G::SZ + (sc + 1);
      const S* src = fin + (size_t)sj * P + sk;
      C post, hsrc;
      if (!edge) {
        post = collide<S>(i, src + i * plane, sRho[fi], sVz[fi], sVr[fi], omega, rref);
        hsrc = source<C>(i, sS[si], sHz[si], sHr[si]);
      } else {
        post = C(0); hsrc = C(0);
#pragma unroll
        for (int q = 0; q < 9; ++q)
          if (q == ii) {
            post = collide<S>(q, src + q * plane, sRho[fi], sVz[fi], sVr[fi], omega, rref);
            hsrc = source<C>(q, sS[si], sHz[si], sHr[si]);
          }
      }
      const C fnew = link ? post + C(0.5) * (hsrc + source<C>(i, sS[di], sHz[di], sHr[di]))
                          : post + hsrc;
      const C sh = C(w_(i)) * rref;
      Store<S>::store(fout + i * plane + (size_t)j * P + k, fnew, sh);
      rho_new += Store<S>::round(fnew, sh);
    }
    psout[(size_t)j * P + k] = rho0 * (C(1) - exp_c(-rho_new / rho0));
  }
}

// Density and hydrodynamic velocity of the current state (read-back and diagnostics).
template <class S, int BZ, int BR>
__global__ void __launch_bounds__(NT) macro_kernel(const InstDesc* __restrict__ descs,
                                                   const int* __restrict__ tile_inst, int toff,
                                                   int parity) {
  using C = typename Store<S>::C;
  using G = Geo<C, BZ, BR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int b = blockIdx.x + toff;
  const int inst = tile_inst[b];
  const InstDesc& D = descs[inst];
  const int t = b - D.tile_base;
  const int k0 = (t % D.tiles_z) * BZ, j0 = (t / D.tiles_z) * BR;
  macro_tile<S, BZ, BR>(D, k0, j0, static_cast<const S*>(D.f[parity]),
                        static_cast<const C*>(D.psi[parity]), sm);
  C* sRho = sm + G::nP + G::nD + G::nE;
  C* sUz = sRho + G::nF;
  C* sUr = sUz + G::nF;
  for (int idx = threadIdx.x; idx < BZ * BR; idx += NT) {
    const int lr = idx / BZ, lc = idx - lr * BZ;
    const int j = j0 + lr, k = k0 + lc;
    if (j >= D.Nr || k >= D.Nz) continue;
    const int fi = (lr + G::HF) * G::FZ + (lc + G::HF);
    const size_t o = (size_t)j * D.Nz + k;
    D.rho_out[o] = double(sRho[fi]);
    D.uz_out[o] = double(sUz[fi]);
    D.ur_out[o] = double(sUr[fi]);
  }
}

// f = f^eq(rho, u) (no force shift) and psi of the stored state.
template <class S>
__global__ void init_kernel(const InstDesc* __restrict__ descs, int inst, const double* rho_in,
                            const double* uz_in, const double* ur_in, int parity) {
  using C = typename Store<S>::C;
  const InstDesc& D = descs[inst];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= D.Nz * D.Nr) return;
  const int j = n / D.Nz, k = n - j * D.Nz;
  const size_t plane = (size_t)D.P * D.Nr, o = (size_t)j * D.P + k;
  S* f = static_cast<S*>(D.f[parity]);
  C* psi = static_cast<C*>(D.psi[parity]);
  const C rho = C(rho_in[n]);
  const C uz = uz_in ? C(uz_in[n]) : C(0), ur = ur_in ? C(ur_in[n]) : C(0);
  const C rref = C(D.rho_ref), rho0 = C(D.rho0);
  C rs = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const C v = feq(i, rho, uz, ur);
    const C sh = C(w_(i)) * rref;
    Store<S>::store(f + i * plane + o, v, sh);
    rs += Store<S>::round(v, sh);
  }
  psi[o] = rho0 * (C(1) - exp_c(-rs / rho0));
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
#pragma unroll
  for (int i = 0; i < 9; ++i)
    out[(size_t)i * N + n] = double(Store<S>::load(f + i * plane + o, C(w_(i)) * C(D.rho_ref)));
}

// ----------------------------------------------------------- diagnostics --
constexpr int DIAG_NT = 256;
constexpr int NSUM = 8;  // mass2d mass3d momz3d Eke q2 sumS bad umax

__device__ __forceinline__ double col_radius(const double* rho, int Nz, int Nr, int k, double mid) {
  for (int j = 0; j < Nr; ++j) {
    const double v = rho[(size_t)j * Nz + k];
    if (v < mid) {
      if (j == 0) return 0.0;
      const double v0 = rho[(size_t)(j - 1) * Nz + k];
      return (j - 1 + 0.5) + (v0 - mid) / (v0 - v);
    }
  }
  return double(Nr);
}

__global__ void __launch_bounds__(DIAG_NT) diag_partial_kernel(const InstDesc* __restrict__ descs,
                                                               int inst, double zc, double rho_l,
                                                               double rho_v, double* partials,
                                                               double* cols) {
  const InstDesc& D = descs[inst];
  const int Nz = D.Nz, Nr = D.Nr, N = Nz * Nr;
  const double pi = 3.14159265358979323846;
  double acc[NSUM] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int n = blockIdx.x * DIAG_NT + threadIdx.x; n < N; n += gridDim.x * DIAG_NT) {
    const int j = n / Nz, k = n - j * Nz;
    const double r = j + 0.5, rho = D.rho_out[n], uz = D.uz_out[n], ur = D.ur_out[n];
    const double u2 = uz * uz + ur * ur;
    acc[0] += rho;
    acc[1] += 2 * pi * r * rho;
    acc[2] += 2 * pi * r * rho * uz;
    acc[3] += pi * r * rho * u2;
    const double dz = k - zc;
    acc[4] += 2 * pi * r * (rho - rho_v) / (rho_l - rho_v) * (dz * dz - 0.5 * r * r);
    acc[5] += -rho * ur / r;
    const bool bad = !(rho > 0) || !isfinite(rho) || !isfinite(u2);
    acc[6] += bad ? 1.0 : 0.0;
    acc[7] = fmax(acc[7], bad ? 0.0 : sqrt(u2));
  }
  __shared__ double red[NSUM][DIAG_NT];
#pragma unroll
  for (int q = 0; q < NSUM; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = DIAG_NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < NSUM - 1; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
      red[NSUM - 1][threadIdx.x] = fmax(red[NSUM - 1][threadIdx.x], red[NSUM - 1][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < NSUM) partials[blockIdx.x * NSUM + threadIdx.x] = red[threadIdx.x][0];
  const double mid = 0.5 * (rho_l + rho_v);
  for (int k = blockIdx.x * DIAG_NT + threadIdx.x; k < Nz; k += gridDim.x * DIAG_NT)
    cols[k] = col_radius(D.rho_out, Nz, Nr, k, mid);
}

template <class C>
__global__ void __launch_bounds__(DIAG_NT) diag_final_kernel(const InstDesc* __restrict__ descs,
                                                             int inst, int parity, double zc,
                                                             double R, const double* partials,
                                                             int nblk, const double* cols,
                                                             double* out) {
  const InstDesc& D = descs[inst];
  const int Nz = D.Nz, Nr = D.Nr;
  __shared__ double red[NSUM + 1][DIAG_NT];
  double acc[NSUM + 1] = {0, 0, 0, 0, 0, 0, 0, 0, 1e300};
  for (int b = threadIdx.x; b < nblk; b += DIAG_NT) {
#pragma unroll
    for (int q = 0; q < NSUM - 1; ++q) acc[q] += partials[b * NSUM + q];
    acc[NSUM - 1] = fmax(acc[NSUM - 1], partials[b * NSUM + NSUM - 1]);
  }
  for (int k = threadIdx.x; k < Nz; k += DIAG_NT) acc[NSUM] = fmin(acc[NSUM], cols[k]);
#pragma unroll
  for (int q = 0; q <= NSUM; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = DIAG_NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < NSUM - 1; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
      red[NSUM - 1][threadIdx.x] = fmax(red[NSUM - 1][threadIdx.x], red[NSUM - 1][threadIdx.x + s]);
      red[NSUM][threadIdx.x] = fmin(red[NSUM][threadIdx.x], red[NSUM][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double pi = 3.14159265358979323846;
    out[0] = red[0][0];
    out[1] = red[1][0];
    out[2] = red[2][0];
    out[3] = red[3][0];
    out[4] = red[7][0];
    out[5] = 5.0 * red[4][0] / (4.0 * pi * pow(R, 5.0));
    int kc = (int)llround(zc);
    kc %= Nz;
    if (kc < 0) kc += Nz;
    out[6] = cols[kc];
    out[7] = red[NSUM][0];
    const C* psi = static_cast<const C*>(D.psi[parity]);
    const double G = D.G;
    auto pres = [&](int k, int j) {
      const double rho = D.rho_out[(size_t)j * Nz + k], ps = double(psi[(size_t)j * D.P + k]);
      return rho / 3.0 + G * ps * ps / 6.0;
    };
    int ko = (kc + Nz / 2) % Nz;
    out[8] = pres(kc, 0);
    out[9] = pres(ko, Nr - 1);
    out[10] = out[8] - out[9];
    out[11] = red[6][0];
    out[12] = red[5][0];
  }
}

template <class S, int BZ, int BR>
cudaError_t launch_step_t(const InstDesc* d, const int* ti, int ntiles, int toff, int parity,
                          cudaStream_t s) {
  using C = typename Store<S>::C;
  constexpr size_t smem = Geo<C, BZ, BR>::bytes;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(step_kernel<S, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(macro_kernel<S, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  step_kernel<S, BZ, BR><<<ntiles, NT, smem, s>>>(d, ti, toff, parity);
  return cudaGetLastError();
}
template <class S, int BZ, int BR>
cudaError_t launch_macro_t(const InstDesc* d, const int* ti, int ntiles, int toff, int parity,
                           cudaStream_t s) {
  using C = typename Store<S>::C;
  constexpr size_t smem = Geo<C, BZ, BR>::bytes;
  cudaFuncSetAttribute(macro_kernel<S, BZ, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  macro_kernel<S, BZ, BR><<<ntiles, NT, smem, s>>>(d, ti, toff, parity);
  return cudaGetLastError();
}

// Tile shapes compiled for each storage form.
struct TileEntry { int storage, tz, tr; };
constexpr TileEntry kTiles[] = {
    {AMLBM_STORE_F64, 32, 8},  {AMLBM_STORE_F64, 64, 8},
    {AMLBM_STORE_F32, 32, 8},  {AMLBM_STORE_F32, 64, 8},  {AMLBM_STORE_F32, 128, 8},  {AMLBM_STORE_F32, 64, 16},
    {AMLBM_STORE_F16, 32, 8},  {AMLBM_STORE_F16, 64, 8},  {AMLBM_STORE_F16, 128, 8},  {AMLBM_STORE_F16, 64, 16},
    {AMLBM_STORE_BF16, 32, 8}, {AMLBM_STORE_BF16, 64, 8}, {AMLBM_STORE_BF16, 128, 8}, {AMLBM_STORE_BF16, 64, 16},
};

template <class S>
cudaError_t dispatch(bool macro, int tz, int tr, const InstDesc* d, const int* ti, int nt, int toff,
                     int par, cudaStream_t s) {
  if (nt <= 0) return cudaSuccess;
#define AMLBM_TILE(TZ, TR)                                                       \
  if (tz == TZ && tr == TR)                                                      \
    return macro ? launch_macro_t<S, TZ, TR>(d, ti, nt, toff, par, s)            \
                 : launch_step_t<S, TZ, TR>(d, ti, nt, toff, par, s);
  AMLBM_TILE(32, 8)
  AMLBM_TILE(64, 8)
  if constexpr (!std::is_same<S, double>::value) {
    AMLBM_TILE(128, 8)
    AMLBM_TILE(64, 16)
  }
#undef AMLBM_TILE
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_storage(int storage, bool macro, int tz, int tr, const InstDesc* d,
                             const int* ti, int nt, int toff, int par, cudaStream_t s) {
  switch (storage) {
    case AMLBM_STORE_F64: return dispatch<double>(macro, tz, tr, d, ti, nt, toff, par, s);
    case AMLBM_STORE_F32: return dispatch<float>(macro, tz, tr, d, ti, nt, toff, par, s);
    case AMLBM_STORE_F16: return dispatch<__half>(macro, tz, tr, d, ti, nt, toff, par, s);
    case AMLBM_STORE_BF16: return dispatch<__nv_bfloat16>(macro, tz, tr, d, ti, nt, toff, par, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool tile_supported(int storage, int tz, int tr) {
  for (const auto& e : kTiles)
    if (e.storage == storage && e.tz == tz && e.tr == tr) return true;
  return false;
}

int tile_list(int storage, int* tz, int* tr, int cap) {
  int n = 0;
  for (const auto& e : kTiles)
    if (e.storage == storage) {
      if (n < cap && tz && tr) { tz[n] = e.tz; tr[n] = e.tr; }
      ++n;
    }
  return n;
}

size_t step_smem_bytes(int storage, int tz, int tr) {
  const size_t c = storage == AMLBM_STORE_F64 ? 8 : 4;
  const int nP = (tz + 14) * (tr + 14), nD = (tz + 10) * (tr + 10), nE = (tz + 10) * (tr + 6);
  const int nF = (tz + 6) * (tr + 6);
  return c * (size_t)(nP + nD + nE + 5 * nF);
}

cudaError_t launch_step(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                        int toff, int parity, cudaStream_t s) {
  return dispatch_storage(storage, false, tz, tr, d, ti, nt, toff, parity, s);
}
cudaError_t launch_macro(int storage, int tz, int tr, const InstDesc* d, const int* ti, int nt,
                         int toff, int parity, cudaStream_t s) {
  return dispatch_storage(storage, true, tz, tr, d, ti, nt, toff, parity, s);
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
  (void)Nr;
  diag_partial_kernel<<<nblk, DIAG_NT, 0, s>>>(d, inst, zc, rho_l, rho_v, partials, cols);
  if (storage == AMLBM_STORE_F64)
    diag_final_kernel<double><<<1, DIAG_NT, 0, s>>>(d, inst, parity, zc, R, partials, nblk, cols, out);
  else
    diag_final_kernel<float><<<1, DIAG_NT, 0, s>>>(d, inst, parity, zc, R, partials, nblk, cols, out);
  (void)Nz;
  return cudaGetLastError();
}

}  // namespace amlbm
