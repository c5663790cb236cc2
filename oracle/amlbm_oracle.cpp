// Oracle for the axisymmetric Shan-Chen lattice Boltzmann step
// (Srivastava, Perlekar, ten Thije Boonkkamp, Verma, Toschi, arXiv:1310.1871).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, loop-by-loop CPU
// restatement of the paper's per-timestep update in FP64.  Only the tests, the
// smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
// code, header, table or constant with the CUDA library; the two are written
// independently from the paper.
//
// The scalar type is a template parameter so that std::complex<double> gives
// complex-step derivatives (Squire & Trapp 1998) of the whole discrete map:
// that is the oracle's "FP64 adjoint" for the gradient checks.
//
// Readings of passages that the paper leaves garbled or open are marked
// "reading:" at the place they are used.
//
// Lattice: D2Q9 on the meridional (z, r) plane, delta t = delta z = delta r = 1
// (Sec. II.E).  Nodes sit at z_k = k, r_j = j + 1/2, so the axis r = 0 lies
// half-way between row 0 and its mirror row -1 (mid-grid specular reflection,
// Sec. II.E; the drop centre (160, 0.5) of Sec. IV.2).  A lattice that does not
// reach the axis (the flow between two discs of Sec. III.2, R_i <= r <= R) has
// its rows shifted outwards: r_j = j + 1/2 + r_off.
//
// Memory layout of every field array: a[j * Nz + k] (row j = radial index,
// k = axial index), populations f[i][j][k].

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// Built twice: serially, and with -fopenmp for the all-cores CPU baseline.  In
// the second build the site loops below run their rows (or sites) on several
// threads; every iteration writes only its own outputs and computes them with
// the same operations in the same order, so both builds give identical bits.
#define ORC_PAR _Pragma("omp parallel for schedule(static)")

namespace orc {

constexpr int Q = 9;
// Lattice velocities (c_z, c_r).  c_1, c_3 = +-z and c_2, c_4 = +-r (the
// numbering used by the 1D stencils of Sec. II.D).  Reading: the diagonals are
// numbered c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1), c_8 = (1,-1) (the figure
// that shows them is missing); only the order of f_i in dumps depends on it.
constexpr int CZ[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int CR[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
// Weights W_0 = 4/9, W_1..4 = 1/9, W_5..8 = 1/36 (App. A, after Eq. e_distribution).
const double W[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
// Speed of sound squared c_s^2 = 1/3 (Sec. II.A).
const double CS2 = 1.0 / 3.0;
const double CS4 = 1.0 / 9.0;

// Direction with the radial component flipped (specular reflection) and the
// fully reversed direction (bounce-back).
constexpr int MIRROR_R[Q] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
constexpr int OPPOSITE[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

enum { WALL_FREESLIP = 0, WALL_NOSLIP = 1, WALL_OUTLET = 2 };
enum { SRC_LOCAL = 0, SRC_LINK = 1 };
enum { Z_PERIODIC = 0, Z_NOSLIP = 1 };
enum { RLO_AXIS = 0, RLO_INLET = 1 };
enum { FORCE_SHIFT = 0, FORCE_GUO = 1 };

template <class T>
struct Params {
  int Nz, Nr;
  T tau, G, rho0, gz;
  int wall;      // outer radial boundary: 0 free-slip (mid-grid specular), 1 no-slip
                 // (mid-grid bounce-back), 2 outlet (equilibrium row, see step)
  int axisym;    // 1: axisymmetric terms on; 0: planar 2D Shan-Chen (Table I "2D" columns)
  int src_mode;  // how h_i(x + c_i/2, t + 1/2) of Eq. lbm2d_mod_new is discretised (SRC_*)
  int zbc;       // axial ends: 0 periodic, 1 no-slip walls (mid-grid bounce-back) at z = -1/2, Nz - 1/2
  int rlo;       // lower radial boundary: 0 the axis, 1 inlet (equilibrium row, see step)
  double r_off;  // r_j = j + 1/2 + r_off (0 with the axis)
  double rho_out;            // density imposed on the outlet row
  const double* inlet_uz;    // velocity imposed on the inlet row, [Nz] each
  const double* inlet_ur;
  int forcing;   // FORCE_SHIFT: the Shan-Chen velocity shift (Eq. ueq, the paper's
                 // scheme); FORCE_GUO: the forcing of Guo, Zheng & Shi (2002) that
                 // Sec. IV.1 compares it with (Table I, Laplace test)
};

// Padded scalar field with explicit ghost cells of width g on every side.
template <class T>
struct Pad {
  int Nz, Nr, g, W_;
  std::vector<T> v;
  Pad(int nz, int nr, int gg) : Nz(nz), Nr(nr), g(gg), W_(nz + 2 * gg),
                                v((size_t)(nr + 2 * gg) * (nz + 2 * gg), T(0)) {}
  T& operator()(int k, int j) { return v[(size_t)(j + g) * W_ + (k + g)]; }
  const T& operator()(int k, int j) const { return v[(size_t)(j + g) * W_ + (k + g)]; }
};

static inline int wrap_z(int k, int Nz) { int m = k % Nz; return m < 0 ? m + Nz : m; }
// Row of the real site that a ghost row mirrors: about r = 0 (between rows -1
// and 0) and about the outer wall r = Nr (between rows Nr-1 and Nr).
static inline int mirror_row(int j, int Nr) {
  if (j < 0) return -1 - j;
  if (j >= Nr) return 2 * Nr - 1 - j;
  return j;
}
// The same for any boundary: mid-grid walls and the axis mirror about the
// half-way point, inlet and outlet rows about the boundary row itself.
template <class T>
static inline int ghost_row(const Params<T>& P, int j) {
  if (j < 0) return P.rlo == RLO_INLET ? -j : -1 - j;
  if (j >= P.Nr) return P.wall == WALL_OUTLET ? 2 * (P.Nr - 1) - j : 2 * P.Nr - 1 - j;
  return j;
}
// Column of a ghost column: periodic wrap, or the mirror about a wall at
// z = -1/2 or z = Nz - 1/2.
template <class T>
static inline int ghost_col(const Params<T>& P, int k) {
  if (P.zbc == Z_PERIODIC) return wrap_z(k, P.Nz);
  if (k < 0) return -1 - k;
  if (k >= P.Nz) return 2 * P.Nz - 1 - k;
  return k;
}
static inline double r_of(int j) { return j + 0.5; }
template <class T>
static inline double r_at(const Params<T>& P, int j) { return j + 0.5 + P.r_off; }

// Equilibrium distribution, App. A Eq. e_distribution, to second order in the
// velocity.  Reading: the printed equation mixes u (linear term) and u^eq
// (quadratic terms); Eq. lbm2d evaluates f^eq at (rho, u^eq), so every term
// uses the same velocity v here.
template <class T>
static inline T feq(int i, const T& rho, const T& vz, const T& vr) {
  T cv = double(CZ[i]) * vz + double(CR[i]) * vr;
  T vv = vz * vz + vr * vr;
  return W[i] * rho * (1.0 + cv / CS2 + (cv * cv) / (2.0 * CS4) - vv / (2.0 * CS2));
}

// Pseudopotential psi(rho) = rho0 (1 - exp(-rho/rho0)), Sec. II.A.
template <class T>
static inline T psi_of(const T& rho, const T& rho0) { return rho0 * (1.0 - std::exp(-rho / rho0)); }

// Isotropic first derivative along r (alpha = 1) or z (alpha = 0), Sec. II.D
// Eq. forthorder_firstderivativex:
//   d_r phi(x) = 1/36 sum_{i=1..8} (8 phi(x + c_i) - phi(x + 2 c_i)) c_ir.
// The z version replaces c_ir by c_iz (reading: the paper prints only d_r; the
// velocity gradients d_z u_r use the same stencil rotated).
template <class T>
static inline T iso_d(const Pad<T>& p, int k, int j, int alpha) {
  T s = T(0);
  for (int i = 1; i < Q; ++i) {
    const int c = alpha ? CR[i] : CZ[i];
    s += (8.0 * p(k + CZ[i], j + CR[i]) - p(k + 2 * CZ[i], j + 2 * CR[i])) * double(c);
  }
  return s / 36.0;
}

// One-dimensional fourth-order central difference along r (Sec. II.D, the
// d_r used inside the mixed derivative) and along z (the outer operator of
// Eq. forthorder_mixedderivative).
template <class T>
static inline T d1_r(const Pad<T>& p, int k, int j) {
  return (-p(k, j + 2) + 8.0 * p(k, j + 1) - 8.0 * p(k, j - 1) + p(k, j - 2)) / 12.0;
}
template <class T>
static inline T d1_z(const Pad<T>& p, int k, int j) {
  return (-p(k + 2, j) + 8.0 * p(k + 1, j) - 8.0 * p(k - 1, j) + p(k - 2, j)) / 12.0;
}

// Every per-site intermediate of one step, kept for the unit tests.
template <class T>
struct Macro {
  int N;
  std::vector<T> rho, jz, jr, psi, Fsc_z, Fsc_r, Dr, Drr, Dzr, Fg_z, Fg_r, Fz, Fr,
      uz, ur, ueqz, ueqr, druz, dzur, drur, S, Hz, Hr;
  explicit Macro(int n) : N(n) {
    for (auto* a : all()) a->assign(n, T(0));
  }
  std::vector<std::vector<T>*> all() {
    return {&rho, &jz, &jr, &psi, &Fsc_z, &Fsc_r, &Dr, &Drr, &Dzr, &Fg_z, &Fg_r, &Fz, &Fr,
            &uz, &ur, &ueqz, &ueqr, &druz, &dzur, &drur, &S, &Hz, &Hr};
  }
};

// Steps 1-8 of the update: moments, pseudopotential, forces, velocities,
// velocity gradients and axisymmetric sources at every real site.
template <class T>
static void macro(const Params<T>& P, const T* f, Macro<T>& M) {
  const int Nz = P.Nz, Nr = P.Nr, N = Nz * Nr;
  // 1. Moments rho = sum_i f_i, rho u = sum_i c_i f_i (App. A Eq. hydro_var).
  ORC_PAR
  for (int n = 0; n < N; ++n) {
    T rho = T(0), jz = T(0), jr = T(0);
    for (int i = 0; i < Q; ++i) {
      const T fi = f[(size_t)i * N + n];
      rho += fi;
      jz += double(CZ[i]) * fi;
      jr += double(CR[i]) * fi;
    }
    M.rho[n] = rho; M.jz[n] = jz; M.jr[n] = jr;
    // 2. Pseudopotential (Sec. II.A).
    M.psi[n] = psi_of(rho, P.rho0);
  }
  // 3. psi with ghost cells of depth 4: periodic in z; even mirror about the
  // axis (symmetry condition for the derivatives at the axis, Sec. II.E) and,
  // reading, also about the outer wall, the z walls, and the inlet and outlet
  // rows (zero normal derivative there, the paper's rule for the non-axis
  // boundaries).
  const int g = 4;
  Pad<T> ps(Nz, Nr, g);
  ORC_PAR
  for (int j = -g; j < Nr + g; ++j)
    for (int k = -g; k < Nz + g; ++k)
      ps(k, j) = M.psi[(size_t)ghost_row(P, j) * Nz + ghost_col(P, k)];

  // 5a. Isotropic d_r psi on the real rows and on two ghost rows each side,
  // evaluated from the ghost-extended psi, and the 1D d_r psi used inside the
  // mixed derivative.
  Pad<T> dr(Nz, Nr, 2), dr1(Nz, Nr, 2);
  ORC_PAR
  for (int j = -2; j < Nr + 2; ++j)
    for (int k = -2; k < Nz + 2; ++k) {
      dr(k, j) = iso_d(ps, k, j, 1);
      dr1(k, j) = d1_r(ps, k, j);
    }

  ORC_PAR
  for (int j = 0; j < Nr; ++j) {
    const double r = r_at(P, j);
    for (int k = 0; k < Nz; ++k) {
      const size_t n = (size_t)j * Nz + k;
      const T psi = ps(k, j);
      // 4. Two-dimensional Shan-Chen force, Eq. scforce / Eq. sc2d:
      //    F(x) = -G psi(x) sum_i W_i psi(x + c_i) c_i.
      T sz = T(0), sr = T(0);
      for (int i = 1; i < Q; ++i) {
        sz += W[i] * ps(k + CZ[i], j + CR[i]) * double(CZ[i]);
        sr += W[i] * ps(k + CZ[i], j + CR[i]) * double(CR[i]);
      }
      M.Fsc_z[n] = -P.G * psi * sz;
      M.Fsc_r[n] = -P.G * psi * sr;
      // 5b. d_rr psi = isotropic d_r applied to d_r psi
      // (Eq. forthorder_secondderivativex); d_zr psi = 1D d_z of 1D d_r psi
      // (Eq. forthorder_mixedderivative).
      const T Dr = dr(k, j);
      const T Drr = iso_d(dr, k, j, 1);
      const T Dzr = d1_z(dr1, k, j);
      M.Dr[n] = Dr; M.Drr[n] = Drr; M.Dzr[n] = Dzr;
      // Axisymmetric surface-tension force, Eq. scAxisExtra, delta t = 1:
      //   F_z = -(G/2) c_s^4 psi r^-1 d_zr psi
      //   F_r = -(G/2) c_s^4 psi (r^-1 d_rr psi - r^-2 d_r psi).
      if (P.axisym) {
        M.Fg_z[n] = -(P.G / 2.0) * CS4 * psi * Dzr / r;
        M.Fg_r[n] = -(P.G / 2.0) * CS4 * psi * (Drr / r - Dr / (r * r));
      } else {
        M.Fg_z[n] = T(0);
        M.Fg_r[n] = T(0);
      }
      // 6. Total force with the constant body force rho g along z (Sec. III.1),
      // hydrodynamic velocity (Eq. uhydro) and the shifted equilibrium
      // velocity of the Shan-Chen forcing (Eq. ueq).
      const T rho = M.rho[n];
      const T Fz = M.Fsc_z[n] + M.Fg_z[n] + rho * P.gz;
      const T Fr = M.Fsc_r[n] + M.Fg_r[n];
      M.Fz[n] = Fz; M.Fr[n] = Fr;
      M.uz[n] = (M.jz[n] + Fz / 2.0) / rho;
      M.ur[n] = (M.jr[n] + Fr / 2.0) / rho;
      M.ueqz[n] = (M.jz[n] + P.tau * Fz) / rho;
      M.ueqr[n] = (M.jr[n] + P.tau * Fr) / rho;
    }
  }

  // 7. Velocity with ghost cells of depth 2: periodic in z; about the axis
  // u_z is even and u_r odd; at the outer wall (reading of "derivatives
  // zero", Sec. II.E: mirror ghosts by the wall's own symmetry) free-slip
  // keeps u_z even and u_r odd, no-slip makes both odd; at the no-slip z walls
  // both are odd.  Beyond an inlet or outlet row b the velocity continues
  // linearly, u(b - m) = 2 u(b) - u(b + m) (reading: an open boundary with a
  // zero derivative would halve the viscous term of a u_r ~ 1/r outflow in
  // the rows next to it).  Ghost columns are filled first, then ghost rows
  // from the column-extended real rows.
  Pad<T> uzp(Nz, Nr, 2), urp(Nz, Nr, 2);
  ORC_PAR
  for (int j = 0; j < Nr; ++j)
    for (int k = -2; k < Nz + 2; ++k) {
      const size_t n = (size_t)j * Nz + ghost_col(P, k);
      const double sgn = (P.zbc == Z_NOSLIP && (k < 0 || k >= Nz)) ? -1.0 : 1.0;
      uzp(k, j) = sgn * M.uz[n];
      urp(k, j) = sgn * M.ur[n];
    }
  for (int m = 1; m <= 2; ++m)
    for (int k = -2; k < Nz + 2; ++k) {
      // below row 0
      if (P.rlo == RLO_INLET) {
        uzp(k, -m) = 2.0 * uzp(k, 0) - uzp(k, m);
        urp(k, -m) = 2.0 * urp(k, 0) - urp(k, m);
      } else {
        uzp(k, -m) = uzp(k, m - 1);
        urp(k, -m) = -urp(k, m - 1);
      }
      // beyond row Nr - 1
      const int b = Nr - 1;
      if (P.wall == WALL_OUTLET) {
        uzp(k, b + m) = 2.0 * uzp(k, b) - uzp(k, b - m);
        urp(k, b + m) = 2.0 * urp(k, b) - urp(k, b - m);
      } else {
        const double sgn_z = P.wall == WALL_NOSLIP ? -1.0 : 1.0;
        uzp(k, b + m) = sgn_z * uzp(k, Nr - m);
        urp(k, b + m) = -urp(k, Nr - m);
      }
    }

  ORC_PAR
  for (int j = 0; j < Nr; ++j) {
    const double r = r_at(P, j);
    for (int k = 0; k < Nz; ++k) {
      const size_t n = (size_t)j * Nz + k;
      // Velocity gradients with the 1D fourth-order central differences of
      // Sec. II.D (reading: the paper names no stencil for them).  The
      // isotropic stencil is not usable here: on a mode that alternates in z
      // its diagonal taps reverse the sign of d_r u_z, so the viscous source
      // mu d_r u_z / r amplifies that mode next to a no-slip wall (it grows
      // from rounding noise at tau = 1 and blows up at tau = 1.5), whereas
      // Sec. III.1 reports a steady state whose kinetic energy is constant to
      // machine precision.
      const T druz = d1_r(uzp, k, j);
      const T dzur = d1_z(urp, k, j);
      const T drur = d1_r(urp, k, j);
      M.druz[n] = druz; M.dzur[n] = dzur; M.drur[n] = drur;
      // 8. Axisymmetric sources, Eq. condition_h and App. A
      // Eqs. corr_cty_eqn, corr_r_ns_eqn, corr_z_ns_eqn, with mu = nu rho and
      // nu = c_s^2 (tau - 1/2).  Reading: Eq. H_terms prints an extra c_iz
      // (c_ir) factor in H_z (H_r); it is dropped, because with it
      // sum_i c_i h_i would vanish instead of giving the App. A moments.
      if (P.axisym) {
        const T rho = M.rho[n], uz = M.uz[n], ur = M.ur[n];
        const T mu = rho * CS2 * (P.tau - 0.5);
        M.S[n] = -rho * ur / r;
        M.Hz[n] = (mu * (druz + dzur) - rho * ur * uz) / r;
        M.Hr[n] = (2.0 * mu * (drur - ur / r) - rho * ur * ur) / r;
      } else {
        M.S[n] = T(0); M.Hz[n] = T(0); M.Hr[n] = T(0);
      }
    }
  }
}

// Source term h_i = W_i (S + (c_iz H_z + c_ir H_r)/c_s^2), Eq. condition_h.
template <class T>
static inline T h_of(int i, const T& S, const T& Hz, const T& Hr) {
  return W[i] * (S + (double(CZ[i]) * Hz + double(CR[i]) * Hr) / CS2);
}

// One full timestep f(t) -> f(t+1), Eq. lbm2d_mod_new, with the boundary
// conditions of Sec. II.E applied to the streaming step.
template <class T>
static void step(const Params<T>& P, const T* f, T* fn, Macro<T>* keep) {
  const int Nz = P.Nz, Nr = P.Nr, N = Nz * Nr;
  Macro<T> M(N);
  macro(P, f, M);
  // 9. BGK collision towards f^eq(rho, u^eq) (Eq. lbm2d) and the source of
  // every population at its own site.
  // With the Guo forcing (Guo, Zheng & Shi 2002, restated from its definition):
  // f^eq at the hydrodynamic u, plus (1 - 1/(2 tau)) times the discrete force
  // W_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . F, whose zeroth moment is 0
  // and first moment F.
  std::vector<T> fs((size_t)Q * N), h((size_t)Q * N);
  ORC_PAR
  for (int n = 0; n < N; ++n)
    for (int i = 0; i < Q; ++i) {
      const T fi = f[(size_t)i * N + n];
      if (P.forcing == FORCE_GUO) {
        const T uz = M.uz[n], ur = M.ur[n], Fz = M.Fz[n], Fr = M.Fr[n];
        const T cu = double(CZ[i]) * uz + double(CR[i]) * ur;
        const T cF = double(CZ[i]) * Fz + double(CR[i]) * Fr;
        const T uF = uz * Fz + ur * Fr;
        const T Si = W[i] * ((cF - uF) / CS2 + cu * cF / CS4);
        fs[(size_t)i * N + n] = fi - (fi - feq(i, M.rho[n], uz, ur)) / P.tau + (1.0 - 0.5 / P.tau) * Si;
      } else {
        fs[(size_t)i * N + n] = fi - (fi - feq(i, M.rho[n], M.ueqz[n], M.ueqr[n])) / P.tau;
      }
      h[(size_t)i * N + n] = h_of(i, M.S[n], M.Hz[n], M.Hr[n]);
    }
  // Inlet and outlet rows (Sec. II.E: a prescribed velocity or pressure is set
  // by the equilibrium of the wanted density and hydrodynamic velocity,
  // imposed before streaming).  Reading: the inlet row holds
  // f^eq(rho of row 1, u_in(z)) (velocity prescribed, density free), the
  // outlet row f^eq(rho_out, u of row Nr - 2) (density prescribed, the
  // velocity leaves freely); both from the moments at time t, without source.
  // These populations stream out of the boundary row and also become its own
  // state at t + 1.
  auto set_boundary_row = [&](int j, int jn, bool inlet) {
    for (int k = 0; k < Nz; ++k) {
      const size_t n = (size_t)j * Nz + k, nn = (size_t)jn * Nz + k;
      const T rho = inlet ? M.rho[nn] : T(P.rho_out);
      const T uz = inlet ? T(P.inlet_uz[k]) : M.uz[nn];
      const T ur = inlet ? T(P.inlet_ur[k]) : M.ur[nn];
      for (int i = 0; i < Q; ++i) {
        fs[(size_t)i * N + n] = feq(i, rho, uz, ur);
        h[(size_t)i * N + n] = T(0);
      }
    }
  };
  if (P.rlo == RLO_INLET) set_boundary_row(0, 1, true);
  if (P.wall == WALL_OUTLET) set_boundary_row(Nr - 1, Nr - 2, false);
  auto boundary_row = [&](int j) {
    return (j == 0 && P.rlo == RLO_INLET) || (j == Nr - 1 && P.wall == WALL_OUTLET);
  };
  // 10. Pull streaming.  Population i arriving at x left its source site
  // x_s = x - c_i in direction i' = i, except where the link crosses a wall:
  //  - axis r = 0 (mid-grid specular reflection): a population arriving at
  //    row 0 with c_ir = +1 left row 0 at z - c_iz in the mirrored direction;
  //  - outer wall, free-slip (mid-grid specular): the same about r = Nr;
  //  - outer wall, no-slip (mid-grid bounce-back): it left x itself in -c_i.
  // Reading of h_i(x + c_i/2, t + 1/2): the value at the departure site
  // h_i'(x_s, t) (SRC_LOCAL, the default), or the link average
  // (h_i'(x_s) + h_i(x)) / 2 at time t (SRC_LINK).  The link average leaves
  // the odd-even radial mode without a mass source on radial links and, in
  // the oracle, grows an odd-even u_r oscillation from the axis within a few
  // thousand steps (flat interface of Table I, static drop); the
  // departure-site value is stable there.
  //  - z walls (no-slip, mid-grid bounce-back at z = -1/2 and Nz - 1/2): a
  //    population whose departure column lies beyond a wall left x itself in
  //    -c_i; this takes precedence over the radial maps at the corners.
  //  - inlet and outlet rows are not streamed into: they take their own
  //    boundary populations.
  ORC_PAR
  for (int j = 0; j < Nr; ++j)
    for (int k = 0; k < Nz; ++k)
      for (int i = 0; i < Q; ++i) {
        if (boundary_row(j)) {
          const size_t d = (size_t)i * N + (size_t)j * Nz + k;
          fn[d] = fs[d];
          continue;
        }
        int sk = k - CZ[i], sj = j - CR[i], ii = i;
        if (P.zbc == Z_NOSLIP && (sk < 0 || sk >= Nz)) {
          sk = k; sj = j; ii = OPPOSITE[i];
        } else if (sj < 0) {
          sj = 0; ii = MIRROR_R[i];
        } else if (sj >= Nr) {
          if (P.wall == WALL_NOSLIP) { sk = k; sj = Nr - 1; ii = OPPOSITE[i]; }
          else { sj = Nr - 1; ii = MIRROR_R[i]; }
        }
        const size_t src = (size_t)ii * N + (size_t)sj * Nz + wrap_z(sk, Nz);
        const size_t dst = (size_t)i * N + (size_t)j * Nz + k;
        if (P.src_mode == SRC_LINK)
          fn[dst] = fs[src] + 0.5 * h[src] + 0.5 * h[dst];
        else
          fn[dst] = fs[src] + h[src];
      }
  if (keep) *keep = M;
}

// Initial populations f_i = f^eq_i(rho, u) (no force shift).
template <class T>
static void init(const Params<T>& P, const T* rho, const T* uz, const T* ur, T* f) {
  const int N = P.Nz * P.Nr;
  for (int n = 0; n < N; ++n)
    for (int i = 0; i < Q; ++i) f[(size_t)i * N + n] = feq(i, rho[n], uz[n], ur[n]);
}

// Legendre polynomial P_l(x) by the three-term recurrence.
template <class T>
static T legendre(int l, const T& x) {
  T p0 = T(1.0), p1 = x;
  if (l == 0) return p0;
  for (int m = 1; m < l; ++m) {
    T p2 = ((2.0 * m + 1.0) * x * p1 - double(m) * p0) / double(m + 1);
    p0 = p1; p1 = p2;
  }
  return p1;
}

// Shape-perturbed drop: rho = rho_v + (rho_l - rho_v)/2 (1 - tanh((d - R_s)/w))
// with d the distance from (zc, 0) and R_s(theta) = R (1 + sum_m a_m P_{l0+m}(cos theta)).
template <class T>
static void drop_rho(int Nz, int Nr, double zc, double R, double w, double rho_l, double rho_v,
                     int l0, int namp, const T* amp, T* rho) {
  for (int j = 0; j < Nr; ++j)
    for (int k = 0; k < Nz; ++k) {
      const double dz = k - zc, r = r_of(j);
      const double d = std::sqrt(dz * dz + r * r);
      const double ct = dz / d;
      T s = T(0);
      for (int m = 0; m < namp; ++m) s += amp[m] * legendre(l0 + m, T(ct));
      const T Rs = R * (1.0 + s);
      rho[(size_t)j * Nz + k] = rho_v + 0.5 * (rho_l - rho_v) * (1.0 - std::tanh((d - Rs) / w));
    }
}

// Smooth shape measures that are linear in rho (used as objectives):
//  - quadrupole amplitude a_2 = 5/(4 pi R^5) sum 2 pi r phi ((z-zc)^2 - r^2/2),
//    with phi = (rho - rho_v)/(rho_l - rho_v): the P_2 moment of the liquid
//    indicator, normalised so that a drop r_s = R (1 + e P_2) gives a_2 ~ e;
//  - neck radius r_n = sqrt(2 sum_j r_j phi(z*, j)) on the column z*.
template <class T>
static T objective(int kind, int Nz, int Nr, const T* rho, double zc, double R,
                   double rho_l, double rho_v, int kstar) {
  const double pi = 3.14159265358979323846;
  if (kind == 0) {
    T q = T(0);
    for (int j = 0; j < Nr; ++j)
      for (int k = 0; k < Nz; ++k) {
        const double dz = k - zc, r = r_of(j);
        const T phi = (rho[(size_t)j * Nz + k] - rho_v) / (rho_l - rho_v);
        q += 2.0 * pi * r * phi * (dz * dz - 0.5 * r * r);
      }
    const T a2 = 5.0 * q / (4.0 * pi * std::pow(R, 5));
    return a2 * a2;
  }
  T s = T(0);
  for (int j = 0; j < Nr; ++j)
    s += r_of(j) * (rho[(size_t)j * Nz + kstar] - rho_v) / (rho_l - rho_v);
  return std::sqrt(2.0 * s);
}

}  // namespace orc

// ---------------------------------------------------------------------------
// C entry points (loaded with ctypes by the tests and the benchmark's CPU leg).
// ---------------------------------------------------------------------------
using cplx = std::complex<double>;

struct orc_params {
  int Nz, Nr;
  double tau, G, rho0, gz;
  int wall, axisym, src_mode;
  int zbc, rlo;
  double r_off, rho_out;
  const double* inlet_uz;  // [Nz], read when rlo is the inlet
  const double* inlet_ur;
  int forcing;
};

static orc::Params<double> to_p(const orc_params* p) {
  return {p->Nz, p->Nr, p->tau, p->G, p->rho0, p->gz, p->wall, p->axisym, p->src_mode,
          p->zbc, p->rlo, p->r_off, p->rho_out, p->inlet_uz, p->inlet_ur, p->forcing};
}
// Sizes are such that every ghost cell of depth 4 mirrors a real site.
static int check(const orc_params* p) {
  if (!p || p->Nz < 1 || p->Nr < 4 || !(p->tau > 0.5) || !(p->rho0 > 0)) return -1;
  if (p->wall < 0 || p->wall > 2 || p->zbc < 0 || p->zbc > 1 || p->rlo < 0 || p->rlo > 1) return -1;
  if (p->zbc == 1 && p->Nz < 4) return -1;
  if ((p->rlo == 1 || p->wall == 2) && p->Nr < 6) return -1;
  if (p->rlo == 0 && p->r_off != 0.0) return -1;
  if (!(p->r_off >= 0.0)) return -1;
  if (p->rlo == 1 && (!p->inlet_uz || !p->inlet_ur)) return -1;
  if (p->wall == 2 && !(p->rho_out > 0)) return -1;
  if (p->forcing != 0 && p->forcing != 1) return -1;
  return 0;
}

extern "C" {

int orc_num_fields(void) { return 23; }

// Threads of the site loops: n > 0 sets them (OpenMP build only); returns the
// number a parallel loop uses now (1 in the serial build).
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// f = f^eq(rho, u), arrays [Nr][Nz], f [9][Nr][Nz].
int orc_init(const orc_params* p, const double* rho, const double* uz, const double* ur, double* f) {
  if (check(p)) return -1;
  orc::init(to_p(p), rho, uz, ur, f);
  return 0;
}

// Advance f in place by nsteps steps.
int orc_run(const orc_params* p, double* f, int nsteps) {
  if (check(p) || nsteps < 0) return -1;
  const orc::Params<double> P = to_p(p);
  const size_t n = (size_t)9 * P.Nz * P.Nr;
  std::vector<double> tmp(n);
  for (int s = 0; s < nsteps; ++s) {
    orc::step(P, f, tmp.data(), (orc::Macro<double>*)nullptr);
    std::memcpy(f, tmp.data(), n * sizeof(double));
  }
  return 0;
}

// All 23 per-site intermediates of one step, out[23][Nr][Nz], in the order
// rho jz jr psi Fsc_z Fsc_r Dr Drr Dzr Fg_z Fg_r Fz Fr uz ur ueqz ueqr
// druz dzur drur S Hz Hr.
int orc_fields(const orc_params* p, const double* f, double* out) {
  if (check(p)) return -1;
  const orc::Params<double> P = to_p(p);
  const int N = P.Nz * P.Nr;
  orc::Macro<double> M(N);
  orc::macro(P, f, M);
  int q = 0;
  for (auto* a : M.all()) { std::memcpy(out + (size_t)q * N, a->data(), N * sizeof(double)); ++q; }
  return 0;
}

// Stencil operators on a caller-supplied padded array (pad cells on each
// side), for the polynomial-exactness tests.  op: 0 iso d_z, 1 iso d_r,
// 2 1D d_r, 3 1D d_z, 4 iso d_r(iso d_r), 5 1D d_z(1D d_r).  out is
// [Nr][Nz] at the interior sites.
int orc_stencil(int Nz, int Nr, int pad, const double* padded, int op, double* out) {
  if (pad < 4) return -1;
  orc::Pad<double> a(Nz, Nr, pad);
  std::memcpy(a.v.data(), padded, a.v.size() * sizeof(double));
  orc::Pad<double> t(Nz, Nr, pad);
  if (op >= 4) {
    for (int j = -2; j < Nr + 2; ++j)
      for (int k = -2; k < Nz + 2; ++k) t(k, j) = op == 4 ? orc::iso_d(a, k, j, 1) : orc::d1_r(a, k, j);
  }
  for (int j = 0; j < Nr; ++j)
    for (int k = 0; k < Nz; ++k) {
      double v = 0;
      switch (op) {
        case 0: v = orc::iso_d(a, k, j, 0); break;
        case 1: v = orc::iso_d(a, k, j, 1); break;
        case 2: v = orc::d1_r(a, k, j); break;
        case 3: v = orc::d1_z(a, k, j); break;
        case 4: v = orc::iso_d(t, k, j, 1); break;
        case 5: v = orc::d1_z(t, k, j); break;
        default: return -1;
      }
      out[(size_t)j * Nz + k] = v;
    }
  return 0;
}

// The source moments at every site for the identity tests: h[9][Nr][Nz].
int orc_sources(const orc_params* p, const double* f, double* h) {
  if (check(p)) return -1;
  const orc::Params<double> P = to_p(p);
  const int N = P.Nz * P.Nr;
  orc::Macro<double> M(N);
  orc::macro(P, f, M);
  for (int n = 0; n < N; ++n)
    for (int i = 0; i < 9; ++i) h[(size_t)i * N + n] = orc::h_of(i, M.S[n], M.Hz[n], M.Hr[n]);
  return 0;
}

// Shape-perturbed drop density (see drop_rho); amplitudes of P_l0 .. P_{l0+namp-1}.
int orc_drop_rho(int Nz, int Nr, double zc, double R, double w, double rho_l, double rho_v,
                 int l0, int namp, const double* amp, double* rho) {
  orc::drop_rho<double>(Nz, Nr, zc, R, w, rho_l, rho_v, l0, namp, amp, rho);
  return 0;
}

// Objective J of the differentiable runs: the drop quadrupole a_2 squared
// (kind 0) or the neck radius on column kstar (kind 1), at the density rho.
double orc_objective(int kind, int Nz, int Nr, const double* rho, double zc, double R,
                     double rho_l, double rho_v, int kstar) {
  return orc::objective<double>(kind, Nz, Nr, rho, zc, R, rho_l, rho_v, kstar);
}

// Differentiable end-to-end run: drop_rho(amplitudes) -> f = f^eq(rho, 0) ->
// T steps -> J.  Returns J and, by complex-step differentiation with step
// h = 1e-30 along each of the (2 + namp) parameters (G, tau, amplitudes),
// the exact derivative of the discrete map.  grad may be null (J only).
int orc_grad(const orc_params* p, int T, double zc, double R, double w, double rho_l,
             double rho_v, int l0, int namp, const double* amp, int kind, double objR, int kstar,
             double* J, double* grad) {
  if (check(p) || T < 0 || namp < 0) return -1;
  const int Nz = p->Nz, Nr = p->Nr, N = Nz * Nr;
  const int npar = 2 + namp;
  const double hstep = 1e-30;
  // Run q = -1 is the unperturbed run (J only); runs q >= 0 perturb one parameter.
  const int qfirst = grad ? 0 : -1, qlast = grad ? npar - 1 : -1;
  for (int q = qfirst; q <= qlast; ++q) {
    orc::Params<cplx> P{Nz, Nr, cplx(p->tau), cplx(p->G), cplx(p->rho0), cplx(p->gz),
                        p->wall, p->axisym, p->src_mode, p->zbc, p->rlo, p->r_off,
                        p->rho_out, p->inlet_uz, p->inlet_ur, p->forcing};
    std::vector<cplx> a(namp);
    for (int m = 0; m < namp; ++m) a[m] = cplx(amp[m]);
    if (q == 0) P.G += cplx(0, hstep);
    if (q == 1) P.tau += cplx(0, hstep);
    if (q >= 2) a[q - 2] += cplx(0, hstep);
    std::vector<cplx> rho(N), zero(N, cplx(0)), f((size_t)9 * N), fn((size_t)9 * N);
    orc::drop_rho<cplx>(Nz, Nr, zc, R, w, rho_l, rho_v, l0, namp, a.data(), rho.data());
    orc::init(P, rho.data(), zero.data(), zero.data(), f.data());
    for (int s = 0; s < T; ++s) {
      orc::step(P, f.data(), fn.data(), (orc::Macro<cplx>*)nullptr);
      f.swap(fn);
    }
    for (int n = 0; n < N; ++n) {
      cplx s = 0;
      for (int i = 0; i < 9; ++i) s += f[(size_t)i * N + n];
      rho[n] = s;
    }
    const cplx Jc = orc::objective<cplx>(kind, Nz, Nr, rho.data(), zc, objR, rho_l, rho_v, kstar);
    if (q <= 0 && J) *J = Jc.real();
    if (q >= 0) grad[q] = Jc.imag() / hstep;
  }
  return 0;
}

// Diagnostics of a state (FP64 sums over real sites), out[16]:
//  0 mass2d = sum rho          1 mass3d = sum 2 pi r rho
//  2 momz3d = sum 2 pi r rho u_z (hydrodynamic u)
//  3 E_ke = pi sum r rho |u|^2 (Sec. III)      4 max |u|
//  5 a_2 (quadrupole, about zc, radius objR)   6 A: r-intercept on column kc
//  7 neck: min over z of the interface radius  8 p_in  9 p_out
//  10 dp = p_in - p_out   11 count of non-finite or non-positive rho
//  12 sum of S (discrete mass source of the step that starts from f)
// Interface radius of a column: first row (from the axis) where rho drops
// below (rho_l + rho_v)/2, linearly interpolated; Nr when it never does.
// Pressure from Eq. pressure, p = c_s^2 rho + c_s^2 G psi^2/2, taken at
// (kc, row 0) (p_in) and at (kc + Nz/2, row Nr-1) (p_out).
int orc_diag(const orc_params* p, const double* f, double zc, double objR, double rho_l,
             double rho_v, double* out) {
  if (check(p)) return -1;
  const orc::Params<double> P = to_p(p);
  const int Nz = P.Nz, Nr = P.Nr, N = Nz * Nr;
  const double pi = 3.14159265358979323846;
  orc::Macro<double> M(N);
  orc::macro(P, f, M);
  for (int q = 0; q < 16; ++q) out[q] = 0;
  double umax = 0, q2 = 0, sumS = 0;
  int bad = 0;
  for (int j = 0; j < Nr; ++j)
    for (int k = 0; k < Nz; ++k) {
      const int n = j * Nz + k;
      const double r = orc::r_at(P, j), rho = M.rho[n], uz = M.uz[n], ur = M.ur[n];
      const double u2 = uz * uz + ur * ur;
      out[0] += rho;
      out[1] += 2 * pi * r * rho;
      out[2] += 2 * pi * r * rho * uz;
      out[3] += pi * r * rho * u2;
      if (std::sqrt(u2) > umax) umax = std::sqrt(u2);
      const double dz = k - zc;
      q2 += 2 * pi * r * (rho - rho_v) / (rho_l - rho_v) * (dz * dz - 0.5 * r * r);
      sumS += M.S[n];
      if (!(rho > 0) || !std::isfinite(rho) || !std::isfinite(u2)) ++bad;
    }
  out[4] = umax;
  out[5] = 5 * q2 / (4 * pi * std::pow(objR, 5));
  const double mid = 0.5 * (rho_l + rho_v);
  auto radius = [&](int k) {
    for (int j = 0; j < Nr; ++j) {
      const double rho = M.rho[(size_t)j * Nz + k];
      if (rho < mid) {
        if (j == 0) return P.r_off;
        const double r0 = M.rho[(size_t)(j - 1) * Nz + k];
        return orc::r_at(P, j - 1) + (r0 - mid) / (r0 - rho);
      }
    }
    return Nr + P.r_off;
  };
  int kc = (int)std::lround(zc);
  kc = orc::wrap_z(kc, Nz);
  out[6] = radius(kc);
  double neck = 1e300;
  for (int k = 0; k < Nz; ++k) neck = std::min(neck, radius(k));
  out[7] = neck;
  auto pres = [&](int k, int j) {
    const double rho = M.rho[(size_t)j * Nz + k], psi = M.psi[(size_t)j * Nz + k];
    return orc::CS2 * rho + orc::CS2 * P.G * psi * psi / 2;
  };
  out[8] = pres(kc, 0);
  out[9] = pres(orc::wrap_z(kc + Nz / 2, Nz), Nr - 1);
  out[10] = out[8] - out[9];
  out[11] = bad;
  out[12] = sumS;
  return 0;
}

}  // extern "C"
