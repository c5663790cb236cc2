"""Pins of the oracle's diagnostics (orc_diag) to closed forms.

The GPU diagnostics are compared with these outputs, so each one is tied here to
something the mathematics fixes independently of the oracle's code: sums with a
closed form on uniform states, crossings of a tanh profile whose half-density
radius is known exactly, the ideal-gas limit and the paper's coexistence pair for
the pressure of Sec. II.A, and counts planted by the test.  Each test names the
slip it is there to catch.

States are f = f^eq(rho, u) (the oracle's init); at G = 0 and g_z = 0 no force
acts, so the hydrodynamic velocity of Eq. uhydro is the prescribed u to rounding.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I

NZ, NR = 20, 12


def _uniform(rho0, U=0.0, V=0.0, G=0.0):
    o = O.Oracle(NZ, NR, tau=1.0, G=G)
    shp = (NR, NZ)
    f = o.init(np.full(shp, rho0), np.full(shp, U), np.full(shp, V))
    return o, f


def test_mass_momentum_energy_of_a_uniform_flow():
    """Sec. II.C and Sec. III: mass2d = sum rho, mass3d = sum 2 pi r rho,
    momz3d = sum 2 pi r rho u_z, E_ke = pi sum r rho |u|^2 with r_j = j + 1/2.
    For a uniform state sum_j (j + 1/2) = Nr^2 / 2, so
      mass2d = rho Nz Nr,  mass3d = pi rho Nz Nr^2,
      momz3d = pi rho U Nz Nr^2,  E_ke = (pi / 2) rho (U^2 + V^2) Nz Nr^2.
    Catches a dropped 2 pi, r at j instead of j + 1/2, u_r in the axial momentum,
    or a factor 1/2 in the energy."""
    rho0, U, V = 1.3, 0.021, -0.013
    o, f = _uniform(rho0, U, V)
    d = o.diag(f)
    assert abs(d["mass2d"] / (rho0 * NZ * NR) - 1) < 1e-14
    assert abs(d["mass3d"] / (np.pi * rho0 * NZ * NR ** 2) - 1) < 1e-14
    assert abs(d["momz3d"] / (np.pi * rho0 * U * NZ * NR ** 2) - 1) < 1e-12
    assert abs(d["Eke"] / (0.5 * np.pi * rho0 * (U * U + V * V) * NZ * NR ** 2) - 1) < 1e-12


def test_mass3d_of_a_drop_closed_form():
    """The 3D mass of a tanh drop: the vapour filling the cylinder pi Nr^2 Nz plus
    (rho_l - rho_v) times the liquid indicator's volume 4/3 pi (R^3 + pi^2 R w^2 / 4)
    (first two moments of the sech^2 profile).  Catches a wrong radius in the weight."""
    Nz, Nr, R, w, rl, rv = 96, 48, 15.0, 2.0, 1.9, 0.2
    rho = I.drop(Nz, Nr, 48.0, R, rl, rv, w=w)[0]
    o = O.Oracle(Nz, Nr, tau=1.0, G=0.0)
    d = o.diag(o.init(rho))
    want = rv * np.pi * Nr ** 2 * Nz + (rl - rv) * 4 / 3 * np.pi * (R ** 3 + np.pi ** 2 * R * w ** 2 / 4)
    assert abs(d["mass3d"] / want - 1) < 2e-3


def test_umax_is_the_largest_speed():
    """max |u| = max sqrt(u_z^2 + u_r^2).  Three planted sites: (0.03, 0), (0.025,
    0.025) and (0, 0.031) on a fluid at rest; the answer is 0.025 sqrt 2, which
    neither max |u_z| (0.03), max |u_r| (0.031) nor |u_z| + |u_r| (0.05) gives."""
    o = O.Oracle(NZ, NR, tau=1.0, G=0.0)
    uz, ur = np.zeros((NR, NZ)), np.zeros((NR, NZ))
    uz[3, 4] = 0.03
    uz[7, 11], ur[7, 11] = 0.025, 0.025
    ur[10, 17] = 0.031
    d = o.diag(o.init(np.full((NR, NZ), 1.1), uz, ur))
    assert abs(d["umax"] - 0.025 * np.sqrt(2)) < 1e-15


@pytest.mark.parametrize("R", [9.5, 12.3, 17.81])
def test_r_intercept_of_a_sphere(R):
    """Sec. IV.2: A(t) is the radius where rho crosses (rho_l + rho_v)/2 on the column
    through the drop's centre.  The tanh profile crosses half density exactly at
    d = R, so A = R up to the linear interpolation between the two rows around it
    (at most 0.01 for width 2).  Catches r at j instead of j + 1/2 (an error of
    1/2), interpolating towards the wrong row, or the wrong column."""
    Nz, Nr, rl, rv = 64, 32, 1.93, 0.16
    rho = I.drop(Nz, Nr, 32.0, R, rl, rv)[0]
    o = O.Oracle(Nz, Nr, tau=1.0, G=0.0)
    d = o.diag(o.init(rho), 32.0, R, rl, rv)
    assert abs(d["A"] - R) < 0.01, d["A"]


def test_neck_of_a_thread():
    """The neck (Sec. IV.3) is the smallest interface radius over the columns.  A thread
    R(z) = R0 (1 + eps cos(2 pi z / lambda)) has it at z = lambda / 2, R0 (1 - eps),
    up to the interpolation (0.01 at width 2); the widest column gives R0 (1 + eps).
    Catches a maximum for a minimum, a column offset, or r at j instead of j + 1/2."""
    Nz, Nr, R0, eps, rl, rv = 40, 48, 20.0, 0.15, 1.93, 0.16
    rho = I.thread(Nz, Nr, R0=R0, eps=eps, rho_l=rl, rho_v=rv)[0]
    o = O.Oracle(Nz, Nr, tau=1.0, G=0.0)
    f = o.init(rho)
    d = o.diag(f, 0.0, R0, rl, rv)
    assert abs(d["neck"] - R0 * (1 - eps)) < 0.01, d["neck"]
    assert abs(d["A"] - R0 * (1 + eps)) < 0.01, d["A"]  # column kc = 0 is the widest
    d2 = o.diag(f, Nz / 2, R0, rl, rv)
    assert abs(d2["A"] - d["neck"]) < 1e-12  # the column through z = lambda/2 is the neck


def test_interface_radius_without_a_crossing():
    """A column that never drops below half density reports the lattice height; a
    lattice entirely below it reports the axis (0)."""
    o = O.Oracle(NZ, NR, tau=1.0, G=0.0)
    d = o.diag(o.init(np.full((NR, NZ), 1.9)), 0.0, 1.0, 1.93, 0.16)
    assert d["A"] == NR and d["neck"] == NR
    d = o.diag(o.init(np.full((NR, NZ), 0.2)), 0.0, 1.0, 1.93, 0.16)
    assert d["A"] == 0.0 and d["neck"] == 0.0


def test_pressure_ideal_gas_limit_and_sites():
    """Eq. pressure, p = c_s^2 rho + c_s^2 G psi^2 / 2: at G = 0 the ideal gas
    p = rho / 3.  p_in is read at (kc, row 0), p_out at (kc + Nz/2, row Nr - 1):
    planted densities there give p_in = a/3 and p_out = b/3 exactly.  Catches the
    wrong c_s^2 and the wrong sites."""
    o = O.Oracle(NZ, NR, tau=1.0, G=0.0)
    rho = np.ones((NR, NZ))
    kc = 7
    rho[0, kc], rho[NR - 1, (kc + NZ // 2) % NZ] = 1.7, 0.4
    d = o.diag(o.init(rho), float(kc), 1.0, 2.0, 0.1)
    assert abs(d["p_in"] - 1.7 / 3) < 1e-15
    assert abs(d["p_out"] - 0.4 / 3) < 1e-15
    assert abs(d["dp"] - 1.3 / 3) < 1e-15


def test_pressure_equal_at_the_papers_coexistence_pair():
    """Sec. IV.2 prints the G = -6 coexistence densities 2.65 / 0.075.  A flat
    interface carries no pressure jump, so Eq. pressure must give the liquid and the
    vapour the same p to the printed precision (measured 0.7 %); with the wrong sign
    of G, a missing c_s^2 on the psi^2 term or psi = rho the two differ by O(1)."""
    o = O.Oracle(NZ, NR, tau=1.0, G=-6.0)
    rho = np.full((NR, NZ), 0.075)
    rho[0, 0] = 2.65
    d = o.diag(o.init(rho), 0.0, 1.0, 2.65, 0.075)
    assert d["p_in"] > 0 and d["p_out"] > 0
    assert abs(d["dp"]) < 0.01 * d["p_out"], (d["p_in"], d["p_out"])


def test_a2_of_a_shaped_drop():
    """The quadrupole amplitude a_2 of a drop with surface R(1 + e P_2) is e to first
    order and 0 for a sphere (up to the lattice).  Catches the wrong normalisation,
    the sign of (dz^2 - r^2/2), or the indicator phi taken from rho unscaled."""
    Nz, Nr, R, rl, rv = 96, 48, 16.0, 1.93, 0.16
    o = O.Oracle(Nz, Nr, tau=1.0, G=0.0)
    d0 = o.diag(o.init(I.drop(Nz, Nr, 48.0, R, rl, rv, w=1.0)[0]), 48.0, R, rl, rv)
    assert abs(d0["a2"]) < 2e-3
    for e in (0.02, -0.03):
        d = o.diag(o.init(I.drop(Nz, Nr, 48.0, R, rl, rv, w=1.0, amps=(e,))[0]), 48.0, R, rl, rv)
        assert abs(d["a2"] / e - 1) < 0.06, (e, d["a2"])


def test_bad_counts_planted_sites():
    """'bad' counts the sites whose density is not positive (or whose density or
    velocity is not finite).  At G = 0 no force reaches a neighbour, so two planted
    sites (rho = -1 and rho = 0) count exactly 2; a NaN population makes at least its
    own site bad."""
    o = O.Oracle(NZ, NR, tau=1.0, G=0.0)
    f = o.init(np.ones((NR, NZ)))
    f[:, 2, 3] *= -1.0          # rho = -1
    f[:, 9, 1] = 0.0            # rho = 0
    assert o.diag(f)["bad"] == 2
    g = o.init(np.ones((NR, NZ)))
    assert o.diag(g)["bad"] == 0
    g[0, 5, 6] = np.nan
    assert o.diag(g)["bad"] >= 1


def test_sumS_of_a_uniform_radial_flow():
    """S = -rho u_r / r (Eq. corr_cty_eqn): for uniform rho0 and u_r = V the sum over
    the lattice is -rho0 V Nz sum_j 1/(j + 1/2); with u_r = 0 it vanishes.  (The
    step's own mass budget pins sumS against the change of sum rho as well.)"""
    rho0, V = 0.9, 0.004
    o, f = _uniform(rho0, 0.0, V)
    want = -rho0 * V * NZ * sum(1.0 / (j + 0.5) for j in range(NR))
    assert abs(o.diag(f)["sumS"] / want - 1) < 1e-12
    o, f = _uniform(rho0, 0.01, 0.0)
    assert abs(o.diag(f)["sumS"]) < 1e-15
