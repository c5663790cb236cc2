"""Pins of the oracle's differentiable pieces: the shape-perturbed drop (the map from
Legendre amplitudes to the initial density), the two objectives, and the complex-step
derivative of the whole discrete run (the reference for the GPU adjoint)."""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I


def test_drop_volume_closed_form():
    """The liquid indicator of an unperturbed tanh drop has the 3D volume
    4/3 pi (R^3 + pi^2 R w^2 / 4) (first two moments of the sech^2 profile)."""
    Nz, Nr, R, w = 96, 48, 15.0, 2.0
    rho = O.drop_rho(Nz, Nr, 48.0, R, w, 1.0, 0.0, np.zeros(3))
    r = (np.arange(Nr) + 0.5)[:, None]
    V = np.sum(2 * np.pi * r * rho)
    assert abs(V / (4 / 3 * np.pi * (R ** 3 + np.pi ** 2 * R * w ** 2 / 4)) - 1) < 2e-3


def test_drop_surface_follows_legendre_shape():
    """With an l = 2 amplitude e the interface sits at R(1 + e) on the axis and at
    R(1 - e/2) in the equatorial plane (P_2(1) = 1, P_2(0) = -1/2)."""
    Nz, Nr, R, e = 96, 48, 20.0, 0.1
    rho = O.drop_rho(Nz, Nr, 48.0, R, 2.0, 1.0, 0.0, np.array([e]))
    # half-density crossing along the axis row and along the column z = zc
    row = rho[0]
    k = np.where(row[48:] < 0.5)[0][0] + 48
    z_cross = (k - 1) + (row[k - 1] - 0.5) / (row[k - 1] - row[k])
    col = rho[:, 48]
    j = np.where(col < 0.5)[0][0]
    r_cross = (j - 0.5) + (col[j - 1] - 0.5) / (col[j - 1] - col[j])
    assert abs((z_cross - 48.0) - R * (1 + e)) < 0.05
    assert abs(r_cross - R * (1 - e / 2)) < 0.05


def test_quadrupole_objective_measures_the_amplitude():
    """a_2 of a drop with surface R(1 + e P_2) is e to first order (J = a_2^2), and a
    sphere has a_2 = 0 up to the lattice."""
    Nz, Nr, R = 96, 48, 16.0
    J0 = O.objective(0, O.drop_rho(Nz, Nr, 48.0, R, 1.0, 1.0, 0.0, np.zeros(1)), 48.0, R, 1.0, 0.0)
    assert np.sqrt(J0) < 2e-3
    for e in (0.01, 0.03):
        J = O.objective(0, O.drop_rho(Nz, Nr, 48.0, R, 1.0, 1.0, 0.0, np.array([e])), 48.0, R, 1.0, 0.0)
        assert abs(np.sqrt(J) / e - 1) < 0.06


def test_neck_objective_of_a_cylinder():
    """r_n = sqrt(2 sum_j r_j phi) of a liquid cylinder of radius R0 with a tanh wall
    of width w is sqrt(R0^2 + pi^2 w^2 / 12)."""
    rho, _, _ = I.thread(32, 64, R0=20.0, eps=0.0, rho_l=1.0, rho_v=0.0, w=2.0)
    rn = O.objective(1, rho, 0.0, 1.0, 1.0, 0.0, kstar=5)
    assert abs(rn / np.sqrt(20.0 ** 2 + np.pi ** 2 * 4 / 12) - 1) < 1e-3


@pytest.mark.parametrize("kind", [0, 1])
def test_complex_step_gradient_matches_central_differences(kind):
    """The complex-step derivative (Squire & Trapp) of drop_rho -> f^eq -> T steps -> J
    with respect to G, tau and the amplitudes equals central finite differences of the
    real-valued run to 1e-6 relative."""
    Nz, Nr, T, h = 32, 16, 30, 1e-6
    amps = I.legendre_amplitudes(3, 0.03, seed=7)
    kw = dict(kind=kind, kstar=16) if kind else dict(kind=kind)

    def J(G=-5.0, tau=0.9, a=amps):
        return O.Oracle(Nz, Nr, tau=tau, G=G).grad(T, 16.0, 7.0, 2.0, 1.93, 0.16, a, with_grad=False,
                                                   **kw)[0]

    J0, g = O.Oracle(Nz, Nr, tau=0.9, G=-5.0).grad(T, 16.0, 7.0, 2.0, 1.93, 0.16, amps, **kw)
    assert abs(J0 - J()) <= 1e-14 * abs(J0)
    fd = [(J(G=-5 + h) - J(G=-5 - h)) / (2 * h), (J(tau=0.9 + h) - J(tau=0.9 - h)) / (2 * h)]
    for m in range(len(amps)):
        ap, am = amps.copy(), amps.copy()
        ap[m] += h
        am[m] -= h
        fd.append((J(a=ap) - J(a=am)) / (2 * h))
    fd = np.array(fd)
    assert np.all(np.abs(fd - g) <= 1e-6 * np.abs(g).max())
