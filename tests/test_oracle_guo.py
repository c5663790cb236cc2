"""Pins of the oracle's Guo forcing (Guo, Zheng & Shi 2002), the alternative to the
Shan-Chen velocity shift that Sec. IV.1 compares it with.  The paper prints no
formula for it; the oracle restates the published scheme: f^eq at the hydrodynamic
u, plus (1 - 1/(2 tau)) W_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . F.

What fixes each expected value:
  - an independently written NumPy restatement (8 x 8 grids, 30 steps, 1e-13);
  - exact planar mass conservation (the discrete force has zero zeroth moment);
  - Table I's "Guo" columns, gamma of Eq. st on the flat interface, and their ratio
    to the "SC" columns;
  - the Laplace test of Sec. IV.1: the paper reports a maximum relative error of 2 %
    for the Guo scheme against 20 % for the shift.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I
from tests import np_oracle as NPO


@pytest.mark.parametrize("axisym,wall,src,G,gz", [(1, 0, 0, -5.0, 0.0), (1, 1, 1, -4.7, 1e-4), (0, 0, 0, -5.2, 0.0)])
def test_brute_force_guo_against_numpy_restatement(axisym, wall, src, G, gz):
    Nz = Nr = 8
    rho, uz, ur = I.noisy(Nz, Nr, seed=31 + wall, base=1.2, amp=0.2, uamp=0.02)
    o = O.Oracle(Nz, Nr, tau=0.9, G=G, gz=gz, wall=wall, axisym=axisym, src_mode=src, forcing=O.FORCE_GUO)
    f = o.init(rho, uz, ur)
    g = NPO.equilibrium(rho, uz, ur)
    for _ in range(30):
        g = NPO.step(g, 0.9, G, gz=gz, wall=wall, axisym=axisym, src_mode=src, forcing=1)
    f = o.run(f, 30)
    assert np.abs(f - g).max() <= 1e-13 * np.abs(g).max()


def test_guo_planar_mass_is_exact():
    o = O.Oracle(32, 16, tau=0.8, G=-5.0, axisym=0, forcing=O.FORCE_GUO)
    f = o.init(I.drop(32, 16, 16.0, 6.0)[0])
    m0 = f.sum()
    assert abs(o.run(f, 300).sum() / m0 - 1) < 1e-13


def _flat(G, axisym, forcing):
    rl, rv = I.coexistence(G)
    o = O.Oracle(1, 64, tau=1.0, G=G, axisym=axisym, forcing=forcing)
    F = o.fields(o.run(o.init(I.slab(1, 64, 32.0, rl, rv)[0]), 20000))
    gam = -(G / 18) * np.sum(F["Dr"] ** 2)
    return gam, gam + 0.25 * np.sum(F["Fr"] ** 2 / F["rho"])


@pytest.mark.parametrize("G,sc,guo2d,guoax", [(-4.5, 0.0220, 0.0135, 0.0136), (-5.0, 0.0579, 0.0376, 0.0378),
                                              (-5.5, 0.0995, 0.0681, 0.0683)])
def test_table_I_guo_columns(G, sc, guo2d, guoax):
    """gamma (Eq. st) of the Guo flat interface within 6 % of Table I (measured: 0.6, 2.8,
    5.1 % low in 2D; 1.1, 3.1, 5.5 % axisymmetric), and the Guo / SC ratio within 4 %
    of the printed ratio (measured 0.3, 1.6, 3.1 %).  The deviation grows with |G|;
    the paper does not print the Guo scheme's densities or profile to compare."""
    g2, _ = _flat(G, 0, O.FORCE_GUO)
    ga, _ = _flat(G, 1, O.FORCE_GUO)
    _, sc_t = _flat(G, 0, O.FORCE_SHIFT)
    assert abs(g2 / guo2d - 1) < 0.06
    assert abs(ga / guoax - 1) < 0.06
    assert abs((g2 / sc_t) / (guo2d / sc) - 1) < 0.04


@pytest.mark.slow
def test_laplace_guo_much_closer_than_shift():
    """Sec. IV.1: with the Guo forcing the in-out pressure difference of a static drop
    (G = -5, tau = 1, Eq. pressure) is far closer to 2 gamma / R than with the shift.
    Against the printed gamma = 0.0378 the deviation is 5.5-8.3 % at these small radii
    (the shift's, in the SC Laplace test, 23.5-26 %), shrinking with R; at R = 16-64 on
    the GPU (test_gpu_laplace_scale.py, each scheme's own gamma) the deviations come down
    to the paper's figures: Guo 3.8 -> 1.2 %, the shift 23 -> 21.6 %."""
    gam = 0.0378
    errs = []
    for (Nz, Nr, R) in [(64, 32, 10), (64, 32, 14), (128, 64, 24)]:
        rl, rv = I.coexistence(-5.0)
        o = O.Oracle(Nz, Nr, tau=1.0, G=-5.0, forcing=O.FORCE_GUO)
        d = o.diag(o.run(o.init(I.drop(Nz, Nr, Nz / 2, R, rl, rv)[0]), 4000), Nz / 2, R, rl, rv)
        errs.append(d["dp"] / (2 * gam / d["A"]) - 1)
    errs = np.array(errs)
    assert (errs < 0).all() and (errs > -0.09).all()
    assert errs[-1] > errs[0]  # closer for the larger drop
