"""Dynamic physics pins of the oracle (Sec. IV): the l = 2 oscillation frequency of a
drop against Miller & Scriven (Eq. freq-drop-miller) and the Rayleigh-Plateau
instability of a liquid thread (breakup iff kappa* = 2 pi R_C / lambda < 1, growth
rate against the linear dispersion of a viscous thread).  Reduced sizes so that the
CPU suite stays within minutes."""
import numpy as np
import pytest
from scipy.optimize import curve_fit

import oracle as O
from paper_1310_1871_gb300 import inputs as I


def _flat_gamma(G):
    rl, rv = I.coexistence(G)
    o = O.Oracle(1, 64, tau=1.0, G=G, axisym=0)
    F = o.fields(o.run(o.init(I.slab(1, 64, 32.0, rl, rv)[0]), 20000))
    return -(G / 18) * np.sum(F["Dr"] ** 2) + 0.25 * np.sum(F["Fr"] ** 2 / F["rho"]), rl, rv


def _crossing(values, mid, start):
    """Position (from start) where a decreasing profile crosses mid, linearly interpolated."""
    i = np.argmax(values[start:] < mid) + start
    return (i - 1) + (values[i - 1] - mid) / (values[i - 1] - values[i])


def miller_scriven(gam, R, rl, rv, nu):
    """Eq. freq-drop-miller with equal kinematic viscosities inside and outside."""
    ws = np.sqrt(24 * gam / (R ** 3 * (2 * rv + 3 * rl)))
    al = 25 * nu * rl * rv / (np.sqrt(2) * R * (2 * rv + 3 * rl) * (np.sqrt(nu) * rl + np.sqrt(nu) * rv))
    return ws - 0.5 * al * np.sqrt(ws) + 0.25 * al * al


@pytest.mark.slow
def test_drop_oscillation_frequency():
    """A G = -5 drop (128 x 64, R = 20 with a 0.08 P_2 shape, tau = 0.7) oscillates at the
    Miller-Scriven l = 2 frequency (gamma~ of the flat interface, equilibrium radius and
    densities from the run) to within 8%; measured -5.8%.  (At the paper's size, R ~ 44 at
    G = -6, the GPU test gives -2%; the paper reports ~1%.)  The signal is the difference
    of the polar and equatorial intercepts, which the breathing mode does not move."""
    G, tau, Nz, Nr, R = -5.0, 0.7, 128, 64, 20.0
    gam, rl, rv = _flat_gamma(G)
    o = O.Oracle(Nz, Nr, tau=tau, G=G)
    zc, mid = Nz / 2, 0.5 * (rl + rv)
    f = o.init(I.drop(Nz, Nr, zc, R, rl, rv, amps=(0.08,))[0])
    ts, D, Rm = [], [], []
    for n in range(0, 6000, 20):
        rho = f.sum(0)
        ap = _crossing(rho[0], mid, int(zc)) - zc
        r_eq = _crossing(rho[:, int(zc)], mid, 0) + 0.5
        ts.append(n)
        D.append(ap - r_eq)
        Rm.append((ap * r_eq * r_eq) ** (1 / 3))
        f = o.run(f, 20)
    ts, D = np.array(ts, float), np.array(D)
    Rd = float(np.mean(Rm[len(Rm) // 2:]))
    w_ms = miller_scriven(gam, Rd, rl, rv, (tau - 0.5) / 3)
    model = lambda t, a, b, w, ph, c: a * np.exp(-b * t) * np.sin(w * t + ph) + c
    m = ts > 50
    p, _ = curve_fit(model, ts[m], D[m], p0=[D[m][0] - D[m][-1], 1e-4, w_ms, np.pi / 2, D[m][-1]],
                     maxfev=50000)
    rel = abs(p[2]) / w_ms - 1
    print(f"drop l=2 frequency: fit {abs(p[2]):.4e}, Miller-Scriven {w_ms:.4e}, rel {rel:+.4f}, R_D {Rd:.2f}")
    assert abs(rel) < 0.08, rel
    assert abs(p[2]) * ts[-1] / (2 * np.pi) > 2.5  # several periods were fitted


def _thread_amplitude(lam, R0, Nr, steps, every=50):
    gam, rl, rv = _GAM
    o = O.Oracle(lam, Nr, tau=1.0, G=-5.0)
    f = o.init(I.thread(lam, Nr, R0, 0.02, rl, rv)[0])
    mid = 0.5 * (rl + rv)
    ts, amp = [], []
    for n in range(0, steps, every):
        rho = f.sum(0)
        crest = _crossing(rho[:, 0], mid, 0)
        trough = _crossing(rho[:, lam // 2], mid, 0) if rho[0, lam // 2] > mid else 0.0
        ts.append(n)
        amp.append(0.5 * (crest - trough))
        if trough < 0.25 * R0:
            break
        f = o.run(f, every)
    return np.array(ts, float), np.array(amp), gam, rl


_GAM = None


@pytest.fixture(scope="module", autouse=True)
def _gamma():
    global _GAM
    _GAM = _flat_gamma(-5.0)


@pytest.mark.slow
def test_rayleigh_plateau_breakup_criterion():
    """Sec. IV.3: a thread breaks up iff lambda > 2 pi R_C.  R_0 = 10 (G = -5, tau = 1):
    kappa* = 1.26 (lambda = 50) relaxes back to a cylinder, kappa* = 0.63 (lambda = 100)
    grows to pinch-off."""
    ts, amp, _, _ = _thread_amplitude(50, 10.0, 40, 3000)
    assert amp[-1] < 0.2 * amp[1]
    ts, amp, _, _ = _thread_amplitude(100, 10.0, 40, 12000)
    assert amp[-1] > 2.0 and ts[-1] < 11950  # pinched before the end of the run


@pytest.mark.slow
def test_rayleigh_plateau_growth_rate():
    """Growth rate of a long-wave perturbation (kappa* = 0.31, R_0 = 10, lambda = 200) in
    the linear regime against the dispersion of a viscous thread (Weber 1931, the
    long-wave limit of Rayleigh's with viscosity; Oh ~ 0.2 here): within [0.5, 1.0] of
    it (measured ~0.8 on the GPU at R_0 = 12).  Inviscid Rayleigh would be ~25% larger
    still."""
    lam, R0 = 200, 10.0
    ts, amp, gam, rl = _thread_amplitude(lam, R0, 40, 14000)
    ok = (amp > 3 * amp[0]) & (amp < 0.3 * R0)
    assert ok.sum() > 5
    sigma = np.polyfit(ts[ok], np.log(amp[ok]), 1)[0]
    nu, k = 1.0 / 6.0, 2 * np.pi / lam
    x = k * R0
    weber = np.sqrt(gam / (2 * rl * R0 ** 3) * x * x * (1 - x * x) + 2.25 * nu * nu * k ** 4) - 1.5 * nu * k * k
    print(f"RP growth rate: {sigma:.4e}, viscous (Weber) {weber:.4e}, ratio {sigma / weber:.3f}")
    assert 0.5 < sigma / weber < 1.0, sigma / weber
