"""Physics of the CUDA path at the paper's sizes (FP64 storage), against the closed
forms the paper compares with: the Miller-Scriven l = 2 drop frequency
(Eq. freq-drop-miller) and the Rayleigh-Plateau breakup criterion with the growth rate
of a viscous thread."""
import numpy as np
import pytest
from scipy.optimize import curve_fit

from paper_1310_1871_gb300 import inputs as I
from tests.test_oracle_physics import _crossing, _flat_gamma, miller_scriven

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402


def test_drop_frequency_at_paper_size():
    """Sec. IV.2 setup: 320 x 128, G = -6, tau = 1, drop on the axis at z = 160 with a
    0.1 P_2 shape, R = 45.  The fitted frequency is within 3% of Miller-Scriven
    (measured -2.1%; the paper reports ~1%)."""
    G, tau, Nz, Nr, R = -6.0, 1.0, 320, 128, 45.0
    gam, rl, rv = _flat_gamma(G)
    lat = amlbm.Lattice(Nz, Nr, tau=tau, G=G, storage="f64")
    zc, mid = Nz / 2, 0.5 * (rl + rv)
    lat.init_fields(*I.drop(Nz, Nr, zc, R, rl, rv, amps=(0.1,)))
    ts, D, Rm = [], [], []
    for n in range(0, 9000, 20):
        rho, _, _ = lat.read()
        ap = _crossing(rho[0], mid, int(zc)) - zc
        r_eq = _crossing(rho[:, int(zc)], mid, 0) + 0.5
        ts.append(n)
        D.append(ap - r_eq)
        Rm.append((ap * r_eq * r_eq) ** (1 / 3))
        lat.step(20)
    lat.close()
    ts, D = np.array(ts, float), np.array(D)
    Rd = float(np.mean(Rm[len(Rm) // 2:]))
    w_ms = miller_scriven(gam, Rd, rl, rv, (tau - 0.5) / 3)
    model = lambda t, a, b, w, ph, c: a * np.exp(-b * t) * np.sin(w * t + ph) + c
    m = ts > 50
    p, _ = curve_fit(model, ts[m], D[m], p0=[D[m][0] - D[m][-1], 1e-4, w_ms, np.pi / 2, D[m][-1]],
                     maxfev=50000)
    rel = abs(p[2]) / w_ms - 1
    print(f"paper-size drop: R_D {Rd:.2f}, fit {abs(p[2]):.4e}, Miller-Scriven {w_ms:.4e}, rel {rel:+.4f}")
    assert abs(rel) < 0.03


@pytest.mark.parametrize("lam,breaks", [(120, False), (400, True)])
def test_thread_breakup_at_workload_size(lam, breaks):
    """The capillary-thread workload (R_0 = 25, 128 rows, G = -5, tau = 1): kappa* = 1.31
    (lambda = 120) relaxes, kappa* = 0.39 (lambda = 400) pinches off, growing at 0.5-1.0
    of the viscous (Weber) long-wave rate in the linear regime."""
    gam, rl, rv = _flat_gamma(-5.0)
    R0, Nr = 25.0, 128
    lat = amlbm.Lattice(lam, Nr, tau=1.0, G=-5.0, storage="f64")
    lat.init_fields(*I.thread(lam, Nr, R0, 0.02, rl, rv))
    mid = 0.5 * (rl + rv)
    ts, amp = [], []
    for n in range(0, 30000, 100):
        rho, _, _ = lat.read()
        crest = _crossing(rho[:, 0], mid, 0)
        trough = _crossing(rho[:, lam // 2], mid, 0) if rho[0, lam // 2] > mid else 0.0
        ts.append(n)
        amp.append(0.5 * (crest - trough))
        if trough < 0.25 * R0:
            break
        lat.step(100)
    lat.close()
    ts, amp = np.array(ts, float), np.array(amp)
    if not breaks:
        assert amp[-1] < 0.2 * amp[1] and ts[-1] == 29900
        return
    assert ts[-1] < 29900
    ok = (amp > 3 * amp[0]) & (amp < 0.3 * R0)
    sigma = np.polyfit(ts[ok], np.log(amp[ok]), 1)[0]
    nu, k = 1.0 / 6.0, 2 * np.pi / lam
    x = k * R0
    weber = np.sqrt(gam / (2 * rl * R0 ** 3) * x * x * (1 - x * x) + 2.25 * nu * nu * k ** 4) - 1.5 * nu * k * k
    print(f"thread lambda={lam}: pinch at {ts[-1]:.0f} steps, sigma {sigma:.4e}, Weber {weber:.4e}, ratio {sigma / weber:.3f}")
    assert 0.5 < sigma / weber < 1.0
