"""The workload configurations at their full sizes on the GPU, against the FP64 form
and the closed forms the paper compares with:

- the oscillating drop (256 x 128, R = 40, 5 % P_2 shape, G = -5) at tau = 1.0 for
  20,000 steps: l = 2 period against Miller-Scriven (Eq. freq-drop-miller, Sec. IV.2)
  with the surface tension from the flat-interface tool, FP64 and FP32 storage;
- the capillary threads (lambda x 128, R_0 = 25, 10 % perturbation, Sec. IV.3) at
  lambda = 400 and 800, tau = 1.0 and 0.65: pinch-off time of FP32 storage against
  FP64; lambda = 200 (kappa* = 0.79) run to the 50,000-step limit; tau = 0.6, where
  the scheme itself is unstable with this initial state (the FP64 oracle goes
  non-finite within 500 steps at lambda = 400 and 800), checked to fail the same way;
- the differentiable drop (512 x 128, R = 48, 16 Legendre amplitudes, J = a_2(T)^2,
  T = 10,000, checkpoints every 100): the FP64 adjoint's dJ/dG, dJ/dtau and two
  amplitude derivatives against fourth-order central differences of the FP64
  forward run, and the FP32 adjoint's error against the same differences.

Every run prints what it measured."""
import numpy as np
import pytest
from scipy.optimize import curve_fit

from paper_1310_1871_gb300 import inputs as I
from tests.test_oracle_physics import _crossing, miller_scriven

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402

# The accuracy target on the oscillation period and the pinch-off time of the FP32 form (0.5 %).
PHYS_TOL = 5e-3


def _drop_run(storage, tau=1.0, steps=20000, every=20):
    """Polar minus equatorial interface intercept D(t) of the 256 x 128 drop, and the
    volume-equivalent radius (mean over the second half of the run)."""
    Nz, Nr, R, zc = 256, 128, 40.0, 128.0
    rl, rv = I.coexistence(-5.0)
    lat = amlbm.Lattice(Nz, Nr, tau=tau, G=-5.0, storage=storage)
    lat.init_fields(*I.drop(Nz, Nr, zc, R, rl, rv, amps=(0.05,)))
    mid = 0.5 * (rl + rv)
    ts, D, Rm = [], [], []
    for n in range(0, steps, every):
        rho, _, _ = lat.read()
        ap = _crossing(rho[0], mid, int(zc)) - zc
        r_eq = _crossing(rho[:, int(zc)], mid, 0) + 0.5
        ts.append(n)
        D.append(ap - r_eq)
        Rm.append((ap * r_eq * r_eq) ** (1 / 3))
        lat.step(every)
    lat.close()
    return np.array(ts, float), np.array(D), float(np.mean(Rm[len(Rm) // 2:]))


def _fit_omega(ts, D, w0):
    model = lambda t, a, b, w, ph, c: a * np.exp(-b * t) * np.sin(w * t + ph) + c
    m = ts > 50
    p, _ = curve_fit(model, ts[m], D[m], p0=[D[m][0] - D[m][-1], 3e-4, w0, np.pi / 2, D[m][-1]],
                     maxfev=50000)
    return abs(p[2])


def test_oscillating_drop_tau1_period():
    """256 x 128 drop at tau = 1.0, 20,000 steps.  FP32 storage gives the FP64 period
    within 0.5 % (measured 6.6e-6).  The FP64 frequency lies 5.5 % below Miller-Scriven
    with gamma~ of the flat-interface tool; the bound is 6 %.  The paper reports ~1 %
    for its drop (G = -6, R ~ 45), where this build measures -2.1 %: at G = -5 the
    interface (4-5 sites) is a larger fraction of R = 40, and the velocity shift's
    curvature deficit (the Laplace test's -22 %) lowers the restoring pressure."""
    gam = amlbm.flat_interface(-5.0)["gamma_tilde"]
    rl, rv = I.coexistence(-5.0)
    nu = (1.0 - 0.5) / 3
    ts, D64, R64 = _drop_run("f64")
    w_ms = miller_scriven(gam, R64, rl, rv, nu)
    w64 = _fit_omega(ts, D64, w_ms)
    ts, D32, _ = _drop_run("f32")
    w32 = _fit_omega(ts, D32, w_ms)
    rel_ms = w64 / w_ms - 1
    rel32 = w64 / w32 - 1  # period ratio T32 / T64 - 1
    print(f"C2 tau=1.0: R_D {R64:.2f}, gamma~ {gam:.5f}, period FP64 {2 * np.pi / w64:.1f} "
          f"(Miller-Scriven {2 * np.pi / w_ms:.1f}, omega rel {rel_ms:+.4f}), "
          f"FP32 period rel to FP64 {rel32:+.2e}, max |D32 - D64| {np.abs(D32 - D64).max():.2e}")
    assert abs(rel32) < PHYS_TOL
    assert abs(rel_ms) < 0.06


def _pinch(storage, lam, tau, limit=50000, every=20, eps=0.1):
    """Step at which the neck first falls below R_0/5 (linear interpolation between
    samples), or None when it does not by `limit`; and the last neck radius."""
    Nr, R0 = 128, 25.0
    rl, rv = I.RHO_L_G5, I.RHO_V_G5
    lat = amlbm.Lattice(lam, Nr, tau=tau, G=-5.0, storage=storage)
    lat.init_fields(*I.thread(lam, Nr, R0, eps))
    prev_t = prev_n = None
    try:
        for n in range(0, limit + 1, every):
            d = lat.diagnostics(zc=lam / 2, R=R0, rho_l=rl, rho_v=rv, check=False)
            if d["neck"] < 0.2 * R0:
                return prev_t + (n - prev_t) * (prev_n - 0.2 * R0) / (prev_n - d["neck"]), d["neck"]
            prev_t, prev_n = n, d["neck"]
            if n < limit:
                lat.step(every)
        return None, prev_n
    finally:
        lat.close()


@pytest.mark.parametrize("lam,tau", [(400, 1.0), (800, 1.0), (400, 0.65), (800, 0.65)])
def test_thread_pinch_off_fp32_vs_fp64(lam, tau):
    """The thread pinches off within 50,000 steps and FP32 storage gives the FP64
    pinch-off time within 0.5 %."""
    t64, _ = _pinch("f64", lam, tau)
    t32, _ = _pinch("f32", lam, tau)
    print(f"C3 lambda={lam} tau={tau}: pinch-off FP64 {t64}, FP32 {t32}")
    assert t64 is not None and t32 is not None
    assert abs(t32 / t64 - 1) < PHYS_TOL


@pytest.mark.parametrize("lam", [400, 800])
def test_thread_tau06_is_unstable_as_in_the_oracle(lam):
    """The viscosity sweep's tau = 0.6 (nu = 1/30) at G = -5 with the tanh initial
    state: the FP64 oracle's state goes non-finite between steps 400 and 500 (the
    initial spurious currents, max |u| = 0.10, grow to 0.47 by step 400).  Both GPU
    forms fail within 600 steps as well.  The viscosity sweep runs at tau = 0.65
    instead (test above), the nearest value at which the oracle stays finite (0.65
    and 0.7 checked over 3,000 steps)."""
    rl, rv = I.RHO_L_G5, I.RHO_V_G5
    for storage in ("f64", "f32"):
        lat = amlbm.Lattice(lam, 128, tau=0.6, G=-5.0, storage=storage)
        lat.init_fields(*I.thread(lam, 128, 25.0, 0.1))
        d0 = lat.diagnostics(zc=lam / 2, R=25.0, rho_l=rl, rho_v=rv)
        lat.step(600)
        d = lat.diagnostics(zc=lam / 2, R=25.0, rho_l=rl, rho_v=rv, check=False)
        lat.close()
        print(f"tau=0.6 lambda={lam} {storage}: bad sites after 600 steps {d['bad']:.0f}, "
              f"initial max |u| {d0['umax']:.3f}")
        assert d0["bad"] == 0 and d["bad"] > 0


def test_thread_lambda200_to_the_step_limit():
    """lambda = 200 (kappa* = 2 pi 25 / 200 = 0.79 < 1 by the paper's criterion) does
    not pinch off within the 50,000-step limit in this scheme, in FP64 or FP32: the
    diffuse interface (4-5 sites at G = -5) moves the effective cutoff of an R_0 = 25
    thread below kappa* = 0.79 (the paper's threads have R_C = 80).  The two forms end
    at the same neck radius within 0.5 %."""
    t64, n64 = _pinch("f64", 200, 1.0)
    t32, n32 = _pinch("f32", 200, 1.0)
    print(f"C3 lambda=200 tau=1.0: pinch FP64 {t64}, FP32 {t32}; neck at 50,000 steps FP64 {n64:.3f}, "
          f"FP32 {n32:.3f} (R_0 = 25)")
    assert t64 is None and t32 is None
    assert abs(n32 / n64 - 1) < PHYS_TOL


def test_differentiable_drop_adjoint_vs_central_differences():
    """512 x 128, R = 48, 16 amplitudes ~ N(0, 0.02^2) (seed 2024), J = a_2(T)^2,
    T = 10,000, checkpoints every 100.  FP64 adjoint against fourth-order central
    differences of the FP64 forward run, component by component, for dJ/dG, dJ/dtau
    and the P_2 and P_4 amplitudes: 1e-6 relative.  The FP32 adjoint's error against
    the same differences is printed (bounded at 5e-2)."""
    Nz, Nr, T, R, zc = 512, 128, 10000, 48.0, 256.0
    amps = I.legendre_amplitudes(16, 0.02, seed=2024)
    lat = amlbm.Lattice(Nz, Nr, tau=1.0, G=-5.0, storage="f64")
    J, dG, dT, dA = lat.adjoint(T, amps, zc, R, ckpt_every=100)

    def Jf(G=-5.0, tau=1.0, a=amps):
        lat2 = amlbm.Lattice(Nz, Nr, tau=tau, G=G, storage="f64")
        v = lat2.objective(T, a, zc, R)
        lat2.close()
        return v

    def d4(fun, h):
        return (8 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12 * h)

    fd = [d4(lambda h: Jf(G=-5.0 + h), 1e-4), d4(lambda h: Jf(tau=1.0 + h), 1e-4)]
    for m in (0, 2):
        def fa(h, m=m):
            a = amps.copy()
            a[m] += h
            return Jf(a=a)
        fd.append(d4(fa, 1e-4))
    adj = np.array([dG, dT, dA[0], dA[2]])
    fd = np.array(fd)
    rel = np.abs(adj - fd) / np.abs(fd)
    lat32 = amlbm.Lattice(Nz, Nr, tau=1.0, G=-5.0, storage="f32")
    J32, dG32, dT32, dA32 = lat32.adjoint(T, amps, zc, R, ckpt_every=100)
    lat32.close()
    lat.close()
    rel32 = np.abs(np.array([dG32, dT32, dA32[0], dA32[2]]) - fd) / np.abs(fd)
    print(f"C5: J {J:.6e}; dJ/d(G, tau, a2, a4) adjoint {adj}, FD {fd}; FP64 rel {rel}; "
          f"FP32 rel {rel32} (J32 rel {abs(J32 / J - 1):.2e})")
    assert np.all(rel < 1e-6), rel
    assert np.all(rel32 < 5e-2), rel32
