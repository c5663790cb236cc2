"""The Laplace test of Sec. IV.1 at radii the oracle cannot reach: static drops of
R = 16 ... 64 (G = -5, tau = 1, FP64 storage) with the paper's velocity-shift forcing and
with the Guo forcing, all in one batch on the GPU.  Delta p from Eq. pressure (inside on
the axis at the centre, outside in the far corner) against 2 gamma / R_D, with R_D the
equatorial interface radius and gamma from the flat-interface tool (gamma~ of Eq. stc for
the shift, gamma of Eq. st for Guo, as Table I pairs them).

Measured (converged: the 30,000- and 40,000-step values agree to 1e-4): the shift
-23.2, -22.5, -22.1, -21.8, -21.6 % for R = 16, 24, 32, 48, 64, levelling off near the 20 %
the paper reports for it; Guo -3.8, -2.6, -2.1, -1.4, -1.2 %, through the paper's 2 % at
R ~ 30 and shrinking with R (a finite-interface-width effect).  Pins: the shift within
-24 % ... -19 % at every radius; Guo within 4 % at every radius, within 2.5 % from R = 32,
decreasing in magnitude with R."""
import numpy as np
import pytest

from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402

RADII = [16, 24, 32, 48, 64]
G = -5.0


def test_laplace_deviation_against_radius():
    gam = {"shift": amlbm.flat_interface(G, axisym=False)["gamma_tilde"],
           "guo": amlbm.flat_interface(G, axisym=False, forcing="guo")["gamma"]}
    rl, rv = I.coexistence(G)
    cases = [(R, fc) for fc in ("shift", "guo") for R in RADII]
    specs, fields, params = [], [], []
    for R, fc in cases:
        Nz, Nr = 4 * R + 16, 2 * R + 8
        specs.append(amlbm.InstanceSpec(Nz, Nr, 1.0, G, forcing=fc))
        fields.append(I.drop(Nz, Nr, Nz / 2, float(R), rl, rv))
        params.append([Nz / 2, float(R), rl, rv])
    b = amlbm.Batch(specs, storage="f64", tile=(32, 8), schedule="fused")
    b.init_all([f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields])
    snaps = []
    for steps in (30000, 10000):  # the interior density of a large drop settles slowly
        b.step(steps)
        d = b.diagnostics_all(np.array(params), as_array=True)
        snaps.append({c: d[q, 10] / (2 * gam[c[1]] / d[q, 6]) - 1 for q, c in enumerate(cases)})
    b.close()
    rel = snaps[-1]
    for s in snaps:
        print("Laplace deviation", {f"{R}/{fc}": round(float(v), 4) for (R, fc), v in s.items()})
    print("gamma", gam)
    for c in cases:
        assert abs(snaps[-1][c] - snaps[-2][c]) < 1e-3, c  # equilibrated
    for R in RADII:
        assert -0.24 < rel[(R, "shift")] < -0.19, (R, rel[(R, "shift")])
        assert abs(rel[(R, "guo")]) < (0.025 if R >= 32 else 0.04), (R, rel[(R, "guo")])
    guo = [abs(rel[(R, "guo")]) for R in RADII]
    assert all(a > b for a, b in zip(guo, guo[1:]))
