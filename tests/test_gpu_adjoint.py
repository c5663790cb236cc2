"""The hand-written discrete adjoint (amlbm_adjoint) against the oracle's complex-step
derivative of the same discrete run and against central finite differences of the GPU
forward run.  Bar: 1e-6 relative (FP64); the FP32 adjoint's error is measured."""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402


def oracle_grad(Nz, Nr, T, amps, tau, G, wall=0, gz=0.0, axisym=1, kind=0, kstar=0, zc=None, R=7.0):
    o = O.Oracle(Nz, Nr, tau=tau, G=G, wall=wall, gz=gz, axisym=axisym)
    zc = Nz / 2 if zc is None else zc
    return o.grad(T, zc, R, 2.0, 1.93, 0.16, amps, kind=kind, kstar=kstar)


def gpu_grad(Nz, Nr, T, amps, tau, G, wall="freeslip", gz=0.0, axisym=True, kind="a2sq", kstar=0,
             storage="f64", ckpt=None, zc=None, R=7.0):
    lat = amlbm.Lattice(Nz, Nr, tau=tau, G=G, wall=wall, gz=gz, axisym=axisym, storage=storage)
    zc = Nz / 2 if zc is None else zc
    out = lat.adjoint(T, amps, zc, R, objective=kind, kstar=kstar, ckpt_every=ckpt)
    lat.close()
    return out


def rel_err(g_gpu, g_ref):
    return np.abs(np.asarray(g_gpu) - np.asarray(g_ref)).max() / np.abs(g_ref).max()


def comp_err(g_gpu, g_ref, floor=1e-3):
    """Largest per-component relative error, each component against its own size
    (with a floor of `floor` times the largest component, so that a component that
    is zero to rounding is held to an absolute bar)."""
    g_gpu, g_ref = np.asarray(g_gpu), np.asarray(g_ref)
    den = np.maximum(np.abs(g_ref), floor * np.abs(g_ref).max())
    return float((np.abs(g_gpu - g_ref) / den).max())


@pytest.mark.parametrize("case", [
    dict(),                                   # free-slip drop, a2^2
    dict(wall=1, gz=2e-5, tau=0.8),           # no-slip wall, body force
    dict(axisym=0, G=-4.8),                   # planar model
    dict(kind=1, kstar=9, tau=0.95),          # neck objective on column 9
])
def test_fp64_adjoint_matches_oracle_complex_step(case):
    Nz, Nr, T = 32, 16, 30
    amps = I.legendre_amplitudes(3, 0.03, seed=11)
    tau, G = case.get("tau", 0.9), case.get("G", -5.0)
    wall, gz, axisym, kind, kstar = (case.get("wall", 0), case.get("gz", 0.0), case.get("axisym", 1),
                                     case.get("kind", 0), case.get("kstar", 0))
    J_ref, g_ref = oracle_grad(Nz, Nr, T, amps, tau, G, wall, gz, axisym, kind, kstar)
    J, dG, dT, dA = gpu_grad(Nz, Nr, T, amps, tau, G, ("freeslip", "noslip")[wall], gz, bool(axisym),
                             ("a2sq", "neck")[kind], kstar, ckpt=7)
    g = np.concatenate([[dG, dT], dA])
    print(case, "J", J, J_ref, "rel grad err", rel_err(g, g_ref), "per component", comp_err(g, g_ref))
    assert abs(J / J_ref - 1) < 1e-11
    assert rel_err(g, g_ref) < 1e-6
    assert comp_err(g, g_ref) < 1e-6


def test_fp64_adjoint_matches_gpu_finite_differences():
    Nz, Nr, T, h = 40, 20, 40, 1e-6
    amps = I.legendre_amplitudes(2, 0.03, seed=3)
    J, dG, dT, dA = gpu_grad(Nz, Nr, T, amps, 0.85, -5.0, ckpt=8, R=8.0)

    def Jf(G=-5.0, tau=0.85, a=amps):
        lat = amlbm.Lattice(Nz, Nr, tau=tau, G=G)
        v = lat.objective(T, a, Nz / 2, 8.0)
        lat.close()
        return v

    fd = [(Jf(G=-5 + h) - Jf(G=-5 - h)) / (2 * h), (Jf(tau=0.85 + h) - Jf(tau=0.85 - h)) / (2 * h)]
    for m in range(len(amps)):
        ap, am = amps.copy(), amps.copy()
        ap[m] += h
        am[m] -= h
        fd.append((Jf(a=ap) - Jf(a=am)) / (2 * h))
    g = np.concatenate([[dG, dT], dA])
    assert rel_err(g, fd) < 1e-6
    assert comp_err(g, fd) < 1e-6


def test_checkpoint_spacing_does_not_change_the_gradient():
    amps = I.legendre_amplitudes(2, 0.03, seed=5)
    a = gpu_grad(32, 16, 25, amps, 0.9, -5.0, ckpt=1)
    b = gpu_grad(32, 16, 25, amps, 0.9, -5.0, ckpt=25)
    c = gpu_grad(32, 16, 25, amps, 0.9, -5.0, ckpt=6)
    for x, y in ((a, b), (a, c)):
        assert x[0] == y[0] and x[1] == y[1] and x[2] == y[2] and np.array_equal(x[3], y[3])


def test_fp32_adjoint_error_against_oracle():
    """FP32 forward and adjoint (FP64 parameter accumulation): the measured relative
    gradient error is printed and bounded at 1e-2."""
    Nz, Nr, T = 64, 32, 100
    amps = I.legendre_amplitudes(4, 0.02, seed=2024)
    J_ref, g_ref = oracle_grad(Nz, Nr, T, amps, 1.0, -5.0, R=12.0)
    J, dG, dT, dA = gpu_grad(Nz, Nr, T, amps, 1.0, -5.0, storage="f32", R=12.0)
    g = np.concatenate([[dG, dT], dA])
    e = rel_err(g, g_ref)
    print("fp32 adjoint rel err", e, "J rel", abs(J / J_ref - 1))
    assert e < 1e-2


def test_autograd_function():
    run = amlbm.DropRun(Nz=32, Nr=16, T=20, zc=16.0, R=7.0)
    amps = torch.tensor(I.legendre_amplitudes(3, 0.03, seed=1), dtype=torch.float64, requires_grad=True)
    G = torch.tensor(-5.0, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    J = amlbm.drop_objective(amps, G, tau, run)
    J.backward()
    J_ref, g_ref = oracle_grad(32, 16, 20, amps.detach().numpy(), 0.9, -5.0)
    assert abs(J.item() / J_ref - 1) < 1e-11
    g = np.concatenate([[G.grad.item(), tau.grad.item()], amps.grad.numpy()])
    assert rel_err(g, g_ref) < 1e-6
