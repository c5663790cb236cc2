"""Parity of the bounded-domain forms (no-slip z walls, inlet and outlet rows,
lattices off the axis; Sec. II.E, Sec. III.2) between the CUDA path, through the
C ABI, and the FP64 CPU oracle.

Bars as for the periodic lattice: FP64 storage to a max relative error of 1e-11
(f pointwise, rho pointwise, u normwise: max|du| / max|u|); FP32 storage to 1e-4
relative in rho after 200 steps; every tiling, and a batch that mixes bounded and
periodic lattices, bit-identical to a lone run.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402

ORC_WALL = {"freeslip": O.WALL_FREESLIP, "noslip": O.WALL_NOSLIP, "outlet": O.WALL_OUTLET}


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


class Case:
    """A bounded lattice: its oracle and its CUDA instance spec."""

    def __init__(self, Nz, Nr, tau=0.9, G=-5.0, wall="noslip", z_bc="noslip", r_lo="axis", r_off=0.0,
                 rho_out=1.0, inlet=None, src="local", gz=0.0):
        self.Nz, self.Nr = Nz, Nr
        self.inlet = inlet if inlet is not None else (np.zeros(Nz), np.zeros(Nz))
        self.o = O.Oracle(Nz, Nr, tau=tau, G=G, gz=gz, wall=ORC_WALL[wall],
                          src_mode=O.SRC_LINK if src == "link" else O.SRC_LOCAL,
                          zbc=O.Z_NOSLIP if z_bc == "noslip" else O.Z_PERIODIC,
                          rlo=O.RLO_INLET if r_lo == "inlet" else O.RLO_AXIS, r_off=r_off,
                          rho_out=rho_out, inlet=self.inlet)
        self.spec = amlbm.InstanceSpec(Nz, Nr, tau, G, 1.0, wall, True, src, gz, 1.0, "default",
                                       "nearest", z_bc, r_lo, r_off, rho_out)

    def gpu(self, fields, steps, storage="f64", tile=None, schedule="auto", extra=()):
        """Run on the GPU (alone, or as instance 0 of a batch with `extra` specs)."""
        b = amlbm.Batch([self.spec] + [s for s, _ in extra], storage=storage, tile=tile,
                        schedule=schedule)
        b.init_fields(0, *fields)
        for q, (_, fx) in enumerate(extra):
            b.init_fields(q + 1, *fx)
        if self.spec.r_lo == "inlet":
            b.set_inlet(0, *self.inlet)
        b.step(steps)
        out = b.read_f(0), b.read(0)
        b.close()
        return out

    def oracle(self, fields, steps):
        f = self.o.run(self.o.init(*fields), steps)
        return f, self.o.fields(f)


def check_fp64(gpu, ref, tol=1e-11):
    """u = (sum_i c_i f_i + F/2) / rho is a difference of populations, so its rounding
    floor is that of the populations: a flow far slower than max f (the flow between
    discs, |u| ~ 4e-4 against f ~ 0.4) is held to tol times max f instead of max |u|."""
    (f_gpu, (rho, uz, ur)), (f_ref, F) = gpu, ref
    assert np.isfinite(f_gpu).all()
    assert rel(f_gpu, f_ref) < tol
    assert np.abs(rho / F["rho"] - 1).max() < tol
    scale = max(np.abs(F["uz"]).max(), np.abs(F["ur"]).max(), np.abs(f_ref).max())
    assert max(np.abs(uz - F["uz"]).max(), np.abs(ur - F["ur"]).max()) / scale < tol


def disc_case(H=32, R_i=9.5, Nr=111, U2=3.93e-4):
    inp = I.disc_flow(H, R_i, Nr, U2)
    return Case(H, Nr, tau=1.0, G=0.0, wall="outlet", z_bc="noslip", r_lo="inlet", r_off=inp.r_off,
                inlet=(np.zeros(H), inp.u_in)), inp


def test_fp64_disc_flow_paper_size_1000_steps():
    """Sec. III.2 at the paper's 32 x 120 (111 rows from R_i = 9.5), 1000 steps."""
    c, inp = disc_case()
    fields = inp.fields()
    check_fp64(c.gpu(fields, 1000), c.oracle(fields, 1000))


def test_fp64_disc_flow_steady_state_against_middleman():
    """The GPU run to steady state (16,000 steps) is the oracle's steady state, and
    within 4 % of U_2 of Middleman's profile (the oracle's own pin)."""
    c, inp = disc_case()
    fields = inp.fields()
    (f_gpu, (rho, uz, ur)), (f_ref, F) = c.gpu(fields, 16000), c.oracle(fields, 16000)
    assert rel(f_gpu, f_ref) < 1e-10
    assert np.abs(ur - inp.analytic()).max() / inp.U2 < 0.04
    assert np.abs(uz).max() < 0.005 * inp.U2


@pytest.mark.parametrize("kw", [
    dict(wall="noslip", z_bc="noslip"),                                   # closed box on the axis
    dict(wall="freeslip", z_bc="noslip", src="link", gz=1e-3),            # z walls, link source, gravity
    dict(wall="outlet", z_bc="periodic", r_lo="inlet", r_off=3.0, G=-4.8,  # two-phase inflow / outflow
         rho_out=1.05),
    dict(wall="noslip", z_bc="noslip", r_lo="inlet", r_off=2.0, G=-4.6, src="link")])
def test_fp64_bounded_forms(kw):
    """Every bounded form with a two-phase state, 300 steps, several tiles with a
    ragged tail in z and r (70 x 45, tiles of 32 x 8)."""
    Nz, Nr = 70, 45
    inlet = (0.01 * np.sin(np.arange(Nz) / 5.0), 0.02 + 0.005 * np.cos(np.arange(Nz) / 7.0))
    c = Case(Nz, Nr, inlet=inlet, **kw)
    if kw.get("r_lo") == "inlet":
        fields = I.noisy(Nz, Nr, seed=7, base=1.0, amp=0.05, uamp=0.01)
    else:
        fields = I.drop(Nz, Nr, 34.5, 12.0, amps=(0.08,))
    check_fp64(c.gpu(fields, 300, tile=(32, 8)), c.oracle(fields, 300))


@pytest.mark.parametrize("Nz,Nr", [(4, 16), (5, 6), (33, 7)])
def test_fp64_bounded_small_sizes(Nz, Nr):
    """The smallest lattices the bounded forms take (Nz = 4 between walls, Nr = 6 with
    an inlet and an outlet) and one-column ragged tails."""
    inlet = (np.zeros(Nz), 0.01 + 0.002 * np.arange(Nz))
    c = Case(Nz, Nr, G=-4.7, wall="outlet", z_bc="noslip", r_lo="inlet", r_off=4.0, inlet=inlet)
    fields = I.noisy(Nz, Nr, seed=Nz + Nr, base=1.0, amp=0.05, uamp=0.01)
    check_fp64(c.gpu(fields, 200), c.oracle(fields, 200))


@pytest.mark.parametrize("storage,shift", [("f32", "default"), ("bf16", "equilibrium")])
def test_reduced_storage_bounded(storage, shift):
    """FP32 storage within 1e-4 of the oracle's density after 200 steps of a closed
    two-phase box; BF16 with the equilibrium shift within 5e-3."""
    Nz, Nr = 70, 45
    c = Case(Nz, Nr, wall="noslip", z_bc="noslip")
    c.spec.shift = shift
    fields = I.drop(Nz, Nr, 34.5, 12.0, amps=(0.08,))
    (_, (rho, _, _)), (_, F) = c.gpu(fields, 200, storage=storage), c.oracle(fields, 200)
    bound = 1e-4 if storage == "f32" else 5e-3
    assert np.abs(rho / F["rho"] - 1).max() < bound


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_tilings_and_batch_bit_identical(storage):
    """Every compiled fused tile gives the same bits on a bounded lattice, and so does
    the lattice as instance 0 of a batch with a periodic drop beside it."""
    Nz, Nr = 70, 45
    c = Case(Nz, Nr, G=-4.8, wall="outlet", z_bc="noslip", r_lo="inlet", r_off=5.0,
             inlet=(np.zeros(Nz), 0.01 * np.ones(Nz)))
    fields = I.noisy(Nz, Nr, seed=3, base=1.0, amp=0.05, uamp=0.01)
    ref = c.gpu(fields, 100, storage=storage, tile=(32, 8), schedule="fused")[0]
    for tz, tr in amlbm.tiles(storage, "fused"):
        got = c.gpu(fields, 100, storage=storage, tile=(tz, tr), schedule="fused")[0]
        assert np.array_equal(got, ref), (tz, tr)
    drop = amlbm.InstanceSpec(48, 24, 0.9, -5.0)
    got = c.gpu(fields, 100, storage=storage, tile=(32, 8), schedule="fused",
                extra=[(drop, I.drop(48, 24, 24.0, 8.0))])[0]
    assert np.array_equal(got, ref)


def test_diagnostics_off_axis_match_oracle():
    """Mass, 3D mass, momentum, kinetic energy and the mass source use r_j = j + 1/2 + r_off."""
    c, inp = disc_case(16, 4.5, 40)
    fields = inp.fields()
    lat = amlbm.Lattice(16, 40, tau=1.0, G=0.0, wall="outlet", z_bc="noslip", r_lo="inlet",
                        r_off=inp.r_off)
    lat.set_inlet(*c.inlet)
    lat.init_fields(*fields)
    lat.step(500)
    d = lat.diagnostics(zc=8.0, R=10.0, rho_l=2.0, rho_v=0.1)
    f = c.o.run(c.o.init(*fields), 500)
    ref = c.o.diag(f, zc=8.0, objR=10.0, rho_l=2.0, rho_v=0.1)
    # In a flow this slow (|u| ~ 4e-4) u carries the rounding of the populations
    # (max f ~ 0.4, see check_fp64), so momz3d = sum 2 pi r rho u_z (which also
    # cancels to round-off here: the flow is symmetric in z) and E_ke = pi sum r rho
    # |u|^2, whose rounding is at most sum 2 pi r rho |u| |du|, are held to the scale
    # mass3d * umax of their terms.
    scale = dict(momz3d=ref["mass3d"] * ref["umax"], Eke=ref["mass3d"] * ref["umax"])
    for key in ("mass2d", "mass3d", "momz3d", "Eke", "sumS", "a2"):
        assert abs(d[key] - ref[key]) <= 1e-11 * scale.get(key, abs(ref[key])), key
    lat.close()


def test_inlet_and_adjoint_misuse_rejected():
    """set_inlet on a lattice without an inlet and the adjoint of a bounded lattice are EINVAL."""
    lat = amlbm.Lattice(32, 16, tau=0.9, G=-5.0)
    with pytest.raises(amlbm.AmlbmError) as e:
        lat.set_inlet(np.zeros(32), np.zeros(32))
    assert e.value.code == amlbm.EINVAL
    lat.close()
    box = amlbm.Lattice(48, 24, tau=0.9, G=-5.0, storage="f64", z_bc="noslip")
    with pytest.raises(amlbm.AmlbmError) as e:
        box.adjoint(4, I.legendre_amplitudes(4), 24.0, 8.0)
    assert e.value.code == amlbm.EINVAL
    box.close()


@pytest.mark.parametrize("storage,shift,bound", [("f16", "equilibrium", 1e-3), ("f16", "local", 2e-2)])
def test_fp16_bounded_disc_flow(storage, shift, bound):
    """The flow between discs with FP16 storage: density within the bound after 2000 steps,
    and the radial velocity within 2 % of U_2 of the FP64 oracle's."""
    c, inp = disc_case()
    c.spec.shift = shift
    fields = inp.fields()
    (_, (rho, _, ur)), (_, F) = c.gpu(fields, 2000, storage=storage), c.oracle(fields, 2000)
    assert np.abs(rho / F["rho"] - 1).max() < bound
    assert np.abs(ur - F["ur"]).max() < 0.02 * inp.U2
