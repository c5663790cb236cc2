"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: FP64 storage matches the oracle to a max relative error of 1e-11 after up
to 1000 steps (f pointwise, rho pointwise, u normwise: max|du| / max|u|).  The
reduced-precision forms are held to the bounds stated at their test.
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

WALLS = {0: "freeslip", 1: "noslip"}


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def run_pair(Nz, Nr, steps, fields, tau=1.0, G=-5.0, wall=0, axisym=1, src=0, gz=0.0,
             storage="f64", tile=None, rho_ref=1.0, shift="default", rounding="nearest"):
    rho, uz, ur = fields
    o = O.Oracle(Nz, Nr, tau=tau, G=G, gz=gz, wall=wall, axisym=axisym, src_mode=src)
    f_ref = o.run(o.init(rho, uz, ur), steps)
    spec = amlbm.InstanceSpec(Nz, Nr, tau, G, 1.0, WALLS[wall], bool(axisym),
                              "link" if src else "local", gz, rho_ref, shift, rounding)
    b = amlbm.Batch([spec], storage=storage, tile=tile)
    b.init_fields(0, rho, uz, ur)
    b.step(steps)
    f_gpu = b.read_f(0)
    rho_g, uz_g, ur_g = b.read(0)
    b.close()
    F = o.fields(f_ref)
    return f_gpu, f_ref, (rho_g, uz_g, ur_g), F


def check_fp64(res, tol=1e-11):
    f_gpu, f_ref, (rho, uz, ur), F = res
    assert np.isfinite(f_gpu).all()
    assert rel(f_gpu, f_ref) < tol
    assert np.abs(rho / F["rho"] - 1).max() < tol
    umax = max(np.abs(F["uz"]).max(), np.abs(F["ur"]).max())
    if umax > 0:
        assert max(np.abs(uz - F["uz"]).max(), np.abs(ur - F["ur"]).max()) / umax < tol


def test_fp64_static_drop_1000_steps():
    """The static-drop workload: 64 x 32, G = -5, tau = 1, R = 12 at (32, 0), 1000 steps."""
    check_fp64(run_pair(64, 32, 1000, I.drop(64, 32, 32.0, 12.0)))


@pytest.mark.parametrize("wall,src,axisym,gz,tau,G", [
    (0, 0, 1, 0.0, 0.8, -5.0), (1, 0, 1, 1e-4, 1.0, -4.6), (0, 1, 1, 0.0, 0.9, -5.0),
    (1, 1, 1, 0.0, 0.7, -4.8), (0, 0, 0, 0.0, 1.0, -5.5), (1, 0, 0, 5e-5, 0.6, 0.0)])
def test_fp64_flag_combinations(wall, src, axisym, gz, tau, G):
    fields = I.drop(40, 20, 17.0, 7.0, amps=(0.1,)) if G else I.noisy(40, 20, seed=4)
    check_fp64(run_pair(40, 20, 200, fields, tau=tau, G=G, wall=wall, axisym=axisym, src=src, gz=gz))


@pytest.mark.parametrize("tile", [(32, 8), (64, 8)])
def test_fp64_ragged_tiles(tile):
    """Sizes that are not multiples of the tile (ragged tail in z and r, several tiles)."""
    check_fp64(run_pair(70, 21, 300, I.drop(70, 21, 30.0, 9.0, amps=(0.08,)), tau=0.85, tile=tile))


@pytest.mark.parametrize("Nz,Nr", [(1, 64), (3, 4), (5, 9), (33, 4)])
def test_fp64_degenerate_sizes(Nz, Nr):
    """Single-column lattice (the flat interface of Table I), minimum Nr and odd sizes."""
    fields = I.slab(Nz, Nr, Nr / 2, 1.93, 0.16) if Nz == 1 else I.noisy(Nz, Nr, seed=Nz)
    check_fp64(run_pair(Nz, Nr, 300, fields, tau=0.9))


def test_fp64_oscillating_drop_full_size():
    """The oscillating-drop workload at full size: 256 x 128, R = 40 with 5% P2, tau = 0.8."""
    check_fp64(run_pair(256, 128, 1000, I.drop(256, 128, 128.0, 40.0, amps=(0.05,)), tau=0.8))


def test_fp64_thread_full_size():
    """The capillary-thread workload: lambda = 200 x 128, R0 = 25, 10% cos perturbation."""
    check_fp64(run_pair(200, 128, 1000, I.thread(200, 128, 25.0, 0.1)))


# Max relative error in rho after 1000 steps of the static-drop workload against
# the FP64 oracle, per storage form, shift and rounding.
#
# Forms held to the stated accuracy target, 1e-4:
TARGET_FORMS = [("f32", "none", "nearest"), ("f32", "local", "nearest"), ("f32", "equilibrium", "nearest")]
#
# Forms that do NOT meet the 1e-4 target.  Their bounds are measured findings with
# margin, kept as regression bounds on the measured error, not the specification.
# The 16-bit errors are random walks whose maximum over the sites varies with the
# drop's placement: over four placements BF16 measured 1.0e-2 .. 6.2e-2 rounded to
# nearest and 4.3e-3 .. 1.8e-2 with stochastic rounding, FP16 7e-4 .. 3.4e-3 either
# way; with the equilibrium shift (the 16-bit value holds f_i - f^eq_i) FP16 1.1e-5 ..
# 1.1e-4 (nearest), BF16 2.2e-4 .. 1.5e-3 (nearest) and 2.0e-4 .. 2.0e-3 (stochastic).
BELOW_TARGET_FINDINGS = [
    ("f16", "local", "nearest", 5e-3), ("bf16", "local", "nearest", 1.5e-1),
    ("f16", "local", "stochastic", 5e-3), ("bf16", "local", "stochastic", 3e-2),
    ("f16", "global", "nearest", 1.0), ("bf16", "global", "nearest", 1.0),
    ("f16", "equilibrium", "nearest", 2.5e-4), ("bf16", "equilibrium", "nearest", 4e-3),
    ("bf16", "equilibrium", "stochastic", 5e-3),
]


def drop_rho_error(storage, shift, rounding):
    _, _, (rho, uz, ur), F = run_pair(64, 32, 1000, I.drop(64, 32, 32.0, 12.0), storage=storage,
                                      tile=(32, 8), shift=shift, rounding=rounding)
    err = np.abs(rho / F["rho"] - 1).max()
    uerr = max(np.abs(uz - F["uz"]).max(), np.abs(ur - F["ur"]).max()) / np.abs(F["uz"]).max()
    print(f"{storage}/{shift}/{rounding}: rho max rel err {err:.3e}, u normwise {uerr:.3e}")
    assert np.isfinite(rho).all()
    return err


@pytest.mark.parametrize("storage,shift,rounding", TARGET_FORMS)
def test_forms_meeting_the_accuracy_target(storage, shift, rounding):
    """FP32 arithmetic and FP32 storage against the FP64 oracle: within 1e-4."""
    assert drop_rho_error(storage, shift, rounding) <= 1e-4


@pytest.mark.parametrize("storage,shift,rounding,bound", BELOW_TARGET_FINDINGS)
def test_forms_below_the_target_stay_at_their_measured_error(storage, shift, rounding, bound):
    """16-bit storage of f_i - W_i s (or of f_i - f^eq_i): these miss the 1e-4 target;
    the bound only keeps their measured error from growing."""
    assert drop_rho_error(storage, shift, rounding) < bound


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("case", [dict(), dict(wall="noslip", gz=1e-4), dict(src="link"), dict(axisym=False),
                                  dict(rounding="stochastic"), dict(shift="equilibrium")])
def test_split_schedule_equals_fused_bitwise(storage, case):
    """The two-kernel schedule performs the fused kernel's arithmetic operation for
    operation: states after 120 steps are bit-identical (ragged 70 x 21 lattice)."""
    if storage == "f64" and case.get("shift"):
        pytest.skip("FP64 storage is never shifted")
    spec = amlbm.InstanceSpec(70, 21, 0.8, -5.0, **case)
    fl = I.drop(70, 21, 30.0, 9.0, amps=(0.08,))
    out = []
    for sched, tile in (("fused", (32, 8)), ("split", (32, 8)), ("split", (64, 8)), ("split", (32, 16))):
        b = amlbm.Batch([spec], storage=storage, tile=tile, schedule=sched)
        b.init_fields(0, *fl)
        b.step(120)
        out.append(b.read_f(0))
        b.close()
    for x in out[1:]:
        assert np.array_equal(out[0], x)


def test_batch_equals_single_instances_bitwise():
    """Uneven instances in one launch give bit-identical results to separate runs."""
    specs = [amlbm.InstanceSpec(48, 24, 0.9, -5.0), amlbm.InstanceSpec(70, 21, 0.75, -4.7, wall="noslip"),
             amlbm.InstanceSpec(33, 16, 1.1, -5.3, src="link")]
    fields = [I.drop(48, 24, 24.0, 8.0, amps=(0.05,)), I.drop(70, 21, 35.0, 9.0),
              I.drop(33, 16, 16.0, 6.0, amps=(0.02,))]
    for storage in ("f64", "f32", "bf16", "f16"):
        if storage in ("bf16", "f16"):
            for sp in specs:
                sp.rounding = "stochastic"
        b = amlbm.Batch(specs, storage=storage, tile=(32, 8))
        for k, fl in enumerate(fields):
            b.init_fields(k, *fl)
        b.step(150)
        for k, (s, fl) in enumerate(zip(specs, fields)):
            one = amlbm.Batch([s], storage=storage, tile=(32, 8))
            one.init_fields(0, *fl)
            one.step(150)
            assert np.array_equal(one.read_f(0), b.read_f(k)), (storage, k)
            one.close()
        b.close()


def test_graph_chunks_equal_direct_launches():
    s = [amlbm.InstanceSpec(64, 32, 0.9, -5.0)]
    fl = I.drop(64, 32, 32.0, 10.0, amps=(0.05,))
    out = []
    s[0].rounding = "stochastic"
    for chunk in (0, 16):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            b = amlbm.Batch(s, storage="bf16", graph_chunk=chunk, stream=stream)
            b.init_fields(0, *fl)
            b.step(37)
            out.append(b.read_f(0))
            b.close()
    assert np.array_equal(out[0], out[1])


def test_diagnostics_match_oracle():
    Nz, Nr, zc, R = 64, 32, 32.0, 12.0
    fl = I.drop(Nz, Nr, zc, R, amps=(0.05,))
    lat = amlbm.Lattice(Nz, Nr, tau=0.9, G=-5.0)
    lat.init_fields(*fl)
    lat.step(200)
    d = lat.diagnostics(zc=zc, R=R, rho_l=1.93, rho_v=0.16)
    o = O.Oracle(Nz, Nr, tau=0.9, G=-5.0)
    f = o.run(o.init(*fl), 200)
    e = o.diag(f, zc, R, 1.93, 0.16)
    for k in ("mass2d", "mass3d", "Eke", "umax", "a2", "A", "neck", "p_in", "p_out", "dp"):
        assert abs(d[k] - e[k]) <= 1e-10 * abs(e[k]), (k, d[k], e[k])
    # near-zero sums: bound the difference by the scale of their terms
    assert abs(d["momz3d"] - e["momz3d"]) <= 1e-10 * e["mass3d"] * e["umax"]
    assert abs(d["sumS"] - e["sumS"]) <= 1e-10 * e["mass2d"] * e["umax"]
    assert d["bad"] == 0 and d["steps"] == 200
    lat.close()


def test_diagnostics_flag_unstable_state():
    lat = amlbm.Lattice(16, 8, tau=1.0, G=-5.0)
    rho = torch.ones(8, 16, dtype=torch.float64, device="cuda")
    rho[3, 5] = -1.0
    lat.init_fields_device(rho)
    d = lat.diagnostics(check=False)
    assert d["bad"] == 1
    with pytest.raises(amlbm.AmlbmError) as e:
        lat.diagnostics()
    assert e.value.code == amlbm.EUNSTABLE
    lat.close()


@pytest.mark.parametrize("storage,shift", [("f32", "default"), ("bf16", "equilibrium")])
def test_save_load_state_roundtrip(storage, shift):
    """The saved state (populations, psi and, for the equilibrium shift, the stored
    velocity) restarts the run bit for bit."""
    fl = I.drop(40, 20, 20.0, 7.0, amps=(0.05,))
    lat = amlbm.Lattice(40, 20, tau=0.9, G=-5.0, storage=storage, shift=shift)
    lat.init_fields(*fl)
    lat.step(30)
    state = lat.save_state()
    lat.step(40)
    a = lat.read_f()
    lat.load_state(state)
    lat.step(40)
    assert np.array_equal(lat.read_f(), a)
    lat.close()


def test_device_init_equals_host_init():
    fl = I.drop(40, 20, 20.0, 7.0)
    a = amlbm.Lattice(40, 20)
    a.init_fields(*fl)
    b = amlbm.Lattice(40, 20)
    b.init_fields_device(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in fl))
    assert np.array_equal(a.read_f(), b.read_f())
    a.close()
    b.close()


def test_batch_sweep_sampled_against_oracle():
    """The 64-drop batch sweep at full size (FP64 storage), 20 steps; three instances
    (smallest, largest, one oscillating) are checked against the oracle."""
    inst = I.batch_sweep(64)
    specs = [amlbm.InstanceSpec(x.Nz, x.Nr, x.tau, x.G) for x in inst]
    b = amlbm.Batch(specs, storage="f64")
    for k, x in enumerate(inst):
        b.init_fields(k, *x.make_fields())
    b.step(20)
    sizes = [x.Nz * x.Nr for x in inst]
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), 1}
    for k in picks:
        x = inst[k]
        o = O.Oracle(x.Nz, x.Nr, tau=x.tau, G=x.G)
        f_ref = o.run(o.init(*x.make_fields()), 20)
        assert rel(b.read_f(k), f_ref) < 1e-12, k
    b.close()
