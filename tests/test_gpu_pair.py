"""The pair schedule (two adjacent z-sites per thread, amlbm_step_pair.cu) against
the fused schedule and the FP64 oracle.

It performs the fused schedule's arithmetic on the same values, so states after
many steps must be bit-identical for every storage form, boundary option and
compiled tile, on ragged and on very small lattices; the FP64 form is also held
to the oracle at 1e-11 after 1000 steps.  Lattices outside its scope are
rejected with EINVAL."""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402


def run(specs, fields, storage, sched, tile, steps):
    b = amlbm.Batch(specs, storage=storage, tile=tile, schedule=sched)
    for k, fl in enumerate(fields):
        b.init_fields(k, *fl)
    b.step(steps)
    out = [b.read_f(k) for k in range(len(specs))]
    b.close()
    return out


CASES = [dict(), dict(wall="noslip", gz=1e-4), dict(axisym=False), dict(rounding="stochastic"),
         dict(shift="equilibrium"), dict(forcing="guo"), dict(shift="global", rho_ref=0.9)]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("case", CASES)
def test_pair_equals_fused_bitwise(storage, case):
    """Ragged 70 x 21 lattice (several tiles, ragged in z and r), 150 steps."""
    if storage == "f64" and (case.get("shift") or case.get("rounding")):
        pytest.skip("FP64 storage is neither shifted nor rounded")
    spec = amlbm.InstanceSpec(70, 21, 0.8, -5.0, **case)
    fl = I.drop(70, 21, 30.0, 9.0, amps=(0.08,))
    ref = run([spec], [fl], storage, "fused", (32, 8), 150)[0]
    tiles = amlbm.tiles(storage, "pair")
    assert tiles
    for tile in tiles:
        got = run([spec], [fl], storage, "pair", tile, 150)[0]
        assert np.array_equal(ref, got), (tile, np.abs(ref - got).max())


@pytest.mark.parametrize("Nz,Nr", [(2, 8), (8, 12), (16, 9), (40, 20), (130, 9)])
def test_pair_small_and_odd_shapes_bitwise(Nz, Nr):
    """Lattices narrower than a tile's halo (the periodic seam wraps more than once)
    and ragged shapes, FP32 and FP64."""
    fl = I.noisy(Nz, Nr, seed=Nz + Nr)
    for storage in ("f32", "f64"):
        spec = amlbm.InstanceSpec(Nz, Nr, 0.9, -4.8)
        ref = run([spec], [fl], storage, "fused", (32, 8), 100)[0]
        for tile in amlbm.tiles(storage, "pair"):
            got = run([spec], [fl], storage, "pair", tuple(tile), 100)[0]
            assert np.array_equal(ref, got), (storage, tile, np.abs(ref - got).max())


def test_pair_fp64_matches_oracle_1000_steps():
    """The static-drop workload (64 x 32, G = -5, tau = 1, R = 12), 1000 steps: max
    relative error 1e-11 in f against the FP64 oracle."""
    fl = I.drop(64, 32, 32.0, 12.0)
    o = O.Oracle(64, 32, tau=1.0, G=-5.0)
    f_ref = o.run(o.init(*fl), 1000)
    got = run([amlbm.InstanceSpec(64, 32, 1.0, -5.0)], [fl], "f64", "pair", (32, 8), 1000)[0]
    err = np.abs(got - f_ref).max() / np.abs(f_ref).max()
    print(f"pair FP64 vs oracle after 1000 steps: {err:.2e}")
    assert err < 1e-11


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_pair_sweep_equals_fused_bitwise(storage):
    """The 64-drop sweep (uneven lattices, one persistent launch per step), 60 steps, on
    the default pair tile and two others."""
    inst = I.batch_sweep(64)
    specs = [amlbm.InstanceSpec(x.Nz, x.Nr, x.tau, x.G) for x in inst]
    fields = [x.make_fields() for x in inst]
    a = run(specs, fields, storage, "fused", (26, 16), 60)
    for tile in ((64, 24), (40, 24), (32, 16)):
        b = run(specs, fields, storage, "pair", tile, 60)
        for k in range(len(specs)):
            assert np.array_equal(a[k], b[k], equal_nan=True), (tile, k)


@pytest.mark.parametrize("kw,Nz", [(dict(src="link"), 32), (dict(), 33), (dict(z_bc="noslip"), 32),
                                   (dict(wall="outlet"), 32)])
def test_pair_rejects_lattices_outside_its_scope(kw, Nz):
    spec = amlbm.InstanceSpec(Nz, 16, 0.9, -5.0, **kw)
    with pytest.raises(amlbm.AmlbmError) as e:
        amlbm.Batch([spec], storage="f32", tile=(32, 16), schedule="pair")
    assert e.value.code == amlbm.EINVAL
