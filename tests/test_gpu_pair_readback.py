"""The pair schedule's read-back (rho and u of the current state, the input of the
diagnostics, amlbm_step_pair.cu) against the fused schedule's read-back: the
same operations on the same state, so rho, u and every diagnostic must be
bit-identical, per instance and for the whole batch, for each storage form and
option the pair schedule takes, on ragged and very small lattices."""
import numpy as np
import pytest

from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402

CASES = [dict(), dict(wall="noslip", gz=1e-4), dict(axisym=False), dict(shift="equilibrium"),
         dict(forcing="guo"), dict(rounding="stochastic")]


def batches(specs, fields, storage, pair_tile, steps):
    out = []
    for sched, tile in (("fused", (32, 8)), ("pair", pair_tile)):
        b = amlbm.Batch(specs, storage=storage, tile=tile, schedule=sched)
        for k, fl in enumerate(fields):
            b.init_fields(k, *fl)
        b.step(steps)
        out.append(b)
    return out


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16", "f64"])
@pytest.mark.parametrize("case", CASES)
def test_pair_readback_equals_fused_bitwise(storage, case):
    if storage == "f64" and (case.get("shift") or case.get("rounding")):
        pytest.skip("FP64 storage is neither shifted nor rounded")
    dims = [(70, 21), (48, 30), (8, 12)]
    specs = [amlbm.InstanceSpec(Nz, Nr, 0.85, -5.0, **case) for Nz, Nr in dims]
    fields = [I.drop(Nz, Nr, Nz / 2, min(Nz, 2 * Nr) / 4.0, amps=(0.05,)) for Nz, Nr in dims]
    for tile in amlbm.tiles(storage, "pair"):
        a, b = batches(specs, fields, storage, tuple(tile), 40)
        for k in range(len(dims)):
            for x, y in zip(a.read(k), b.read(k)):
                assert np.array_equal(x, y), (tile, k)
            da, db = a.diagnostics(k, check=False), b.diagnostics(k, check=False)
            assert da.keys() == db.keys()
            assert np.array_equal(np.array([float(da[q]) for q in da]), np.array([float(db[q]) for q in da]),
                                  equal_nan=True), (tile, k)
        da = a.diagnostics_all(check=False, as_array=True)
        db = b.diagnostics_all(check=False, as_array=True)
        assert np.array_equal(da, db, equal_nan=True), tile
        a.close()
        b.close()


def test_pair_readback_on_the_sweep():
    """The 64-drop sweep on the default pair tile: whole-batch diagnostics and every
    instance's rho and u equal the fused schedule's."""
    inst = I.batch_sweep(64)
    specs = [amlbm.InstanceSpec(x.Nz, x.Nr, x.tau, x.G) for x in inst]
    fields = [x.make_fields() for x in inst]
    a, b = batches(specs, fields, "f32", (40, 24), 20)
    params = np.array([[x.zc, x.R, x.rho_l, x.rho_v] for x in inst], dtype=np.float64)
    assert np.array_equal(a.diagnostics_all(params, check=False, as_array=True),
                          b.diagnostics_all(params, check=False, as_array=True), equal_nan=True)
    for k in range(0, 64, 9):
        for x, y in zip(a.read(k), b.read(k)):
            assert np.array_equal(x, y), k
    a.close()
    b.close()
