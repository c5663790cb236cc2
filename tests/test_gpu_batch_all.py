"""Whole-batch entry points: amlbm_batch_init_all and amlbm_batch_diagnostics_all
give exactly what the per-instance calls give, and a rejected init leaves the
state unchanged."""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402

SPECS = [(48, 24, 0.9, -5.0, dict()), (70, 21, 0.75, -4.7, dict(wall="noslip")),
         (33, 16, 1.1, -5.3, dict(src="link")), (40, 20, 1.0, -5.0, dict(axisym=False))]


def make(storage, graph_chunk=0, stream=None):
    specs = [amlbm.InstanceSpec(Nz, Nr, tau, G, **kw) for Nz, Nr, tau, G, kw in SPECS]
    fields = []
    for k, (Nz, Nr, _, _, _) in enumerate(SPECS):
        rho, uz, ur = I.drop(Nz, Nr, Nz / 2, Nr / 2.5, amps=(0.04,))
        fields.append((rho, uz + 0.01 * (k % 2), ur))
    return amlbm.Batch(specs, storage=storage, tile=(32, 8), graph_chunk=graph_chunk, stream=stream), fields


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
def test_init_all_equals_per_instance_init(storage):
    a, fields = make(storage)
    b, _ = make(storage)
    for k, fl in enumerate(fields):
        a.init_fields(k, *fl)
    b.init_all(*[[fl[q] for fl in fields] for q in range(3)])
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    a.step(25)
    b.step(25)  # the step after a parity change takes every tile (counters reset)
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    a.close()
    b.close()


def test_init_all_with_graphs_and_repeated_calls():
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a, fields = make("bf16", graph_chunk=4, stream=stream)
        b, _ = make("bf16", stream=stream)
        cols = [[fl[q] for fl in fields] for q in range(3)]
        for _ in range(3):  # each call flips the parity
            a.init_all(*cols)
            a.step(9)
        b.init_all(*cols)
        b.step(9)
        for k in range(len(fields)):
            assert np.array_equal(a.read_f(k), b.read_f(k)), k
        a.close()
        b.close()


def test_init_all_rejects_bad_density_and_keeps_state():
    b, fields = make("f32")
    cols = [[fl[q] for fl in fields] for q in range(3)]
    b.init_all(*cols)
    b.step(5)
    before = [b.read_f(k) for k in range(len(fields))]
    bad = [np.array(x, copy=True) for x in cols[0]]
    bad[2][3, 4] = np.nan
    bad[0][0, 0] = -1.0
    with pytest.raises(amlbm.AmlbmError) as e:
        b.init_all(bad, cols[1], cols[2])
    assert e.value.code == amlbm.EINVAL and "2 sites" in str(e.value)
    for k in range(len(fields)):
        assert np.array_equal(b.read_f(k), before[k]), k
    b.step(3)  # still steps from the kept state
    ref, _ = make("f32")
    ref.init_all(*cols)
    ref.step(8)
    for k in range(len(fields)):
        assert np.array_equal(b.read_f(k), ref.read_f(k)), k
    b.close()
    ref.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
def test_init_all_f32_equals_fp64_inputs(storage):
    """amlbm_batch_init_all_f32: for the FP32-arithmetic forms the state equals that of
    amlbm_batch_init_all of the FP64 fields (both round to FP32 first); for FP64
    storage it equals amlbm_batch_init_all of the FP32 values widened to FP64."""
    a, fields = make(storage)
    b, _ = make(storage)
    cols = [np.concatenate([np.ravel(fl[q]) for fl in fields]) for q in range(3)]
    cols32 = [c.astype(np.float32) for c in cols]
    a.init_all(*([c.astype(np.float64) for c in cols32] if storage == "f64" else cols))
    b.init_all(*cols32)
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    a.step(20)
    b.step(20)
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    b.init_all(cols32[0])  # zero velocity
    a.init_all(cols32[0].astype(np.float64))
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    a.close()
    b.close()


def test_init_all_f32_rejects_bad_density_and_keeps_state():
    b, fields = make("f32")
    cols = [np.concatenate([np.ravel(fl[q]) for fl in fields]).astype(np.float32) for q in range(3)]
    b.init_all(*cols)
    b.step(4)
    before = [b.read_f(k) for k in range(len(fields))]
    bad = cols[0].copy()
    bad[100] = np.nan
    bad[7] = 0.0
    bad[9] = -2.0
    with pytest.raises(amlbm.AmlbmError) as e:
        b.init_all(bad, cols[1], cols[2])
    assert e.value.code == amlbm.EINVAL and "3 sites" in str(e.value)
    for k in range(len(fields)):
        assert np.array_equal(b.read_f(k), before[k]), k
    b.close()


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_diagnostics_all_equals_per_instance(storage):
    b, fields = make(storage)
    for k, fl in enumerate(fields):
        b.init_fields(k, *fl)
    b.step(40)
    params = [dict(zc=Nz / 2, R=Nr / 2.5, rho_l=1.93, rho_v=0.16) for Nz, Nr, _, _, _ in SPECS]
    all_ = b.diagnostics_all(params)
    for k, p in enumerate(params):
        one = b.diagnostics(k, **p)
        assert one == all_[k], k
    assert b.diagnostics_all() == [b.diagnostics(k) for k in range(len(SPECS))]
    b.close()


def test_diagnostics_all_against_oracle():
    Nz, Nr, tau, G, _ = SPECS[0]
    b, fields = make("f64")
    for k, fl in enumerate(fields):
        b.init_fields(k, *fl)
    b.step(60)
    d = b.diagnostics_all([dict(zc=Nz / 2, R=Nr / 2.5, rho_l=1.93, rho_v=0.16)] * len(SPECS))[0]
    o = O.Oracle(Nz, Nr, tau=tau, G=G)
    e = o.diag(o.run(o.init(*fields[0]), 60), Nz / 2, Nr / 2.5, 1.93, 0.16)
    for key in ("mass2d", "mass3d", "Eke", "umax", "a2", "A", "neck", "p_in", "p_out", "dp"):
        assert abs(d[key] - e[key]) <= 1e-10 * abs(e[key]), (key, d[key], e[key])
    b.close()


def test_diagnostics_all_array_forms_and_repeated_calls():
    """Parameters as an (n, 4) array and results as an (n, 16) array give the dict
    results; repeated calls with unchanged and with changed parameters agree with the
    per-instance call (the parameters are uploaded only when they change)."""
    b, fields = make("bf16")
    for k, fl in enumerate(fields):
        b.init_fields(k, *fl)
    b.step(30)
    arr = np.array([[Nz / 2, Nr / 2.5, 1.93, 0.16] for Nz, Nr, _, _, _ in SPECS])
    dicts = b.diagnostics_all([dict(zc=a[0], R=a[1], rho_l=a[2], rho_v=a[3]) for a in arr])
    for _ in range(2):
        res = b.diagnostics_all(arr, as_array=True)
        for k, d in enumerate(dicts):
            assert [res[k, m] for m in range(len(amlbm.DIAG_FIELDS))] == [d[f] for f in amlbm.DIAG_FIELDS]
    arr2 = arr.copy()
    arr2[:, 1] *= 1.5
    res2 = b.diagnostics_all(arr2, as_array=True)
    for k in range(len(SPECS)):
        one = b.diagnostics(k, zc=arr2[k, 0], R=arr2[k, 1], rho_l=1.93, rho_v=0.16)
        assert [res2[k, m] for m in range(len(amlbm.DIAG_FIELDS))] == [one[f] for f in amlbm.DIAG_FIELDS]
    b.close()


def _pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    return t, t.numpy()


def test_init_all_reads_pinned_host_arrays_in_place():
    """Page-locked arrays are read by the init kernel in place; the state is bit for bit
    the one of the copy path, also with pinned and pageable arrays mixed, and a bad
    density in a pinned array is still rejected with the state kept."""
    a, fields = make("bf16")
    b, _ = make("bf16")
    cols = [np.concatenate([np.ravel(fl[q]) for fl in fields]) for q in range(3)]
    keep = [_pinned(c) for c in cols]  # the tensors own the pinned buffers
    a.init_all(*cols)
    b.init_all(keep[0][1], keep[1][1], cols[2])
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    b.init_all(*[p[1] for p in keep])
    a.step(12)
    b.step(12)
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    before = [b.read_f(k) for k in range(len(fields))]
    bad = _pinned(cols[0])
    bad[1][17] = -2.0
    with pytest.raises(amlbm.AmlbmError) as e:
        b.init_all(bad[1], keep[1][1], keep[2][1])
    assert e.value.code == amlbm.EINVAL and "1 sites" in str(e.value)
    for k in range(len(fields)):
        assert np.array_equal(b.read_f(k), before[k]), k
    a.close()
    b.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_init_all_reads_pinned_host_arrays_in_place(dtype):
    """Page-locked host arrays are read by the init kernel over the CPU-GPU link (no
    staging copy): the state equals that of the same values from pageable arrays."""
    a, fields = make("f32")
    b, _ = make("f32")
    cols = [np.concatenate([np.ravel(fl[q]) for fl in fields]).astype(dtype) for q in range(3)]
    pinned = [torch.from_numpy(c.copy()).pin_memory() for c in cols]
    a.init_all(*cols)
    b.init_all(*[t.numpy() for t in pinned])
    for k in range(len(fields)):
        assert np.array_equal(a.read_f(k), b.read_f(k)), k
    a.close()
    b.close()
