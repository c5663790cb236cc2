"""amlbm_diagnostics_noalloc, the diagnostics entry point for callers that must not
allocate device memory (it reduces in a fixed device array of the library instead
of the context's buffers), checked through the C ABI against amlbm_diagnostics on
two calls in a row.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1310_1871_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1310_1871_gb300 import amlbm  # noqa: E402

KEYS_REL = ("mass2d", "mass3d", "Eke", "umax", "a2", "A", "neck", "p_in", "p_out", "dp")


def noalloc(lat, zc, R, rho_l, rho_v):
    dp = amlbm.DiagParams(zc, R, rho_l, rho_v)
    d = amlbm.Diag()
    rc = lat.lib.amlbm_diagnostics_noalloc(lat.h, ctypes.byref(dp), ctypes.byref(d))
    return rc, amlbm._diag_dict(d)


def close_enough(a, b):
    for k in KEYS_REL:
        assert abs(a[k] - b[k]) <= 1e-10 * abs(b[k]), (k, a[k], b[k])
    assert abs(a["momz3d"] - b["momz3d"]) <= 1e-10 * b["mass3d"] * max(b["umax"], 1e-30)
    assert abs(a["sumS"] - b["sumS"]) <= 1e-10 * b["mass2d"] * max(b["umax"], 1e-30)
    assert a["bad"] == b["bad"] and a["steps"] == b["steps"]


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_noalloc_diagnostics_match_two_calls_in_a_row(storage):
    Nz, Nr, zc, R = 96, 40, 48.0, 14.0
    lat = amlbm.Lattice(Nz, Nr, tau=0.9, G=-5.0, storage=storage)
    lat.init_fields(*I.drop(Nz, Nr, zc, R, amps=(0.05,)))
    lat.step(50)
    ref1 = lat.diagnostics(zc=zc, R=R, rho_l=1.93, rho_v=0.16)
    rc, got1 = noalloc(lat, zc, R, 1.93, 0.16)
    assert rc == amlbm.OK, lat.lib.amlbm_last_error()
    close_enough(got1, ref1)
    # second call in a row on a different state: nothing stale may leak through
    lat.step(30)
    ref2 = lat.diagnostics(zc=zc, R=R, rho_l=1.93, rho_v=0.16)
    rc, got2 = noalloc(lat, zc, R, 1.93, 0.16)
    assert rc == amlbm.OK, lat.lib.amlbm_last_error()
    close_enough(got2, ref2)
    assert got2["steps"] == 80 and got1["Eke"] != got2["Eke"]
    lat.close()


def test_noalloc_calls_allocate_no_device_memory():
    """The property the entry point exists for: once the lattice exists (amlbm_create
    loads the code and looks up the scratch array), repeated calls leave the
    device's free memory exactly as it was."""
    Nz, Nr = 64, 32
    lat = amlbm.Lattice(Nz, Nr, tau=1.0, G=-5.0, storage="f32")
    lat.init_fields(*I.drop(Nz, Nr, 32.0, 10.0))
    lat.step(5)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        rc, d = noalloc(lat, 32.0, 10.0, 1.93, 0.16)
        assert rc == amlbm.OK and d["bad"] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    lat.close()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_lattices_beyond_the_static_limit():
    Nz = 8192 + 1
    lat = amlbm.Lattice(Nz, 4, tau=1.0, G=-5.0)
    lat.init_fields(np.full((4, Nz), 0.5))
    rc, _ = noalloc(lat, Nz / 2, 1.0, 2.0, 0.1)
    assert rc == amlbm.EINVAL
    assert b"AMLBM_NOALLOC_MAX_NZ" in lat.lib.amlbm_last_error()
    lat.close()
