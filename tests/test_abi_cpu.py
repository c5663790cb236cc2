"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
function include/amlbm.h declares, and rejects bad arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_1310_1871_gb300 import amlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "amlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amlbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return amlbm.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(amlbm.EXPORTS)


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.amlbm_version()
    assert isinstance(lib.amlbm_last_error(), bytes)


@pytest.mark.parametrize("Nz,Nr,tau,G,rho0", [
    (0, 16, 1.0, -5.0, 1.0), (16, 3, 1.0, -5.0, 1.0), (16, 16, 0.5, -5.0, 1.0),
    (16, 16, 1.0, -7.0, 1.0), (16, 16, 1.0, -5.0, 0.0), (16, 16, float("nan"), -5.0, 1.0)])
def test_create_rejects_bad_arguments(lib, Nz, Nr, tau, G, rho0):
    h = ctypes.c_void_p()
    bc = amlbm.make_bc()
    rc = lib.amlbm_create(Nz, Nr, tau, G, rho0, ctypes.byref(bc), None, None, 0, ctypes.byref(h))
    assert rc == amlbm.EINVAL
    assert h.value is None
    assert len(lib.amlbm_last_error()) > 0


def test_bad_flags_and_tiles_rejected(lib):
    h = ctypes.c_void_p()
    for bc in (amlbm.BC(3, 1, 0, 0, 0, 0, 0.0, 1.0), amlbm.BC(0, 2, 0, 0, 0, 0, 0.0, 1.0),
               amlbm.BC(0, 1, 5, 0, 0, 0, 0.0, 1.0), amlbm.BC(0, 1, 0, 9, 0, 0, 0.0, 1.0),
               amlbm.BC(0, 1, 0, 2, 7, 0, 0.0, 1.0), amlbm.BC(0, 1, 0, 0, 3, 0, 0.0, 1.0),
               amlbm.BC(0, 1, 0, 3, 0, 4, 0.0, 1.0), amlbm.BC(0, 1, 0, 3, 0, -1, 0.0, 1.0)):
        assert lib.amlbm_create(16, 16, 1.0, -5.0, 1.0, ctypes.byref(bc), None, None, 0,
                                ctypes.byref(h)) == amlbm.EINVAL
    inst = (amlbm.InstanceC * 1)(amlbm.InstanceC(32, 16, 1.0, -5.0, 1.0, amlbm.make_bc(storage="f64")))
    tune = amlbm.Tune(128, 8, 0)  # not compiled for FP64
    assert lib.amlbm_batch_create(1, inst, ctypes.byref(tune), None, None, 0, ctypes.byref(h)) == amlbm.EINVAL
    assert b"tile" in lib.amlbm_last_error()


@pytest.mark.parametrize("Nz,Nr,kw", [
    (16, 16, dict(z_bc=2)), (16, 16, dict(r_lo=2)), (16, 16, dict(r_off=1.0)),
    (16, 16, dict(r_lo="inlet", r_off=-1.0)), (16, 16, dict(r_lo="inlet", r_off=float("inf"))),
    (16, 16, dict(wall="outlet", rho_out=0.0)), (3, 16, dict(z_bc="noslip")), (16, 16, dict(forcing=2)),
    (16, 5, dict(r_lo="inlet", r_off=2.0)), (16, 5, dict(wall="outlet"))])
def test_bounded_domain_arguments_rejected(lib, Nz, Nr, kw):
    """Walls in z, inlet and outlet rows: bad codes, an off-axis lattice with the
    axis, a non-positive outlet density and too small lattices are EINVAL."""
    h = ctypes.c_void_p()
    bc = amlbm.make_bc(**kw)
    assert lib.amlbm_create(Nz, Nr, 1.0, -5.0, 1.0, ctypes.byref(bc), None, None, 0,
                            ctypes.byref(h)) == amlbm.EINVAL
    assert h.value is None


@pytest.mark.parametrize("kw", [dict(z_bc="noslip", r_lo="inlet", r_off=9.0, wall="outlet"),
                                dict(forcing="guo")])
def test_bounded_domain_and_guo_need_fused_schedule(lib, kw):
    """The split schedule takes periodic lattices on the axis with the velocity shift only."""
    h = ctypes.c_void_p()
    bc = amlbm.make_bc(**kw)
    inst = (amlbm.InstanceC * 1)(amlbm.InstanceC(32, 111, 1.0, 0.0, 1.0, bc))
    tune = amlbm.Tune(32, 8, 0, amlbm.SCHEDULE["split"])
    assert lib.amlbm_batch_create(1, inst, ctypes.byref(tune), None, None, 0, ctypes.byref(h)) == amlbm.EINVAL
    assert b"split" in lib.amlbm_last_error()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures have the size and field offsets of the C header's."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"amlbm_bc": amlbm.BC, "amlbm_instance": amlbm.InstanceC, "amlbm_tune": amlbm.Tune,
               "amlbm_diag": amlbm.Diag, "amlbm_diag_params": amlbm.DiagParams,
               "amlbm_interface": amlbm.Interface}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "amlbm.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


@pytest.mark.parametrize("args", [
    (-5.0, 1.0, 1.0, 0, 0, 2, 64, 100, 2.0, 0.15),   # FP16 storage
    (-5.0, 1.0, 1.0, 0, 0, 0, 7, 100, 2.0, 0.15),    # n < 8
    (-5.0, 1.0, 1.0, 0, 0, 0, 64, -1, 2.0, 0.15),    # steps < 0
    (-5.0, 1.0, 1.0, 0, 0, 0, 64, 100, 0.1, 0.15),   # rho_l0 <= rho_v0
    (-5.0, 1.0, 1.0, 0, 0, 0, 64, 100, 2.0, 0.0),    # rho_v0 <= 0
    (-5.0, 1.0, 1.0, 2, 0, 0, 64, 100, 2.0, 0.15),   # bad axisym
    (-5.0, 1.0, 1.0, 0, 2, 0, 64, 100, 2.0, 0.15)])  # bad forcing
def test_flat_interface_rejects_bad_arguments(lib, args):
    """amlbm_flat_interface validates before any device work."""
    out = amlbm.Interface()
    assert lib.amlbm_flat_interface(*args, None, ctypes.byref(out)) == amlbm.EINVAL
    assert b"flat interface" in lib.amlbm_last_error()


def test_tile_lists_and_workspace_sizes(lib):
    assert (32, 8) in amlbm.tiles("f64") and (128, 8) not in amlbm.tiles("f64")
    assert (58, 8) in amlbm.tiles("bf16") and (26, 16) in amlbm.tiles("f32")
    assert (26, 16) not in amlbm.tiles("f64") and (64, 16) in amlbm.tiles("bf16", "split")
    small = lib.amlbm_workspace_bytes(64, 32, 0)
    big = lib.amlbm_workspace_bytes(256, 128, 0)
    half = lib.amlbm_workspace_bytes(256, 128, 3)
    assert 0 < small < big and half < big
    # populations (two copies) dominate: 2 x 9 x pitch x Nr x 8 bytes for FP64
    assert big >= 2 * 9 * 256 * 128 * 8
    assert lib.amlbm_workspace_bytes(0, 128, 0) == 0
    # the equilibrium shift keeps two velocity planes beside each psi copy
    inst = (amlbm.InstanceC * 1)(amlbm.InstanceC(256, 128, 1.0, -5.0, 1.0,
                                                amlbm.make_bc(storage="bf16", shift="local")))
    loc = lib.amlbm_batch_workspace_bytes(1, inst)
    inst[0].bc.shift = amlbm.SHIFT["equilibrium"]
    eq = lib.amlbm_batch_workspace_bytes(1, inst)
    assert eq - loc == 2 * 2 * 256 * 128 * 4
    assert half >= eq  # a context's workspace fits every shift mode
    inst[0].bc.shift = 5
    assert lib.amlbm_batch_workspace_bytes(1, inst) == 0


def test_workspace_too_small_rejected(lib):
    h = ctypes.c_void_p()
    bc = amlbm.make_bc()
    # a fake (never dereferenced) aligned device address with too few bytes
    rc = lib.amlbm_create(64, 32, 1.0, -5.0, 1.0, ctypes.byref(bc), None, ctypes.c_void_p(1 << 20), 16,
                          ctypes.byref(h))
    assert rc == amlbm.ENOMEM
