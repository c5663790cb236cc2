"""The OpenMP build of the oracle (the all-cores CPU baseline) computes every site
with the same operations as the serial build: identical bits after many steps, on
the lattice shapes of the workloads and with every boundary option."""
import numpy as np
import pytest

import oracle as O
from paper_1310_1871_gb300 import inputs as I


@pytest.mark.parametrize("kw", [
    dict(),
    dict(wall=O.WALL_NOSLIP, gz=1e-5, G=-4.8),
    dict(src_mode=O.SRC_LINK, tau=0.8),
    dict(forcing=O.FORCE_GUO),
    dict(zbc=O.Z_NOSLIP, axisym=1),
])
def test_openmp_build_is_bitwise_serial(kw):
    Nz, Nr = 40, 24
    rho, uz, ur = I.drop(Nz, Nr, Nz / 2, 8.0, amps=(0.06,))
    a = O.Oracle(Nz, Nr, **kw)
    b = O.Oracle(Nz, Nr, omp=True, **kw)
    n = O.threads(4)
    assert n == 4
    f0 = a.init(rho, uz, ur)
    assert np.array_equal(f0, b.init(rho, uz, ur))
    fa, fb = a.run(f0, 40), b.run(f0, 40)
    assert np.array_equal(fa, fb)
    da, db = a.diag(fa, Nz / 2, 8.0, 1.93, 0.16), b.diag(fb, Nz / 2, 8.0, 1.93, 0.16)
    assert da == db
