"""The OpenMP build of the oracle (the CPU baseline timed on all host cores)
returns the serial oracle's R(U) and RK steps bit for bit: its threads split
only the loops over elements and master faces, each iteration writing its own
values with the serial arithmetic."""
import numpy as np
import pytest

from workloads import box_mesh, mms_params, random_state


@pytest.mark.parametrize("flux,source", [(0, 0), (1, 0), (2, 0), (0, 1)])
def test_parallel_oracle_is_bitwise_serial(orc, flux, source):
    N = 4
    mesh = box_mesh(4, N, deform="sinprod", rotate_seed=90 + flux)
    prm = mms_params()
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=0.02, surf_flux=flux, source=source)
    ser = orc.Oracle(mesh, N, **kw)
    par = orc.Oracle(mesh, N, parallel=True, **kw)
    used = orc.set_threads(4)
    assert used == 4 or used == 1   # 1 if the toolchain has no OpenMP
    U = random_state(mesh.n_elems, N, seed=91)
    a, b = ser.time_derivative(U, t=0.3), par.time_derivative(U, t=0.3)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    a, b = ser.rk_steps(U, 0.0, 1e-3, 2), par.rk_steps(U, 0.0, 1e-3, 2)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
