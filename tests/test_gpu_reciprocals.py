"""The reciprocals the operator kernels use instead of IEEE divisions (the
hardware approximation rcp.approx.ftz plus a Newton-Raphson step in FP64)
against correctly rounded division, over random and edge-case positive
values, with the error bounds stated in dgsem.h (dg_check_reciprocals)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _inputs():
    rng = np.random.default_rng(5)
    wide = np.ldexp(rng.uniform(1.0, 2.0, 300000), rng.integers(-1000, 1001, 300000))
    # the operators' own range: densities, pressures, beta = rho/(2p) and their pair sums
    ops = rng.uniform(0.02, 400.0, 200000)
    edge = np.array([1.0, 2.0, 0.5, 3.0, 0.1, 1.0 / 3.0, 7.0, 71.42857142857143, np.nextafter(1.0, 2.0),
                     np.nextafter(1.0, 0.0), np.nextafter(2.0, 1.0), np.ldexp(1.0, -1022), np.ldexp(1.0, 1020),
                     np.ldexp(1.5, -1000), np.ldexp(1.75, 1000)])
    return np.concatenate([wide, ops, edge])


def test_fp64_reciprocals_vs_ieee(dg):
    x = _inputs()
    cub, quad, adj, _, _ = [t.cpu().numpy() for t in dg.check_reciprocals(torch.from_numpy(x).cuda())]
    ref = 1.0 / x
    ulp = np.spacing(ref)
    # cubic refinement: within one ulp of the correctly rounded reciprocal,
    # and exact (correctly rounded) for almost every input
    err_cub = np.abs(cub - ref) / ulp
    assert err_cub.max() <= 1.0, err_cub.max()
    assert np.mean(cub == ref) > 0.99
    # powers of two are exact
    p2 = x == np.ldexp(1.0, np.frexp(x)[1] - 1)
    assert np.array_equal(cub[p2], ref[p2])
    # quadratic refinement: relative error below 2^-38
    assert (np.abs(quad - ref) / ref).max() < 2.0 ** -38
    # the adjoint kernels use the cubic form, bit for bit
    assert np.array_equal(adj.view(np.uint64), cub.view(np.uint64))


def test_fp32_reciprocal_vs_ieee(dg):
    rng = np.random.default_rng(6)
    x = np.concatenate([np.ldexp(rng.uniform(1.0, 2.0, 200000), rng.integers(-120, 121, 200000)),
                        rng.uniform(0.02, 400.0, 100000), [1.0, 3.0, 0.1, 71.42857142857143]])
    _, _, _, f_op, f_q = [t.cpu().numpy() for t in dg.check_reciprocals(torch.from_numpy(x).cuda())]
    xf = x.astype(np.float32)
    ref = np.float32(1.0) / xf                  # correctly rounded in FP32
    err = np.abs(f_op.astype(np.float64) - ref.astype(np.float64)) / np.spacing(ref).astype(np.float64)
    assert err.max() <= 1.0, err.max()
    # both FP32 forms are the bare approximation
    assert np.array_equal(f_op.view(np.uint32), f_q.view(np.uint32))


def test_reciprocals_flush_subnormals(dg):
    """The .ftz approximation flushes subnormals: a reciprocal below the
    smallest normal double becomes 0; a subnormal or zero input gives a
    non-finite result.  Neither occurs for the operators' operands."""
    x = np.array([np.ldexp(1.0, 1023), np.ldexp(1.5, 1023), 5e-324, np.ldexp(1.0, -1060), 0.0])
    cub, quad, adj, _, _ = [t.cpu().numpy() for t in dg.check_reciprocals(torch.from_numpy(x).cuda())]
    for y in (cub, quad, adj):
        assert np.all(y[:2] == 0.0)
        assert not np.isfinite(y[2:]).any()
