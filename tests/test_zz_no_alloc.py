"""The allocation-free entry point (for callers that may not call cudaMalloc
while they run) against the regular dg_integrals, through the C ABI.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from workloads import box_mesh, random_state

torch = pytest.importorskip("torch")


def test_noalloc_rejects_bad_arguments_on_host():
    import paper_2605_28627_gb300 as dg
    L = dg.load()
    p = C.c_void_p(16)
    # more elements than the fixed scratch array holds
    assert L.dg_conserved_totals_noalloc(p, p, 3, dg.NODES_LGL, 131073, p, None) == dg.DG_EINVAL
    assert L.dg_conserved_totals_noalloc(None, None, 3, dg.NODES_LGL, 8, None, None) == dg.DG_EINVAL
    # unknown node set, degree out of range
    assert L.dg_conserved_totals_noalloc(p, p, 3, 7, 8, p, None) == dg.DG_EINVAL
    assert L.dg_conserved_totals_noalloc(p, p, 10, dg.NODES_LGL, 8, p, None) == dg.DG_EUNSUPPORTED


def _check_two_calls(dg, mesh, N, nodes, seeds):
    s = dg.Solver(mesh, N, mu=0.01, nodes=nodes)
    _, J = s.geometry()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for seed in seeds:                        # two calls in a row, different states
        # on Gauss nodes the face values are extrapolated: a narrower range keeps them admissible
        rng = {} if nodes == dg.NODES_LGL else dict(rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
        U = torch.from_numpy(random_state(mesh.n_elems, N, seed=seed, **rng)).cuda()
        ref = s.integrals(U)[:5]
        got = dg.conserved_totals_noalloc(U, J, N, out=out, nodes=nodes)
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-12, atol=1e-13)
    s.close()


# 27 elements: not a multiple of the 8 element-warps of a block.  N = 1 has no
# interior LGL node, even N puts one at the midpoint, N = 9 is the largest
# degree the library builds.
@pytest.mark.gpu
@pytest.mark.parametrize("N", [1, 2, 3, 7, 9])
def test_noalloc_totals_match_integrals_two_calls(N):
    import paper_2605_28627_gb300 as dg
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=77)
    _check_two_calls(dg, mesh, N, dg.NODES_LGL, (1, 2))


# Gauss-node contexts weight with the Gauss quadrature, as dg_integrals does.
@pytest.mark.gpu
@pytest.mark.parametrize("N", [1, 4, 7])
def test_noalloc_totals_gauss_nodes(N):
    import paper_2605_28627_gb300 as dg
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=78)
    _check_two_calls(dg, mesh, N, dg.NODES_LG, (3, 4))


# More elements than the fold block's 256 threads (each thread folds several
# rows), at N = 7; and a mesh near the 131072-element cap.
@pytest.mark.gpu
@pytest.mark.parametrize("K,N", [(7, 7), (50, 1)])
def test_noalloc_totals_large_meshes(K, N):
    import paper_2605_28627_gb300 as dg
    mesh = box_mesh(K, 1, deform="sinprod", rotate_seed=79)
    _check_two_calls(dg, mesh, N, dg.NODES_LGL, (5, 6))
