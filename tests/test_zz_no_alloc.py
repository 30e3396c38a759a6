"""The allocation-free entry point (for callers that may not call cudaMalloc
while they run) against the regular dg_integrals, through the C ABI.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from workloads import box_mesh, random_state

torch = pytest.importorskip("torch")


def test_noalloc_rejects_oversized_mesh_on_host():
    import paper_2605_28627_gb300 as dg
    L = dg.load()
    st = L.dg_conserved_totals_noalloc(C.c_void_p(16), C.c_void_p(16), 3, 131073, C.c_void_p(16), None)
    assert st == dg.DG_EINVAL
    assert L.dg_conserved_totals_noalloc(None, None, 3, 8, None, None) == dg.DG_EINVAL


@pytest.mark.gpu
def test_noalloc_totals_match_integrals_two_calls():
    import paper_2605_28627_gb300 as dg
    N = 3
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=77)
    s = dg.Solver(mesh, N, mu=0.01)
    _, J = s.geometry()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for seed in (1, 2):                       # two calls in a row, different states
        U = torch.from_numpy(random_state(mesh.n_elems, N, seed=seed)).cuda()
        ref = s.integrals(U)[:5]
        got = dg.conserved_totals_noalloc(U, J, N, out=out)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)
    s.close()
