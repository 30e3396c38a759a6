"""Modal troubled-cell indicator (Persson & Peraire 2006, the detector of the
FV sub-cell shock capturing, Sec. 3.1) on the GPU against the oracle, element
by element, through the C ABI: random states (every mode excited), smooth
states (energy shares down to 1e-12), both node sets, N = 1..9, meshes with a
ragged last block; flags against the oracle's FP64 decision.

The two codes reach the modes differently (the oracle inverts the Vandermonde
matrix; the library uses the node set's discrete orthogonality), so eta is
compared with |d eta| <= 1e-12 eta + 1e-14 sqrt(eta): the rounding of the
modal coefficients (1e-16 of the field) enters eta through the top modes,
which are sqrt(eta) of the field."""
import math

import numpy as np
import pytest

from workloads import box_mesh, random_state, tgv_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _close(got, ref):
    return np.abs(got - ref) <= 1e-12 * ref + 1e-14 * np.sqrt(ref)


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_indicator_random_states(orc, dg, N, nodes):
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=200 + N)
    o = orc.Oracle(mesh, N, nodes=nodes)
    s = dg.Solver(mesh, N, nodes=nodes)
    rng = {} if nodes == 0 else dict(rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    U = random_state(mesh.n_elems, N, seed=300 + N, **rng)
    Ud = torch.from_numpy(U).cuda()
    for var in (dg.IND_RHO, dg.IND_P, dg.IND_RHOP):
        ref = o.persson(U, var)
        eta, flag = s.indicator(Ud, var, log10_threshold=-2.0)
        got = eta.cpu().numpy()
        assert _close(got, ref).all(), (var, np.abs(got - ref).max())
        f = flag.cpu().numpy()
        lr = np.log10(np.maximum(ref, 1e-300))
        sure = np.abs(lr + 2.0) > 1e-9
        assert np.array_equal(f[sure], (lr[sure] > -2.0).astype(np.int32)[sure])
    s.close()


@pytest.mark.parametrize("N", [3, 7])
def test_indicator_smooth_and_discontinuous(orc, dg, N):
    """A smooth Taylor-Green state: tiny shares on every element, matched by
    the GPU; the same state with a density jump across a plane marks exactly
    the elements the jump passes through (threshold between the two)."""
    prm = tgv_params(Ma=0.3, Re=1600.0)
    mesh = box_mesh(4, 1, lo=0.0, hi=2 * math.pi)
    o = orc.Oracle(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U = o.initial_state("tgv", prm["p0"])
    ref = o.persson(U, dg.IND_RHOP)
    eta, _ = s.indicator(torch.from_numpy(U).cuda(), dg.IND_RHOP)
    got = eta.cpu().numpy()
    assert ref.max() < 1e-4 and _close(got, ref).all()
    # a jump of the density at x = 2.4 (inside the second column of elements)
    X = o.node_coords().reshape(mesh.n_elems, 3, N + 1, N + 1, N + 1)
    Uj = U.copy()
    scale = np.where(X[:, 0] > 2.4, 1.5, 1.0)
    Uj[:, 0] *= scale
    for a in range(1, 5):
        Uj[:, a] *= scale
    ref_j = o.persson(Uj, dg.IND_RHOP)
    eta_j, flag_j = s.indicator(torch.from_numpy(Uj).cuda(), dg.IND_RHOP, log10_threshold=-3.0)
    assert _close(eta_j.cpu().numpy(), ref_j).all()
    cut = (X[:, 0].min(axis=(1, 2, 3)) < 2.4) & (X[:, 0].max(axis=(1, 2, 3)) > 2.4)
    assert np.array_equal(flag_j.cpu().numpy().astype(bool), cut)
    s.close()


def test_indicator_rejects_bad_arguments(dg):
    mesh = box_mesh(2, 1)
    s = dg.Solver(mesh, 2)
    U = s.initial_state("tgv", 10.0)
    with pytest.raises(dg.DGError):
        s.indicator(U, var=5)
    s.close()
