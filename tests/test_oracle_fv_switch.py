"""Oracle pins for the automatic DG/FV switching (GALAEXI Sec. 3.1: the modal
indicator marks the troubled DG elements that the FV sub-cell operator takes
over; Sec. 3.2.2 lists the switch as a kernel step).  Before each evaluation of
R(U) the Persson indicator of the evaluated state decides: FV above the upper
threshold or where a node's density or pressure is not positive, DG below the
lower threshold with every node admissible, unchanged in between.

Pins: thresholds no indicator reaches give the DG operator bit for bit; the
mask after one evaluation follows the rule from the indicator values (pinned
against numpy's Legendre polynomials in test_oracle_persson.py) and the mask
before it, including the forced switch of an inadmissible element; the totals
stay conserved through steps that switch elements; and on a Sod-type slab the
run stays finite with admissible sub-cell means, where dropping the
admissibility rule lets an element go back to DG with negative nodal
pressures (the run then fails within 25 steps)."""
import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from workloads import box_mesh, random_state

GAMMA = 1.4


def _slab(o, x0=0.43, inside=(1.0, 1.0), outside=(0.125, 0.1)):
    """Density and pressure (inside) for |x| < x0, (outside) elsewhere, at rest."""
    X = o.node_coords()
    sel = np.abs(X[:, 0]) < x0
    rho = np.where(sel, inside[0], outside[0])
    p = np.where(sel, inside[1], outside[1])
    U = np.zeros((o.E, 5, X.shape[-1]))
    U[:, 0] = rho
    U[:, 4] = p / (GAMMA - 1)
    return U.reshape(o.shape)


def _sub_means_matrix(x):
    """V[a][j]: mean of the Lagrange polynomial j of the nodes x over the a-th
    of n equal sub-intervals of [-1, 1] (numpy polynomial integrals)."""
    n = len(x)
    h = 2.0 / n
    V = np.zeros((n, n))
    for j in range(n):
        c = np.array([1.0])
        for m in range(n):
            if m != j:
                c = npoly.polymul(c, np.array([-x[m], 1.0]) / (x[j] - x[m]))
        ci = npoly.polyint(c)
        for a in range(n):
            lo = -1.0 + a * h
            V[a, j] = (npoly.polyval(lo + h, ci) - npoly.polyval(lo, ci)) / h
    return V


def _prims(a):
    rho = a[:, 0]
    p = (GAMMA - 1) * (a[:, 4] - 0.5 * (a[:, 1] ** 2 + a[:, 2] ** 2 + a[:, 3] ** 2) / rho)
    return rho, p


@pytest.mark.parametrize("nodes", [0, 1])
def test_unreachable_thresholds_give_the_dg_operator(orc, nodes):
    m = box_mesh(2, 2, deform="sinprod", rotate_seed=3)
    N = 3
    U = random_state(m.n_elems, N, seed=5, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    ref = orc.Oracle(m, N, mu=0.01, nodes=nodes).rk_steps(U, 0.0, 1e-3, 2)
    o = orc.Oracle(m, N, mu=0.01, nodes=nodes)
    o.set_fv_switch(2, 1.0, 1.0)          # eta <= 1: log10 eta never above 1
    got = o.rk_steps(U, 0.0, 1e-3, 2)
    assert np.array_equal(got, ref)
    assert o.fv_state()[0].sum() == 0


def test_mask_follows_the_rule(orc):
    N = 4
    m = box_mesh(3, 1, rotate_seed=8)
    o = orc.Oracle(m, N, mu=0.01)
    U = random_state(m.n_elems, N, seed=2)
    le = np.log10(o.persson(U, 2))
    up, low = np.quantile(le, 0.7), np.quantile(le, 0.3)
    start = np.random.default_rng(4).integers(0, 2, m.n_elems)
    # one element with a negative pressure at a node, its indicator below low
    bad = int(np.argmin(le))
    Ub = U.reshape(m.n_elems, 5, -1).copy()
    Ub[bad, 4, 7] = 0.1 * (Ub[bad, 1, 7] ** 2 + Ub[bad, 2, 7] ** 2 + Ub[bad, 3, 7] ** 2) / Ub[bad, 0, 7]
    Ub = Ub.reshape(o.shape)
    le = np.log10(o.persson(Ub, 2))
    o.set_fv_mask(start)
    o.set_fv_switch(2, up, low)
    o.time_derivative(Ub)
    mask, margin = o.fv_state()
    want = np.where(le > up, 1, np.where(le < low, 0, start))
    want[bad] = 1
    assert margin > 1e-9
    assert np.array_equal(mask, want), (mask, want)
    assert 0 < (want != start).sum() < m.n_elems and le[bad] < low


@pytest.mark.parametrize("nodes", [0, 1])
def test_switching_steps_conserve(orc, nodes):
    N = 3
    m = box_mesh(8, 1, dims=(8, 2, 2), rotate_seed=4)
    o = orc.Oracle(m, N, mu=1e-3, nodes=nodes)
    o.set_fv_switch(2, -2.0, -3.0)
    U = _slab(o)
    x, w = (orc.basis(N) if nodes == 0 else orc.gauss_basis(N))[:2]
    wq = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    J = o.geometry()[2]
    tot0 = np.einsum("evp,ep->v", U.reshape(o.E, 5, -1), J * wq)
    seen = 0
    for k in range(6):
        U = o.rk_steps(U, k * 1e-3, 1e-3, 1)
        seen = max(seen, int(o.fv_state()[0].sum()))
    tot = np.einsum("evp,ep->v", U.reshape(o.E, 5, -1), J * wq)
    assert seen > 0
    # momentum starts at zero: one scale, the integral of |U| over all variables
    scale = np.einsum("evp,ep->", np.abs(U.reshape(o.E, 5, -1)), J * wq)
    assert (np.abs(tot - tot0) < 1e-14 * scale).all(), (tot - tot0, scale)


@pytest.mark.parametrize("N", [4, 5])
def test_sod_slab_stays_admissible(orc, N):
    """Sod-type slab (density 1 / 0.125, pressure 1 / 0.1) on a rotated
    Cartesian mesh: 60 steps with switching stay finite, the DG elements'
    nodes and the FV elements' sub-cell means admissible."""
    m = box_mesh(8, 1, dims=(8, 2, 2), rotate_seed=4)
    o = orc.Oracle(m, N, mu=1e-4)
    o.set_fv_switch(2, -2.0, -3.0)
    U = _slab(o)
    x = orc.basis(N)[0]
    V = _sub_means_matrix(x)
    n = N + 1
    ever = 0
    for k in range(60):
        U = o.rk_steps(U, k * 1e-3, 1e-3, 1)
        assert np.isfinite(U).all(), k
        mask, _ = o.fv_state()
        ever = max(ever, int(mask.sum()))
        r = U.reshape(o.E, 5, n, n, n)
        M = np.einsum("ai,bj,ck,evkji->evcba", V, V, V, r)     # affine elements: J is constant
        rho_n, p_n = _prims(r[mask == 0])
        rho_m, p_m = _prims(M[mask != 0])
        assert rho_n.min() > 0 and p_n.min() > 0, k
        if mask.any():
            assert rho_m.min() > 0 and p_m.min() > 0, k
    assert ever > 0


def test_switch_rejections(orc):
    from workloads.mesh import refined_box_mesh
    o = orc.Oracle(box_mesh(2, 1), 2)
    with pytest.raises(ValueError):
        o.set_fv_switch(3, -2.0, -3.0)
    with pytest.raises(ValueError):
        o.set_fv_switch(2, -3.0, -2.0)          # upper below lower
    r = np.zeros(8, dtype=bool)
    r[0] = True
    om = orc.Oracle(refined_box_mesh(2, r), 2)
    om.set_fv_switch(2, -2.0, -3.0)           # mortar meshes: elements with a mortar face stay DG
