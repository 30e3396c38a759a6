"""Automatic DG/FV switching on the GPU (dg_set_fv_switch) against the oracle,
through the C ABI: before every evaluation of R(U) the indicator of the
evaluated state sets the FV mask (upper and lower thresholds, admissibility
rule).  Both sides decide in FP64 from indicator values that differ by
rounding only, so each run first checks on the oracle that no indicator value
came within 1e-9 (in log10) of a threshold; then the states after the RK
steps agree within 1e-10 and the final masks are equal."""
import numpy as np
import pytest

from workloads import box_mesh, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAMMA = 1.4


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _slab(X, x0=0.43, inside=(1.0, 1.0), outside=(0.125, 0.1)):
    sel = np.abs(X[:, 0]) < x0
    rho = np.where(sel, inside[0], outside[0])
    p = np.where(sel, inside[1], outside[1])
    U = np.zeros((X.shape[0], 5, X.shape[-1]))
    U[:, 0] = rho
    U[:, 4] = p / (GAMMA - 1)
    return U


@pytest.mark.parametrize("N,nodes,thr", [(3, 0, (-2.0, -3.0)), (4, 0, (-2.0, -3.0)), (5, 0, (-2.7, -3.7)),
                                         (3, 1, (-2.0, -3.0)), (4, 1, (-2.0, -3.0))])
def test_switching_rk_parity(orc, dg, N, nodes, thr):
    m = box_mesh(8, 1, dims=(8, 2, 2), rotate_seed=4)
    o = orc.Oracle(m, N, mu=1e-3, nodes=nodes)
    s = dg.Solver(m, N, mu=1e-3, nodes=nodes)
    U0 = _slab(o.node_coords()).reshape(o.shape)
    o.set_fv_switch(2, *thr)
    s.set_fv_switch(dg.IND_RHOP, *thr)
    ref = U0.copy()
    masks = 0
    for k in range(8):
        ref = o.rk_steps(ref, k * 1e-3, 1e-3, 1)
        mk, margin = o.fv_state()
        assert margin > 1e-9, (k, margin)
        masks = max(masks, int(mk.sum()))
    assert masks > 0
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 3)          # two graphs, the mask carried over
    s.rk_step(Ud, G, 3e-3, 1e-3, 5)
    got = Ud.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-10
    assert np.array_equal(s.fv_mask().cpu().numpy(), o.fv_state()[0])


def test_switching_time_derivative_parity_and_rule(orc, dg):
    """One evaluation from a given mask: the mask follows the rule (hysteresis
    keeps the starting mask between the thresholds), R(U) matches."""
    N = 4
    m = box_mesh(3, 1, deform="sinprod", rotate_seed=8)
    o = orc.Oracle(m, N, mu=0.01)
    s = dg.Solver(m, N, mu=0.01)
    U = random_state(m.n_elems, N, seed=2, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    le = np.log10(o.persson(U, 2))
    up, low = np.quantile(le, 0.75), np.quantile(le, 0.25)
    start = np.random.default_rng(4).integers(0, 2, m.n_elems).astype(np.int32)
    for side in (o, s):
        side.set_fv_mask(start)
    o.set_fv_switch(2, up, low)
    s.set_fv_switch(dg.IND_RHOP, up, low)
    Ro = o.time_derivative(U)
    mo, margin = o.fv_state()
    assert margin > 1e-9
    R = s.time_derivative(_cuda(U)).cpu().numpy()
    mg = s.fv_mask().cpu().numpy()
    assert np.array_equal(mg, mo)
    assert np.array_equal(mo, np.where(le > up, 1, np.where(le < low, 0, start)))
    assert np.abs(R - Ro).max() / np.abs(Ro).max() < 1e-11


def test_switching_off_keeps_the_mask_and_on_again_resets_the_graph(orc, dg):
    N = 3
    m = box_mesh(8, 1, dims=(8, 2, 2), rotate_seed=4)
    s = dg.Solver(m, N, mu=1e-3)
    o = orc.Oracle(m, N, mu=1e-3)
    U0 = _slab(o.node_coords()).reshape(o.shape)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 2)          # all DG, graph captured
    ref = o.rk_steps(U0, 0.0, 1e-3, 2)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
    s.set_fv_switch(dg.IND_RHOP, -2.0, -3.0)
    o.set_fv_switch(2, -2.0, -3.0)
    s.rk_step(Ud, G, 2e-3, 1e-3, 2)         # same pointers and count: the graph must be rebuilt
    ref = o.rk_steps(ref, 2e-3, 1e-3, 2)
    assert o.fv_state()[1] > 1e-9
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
    mask = s.fv_mask().cpu().numpy()
    assert mask.sum() > 0
    s.set_fv_switch(None)                   # off: the last mask stays in effect
    o.set_fv_switch(None)
    s.rk_step(Ud, G, 4e-3, 1e-3, 2)
    ref = o.rk_steps(ref, 4e-3, 1e-3, 2)
    assert np.array_equal(s.fv_mask().cpu().numpy(), mask)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10


def test_switching_rejections(dg):
    from workloads.mesh import refined_box_mesh
    m = box_mesh(2, 1)
    s = dg.Solver(m, 2)
    for args in ((3, -2.0, -3.0), (2, -3.0, -2.0), (2, float("nan"), -3.0)):
        with pytest.raises(dg.DGError):
            s.set_fv_switch(*args)
    with pytest.raises(dg.DGError):
        dg.Solver(m, 2, precision=dg.FP32OP).set_fv_switch(dg.IND_RHOP, -2.0, -3.0)
    r = np.zeros(8, dtype=bool)
    r[0] = True
    dg.Solver(refined_box_mesh(2, r), 2).set_fv_switch(dg.IND_RHOP, -2.0, -3.0)   # allowed on mortar meshes
    s.set_fv_switch(dg.IND_RHOP, -2.0, -3.0)
    U = _cuda(random_state(m.n_elems, 2, seed=1))
    with pytest.raises(dg.DGError):
        s.time_derivative_vjp(U, torch.ones_like(U))
    # switching set before the ensemble: a single-member unit that switches every stage
    ens = dg.Ensemble([s])
    ens.step([U], [torch.empty_like(U)], [0.0], [1e-3])
    ens.close()


def test_time_step_and_diagnostics_skip_inadmissible_fv_nodes(orc, dg):
    """A uniform state with one node of one element at negative pressure: as
    an FV element's node it does not enter dg_max_dt (the step equals that of
    the uniform state) nor, with Sutherland's law, eps (the integrals equal
    the oracle's, which skips it the same way); as a DG element's node it is
    an error."""
    N = 3
    m = box_mesh(2, 1, rotate_seed=2)
    kw = dict(mu=0.01, visc_law=dg.VISC_SUTHERLAND, T_ref=1.0, S_suth=0.4)
    s = dg.Solver(m, N, **kw)
    o = orc.Oracle(m, N, **kw)
    U = np.zeros(s.shape)
    r, u, p = 1.1, np.array([0.3, -0.1, 0.2]), 0.8
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / (GAMMA - 1) + 0.5 * r * u @ u
    U += 1e-3 * random_state(m.n_elems, N, seed=3)   # vorticity for eps
    dt0 = s.max_dt(_cuda(U))
    Ub = U.reshape(m.n_elems, 5, -1).copy()
    e, node = 3, 10
    Ub[e, 4, node] = 0.25 * (Ub[e, 1, node] ** 2 + Ub[e, 2, node] ** 2 + Ub[e, 3, node] ** 2) / Ub[e, 0, node]
    Ub = Ub.reshape(U.shape)
    with pytest.raises(dg.DGError):
        s.max_dt(_cuda(Ub))
    mask = np.zeros(m.n_elems, dtype=np.int32)
    mask[e] = 1
    s.set_fv_mask(mask)
    o.set_fv_mask(mask)
    dt1 = s.max_dt(_cuda(Ub))
    # the skipped node's neighbours keep the bound: within the 1e-3 perturbation
    assert 0 < dt1 and abs(dt1 - dt0) <= 0.02 * dt0
    Ig, Io = s.integrals(_cuda(Ub)), o.integrals(Ub)
    assert np.isfinite(Ig).all()
    np.testing.assert_allclose(Ig, Io, rtol=1e-11, atol=1e-13)
