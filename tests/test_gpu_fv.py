"""FV sub-cell elements on the GPU (dg_set_fv_mask) against the oracle's FV
branch, element by element, through the C ABI.

Both node sets (LGL with the split form, Legendre-Gauss with the weak form).
Bar: the DG operator's, R(U) within 1e-12 relative per variable (scaled by
max |R|), grown with the conditioning of the mesh-sample interpolation as for
the DG tests; RK steps within 1e-10.  The FV residual reaches the nodes
through the inverse means map V3^-1 (||V^-1||_2 = 2.0, 4.0, 8.9, 23, 67 at
N = 1, 3, 5, 7, 9), but relative to max |R| that factor applies to R and to
its rounding alike: the measured differences stay at the DG operator's size
(<= 4.5e-13 at N = 9).  Meshes are curvilinear with random element frames
(all face orientations).
"""
import math

import numpy as np
import pytest

from workloads import box_mesh, mms_params, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_RK = 1e-10


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rtol(N):
    """1e-12, times kappa^3 / 300 where the interpolation of the equispaced
    mesh samples (degree N) to the LGL nodes amplifies their rounding by kappa
    per direction (kappa^3 > 300 from N = 8 on)."""
    import oracle
    x, _, _ = oracle.basis(N)
    xe = np.linspace(-1.0, 1.0, N + 1)
    V = np.array([[np.prod([(xi - xe[m]) / (xe[j] - xe[m]) for m in range(N + 1) if m != j])
                   for j in range(N + 1)] for xi in x])
    return 1e-12 * max(1.0, np.abs(V).sum(1).max() ** 3 / 300.0)


def _rel_err_per_var(got, ref):
    got = got.reshape(got.shape[0], 5, -1)
    ref = ref.reshape(ref.shape[0], 5, -1)
    return np.array([np.abs(got[:, v] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-300) for v in range(5)])


def _state(n_elems, N, seed, nodes=0):
    """Random admissible state of moderate amplitude: its sub-cell means stay
    admissible up to N = 9 (the means map has row sums 1 but |V| row sums up
    to 1.9 per direction); narrower on Gauss nodes, whose face values are
    extrapolated from the nodes."""
    if nodes == 1:
        return random_state(n_elems, N, seed=seed, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    return random_state(n_elems, N, seed=seed, rho=(0.9, 1.1), vel=0.3, p=(0.9, 1.1))


def _checkerboard(K):
    e = np.arange(K ** 3)
    return (((e % K) + (e // K) % K + e // (K * K)) % 2).astype(np.int32)


def _mask(kind, K, seed=0):
    if kind == "checker":
        return _checkerboard(K)
    if kind == "all":
        return np.ones(K ** 3, dtype=np.int32)
    return np.random.default_rng(seed).integers(0, 2, K ** 3).astype(np.int32)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("kind", ["checker", "random", "all"])
def test_fv_time_derivative_parity(orc, dg, N, kind):
    K = 3 if N <= 5 else 2
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=700 + N)
    kw = dict(mu=0.02, surf_flux=N % 3)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    mask = _mask(kind, K, seed=N)
    o.set_fv_mask(mask)
    s.set_fv_mask(_cuda(mask))
    U = _state(mesh.n_elems, N, 800 + N)
    ref = o.time_derivative(U)
    assert np.isfinite(ref).all()
    got = s.time_derivative(_cuda(U)).cpu().numpy()
    err = _rel_err_per_var(got, ref)
    print("FV parity N=%d %s: max rel err %.3e (bar %.1e)" % (N, kind, err.max(), _rtol(N)))
    assert (err < _rtol(N)).all(), err


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9])
@pytest.mark.parametrize("kind", ["checker", "random"])
def test_fv_time_derivative_parity_gauss_nodes(orc, dg, N, kind):
    K = 3 if N <= 5 else 2
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=760 + N)
    kw = dict(mu=0.02, surf_flux=N % 3, nodes=1)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    mask = _mask(kind, K, seed=N + 20)
    o.set_fv_mask(mask)
    s.set_fv_mask(_cuda(mask))
    U = _state(mesh.n_elems, N, 860 + N, nodes=1)
    ref = o.time_derivative(U)
    assert np.isfinite(ref).all()
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), ref)
    print("FV parity (Gauss nodes) N=%d %s: max rel err %.3e (bar %.1e)" % (N, kind, err.max(), _rtol(N)))
    assert (err < _rtol(N)).all(), err


@pytest.mark.parametrize("N", [2, 3])
def test_fv_parity_sutherland_and_roe(orc, dg, N):
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=720 + N)
    kw = dict(mu=0.03, surf_flux=2, visc_law=1, T_ref=1.0, S_suth=0.4)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    mask = _mask("random", 3, seed=11)
    o.set_fv_mask(mask)
    s.set_fv_mask(mask)                       # a host array is copied to the device
    U = _state(mesh.n_elems, N, 820 + N)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < _rtol(N)).all(), err


@pytest.mark.parametrize("nodes", [0, 1])
def test_all_dg_mask_and_mask_off_are_the_dg_operator_bitwise(dg, nodes):
    """Above the latency-kernel size (21952 nodes), where the DG operator runs
    the same kernels with and without a mask."""
    N = 3
    mesh = box_mesh(7, N, deform="sinprod", rotate_seed=31)
    s = dg.Solver(mesh, N, mu=0.01, nodes=nodes)
    U = _cuda(_state(mesh.n_elems, N, 5, nodes))
    R0 = s.time_derivative(U).clone()
    s.set_fv_mask(torch.zeros(mesh.n_elems, dtype=torch.int32, device="cuda"))
    assert torch.equal(s.time_derivative(U), R0)
    s.set_fv_mask(torch.ones(mesh.n_elems, dtype=torch.int32, device="cuda"))
    assert not torch.allclose(s.time_derivative(U), R0)
    s.set_fv_mask(None)
    assert torch.equal(s.time_derivative(U), R0)


@pytest.mark.parametrize("N,nodes", [(3, 0), (5, 0), (3, 1)])
def test_fv_mms_rk_parity_with_mask_changes(orc, dg, N, nodes):
    """LSERK4-5 steps with a checkerboard, then another mask inside the same
    captured graph (the kernels read the mask at run time), then DG again."""
    prm = mms_params()
    K = 3
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=740 + N)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1, nodes=nodes)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    U0 = o.initial_state("mms", 0.0)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    m1, m2 = _mask("checker", K), _mask("random", K, seed=3)
    dt = 1e-3
    o.set_fv_mask(m1)
    ref = o.rk_steps(U0, 0.0, dt, 3)
    o.set_fv_mask(m2)
    ref = o.rk_steps(ref, 3 * dt, dt, 3)
    o.set_fv_mask(None)
    ref = o.rk_steps(ref, 6 * dt, dt, 2)
    s.set_fv_mask(m1)
    s.rk_step(Ud, G, 0.0, dt, 3)
    s.set_fv_mask(m2)
    s.rk_step(Ud, G, 3 * dt, dt, 3)
    s.set_fv_mask(None)
    s.rk_step(Ud, G, 6 * dt, dt, 2)
    got = Ud.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < RTOL_RK


@pytest.mark.parametrize("nodes", [0, 1])
def test_fv_free_stream_and_conservation_on_gpu(orc, dg, nodes):
    N, K = 3, 8
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=77)
    s = dg.Solver(mesh, N, mu=0.01, nodes=nodes)
    s.set_fv_mask(_checkerboard(K))
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = s.time_derivative(_cuda(U))
    assert float(R.abs().max()) < 1e-11
    U = _cuda(_state(mesh.n_elems, N, 9, nodes))
    R = s.time_derivative(U)
    _, J = s.geometry()
    w = (orc.basis(N) if nodes == 0 else orc.gauss_basis(N))[1]
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w).reshape(-1)).cuda()
    tot = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1), J * wq)
    scale = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1).abs(), J * wq)
    assert bool((tot.abs() <= 1e-13 * scale).all()), (tot, scale)


@pytest.mark.parametrize("N,nodes", [(4, 0), (7, 0), (9, 0), (3, 1), (7, 1)])
def test_fv_mixed_free_stream_stays_bounded_on_gpu(dg, N, nodes):
    """A free stream on a DG/FV checkerboard, 200 LSERK4-5 steps at CFL 0.9:
    the rounding-level departure stays bounded (no growing mode at the DG/FV
    interfaces)."""
    K = 4
    mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, mu=1.0 / 1600, nodes=nodes)
    s.set_fv_mask(_checkerboard(K))
    u = (0.1, 0.05, 0.02)
    U = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    U[:, 0] = 1.0
    for a in range(3):
        U[:, 1 + a] = u[a]
    U[:, 4] = 1.0 / 1.4 / 0.4 + 0.5 * sum(c * c for c in u)
    U0 = U.clone()
    G = torch.empty_like(U)
    dt = s.max_dt(U, cfl=0.9, dfl=0.9)
    drift = []
    for blk in range(4):
        s.rk_step(U, G, blk * 50 * dt, dt, 50)
        drift.append(float((U - U0).abs().max() / U0.abs().max()))
    assert max(drift) < 1e-10 and drift[-1] < 3.0 * drift[0], drift


def _shock_state(X, gamma=1.4):
    """A density and pressure jump across a tilted plane on a smooth field."""
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    sw = (0.6 * x + 0.3 * y - 0.2 * z > 0.1).astype(float)
    rho = 1.0 + 0.1 * np.sin(np.pi * x) + 1.5 * sw
    u = np.stack([0.2 + 0.0 * x, 0.1 * np.cos(np.pi * y), 0.0 * x])
    p = 1.0 + 2.0 * sw
    return np.concatenate([rho[:, None], (rho * u).transpose(1, 0, 2), (p / (gamma - 1) + 0.5 * rho * (u * u).sum(0))[:, None]], 1)


def test_indicator_flags_drive_the_fv_operator(orc, dg):
    """The Persson indicator's flags (device) passed to dg_set_fv_mask as
    they are: the flags equal the oracle's, and R equals the oracle's with
    that mask."""
    N, K = 4, 3
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=91)
    o, s = orc.Oracle(mesh, N, mu=0.005), dg.Solver(mesh, N, mu=0.005)
    X = o.node_coords()
    U = _shock_state(X).reshape(o.shape)
    thr = -3.0
    eta_o = o.persson(U, 2)
    flags_o = ((eta_o > 0) & (np.log10(np.maximum(eta_o, 1e-300)) > thr)).astype(np.int32)
    Ud = _cuda(U)
    _, flag = s.indicator(Ud, 2, thr)
    assert 0 < flags_o.sum() < mesh.n_elems
    assert np.array_equal(flag.cpu().numpy(), flags_o)
    s.set_fv_mask(flag)
    o.set_fv_mask(flags_o)
    err = _rel_err_per_var(s.time_derivative(Ud).cpu().numpy(), o.time_derivative(U))
    assert (err < _rtol(N)).all(), err


def test_fv_full_size_sampled_elements_against_oracle_patch(orc, dg):
    """16^3 curved-free Cartesian elements at N=7 with the checkerboard mask
    (the FV launch configuration of the benchmark): R at sampled elements
    equals the oracle's R at the centre of a periodic 5^3 patch holding the
    same states and mask (R reaches two elements out)."""
    N, K = 7, 16
    L = 2 * math.pi
    mesh = box_mesh(K, 1, lo=0.0, hi=L)
    mu = 1.0 / 1600
    s = dg.Solver(mesh, N, mu=mu)
    mask = _checkerboard(K)
    s.set_fv_mask(mask)
    n = N + 1
    U = _state(mesh.n_elems, N, 43).reshape(K, K, K, 5, n, n, n)
    R = s.time_derivative(_cuda(U.reshape(s.shape))).cpu().numpy().reshape(K, K, K, 5, n, n, n)
    patch_mesh = box_mesh(5, 1, lo=0.0, hi=1.0)
    xg_all = mesh.xgeo.reshape(K, K, K, 3, 2, 2, 2)
    m3 = mask.reshape(K, K, K)
    rng = np.random.default_rng(10)
    for _ in range(3):
        cz, cy, cx = rng.integers(0, K, size=3)
        idx = [(np.arange(5) + c - 2) % K for c in (cz, cy, cx)]
        xg = np.ascontiguousarray(xg_all[np.ix_(idx[0], idx[1], idx[2])].reshape(125, 3, 2, 2, 2))
        o = orc.Oracle(type(patch_mesh)(**{**patch_mesh.__dict__, "xgeo": xg}), N, mu=mu)
        o.set_fv_mask(m3[np.ix_(idx[0], idx[1], idx[2])].reshape(125))
        Up = U[np.ix_(idx[0], idx[1], idx[2])].reshape(125, 5, n, n, n)
        Rp = o.time_derivative(Up).reshape(5, 5, 5, 5, n, n, n)
        ref, got = Rp[2, 2, 2], R[cz, cy, cx]
        for v in range(5):
            assert np.abs(got[v] - ref[v]).max() <= _rtol(N) * np.abs(ref[v]).max()


def test_fv_rejections(dg):
    mesh = box_mesh(2, 1)
    s32 = dg.Solver(mesh, 2, precision=1)
    with pytest.raises(dg.DGError):
        s32.set_fv_mask(np.ones(mesh.n_elems, dtype=np.int32))
    s = dg.Solver(mesh, 2, mu=0.01)
    s.set_fv_mask(np.ones(mesh.n_elems, dtype=np.int32))
    U = _cuda(_state(mesh.n_elems, 2, 1))
    with pytest.raises(dg.DGError):
        s.time_derivative_vjp(U, torch.ones_like(U))
    with pytest.raises(ValueError):
        s.set_fv_mask(np.ones(mesh.n_elems + 1, dtype=np.int32))
    # with its FV elements set before the ensemble is created, the member runs
    # as a single-member unit; a tile-table member that gets FV elements later
    # is refused when stepped
    G = torch.empty_like(U)
    ens = dg.Ensemble([s])
    ens.step([U], [G], [0.0], [1e-3], nsteps=1)
    ens.close()
    s.set_fv_mask(None)
    ens = dg.Ensemble([s])
    s.set_fv_mask(np.ones(mesh.n_elems, dtype=np.int32))
    with pytest.raises(dg.DGError):
        ens.step([U], [G], [0.0], [1e-3], nsteps=1)
    s.set_fv_mask(None)
    ens.step([U], [G], [0.0], [1e-3], nsteps=1)
    ens.close()
