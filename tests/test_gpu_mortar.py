"""Mortar faces on the GPU (non-conforming 2:1 meshes, Sec. 3.2.2, Algorithm 1)
against the oracle, through the C ABI.  Bars as for conforming meshes: R(U)
within 1e-12 relative per variable, RK steps within 1e-10."""
import numpy as np
import pytest

from workloads import mms_params, random_state
from workloads.mesh import refined_box_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _refine(K, cells):
    r = np.zeros(K ** 3, dtype=bool)
    r[list(cells)] = True
    return r


def _rel_err_per_var(got, ref):
    got = got.reshape(got.shape[0], 5, -1)
    ref = ref.reshape(ref.shape[0], 5, -1)
    return np.array([np.abs(got[:, v] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-300) for v in range(5)])


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_mortar_time_derivative_parity(orc, dg, N, flux):
    # straight-sided elements: no geometric amplification of the rounding at N = 8, 9
    K = 3 if N <= 7 else 2
    mesh = refined_box_mesh(K, _refine(K, [0, 13] if K == 3 else [0, 7]), rotate_seed=40 + N)
    kw = dict(mu=0.02, surf_flux=flux)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    U = random_state(mesh.n_elems, N, seed=60 + N)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < 1e-12).all(), err


@pytest.mark.parametrize("N", [2, 5])
def test_mortar_mms_rk_parity(orc, dg, N):
    prm = mms_params()
    K = 3
    mesh = refined_box_mesh(K, _refine(K, [4, 13, 22]), rotate_seed=70 + N)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    U0 = o.initial_state("mms", 0.0)
    ref = o.rk_steps(U0, 0.0, 1e-3, 10)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 10)
    got = Ud.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-10


def test_mortar_free_stream_and_conservation(orc, dg):
    N, K = 4, 4
    mesh = refined_box_mesh(K, _refine(K, [0, 21, 42, 63]), rotate_seed=8)
    s = dg.Solver(mesh, N, mu=0.01)
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = s.time_derivative(_cuda(U))
    _, J = s.geometry()
    _, w, _ = orc.basis(N)
    assert float(R.abs().max()) < 2e-15 * 2.0 / (w[0] * float(J.min())) * N ** 3
    U = _cuda(random_state(mesh.n_elems, N, seed=9))
    R = s.time_derivative(U)
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w).reshape(-1)).cuda()
    tot = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1), J * wq)
    scale = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1).abs(), J * wq)
    assert bool((tot.abs() <= 1e-13 * scale).all()), (tot, scale)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_mortar_fp32_operator_vs_oracle(orc, dg, N):
    """FP32 operator arithmetic (FP64 states and maps in the mortar kernels):
    R(U) within the FP32 operator's bar, 2e-5 of max |R| per variable."""
    K = 3 if N <= 5 else 2
    mesh = refined_box_mesh(K, _refine(K, [0, 13] if K == 3 else [0, 7]), rotate_seed=90 + N)
    o = orc.Oracle(mesh, N, mu=0.02)
    s = dg.Solver(mesh, N, mu=0.02, precision=dg.FP32OP)
    U = random_state(mesh.n_elems, N, seed=70 + N)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < 2e-5).all(), err


def test_mortar_fp32_mms_steps_and_conservation(orc, dg):
    prm = mms_params()
    N, K = 4, 3
    mesh = refined_box_mesh(K, _refine(K, [4, 13, 22]), rotate_seed=5)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o = orc.Oracle(mesh, N, **kw)
    s = dg.Solver(mesh, N, precision=dg.FP32OP, **kw)
    U0 = o.initial_state("mms", 0.0)
    ref = o.rk_steps(U0, 0.0, 1e-3, 10)
    Ud = _cuda(U0)
    s.rk_step(Ud, torch.empty_like(Ud), 0.0, 1e-3, 10)
    # the FP32 operator's state bar: FP32 rounding of the stage updates relative to |U|
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-6
    # discrete conservation through the mortars: FP32 flux rounding only
    s2 = dg.Solver(mesh, N, mu=0.02, precision=dg.FP32OP)
    Ur = _cuda(random_state(mesh.n_elems, N, seed=9))
    R = s2.time_derivative(Ur)
    _, J = s2.geometry()
    _, w, _ = orc.basis(N)
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w).reshape(-1)).cuda()
    tot = torch.einsum("evp,ep->v", R.reshape(s2.E, 5, -1), J * wq)
    scale = torch.einsum("evp,ep->v", R.reshape(s2.E, 5, -1).abs(), J * wq)
    assert bool((tot.abs() <= 1e-6 * scale).all()), (tot, scale)


_GAUSS_STATE = dict(rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))   # face values extrapolated from the nodes


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_mortar_time_derivative_parity_gauss_nodes(orc, dg, N, flux):
    K = 3
    mesh = refined_box_mesh(K, _refine(K, [0, 13]), rotate_seed=140 + N)
    kw = dict(mu=0.02, surf_flux=flux, nodes=1)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    U = random_state(mesh.n_elems, N, seed=160 + N, **_GAUSS_STATE)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < 1e-12).all(), err


@pytest.mark.parametrize("N", [3, 6])
def test_mortar_mms_rk_parity_gauss_nodes(orc, dg, N):
    prm = mms_params()
    K = 3
    mesh = refined_box_mesh(K, _refine(K, [4, 13, 22]), rotate_seed=170 + N)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1, nodes=1)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    U0 = o.initial_state("mms", 0.0)
    ref = o.rk_steps(U0, 0.0, 1e-3, 10)
    Ud = _cuda(U0)
    s.rk_step(Ud, torch.empty_like(Ud), 0.0, 1e-3, 10)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10


def test_mortar_free_stream_and_conservation_gauss_nodes(orc, dg):
    N, K = 4, 4
    mesh = refined_box_mesh(K, _refine(K, [0, 21, 42, 63]), rotate_seed=8)
    s = dg.Solver(mesh, N, mu=0.01, nodes=1)
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = s.time_derivative(_cuda(U))
    _, J = s.geometry()
    w = orc.gauss_basis(N)[1]
    assert float(R.abs().max()) < 2e-15 * 2.0 / (w[0] * float(J.min())) * N ** 3
    U = _cuda(random_state(mesh.n_elems, N, seed=9, **_GAUSS_STATE))
    R = s.time_derivative(U)
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w).reshape(-1)).cuda()
    tot = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1), J * wq)
    scale = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1).abs(), J * wq)
    assert bool((tot.abs() <= 1e-13 * scale).all()), (tot, scale)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_mortar_fp32_operator_gauss_nodes_vs_oracle(orc, dg, N):
    """FP32 operator on Gauss nodes (FP32 face values, FP64 maps) with
    mortars: R(U) within the FP32 operator's bar."""
    K = 3
    mesh = refined_box_mesh(K, _refine(K, [0, 13]), rotate_seed=190 + N)
    o = orc.Oracle(mesh, N, mu=0.02, nodes=1)
    s = dg.Solver(mesh, N, mu=0.02, nodes=dg.NODES_LG, precision=dg.FP32OP)
    U = random_state(mesh.n_elems, N, seed=200 + N, **_GAUSS_STATE)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < 2e-5).all(), err


def test_mortar_rejections(dg):
    mesh = refined_box_mesh(2, _refine(2, [0]))
    s = dg.Solver(mesh, 2, mu=0.01)
    U = _cuda(random_state(mesh.n_elems, 2, seed=1))
    with pytest.raises(dg.DGError):
        s.set_fv_mask(np.ones(mesh.n_elems, dtype=np.int32))
    ens = dg.Ensemble([s])        # a mortar mesh runs as a single-member unit of the ensemble
    ens.step([U], [torch.empty_like(U)], [0.0], [1e-3])
    ens.close()
    bad = refined_box_mesh(2, _refine(2, [0]))
    bad.mortars = bad.mortars.copy()
    bad.mortars[0, 2] = bad.mortars[0, 5]
    with pytest.raises(dg.DGError):
        dg.Solver(bad, 2)


def _term_scale(orc, o, U, N):
    """Per variable: max_i sum_m |2 D_im| x 3 max |f(q) . Ja^d| / min J, the
    size of the flux-differencing terms whose sum is R (as in the MMS test of
    the conforming operator)."""
    _, Ja, J = o.geometry()
    _, _, D = orc.basis(N)
    Uf = U.reshape(U.shape[0], 5, -1)
    r = Uf[:, 0]
    u = Uf[:, 1:4] / r[:, None]
    p = 0.4 * (Uf[:, 4] - 0.5 * r * (u ** 2).sum(1))
    out = np.zeros(5)
    for d in range(3):
        un = np.einsum("elp,elp->ep", u, Ja[:, d])
        f = [r * un] + [Uf[:, 1 + a] * un + p * Ja[:, d, a] for a in range(3)] + [(Uf[:, 4] + p) * un]
        for v in range(5):
            out[v] = max(out[v], np.abs(f[v]).max())
    return 3 * out * 2 * np.abs(D).sum(1).max() / J.min()


def test_mortar_bench_mesh_full_size(orc, dg):
    """The 2:1 mesh of the bench (12^3 box, the cells with three even indices
    split: 3240 elements, 1296 mortars, N = 7, MMS source) at its full size,
    every node against the oracle: R(U) of a random state (1e-12 of max |R|),
    R(U) of the manufactured solution (a small residual of cancelling terms:
    1e-12 of the terms' size, the metric terms of the two codes differing by
    their rounding, 1e-13 relative at N = 7), and one RK step."""
    prm = mms_params()
    K, N = 12, 7
    i = np.arange(K ** 3)
    mesh = refined_box_mesh(K, (i % 2 == 0) & ((i // K) % 2 == 0) & ((i // (K * K)) % 2 == 0), rotate_seed=3)
    assert len(mesh.mortars) == 1296
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o, s = orc.Oracle(mesh, N, **kw), dg.Solver(mesh, N, **kw)
    Ur = random_state(mesh.n_elems, N, seed=11)
    err = _rel_err_per_var(s.time_derivative(_cuda(Ur), t=0.0).cpu().numpy(), o.time_derivative(Ur, t=0.0))
    assert (err < 1e-12).all(), err
    U0 = o.initial_state("mms", 0.0)
    d = np.abs(s.time_derivative(_cuda(U0), t=0.0).cpu().numpy() - o.time_derivative(U0, t=0.0))
    assert (d.reshape(mesh.n_elems, 5, -1).max(axis=(0, 2)) < 1e-12 * _term_scale(orc, o, U0, N)).all()
    ref = o.rk_steps(U0, 0.0, 5e-4, 1)
    Ud = _cuda(U0)
    s.rk_step(Ud, torch.empty_like(Ud), 0.0, 5e-4, 1)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
