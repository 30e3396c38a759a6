"""Gauss-node operator (standard weak-form DGSEM, GALAEXI Sec. 3.1 Eqs. 2-3)
on the GPU against the Gauss-node oracle, element by element, through the C
ABI: geometry at Gauss nodes and face points, R(U) for LLF, EC and Roe faces,
the manufactured source, ten LSERK4-5 steps, the integrals, and the options
the Gauss path rejects.  Same bars as the LGL parity tests."""
import math

import numpy as np
import pytest

from workloads import box_mesh, mms_params, random_state, tgv_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_R = 1e-12
RTOL_RK = 1e-10


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _geo_amp(orc, N, ngeo):
    """Rounding growth of the equispaced-sample interpolation (kappa^3 / 300,
    at least 1), as in the LGL parity tests."""
    x, _, _ = orc.basis(N)
    xe = np.linspace(-1.0, 1.0, ngeo + 1)
    V = np.array([[np.prod([(xi - xe[m]) / (xe[j] - xe[m]) for m in range(ngeo + 1) if m != j])
                   for j in range(ngeo + 1)] for xi in x])
    return max(1.0, np.abs(V).sum(1).max() ** 3 / 300.0)


def _state(mesh, N, seed):
    # admissible after extrapolation to the faces (|l_j(+-1)| sums grow with N)
    return random_state(mesh.n_elems, N, seed=seed, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))


def _rel_err(got, ref):
    got = got.reshape(got.shape[0], 5, -1)
    ref = ref.reshape(ref.shape[0], 5, -1)
    return np.array([np.abs(got[:, v] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-300) for v in range(5)])


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9])
def test_gauss_geometry_parity(orc, dg, N):
    mesh = box_mesh(3 if N < 5 else 2, N, deform="sinprod", rotate_seed=800 + N)
    o = orc.Oracle(mesh, N, nodes=1)
    s = dg.Solver(mesh, N, nodes=dg.NODES_LG)
    X, Ja, J = o.geometry()
    Jag, Jg = s.geometry()
    amp = _geo_amp(orc, N, N)
    np.testing.assert_allclose(s.node_coords().cpu().numpy(), X, rtol=0, atol=1e-14 * amp)
    np.testing.assert_allclose(Jg.cpu().numpy(), J, rtol=1e-12 * amp, atol=0)
    scale = np.abs(Ja).max() * max(1.0, np.abs(X).max())
    assert np.abs(Jag.cpu().numpy() - Ja).max() <= 1e-12 * amp * scale


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_gauss_time_derivative_parity(orc, dg, N, flux):
    K = 3 if N <= 4 else 2
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=900 + N)
    o = orc.Oracle(mesh, N, mu=0.02, surf_flux=flux, nodes=1)
    s = dg.Solver(mesh, N, mu=0.02, surf_flux=flux, nodes=dg.NODES_LG)
    U = _state(mesh, N, 1000 + N)
    err = _rel_err(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < RTOL_R * _geo_amp(orc, N, N)).all(), err


def test_gauss_free_stream_on_gpu(dg):
    N = 5
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=71)
    s = dg.Solver(mesh, N, mu=0.01, nodes=dg.NODES_LG)
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    assert np.abs(s.time_derivative(_cuda(U)).cpu().numpy()).max() < 2e-12 * N * N


@pytest.mark.parametrize("N", [3, 7])
def test_gauss_mms_rk_parity(orc, dg, N):
    prm = mms_params()
    mesh = box_mesh(3 if N < 7 else 2, N, deform="sinprod", rotate_seed=20260528)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o = orc.Oracle(mesh, N, nodes=1, **kw)
    s = dg.Solver(mesh, N, nodes=dg.NODES_LG, **kw)
    U0 = o.initial_state("mms", 0.0)
    np.testing.assert_allclose(s.initial_state("mms", 0.0).cpu().numpy(), U0, rtol=1e-14, atol=1e-14)
    ref = o.rk_steps(U0, 0.0, 1e-3, 10)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 4)
    s.rk_step(Ud, G, 4e-3, 1e-3, 6)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < RTOL_RK


def test_gauss_integrals_parity(orc, dg):
    prm = tgv_params(Ma=0.1, Re=1600.0)
    N = 4
    mesh = box_mesh(3, 1, lo=0.0, hi=2 * math.pi)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    o = orc.Oracle(mesh, N, nodes=1, **kw)
    s = dg.Solver(mesh, N, nodes=dg.NODES_LG, **kw)
    U = o.initial_state("tgv", prm["p0"])
    Io, Ig = o.integrals(U), s.integrals(_cuda(U))
    for a in (0, 4, 5, 6, 7):
        assert abs(Ig[a] - Io[a]) <= 1e-12 * abs(Io[a]), (a, Ig[a], Io[a])
    for a in (1, 2, 3):
        assert abs(Ig[a] - Io[a]) <= 1e-12 * abs(Io[0])


def test_gauss_rejections(dg):
    mesh = box_mesh(2, 2)
    s = dg.Solver(mesh, 2, mu=0.01, nodes=dg.NODES_LG)
    U = torch.from_numpy(_state(mesh, 2, 5)).cuda()
    sf = dg.Solver(mesh, 2, mu=0.01, nodes=dg.NODES_LG, precision=dg.FP32OP)   # the adjoint: FP64 operator
    with pytest.raises(dg.DGError):
        sf.time_derivative_vjp(U, torch.ones_like(U))
    ens = dg.Ensemble([s])            # a Gauss-node member runs as a single-member unit
    ens.step([U], [torch.empty_like(U)], [0.0], [1e-3])
    ens.close()


@pytest.mark.parametrize("N", [2, 3, 5, 7])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_gauss_fp32_operator_vs_oracle(orc, dg, N, flux):
    """FP32 operator on Gauss nodes (prolongation, lifting, face fluxes and the
    weak volume integral in FP32; state and RK update FP64) against the FP64
    oracle: the FP32 operator's bar, 2e-5 of max |R| per variable."""
    mesh = box_mesh(3 if N <= 4 else 2, N, deform="sinprod", rotate_seed=1100 + N)
    o = orc.Oracle(mesh, N, mu=0.02, surf_flux=flux, nodes=1)
    s = dg.Solver(mesh, N, mu=0.02, surf_flux=flux, nodes=dg.NODES_LG, precision=dg.FP32OP)
    U = _state(mesh, N, 1200 + N)
    got = s.time_derivative(_cuda(U)).cpu().numpy()
    ref = o.time_derivative(U)
    assert (_rel_err(got, ref) < 2e-5).all(), _rel_err(got, ref)


def test_gauss_fp32_operator_tgv_steps_and_free_stream(orc, dg):
    prm = tgv_params(Ma=0.1, Re=1600.0)
    N = 3
    mesh = box_mesh(4, 1, lo=0.0, hi=2 * math.pi)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], nodes=1)
    o = orc.Oracle(mesh, N, **kw)
    s = dg.Solver(mesh, N, precision=dg.FP32OP, **kw)
    U0 = o.initial_state("tgv", prm["p0"])
    Ud = _cuda(U0)
    dt = s.max_dt(Ud)
    ref = o.rk_steps(U0, 0.0, dt, 10)
    s.rk_step(Ud, torch.empty_like(Ud), 0.0, dt, 10)
    # state: FP32 rounding of the stage residuals relative to |U|; E_k as for the LGL FP32 operator
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-6
    ek_ref, ek = o.integrals(ref)[5], s.integrals(Ud)[5]
    assert abs(ek - ek_ref) / ek_ref < 1e-6
    # free stream: FP32 rounding of O(1) fluxes through the weak operator
    m2 = box_mesh(3, 3, deform="sinprod", rotate_seed=7)
    s2 = dg.Solver(m2, 4, mu=0.01, nodes=dg.NODES_LG, precision=dg.FP32OP)
    U = np.zeros(s2.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    assert float(s2.time_derivative(_cuda(U)).abs().max()) < 1e-3


def _dg1d_radius(w, D, lm, lp, K=8):
    """Spectral radius of the 1-D upwind DG operator of u_t + u_x = 0 on K
    periodic elements (weak form with the node set's quadrature), from the
    eigenvalues."""
    n = len(w)
    A = np.zeros((n * K, n * K))
    for e in range(K):
        el = (e - 1) % K
        for i in range(n):
            for m in range(n):
                A[e * n + i, e * n + m] += w[m] / w[i] * D[m, i] - lp[i] / w[i] * lp[m]
                A[e * n + i, el * n + m] += lm[i] / w[i] * lp[m]
    return np.abs(np.linalg.eigvals(A)).max()


@pytest.mark.parametrize("N", [3, 9])
def test_gauss_time_step_factor_and_stability(orc, dg, N):
    """max_dt on Gauss nodes = the LGL bound times rho_LGL / rho_LG of the 1-D
    upwind DG operators (here from their eigenvalues), and a perturbed uniform
    flow stays bounded over 20 steps at CFL 0.9."""
    n = N + 1
    xl, wl, Dl = orc.basis(N)
    eL, eR = np.zeros(n), np.zeros(n)
    eL[0], eR[-1] = 1.0, 1.0
    _, wg, Dg, lm, lp = orc.gauss_basis(N)
    ratio = _dg1d_radius(wl, Dl, eL, eR) / _dg1d_radius(wg, Dg, lm, lp)
    mesh = box_mesh(3, 1, lo=0.0, hi=2 * math.pi)
    s_l = dg.Solver(mesh, N, mu=1.0 / 1600.0)
    s_g = dg.Solver(mesh, N, mu=1.0 / 1600.0, nodes=dg.NODES_LG)
    U = np.zeros(s_g.shape)
    u = np.array([0.1, 0.05, 0.02])
    U[:, 0] = 1.0
    U[:, 1:4] = u[None, :, None, None, None]
    U[:, 4] = 1.0 / 1.4 / 0.4 + 0.5 * u @ u
    Ud = _cuda(U)
    dt_l, dt_g = s_l.max_dt(Ud, cfl=0.9, dfl=0.9), s_g.max_dt(Ud, cfl=0.9, dfl=0.9)
    assert abs(dt_g / dt_l / ratio - 1.0) < 2e-3, (dt_g / dt_l, ratio)
    rng = np.random.default_rng(N)
    Up = _cuda(U + 1e-10 * rng.standard_normal(U.shape))
    G = torch.empty_like(Up)
    s_g.rk_step(Up, G, 0.0, dt_g, 20)
    assert np.abs(Up.cpu().numpy() - U).max() < 1e-8


def test_gauss_full_size_pid_mesh_properties(dg):
    """At the full size of the free-stream PID run (64^3 elements, N=3, 16.78 M
    DOF, Gauss nodes), properties that hold at any size: a uniform flow stays
    uniform, and with nodal noise on it the five conservation totals do not
    change over two LSERK4-5 steps (periodic box, no source)."""
    N, K = 3, 64
    mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, mu=1.0 / 1600.0, nodes=dg.NODES_LG)
    U = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    u = (0.1, 0.05, 0.02)
    U[:, 0] = 1.0
    for a in range(3):
        U[:, 1 + a] = u[a]
    U[:, 4] = 1.0 / 1.4 / 0.4 + 0.5 * sum(c * c for c in u)
    U0 = U.clone()
    dt = s.max_dt(U, cfl=0.9, dfl=0.9)
    G = torch.empty_like(U)
    s.rk_step(U, G, 0.0, dt, 2)
    assert float((U - U0).abs().max()) < 1e-13 * float(U0.abs().max())
    gen = torch.Generator(device="cuda").manual_seed(7)
    V = U0 * (1.0 + 1e-3 * torch.randn(U0.shape, generator=gen, device="cuda", dtype=torch.float64))
    I0 = s.integrals(V)
    s.rk_step(V, G, 0.0, dt, 2)
    I1 = s.integrals(V)
    for a in range(5):
        assert abs(I1[a] - I0[a]) <= 1e-12 * abs(I0[0] if a in (1, 2, 3) else I0[a]), (a, I0[a], I1[a])
    del U, U0, V, G
    s.close()
