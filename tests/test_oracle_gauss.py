"""Oracle pins for the Legendre-Gauss node set (GALAEXI Sec. 3.1: the weak
form, Eq. 2, and the weak BR1 lifting, Eq. 3, collocated at the N+1 Gauss
points): basis closed forms and quadrature exactness, the Gauss summation-
by-parts identity, free-stream preservation, discrete conservation, exact
lifting of linear fields, manufactured-solution order and the Taylor-Green
closed forms."""
import math

import numpy as np
import pytest

from workloads import box_mesh, mms_params, random_state, tgv_params


def _wq(orc, N):
    _, w, _, _, _ = orc.gauss_basis(N)
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)


def test_gauss_basis_closed_forms(orc):
    x, w, _, _, _ = orc.gauss_basis(1)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=0, atol=3e-16)
    np.testing.assert_allclose(w, [1.0, 1.0], rtol=0, atol=1e-15)
    x, w, _, _, _ = orc.gauss_basis(2)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], rtol=0, atol=3e-16)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], rtol=0, atol=1e-15)
    x, w, _, _, _ = orc.gauss_basis(3)
    a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
    b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    np.testing.assert_allclose(x, [-b, -a, a, b], rtol=0, atol=3e-16)
    wa, wb = (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36
    np.testing.assert_allclose(w, [wb, wa, wa, wb], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9])
def test_gauss_quadrature_and_interpolation_exactness(orc, N):
    x, w, D, lm, lp = orc.gauss_basis(N)
    # quadrature exact up to degree 2N+1
    for k in range(2 * N + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs((w * x ** k).sum() - exact) < 1e-14, k
    # D exact on degree <= N; end values exact on degree <= N
    for k in range(N + 1):
        dk = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(D @ x ** k, dk, atol=1e-12 * max(1, N * N))
        assert abs(lp @ x ** k - 1.0) < 1e-13
        assert abs(lm @ x ** k - (-1.0) ** k) < 1e-13


@pytest.mark.parametrize("N", [1, 3, 6])
def test_gauss_summation_by_parts(orc, N):
    """W D + (W D)^T = l(1) l(1)^T - l(-1) l(-1)^T (discrete integration by
    parts, exact because Gauss quadrature integrates degree 2N-1 exactly)."""
    _, w, D, lm, lp = orc.gauss_basis(N)
    Q = np.diag(w) @ D
    np.testing.assert_allclose(Q + Q.T, np.outer(lp, lp) - np.outer(lm, lm), atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_gauss_free_stream_preservation(orc, N):
    m = box_mesh(3, N, deform="sinprod", rotate_seed=51)
    o = orc.Oracle(m, N, mu=0.01, nodes=1)
    U = np.zeros((m.n_elems, 5) + (N + 1,) * 3)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = o.time_derivative(U)
    assert np.abs(R).max() < 2e-12 * N * N


@pytest.mark.parametrize("N,flux", [(2, 0), (3, 2), (4, 1)])
def test_gauss_discrete_conservation(orc, N, flux):
    m = box_mesh(2, N, deform="sinprod", rotate_seed=52)
    o = orc.Oracle(m, N, mu=0.02, surf_flux=flux, nodes=1)
    # nodal noise of moderate amplitude: face values are extrapolated from the
    # Gauss nodes (|l_j(+-1)| sums grow with N), and must stay admissible
    U = random_state(m.n_elems, N, seed=53, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    _, _, J = o.geometry()
    R = o.time_derivative(U).reshape(o.E, 5, -1)
    tot = np.einsum("evp,ep->v", R, J * _wq(orc, N))
    scale = np.einsum("evp,ep->v", np.abs(R), J * _wq(orc, N))
    assert (np.abs(tot) < 1e-13 * scale).all(), (tot, scale)


def test_gauss_geometry_matches_affine_closed_form(orc):
    """On a rotated affine mesh the Gauss-node positions are the affine map of
    the Gauss points and J a^d, J are constant."""
    N, K = 3, 2
    m = box_mesh(K, 1, rotate_seed=54)
    o = orc.Oracle(m, N, nodes=1)
    X, Ja, J = o.geometry()
    np.testing.assert_allclose(J, (1.0 / K) ** 3, rtol=1e-13)
    np.testing.assert_allclose(np.abs(Ja).max(axis=-1), np.abs(Ja).min(axis=-1), atol=1e-14)
    x, _, _, _, _ = orc.gauss_basis(N)
    # the node coordinates along each reference line are affine images of x
    for e in range(2):
        for c in range(3):
            v = X[e, c].reshape(N + 1, N + 1, N + 1)
            for axis in range(3):
                d = np.diff(np.moveaxis(v, 2 - axis, 0), axis=0)
                ratio = d / np.diff(x)[:, None, None]
                assert np.abs(ratio - ratio[:1]).max() < 1e-13


def test_gauss_lifting_exact_for_linear_fields(orc):
    N, K, g, Rg = 3, 3, 1.4, 1.0
    m = box_mesh(K, 1, rotate_seed=55)
    o = orc.Oracle(m, N, R=Rg, nodes=1)
    X, _, _ = o.geometry()
    A = np.array([[0.1, -0.2, 0.05], [0.3, 0.0, -0.1], [-0.05, 0.2, 0.15]])
    bT = np.array([0.02, -0.01, 0.03])
    vel = np.einsum("ab,ebp->eap", A, X)
    T = 2.0 + np.einsum("b,ebp->ep", bT, X)
    rho = 1.0 + 0.0 * T
    U = np.zeros((m.n_elems, 5, X.shape[-1]))
    U[:, 0] = rho
    U[:, 1:4] = rho[:, None] * vel
    U[:, 4] = rho * Rg * T / (g - 1) + 0.5 * rho * (vel ** 2).sum(1)
    G = o.lifting(U)
    centre = 1 + K * (1 + K * 1)
    for a in range(3):
        for l in range(3):
            np.testing.assert_allclose(G[centre, a * 3 + l], A[a, l], atol=1e-13)
    for l in range(3):
        np.testing.assert_allclose(G[centre, 9 + l], bT[l], atol=1e-13)


def _mms_error(orc, K, N, t_end, cfl=0.5):
    prm = mms_params()
    m = box_mesh(K, N, deform="sinprod", rotate_seed=20260528)
    o = orc.Oracle(m, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1, nodes=1)
    lam = math.sqrt(1.4 / 1.9) + math.sqrt(3.0)
    nsteps = int(math.ceil(t_end / (cfl * (2.0 / K) / ((2 * N + 1) * lam))))
    U = o.rk_steps(o.initial_state("mms", 0.0), 0.0, t_end / nsteps, nsteps)
    ex = o.initial_state("mms", t_end)
    _, _, J = o.geometry()
    err = ((U[:, 0].reshape(o.E, -1) - ex[:, 0].reshape(o.E, -1)) ** 2 * J * _wq(orc, N)).sum()
    return math.sqrt(err)


def test_gauss_mms_convergence_order(orc):
    """Design order N+1 on the curvilinear rotated mesh (t = 0.5, as for LGL)."""
    N, t_end = 3, 0.5
    e = [_mms_error(orc, K, N, t_end) for K in (4, 8)]
    eoc = math.log2(e[0] / e[1])
    assert eoc > N + 1 - 0.4, (e, eoc)
    assert e[1] < 2e-3


def test_gauss_taylor_green_closed_forms(orc):
    prm = tgv_params(Ma=0.05, Re=1600.0)
    N = 5
    m = box_mesh(4, 1, lo=0.0, hi=2 * np.pi)
    o = orc.Oracle(m, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], nodes=1)
    U = o.initial_state("tgv", prm["p0"])
    I = o.integrals(U)
    assert abs(I[5] - 0.125) < 1e-3
    assert abs(I[6] / (0.75 * prm["mu"]) - 1.0) < 0.05, I[6]


@pytest.mark.parametrize("flux,law,mortar", [(0, 0, False), (1, 1, False), (2, 0, False), (0, 1, True)])
def test_gauss_tangent_linear_matches_central_differences(orc, flux, law, mortar):
    """The dual-number path runs the same Gauss-node code (prolongation, weak
    lifting, face fluxes, weak volume integral, and the mortars): its
    tangent-linear of R(U), and dR/dmu, match central differences."""
    N = 3
    if mortar:
        from workloads.mesh import refined_box_mesh
        r = np.zeros(8, dtype=bool)
        r[0] = True
        m = refined_box_mesh(2, r, rotate_seed=11)
    else:
        m = box_mesh(2, 2, deform="sinprod", rotate_seed=12)
    kw = dict(surf_flux=flux, visc_law=law, T_ref=1.0, S_suth=0.4, nodes=1)
    mu, h = 0.03, 1e-6
    o = orc.Oracle(m, N, mu=mu, **kw)
    U = random_state(m.n_elems, N, seed=13, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    dU = np.random.default_rng(14).normal(size=U.shape)
    R, dR = o.time_derivative_tl(U, dU)
    assert np.array_equal(R, o.time_derivative(U))
    fd = (o.time_derivative(U + h * dU) - o.time_derivative(U - h * dU)) / (2 * h)
    assert np.abs(dR - fd).max() < 1e-8 * np.abs(fd).max()
    _, Rmu = o.time_derivative_tl(U, np.zeros_like(U), 1.0)
    fdmu = (orc.Oracle(m, N, mu=mu + h, **kw).time_derivative(U)
            - orc.Oracle(m, N, mu=mu - h, **kw).time_derivative(U)) / (2 * h)
    assert np.abs(Rmu - fdmu).max() < 1e-8 * np.abs(fdmu).max()


def test_gauss_rk_tangent_linear_matches_central_differences(orc):
    """The step tangent-linear on Gauss nodes (the dual numbers through the
    LSERK4-5 stages of the Gauss-node operator) against central differences
    of the steps, for a direction in U and in mu together.  Entropy-
    conservative faces: the LLF speed max(lambda_L, lambda_R) has a kink
    where the two sides' speeds are equal, and over fifteen stages some face
    point of a random state comes within the differences' step of one."""
    N = 2
    m = box_mesh(2, 2, deform="sinprod", rotate_seed=15)
    mu, h, dt, nsteps, dmu = 0.02, 1e-6, 2e-3, 3, 0.3
    kw = dict(nodes=1, surf_flux=1)
    U = random_state(m.n_elems, N, seed=16, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    dU = np.random.default_rng(17).normal(size=U.shape)
    UT, dUT = orc.Oracle(m, N, mu=mu, **kw).rk_steps_tl(U, dU, dmu, 0.0, dt, nsteps)
    assert np.array_equal(UT, orc.Oracle(m, N, mu=mu, **kw).rk_steps(U, 0.0, dt, nsteps))
    fp = orc.Oracle(m, N, mu=mu + h * dmu, **kw).rk_steps(U + h * dU, 0.0, dt, nsteps)
    fm = orc.Oracle(m, N, mu=mu - h * dmu, **kw).rk_steps(U - h * dU, 0.0, dt, nsteps)
    fd = (fp - fm) / (2 * h)
    assert np.abs(dUT - fd).max() < 1e-7 * np.abs(fd).max()
