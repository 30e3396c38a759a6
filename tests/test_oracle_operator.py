"""Oracle pins for the discrete operator R(U) (GALAEXI Sec. 3.1, Eqs. 1-3):
geometry, free-stream preservation, discrete conservation, entropy
conservation, polynomial exactness of the split-form volume term, exactness of
the BR1 lifting on linear fields, manufactured-solution convergence order,
Taylor-Green closed forms and the tangent-linear operator."""
import math

import numpy as np
import pytest

from workloads import ROTATIONS, box_mesh, mms_params, random_state, tgv_params


def _quad_weights(orc, N):
    _, w, _ = orc.basis(N)
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)


def _entropy_vars(U, gamma):
    r = U[:, 0]
    u = U[:, 1:4] / r[:, None]
    p = (gamma - 1) * (U[:, 4] - 0.5 * r * (u ** 2).sum(1))
    s = np.log(p * r ** -gamma)
    return np.concatenate([((gamma - s) / (gamma - 1) - r * (u ** 2).sum(1) / (2 * p))[:, None],
                           r[:, None] * u / p[:, None], (-r / p)[:, None]], 1)


@pytest.mark.parametrize("N", [1, 2, 4])
def test_affine_geometry_is_exact(orc, N):
    K = 3
    m = box_mesh(K, 1, rotate_seed=11)
    o = orc.Oracle(m, N)
    X, Ja, J = o.geometry()
    x, _, _ = orc.basis(N)
    h = 2.0 / K
    xi = np.stack(np.meshgrid(x, x, x, indexing="ij")[::-1], 0).reshape(3, -1)   # local (xi, eta, zeta)
    for e in range(m.n_elems):
        R = ROTATIONS[m.rot[e]]
        ex, ey, ez = e % K, (e // K) % K, e // (K * K)
        c = -1.0 + h * (np.array([ex, ey, ez]) + 0.5)
        np.testing.assert_allclose(X[e], c[:, None] + (h / 2) * R @ xi, atol=1e-14)
        np.testing.assert_allclose(J[e], (h / 2) ** 3, rtol=1e-13)
        for d in range(3):
            for l in range(3):
                np.testing.assert_allclose(Ja[e, d, l], (h / 2) ** 2 * R[l, d], atol=5e-14)


def test_metric_identities_on_curved_mesh(orc):
    N = 5
    m = box_mesh(2, N, deform="sinprod", rotate_seed=5)
    o = orc.Oracle(m, N)
    X, Ja, J = o.geometry()
    _, w, D = orc.basis(N)
    n = N + 1
    assert (J > 0).all()
    for e in range(m.n_elems):
        for l in range(3):
            s = np.zeros((n, n, n))
            for d in range(3):
                f = Ja[e, d, l].reshape(n, n, n)            # [k, j, i]
                ax = 2 - d
                s += np.moveaxis(np.tensordot(D, np.moveaxis(f, ax, 0), axes=(1, 0)), 0, ax)
            assert np.abs(s).max() < 1e-13
    # the curved map is not affine: metrics vary
    assert np.ptp(J) > 1e-3


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_free_stream_preservation(orc, N):
    m = box_mesh(2, N, deform="sinprod", rotate_seed=7)
    o = orc.Oracle(m, N, mu=0.01)
    U = np.zeros(o.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = o.time_derivative(U)
    assert np.abs(R).max() < 2e-12 * N * N


def _conservation(orc, o, U, N):
    _, _, J = o.geometry()
    wq = _quad_weights(orc, N)
    R = o.time_derivative(U).reshape(o.E, 5, -1)
    tot = np.einsum("evp,ep->v", R, J * wq)
    scale = np.einsum("evp,ep->v", np.abs(R), J * wq)
    return tot, scale


@pytest.mark.parametrize("N,flux", [(2, 0), (3, 0), (4, 1), (3, 2)])
def test_discrete_conservation(orc, N, flux):
    m = box_mesh(2, N, deform="sinprod", rotate_seed=13)
    o = orc.Oracle(m, N, mu=0.02, surf_flux=flux)
    U = random_state(m.n_elems, N, seed=3)
    tot, scale = _conservation(orc, o, U, N)
    assert (np.abs(tot) < 1e-13 * scale).all(), (tot, scale)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_entropy_conservation_ec_surface_flux(orc, N):
    """With the two-point flux on faces and mu = 0 the semi-discrete entropy
    production sum w J w(U) . R(U) vanishes (entropy-conservative DGSEM)."""
    m = box_mesh(2, N, deform="sinprod", rotate_seed=17)
    o = orc.Oracle(m, N, mu=0.0, surf_flux=1)
    U = random_state(m.n_elems, N, seed=5)
    _, _, J = o.geometry()
    wq = _quad_weights(orc, N)
    R = o.time_derivative(U).reshape(o.E, 5, -1)
    Uf = U.reshape(o.E, 5, -1)
    W = np.stack([_entropy_vars(Uf[e].T, 1.4).T for e in range(o.E)])
    prod = np.einsum("evp,evp,ep->", W, R, J * wq)
    scale = np.einsum("evp,evp,ep->", np.abs(W), np.abs(R), J * wq)
    assert abs(prod) < 1e-13 * scale, (prod, scale)
    # with LLF on faces entropy is dissipated
    o2 = orc.Oracle(m, N, mu=0.0, surf_flux=0)
    R2 = o2.time_derivative(U).reshape(o.E, 5, -1)
    assert np.einsum("evp,evp,ep->", W, R2, J * wq) < -1e-6 * scale


def test_split_form_volume_term_polynomial_exactness(orc):
    """Central two-point flux: the split form equals the derivative of the
    interpolated flux; for a flux that is a polynomial of degree <= N on an
    affine (rotated) element it equals J div f exactly (closed form)."""
    N, K, g = 4, 2, 1.4
    m = box_mesh(K, 1, rotate_seed=21)
    o = orc.Oracle(m, N)
    o.set_vol_flux(1)
    X, _, J = o.geometry()
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    u = np.array([0.3, -0.2, 0.1])
    p = 1.0 + 0.1 * x * x * y + 0.05 * z ** 3 - 0.02 * x * y * z
    dp = np.stack([0.2 * x * y - 0.02 * y * z, 0.1 * x * x - 0.02 * x * z, 0.15 * z * z - 0.02 * x * y])
    U = np.zeros((m.n_elems, 5, X.shape[-1]))
    U[:, 0] = 1.0
    U[:, 1:4] = u[None, :, None]
    U[:, 4] = p / (g - 1) + 0.5 * u @ u
    V = o.volume_term(U)
    div = np.zeros_like(V)
    div[:, 1:4] = dp.transpose(1, 0, 2)
    div[:, 4] = g / (g - 1) * np.einsum("a,eap->ep", u, dp.transpose(1, 0, 2))
    np.testing.assert_allclose(V / J[:, None], div, atol=1e-12)
    # the entropy-conservative flux gives the same for a constant state
    o.set_vol_flux(0)
    U[:, 4] = 1.0 / (g - 1) + 0.5 * u @ u
    assert np.abs(o.volume_term(U)).max() < 1e-13


def test_lifting_exact_for_linear_fields(orc):
    N, K, g, Rg = 3, 3, 1.4, 1.0
    m = box_mesh(K, 1, rotate_seed=23)
    o = orc.Oracle(m, N, R=Rg)
    X, _, _ = o.geometry()
    A = np.array([[0.1, -0.2, 0.05], [0.3, 0.0, -0.1], [-0.05, 0.2, 0.15]])
    bT = np.array([0.02, -0.01, 0.03])
    vel = np.einsum("ab,ebp->eap", A, X)
    T = 2.0 + np.einsum("b,ebp->ep", bT, X)
    rho = 1.0 + 0.0 * T
    p = rho * Rg * T
    U = np.zeros((m.n_elems, 5, X.shape[-1]))
    U[:, 0] = rho
    U[:, 1:4] = rho[:, None] * vel
    U[:, 4] = p / (g - 1) + 0.5 * rho * (vel ** 2).sum(1)
    G = o.lifting(U)
    centre = 1 + K * (1 + K * 1)          # element not touching the periodic seam
    for a in range(3):
        for l in range(3):
            np.testing.assert_allclose(G[centre, a * 3 + l], A[a, l], atol=1e-13)
    for l in range(3):
        np.testing.assert_allclose(G[centre, 9 + l], bT[l], atol=1e-13)


def _mms_error(orc, K, N, t_end, cfl=0.5):
    prm = mms_params()
    m = box_mesh(K, N, deform="sinprod", rotate_seed=20260528)
    o = orc.Oracle(m, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    lam = math.sqrt(1.4 / 1.9) + math.sqrt(3.0)          # max |u| + c of the exact solution
    nsteps = int(math.ceil(t_end / (cfl * (2.0 / K) / ((2 * N + 1) * lam))))
    U = o.rk_steps(o.initial_state("mms", 0.0), 0.0, t_end / nsteps, nsteps)
    ex = o.initial_state("mms", t_end)
    _, _, J = o.geometry()
    wq = _quad_weights(orc, N)
    err = ((U[:, 0].reshape(o.E, -1) - ex[:, 0].reshape(o.E, -1)) ** 2 * J * wq).sum()
    return math.sqrt(err)


def test_mms_convergence_order(orc):
    """Design order N+1 of the density error under h-refinement on the
    curvilinear, rotated mesh with the analytic source.  Measured at t = 0.5,
    after the start-up transient (at t = 0.1 the rate is still ~N)."""
    N, t_end = 3, 0.5
    e = [_mms_error(orc, K, N, t_end) for K in (4, 8)]
    eoc = math.log2(e[0] / e[1])
    assert eoc > N + 1 - 0.4, (e, eoc)
    assert e[1] < 2e-3


def test_mms_source_matches_symbolic_residual(orc):
    """The hand-derived source equals q_t + div F(q) of the exact solution,
    computed symbolically here (sympy)."""
    sp = pytest.importorskip("sympy")
    prm = mms_params()
    g, Rg, Pr, mu, A = prm["gamma"], prm["R"], prm["Pr"], prm["mu"], prm["amp"]
    x, y, z, t = sp.symbols("x y z t")
    rho = 2 + A * sp.sin(sp.pi * (x + y + z - t))
    u = [sp.Integer(1)] * 3
    p = sp.Integer(1)
    E = p / (g - 1) + rho * sum(ui ** 2 for ui in u) / 2
    T = p / (rho * Rg)
    lam = mu * g * Rg / (g - 1) / Pr
    X = [x, y, z]
    q = [rho, rho * u[0], rho * u[1], rho * u[2], E]
    res = []
    for v in range(5):
        r = sp.diff(q[v], t)
        for j in range(3):
            if v == 0:
                f = rho * u[j]
            elif v < 4:
                f = rho * u[v - 1] * u[j] + (p if v - 1 == j else 0)
            else:
                f = (E + p) * u[j] - lam * sp.diff(T, X[j])
            r += sp.diff(f, X[j])
        res.append(sp.lambdify((x, y, z, t), r, "numpy"))
    # the oracle's R of the exact state at t, on a fine mesh, approaches
    # q_t... instead compare the source through a constant-in-space check:
    m = box_mesh(2, 3, deform="sinprod", rotate_seed=1)
    o = orc.Oracle(m, 3, gamma=g, R=Rg, Pr=Pr, mu=mu, source=1)
    o0 = orc.Oracle(m, 3, gamma=g, R=Rg, Pr=Pr, mu=mu, source=0)
    U = random_state(m.n_elems, 3, seed=9)
    S = o.time_derivative(U, t=0.3) - o0.time_derivative(U, t=0.3)
    Xn = o.node_coords()
    for v in range(5):
        ref = res[v](Xn[:, 0], Xn[:, 1], Xn[:, 2], 0.3) * np.ones_like(Xn[:, 0])
        np.testing.assert_allclose(S[:, v].reshape(o.E, -1), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("nodes", [0, 1])
def test_viscous_terms_match_symbolic_navier_stokes(orc, nodes):
    """With constant mu the viscous part of R is linear in mu, so
    (R_mu(U) - R_0(U)) / mu is the discrete div F_v of Sec. 3.1 (BR1 lifting,
    viscous volume and surface terms). For a smooth compressible state it must
    approach the symbolic div F_v, with F_v = (0, tau, u.tau + lambda grad T) and
    tau = grad u + grad u^T - 2/3 (div u) I, and stay far from the usual slips:
    the transposed gradient dropped, or the bulk term with the wrong sign or left
    out (the Taylor-Green dissipation cannot tell these apart: there div u = 0)."""
    sp = pytest.importorskip("sympy")
    g, Rg, Pr, mu = 1.4, 1.0, 0.72, 0.5
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    rho = 1 + 0.2 * sp.sin(x) * sp.cos(z) + 0.1 * sp.cos(y)
    u = [0.3 * sp.sin(y) + 0.2 * sp.sin(x) * sp.cos(z),
         0.25 * sp.sin(z) + 0.15 * sp.cos(x) * sp.sin(y),
         0.2 * sp.sin(x + y) + 0.1 * sp.cos(z)]
    p = 1 + 0.1 * sp.cos(y) * sp.sin(z) + 0.05 * sp.sin(x)
    T = p / (rho * Rg)
    lam = g * Rg / (g - 1) / Pr          # lambda / mu = c_p / Pr
    div = sum(sp.diff(u[j], X[j]) for j in range(3))

    def div_fv(transpose=1, bulk=sp.Rational(2, 3)):
        tau = [[sp.diff(u[i], X[j]) + transpose * sp.diff(u[j], X[i]) - (bulk * div if i == j else 0)
                for j in range(3)] for i in range(3)]
        out = [sp.Integer(0)] + [sum(sp.diff(tau[i][j], X[j]) for j in range(3)) for i in range(3)]
        out.append(sum(sp.diff(sum(u[i] * tau[i][j] for i in range(3)) + lam * sp.diff(T, X[j]), X[j])
                       for j in range(3)))
        return [sp.lambdify((x, y, z), f, "numpy") for f in out]

    cons = [rho, rho * u[0], rho * u[1], rho * u[2], p / (g - 1) + rho * sum(ui ** 2 for ui in u) / 2]
    cons = [sp.lambdify((x, y, z), f, "numpy") for f in cons]
    exact = div_fv()
    slips = [div_fv(transpose=0), div_fv(bulk=-sp.Rational(2, 3)), div_fv(bulk=0)]

    def at_nodes(f, Xn):
        return f(Xn[:, 0], Xn[:, 1], Xn[:, 2]) * np.ones_like(Xn[:, 0])

    errs = {}
    for N in (5, 7):
        m = box_mesh(4, N, lo=0.0, hi=2 * np.pi, deform="sinprod", rotate_seed=17)
        o1 = orc.Oracle(m, N, gamma=g, R=Rg, Pr=Pr, mu=mu, nodes=nodes)
        o0 = orc.Oracle(m, N, gamma=g, R=Rg, Pr=Pr, mu=0.0, nodes=nodes)
        Xn = o1.node_coords()
        U = np.stack([at_nodes(f, Xn) for f in cons], 1).reshape(o1.shape)
        V = ((o1.time_derivative(U) - o0.time_derivative(U)) / mu).reshape(o1.E, 5, -1)
        assert np.abs(V[:, 0]).max() < 1e-12           # no viscous mass flux
        scale = [np.abs(at_nodes(exact[v], Xn)).max() for v in range(5)]
        errs[N] = [np.abs(V[:, v] - at_nodes(exact[v], Xn)).max() / scale[v] for v in range(1, 5)]
        if N == 7:
            assert max(errs[N]) < 0.02, errs[N]
            for s in slips:
                es = [np.abs(V[:, v] - at_nodes(s[v], Xn)).max() / scale[v] for v in range(1, 4)]
                assert min(es) > 0.15, es
    # the remaining difference is discretisation error: it falls with N
    assert all(e7 < e5 / 5 for e5, e7 in zip(errs[5], errs[7])), errs


@pytest.mark.parametrize("nodes,surf_flux", [(0, 0), (0, 1), (1, 0), (1, 2)])
def test_inviscid_operator_matches_symbolic_euler(orc, nodes, surf_flux):
    """For a smooth state with every primitive varying in all three
    directions, R with mu = 0 approaches -div F_c(q) of the Euler equations
    (Sec. 3.1, Eq. 1: mass, momentum with its pressure, energy (rho E + p) u),
    written out and differentiated symbolically here, spectrally in N on a
    curved rotated mesh."""
    sp = pytest.importorskip("sympy")
    g = 1.4
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    rho = 1 + 0.2 * sp.sin(x) * sp.cos(z) + 0.1 * sp.cos(y)
    u = [0.3 * sp.sin(y) + 0.2 * sp.sin(x) * sp.cos(z),
         0.25 * sp.sin(z) + 0.15 * sp.cos(x) * sp.sin(y),
         0.2 * sp.sin(x + y) + 0.1 * sp.cos(z)]
    p = 1 + 0.1 * sp.cos(y) * sp.sin(z) + 0.05 * sp.sin(x)
    E = p / (g - 1) + rho * sum(ui ** 2 for ui in u) / 2
    cons = [rho, rho * u[0], rho * u[1], rho * u[2], E]

    def flux(v, j):
        if v == 0:
            return rho * u[j]
        if v < 4:
            return rho * u[v - 1] * u[j] + (p if v - 1 == j else 0)
        return (E + p) * u[j]

    exact = [sp.lambdify((x, y, z), -sum(sp.diff(flux(v, j), X[j]) for j in range(3)), "numpy") for v in range(5)]
    cons = [sp.lambdify((x, y, z), f, "numpy") for f in cons]
    errs = {}
    for N in (5, 7):
        m = box_mesh(4, N, lo=0.0, hi=2 * np.pi, deform="sinprod", rotate_seed=17)
        o = orc.Oracle(m, N, gamma=g, mu=0.0, surf_flux=surf_flux, nodes=nodes)
        Xn = o.node_coords()
        U = np.stack([f(Xn[:, 0], Xn[:, 1], Xn[:, 2]) * np.ones_like(Xn[:, 0]) for f in cons], 1).reshape(o.shape)
        R = o.time_derivative(U).reshape(o.E, 5, -1)
        errs[N] = []
        for v in range(5):
            r = exact[v](Xn[:, 0], Xn[:, 1], Xn[:, 2]) * np.ones_like(Xn[:, 0])
            errs[N].append(np.abs(R[:, v] - r).max() / np.abs(r).max())
    # discretisation error only (a dropped or mis-signed flux term is O(1)):
    # below 1e-3 on LGL nodes, 2.2e-3 with the Gauss weak form at N = 7
    assert max(errs[7]) < 5e-3, errs[7]
    assert all(e7 < e5 / 5 for e5, e7 in zip(errs[5], errs[7])), errs


@pytest.mark.parametrize("nodes", [0, 1])
def test_sutherland_viscous_terms_match_symbolic_navier_stokes(orc, nodes):
    """Sutherland's law (Sec. 4.2) at each node's temperature: mu = mu0 s(T),
    s(T) = (T/T_ref)^(3/2) (T_ref + S)/(T + S), lambda = mu c_p / Pr.  The
    viscous part is still linear in mu0, so (R_mu0 - R_0)/mu0 must approach
    the symbolic div F_v with s(T) inside the stress and the heat flux, and
    differ clearly from the constant-viscosity div F_v where T varies."""
    sp = pytest.importorskip("sympy")
    g, Rg, Pr, mu0, T_ref, S = 1.4, 1.0, 0.72, 0.5, 1.0, 110.4 / 273.15
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    rho = 1 + 0.2 * sp.sin(x) * sp.cos(z) + 0.1 * sp.cos(y)
    u = [0.3 * sp.sin(y) + 0.2 * sp.sin(x) * sp.cos(z),
         0.25 * sp.sin(z) + 0.15 * sp.cos(x) * sp.sin(y),
         0.2 * sp.sin(x + y) + 0.1 * sp.cos(z)]
    p = 1 + 0.2 * sp.cos(y) * sp.sin(z) + 0.1 * sp.sin(x)
    T = p / (rho * Rg)
    cp_Pr = g * Rg / (g - 1) / Pr
    div = sum(sp.diff(u[j], X[j]) for j in range(3))

    def div_fv(law):
        tau = [[law * (sp.diff(u[i], X[j]) + sp.diff(u[j], X[i]) - (sp.Rational(2, 3) * div if i == j else 0))
                for j in range(3)] for i in range(3)]
        out = [sp.Integer(0)] + [sum(sp.diff(tau[i][j], X[j]) for j in range(3)) for i in range(3)]
        out.append(sum(sp.diff(sum(u[i] * tau[i][j] for i in range(3)) + law * cp_Pr * sp.diff(T, X[j]), X[j])
                       for j in range(3)))
        return [sp.lambdify((x, y, z), f, "numpy") for f in out]

    exact = div_fv((T / T_ref) ** sp.Rational(3, 2) * (T_ref + S) / (T + S))
    constant = div_fv(sp.Integer(1))
    cons = [rho, rho * u[0], rho * u[1], rho * u[2], p / (g - 1) + rho * sum(ui ** 2 for ui in u) / 2]
    cons = [sp.lambdify((x, y, z), f, "numpy") for f in cons]

    def at_nodes(f, Xn):
        return f(Xn[:, 0], Xn[:, 1], Xn[:, 2]) * np.ones_like(Xn[:, 0])

    errs = {}
    for N in (5, 7):
        m = box_mesh(4, N, lo=0.0, hi=2 * np.pi, deform="sinprod", rotate_seed=17)
        kw = dict(gamma=g, R=Rg, Pr=Pr, visc_law=1, T_ref=T_ref, S_suth=S, nodes=nodes)
        o1 = orc.Oracle(m, N, mu=mu0, **kw)
        o0 = orc.Oracle(m, N, mu=0.0, **kw)
        Xn = o1.node_coords()
        U = np.stack([at_nodes(f, Xn) for f in cons], 1).reshape(o1.shape)
        V = ((o1.time_derivative(U) - o0.time_derivative(U)) / mu0).reshape(o1.E, 5, -1)
        scale = [np.abs(at_nodes(exact[v], Xn)).max() for v in range(5)]
        errs[N] = [np.abs(V[:, v] - at_nodes(exact[v], Xn)).max() / scale[v] for v in range(1, 5)]
        if N == 7:
            assert max(errs[N]) < 0.02, errs[N]
            off = [np.abs(V[:, v] - at_nodes(constant[v], Xn)).max() / scale[v] for v in range(1, 5)]
            assert max(off) > 0.1, off
    assert all(e7 < e5 / 3 for e5, e7 in zip(errs[5], errs[7])), errs


@pytest.mark.parametrize("nodes", [0, 1])
def test_integrals_match_closed_forms(orc, nodes):
    """The diagnostics of Sec. 4.2 for a smooth periodic state on a curved
    rotated mesh: the five conservation totals, E_k = 1/(2|Omega|) int rho |u|^2,
    eps = mu/|Omega| int |omega|^2 and min p.  The references integrate the same
    trigonometric polynomials with the uniform trapezoidal rule on 32^3 points,
    which is exact for them, so they share nothing with the LGL quadrature,
    the Jacobian or the lifted vorticity of the oracle."""
    sp = pytest.importorskip("sympy")
    g, mu, N = 1.4, 0.01, 7
    x, y, z = sp.symbols("x y z")
    rho = 1 + 0.2 * sp.sin(x) * sp.cos(z) + 0.1 * sp.cos(y)
    u = [0.3 * sp.sin(y) + 0.2 * sp.sin(x) * sp.cos(z),
         0.25 * sp.sin(z) + 0.15 * sp.cos(x) * sp.sin(y),
         0.2 * sp.sin(x + y) + 0.1 * sp.cos(z)]
    p = 1 + 0.1 * sp.cos(y) * sp.sin(z) + 0.05 * sp.sin(x)
    cons = [rho, rho * u[0], rho * u[1], rho * u[2], p / (g - 1) + rho * sum(ui ** 2 for ui in u) / 2]
    omega = [sp.diff(u[2], y) - sp.diff(u[1], z), sp.diff(u[0], z) - sp.diff(u[2], x),
             sp.diff(u[1], x) - sp.diff(u[0], y)]
    integrands = cons + [rho * sum(ui ** 2 for ui in u), sum(w ** 2 for w in omega)]
    M = 32
    t1 = 2 * np.pi * np.arange(M) / M
    gx, gy, gz = np.meshgrid(t1, t1, t1, indexing="ij")
    vol = (2 * np.pi) ** 3

    def trapezoid(f):
        vals = sp.lambdify((x, y, z), f, "numpy")(gx, gy, gz) * np.ones_like(gx)
        return vals.mean() * vol, np.abs(vals).mean() * vol

    tr = [trapezoid(f) for f in integrands]
    ref = [tr[v][0] for v in range(5)] + [tr[5][0] / (2 * vol), mu * tr[6][0] / vol]
    scale = [tr[v][1] for v in range(5)] + [ref[5], ref[6]]

    m = box_mesh(4, N, lo=0.0, hi=2 * np.pi, deform="sinprod", rotate_seed=17)
    o = orc.Oracle(m, N, gamma=g, mu=mu, nodes=nodes)
    Xn = o.node_coords()
    U = np.stack([sp.lambdify((x, y, z), f, "numpy")(Xn[:, 0], Xn[:, 1], Xn[:, 2]) * np.ones_like(Xn[:, 0])
                  for f in cons], 1).reshape(o.shape)
    I = o.integrals(U)
    for v in range(7):
        assert abs(I[v] - ref[v]) < 1e-7 * scale[v], (v, I[v], ref[v])
    p_nodes = sp.lambdify((x, y, z), p, "numpy")(Xn[:, 0], Xn[:, 1], Xn[:, 2])
    assert abs(I[7] - p_nodes.min()) < 1e-14


def test_taylor_green_closed_forms(orc):
    """E_k(0) = 1/8 up to O(Ma^2) density variation, and in the
    incompressible limit dE_k/dt(0) = -2 nu |k|^2 E_k = -3 nu / 4."""
    prm = tgv_params(Ma=0.05, Re=1600.0)
    N = 5
    m = box_mesh(4, 1, lo=0.0, hi=2 * np.pi)
    o = orc.Oracle(m, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U = o.initial_state("tgv", prm["p0"])
    I = o.integrals(U)
    assert abs(I[5] - 0.125) < 1e-3
    vol = (2 * np.pi) ** 3
    assert abs(I[0] / vol - 1.0) < 1e-3
    assert np.abs(I[1:4]).max() < 1e-10
    R = o.time_derivative(U)
    _, _, J = o.geometry()
    wq = _quad_weights(orc, N)
    Uf, Rf = U.reshape(o.E, 5, -1), R.reshape(o.E, 5, -1)
    u = Uf[:, 1:4] / Uf[:, 0:1]
    dke = (np.einsum("eap,eap->ep", u, Rf[:, 1:4]) - 0.5 * (u ** 2).sum(1) * Rf[:, 0])
    dEk = (dke * J * wq).sum() / vol
    assert abs(dEk / (-0.75 * prm["mu"]) - 1.0) < 0.05, dEk
    # the dissipation diagnostic equals -dE_k/dt for the incompressible TGV at t=0
    assert abs(I[6] / (0.75 * prm["mu"]) - 1.0) < 0.05, I[6]


def test_tangent_linear_matches_central_differences(orc):
    N = 2
    m = box_mesh(2, N, deform="sinprod", rotate_seed=31)
    o = orc.Oracle(m, N, mu=0.05)
    U = random_state(m.n_elems, N, seed=1)
    V = np.random.default_rng(2).normal(size=U.shape)
    dmu = 0.7
    _, dR = o.time_derivative_tl(U, V, dmu)
    h = 1e-6
    op = orc.Oracle(m, N, mu=0.05 + h * dmu)
    om = orc.Oracle(m, N, mu=0.05 - h * dmu)
    fd = (op.time_derivative(U + h * V) - om.time_derivative(U - h * V)) / (2 * h)
    assert np.abs(fd - dR).max() < 1e-6 * np.abs(dR).max()


@pytest.mark.parametrize("N", [2, 3])
def test_tangent_linear_at_llf_kinks_is_the_mean_derivative(orc, N):
    """A state mirror-symmetric about the planes x = 0 and x = +-1 (normal
    momentum reversed) puts both faces' LLF speeds max(|u.n| + c) at an exact
    tie with a non-zero jump.  There the tangent-linear takes the mean of the
    one-sided derivatives, which is what central differences converge to, at
    the O(h) rate of a kink; a one-sided (primal-branch) derivative stays O(1)
    away (about 5e-2 of max|dR| here)."""
    K = 2
    m = box_mesh(K, 1)
    o = orc.Oracle(m, N, mu=0.02)
    U = random_state(m.n_elems, N, seed=3)
    for e in range(m.n_elems):
        if e % K == 1:
            Vm = U[e - 1][:, :, :, ::-1].copy()
            Vm[1] = -Vm[1]
            U[e] = Vm
    V = np.random.default_rng(1).normal(size=U.shape)
    _, dR = o.time_derivative_tl(U, V, 0.0)
    err = []
    for h in (1e-6, 1e-7):
        fd = (o.time_derivative(U + h * V) - o.time_derivative(U - h * V)) / (2 * h)
        err.append(np.abs(fd - dR).max() / np.abs(dR).max())
    assert err[0] < 2e-6 and err[1] < err[0] / 5, err


@pytest.mark.parametrize("rk", [0, 1])
def test_tangent_linear_of_rk_steps_matches_central_differences(orc, rk):
    """The tangent of several steps of either 2N-storage scheme (the reference
    of the GPU adjoint's dot-product tests) against central differences of the
    primal steps; its primal part is the primal loop bit for bit."""
    N, mu, dt, nsteps = 2, 0.05, 2e-3, 4
    m = box_mesh(2, N, deform="sinprod", rotate_seed=33)
    o = orc.Oracle(m, N, mu=mu, rk=rk)
    U = random_state(m.n_elems, N, seed=4)
    V = np.random.default_rng(6).normal(size=U.shape)
    dmu = 0.3
    UT, dUT = o.rk_steps_tl(U, V, dmu, 0.0, dt, nsteps)
    np.testing.assert_array_equal(UT, o.rk_steps(U, 0.0, dt, nsteps))
    h = 1e-6
    op = orc.Oracle(m, N, mu=mu + h * dmu, rk=rk)
    om = orc.Oracle(m, N, mu=mu - h * dmu, rk=rk)
    fd = (op.rk_steps(U + h * V, 0.0, dt, nsteps) - om.rk_steps(U - h * V, 0.0, dt, nsteps)) / (2 * h)
    assert np.abs(fd - dUT).max() < 1e-6 * np.abs(dUT).max()


def test_bad_meshes_are_rejected(orc):
    m = box_mesh(2, 1, rotate_seed=3)
    bad = m.face_nbr.copy()
    bad[0, 0, 1] = (bad[0, 0, 1] + 1) % 6
    m2 = type(m)(**{**m.__dict__, "face_nbr": bad})
    with pytest.raises(ValueError):
        orc.Oracle(m2, 2)
    inv = m.xgeo.copy()
    inv[0] = inv[0][:, :, :, ::-1]            # mirror one element -> negative Jacobian
    m3 = type(m)(**{**m.__dict__, "xgeo": inv})
    with pytest.raises(ValueError):
        orc.Oracle(m3, 2)


def _uniform_temperature_state(n_elems, N, T1, R=1.0, seed=0):
    """Random density and velocity, pressure p = rho R T1 (uniform T)."""
    U = random_state(n_elems, N, seed=seed)
    r = U[:, 0]
    u = U[:, 1:4] / r[:, None]
    p = r * R * T1
    U[:, 4] = p / 0.4 + 0.5 * r * (u ** 2).sum(1)
    return U


@pytest.mark.parametrize("T1", [1.0, 2.0, 0.6])
def test_sutherland_uniform_temperature(orc, T1):
    """At a uniform temperature T1 Sutherland's law is one constant,
    mu0 (T1/T_ref)^(3/2) (T_ref + S)/(T1 + S) (closed form): R(U) and the
    dissipation diagnostic equal those of the constant law with that mu.
    At T1 = T_ref the two laws coincide."""
    N, T_ref, S = 3, 1.0, 110.4 / 273.15
    m = box_mesh(2, N, deform="sinprod", rotate_seed=21)
    mu0 = 0.03
    factor = (T1 / T_ref) ** 1.5 * (T_ref + S) / (T1 + S)
    o_s = orc.Oracle(m, N, mu=mu0, visc_law=1, T_ref=T_ref, S_suth=S)
    o_c = orc.Oracle(m, N, mu=mu0 * factor)
    U = _uniform_temperature_state(m.n_elems, N, T1, seed=5)
    Rs = o_s.time_derivative(U).reshape(m.n_elems, 5, -1)
    Rc = o_c.time_derivative(U).reshape(m.n_elems, 5, -1)
    for v in range(5):
        assert np.abs(Rs[:, v] - Rc[:, v]).max() <= 1e-12 * np.abs(Rc[:, v]).max(), v
    Is, Ic = o_s.integrals(U), o_c.integrals(U)
    assert abs(Is[6] - Ic[6]) <= 1e-13 * abs(Ic[6])


def test_sutherland_changes_r_where_temperature_varies(orc):
    """With a varying temperature Sutherland's R differs from every constant
    law's (the viscosity follows the nodes' temperatures), while conservation
    still holds to rounding."""
    N = 3
    m = box_mesh(2, N, deform="sinprod", rotate_seed=22)
    o_s = orc.Oracle(m, N, mu=0.03, visc_law=1, T_ref=1.0, S_suth=0.4)
    U = random_state(m.n_elems, N, seed=6)
    tot, scale = _conservation(orc, o_s, U, N)
    assert (np.abs(tot) < 1e-13 * scale).all(), (tot, scale)
    Rs = o_s.time_derivative(U)
    Rc = orc.Oracle(m, N, mu=0.03).time_derivative(U)
    assert np.abs(Rs - Rc).max() > 1e-6 * np.abs(Rc).max()


def test_unknown_viscosity_law_rejected(orc):
    m = box_mesh(2, 2)
    with pytest.raises(ValueError):
        orc.Oracle(m, 2, mu=0.01, visc_law=3)
