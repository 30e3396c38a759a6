"""Oracle pins for the FV sub-cell operator (GALAEXI Sec. 3.1: elements flagged
by the troubled-cell indicator are advanced by a second-order finite-volume
scheme on (N+1)^3 equidistant sub-cells).  The paper fixes the scheme only by
citation; the oracle follows these readings: J-weighted sub-cell means of the
nodal interpolant, sub-face area vectors integrated from the metric terms,
minmod-limited linear reconstruction of the primitive variables, LLF sub-face
fluxes minus the central viscous flux of the sub-cell means, and on a face
between a DG and an FV element the DG side entering with the sub-face means of
its trace and taking the nodal form of the sub-face fluxes as its face flux.

Pins: a one-dimensional MUSCL-LLF finite-volume scheme written here with numpy
polynomials (a Cartesian mesh whose state varies along x only), invariance
under the elements' local frames (24 rotations, eight face orientations),
free-stream preservation and discrete conservation with mixed DG/FV meshes on
curved elements, bounded free-stream rounding over many steps in a mixed mesh,
and that an all-DG mask is the DG operator bit for bit."""
import numpy as np
import pytest

from workloads import box_mesh, random_state

GAMMA, RGAS, PR = 1.4, 1.0, 0.72


def _nodes(orc, N, nodes):
    """Nodes and weights of the node set (0: LGL, 1: Legendre-Gauss)."""
    x, w = (orc.basis(N) if nodes == 0 else orc.gauss_basis(N))[:2]
    return x, w


def _quad_weights(orc, N, nodes=0):
    _, w = _nodes(orc, N, nodes)
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)


def _free_stream(o):
    U = np.zeros(o.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / (GAMMA - 1) + 0.5 * r * u @ u
    return U


def _checkerboard(m, K):
    e = np.arange(m.n_elems)
    return ((e % K) + (e // K) % K + e // (K * K)) % 2


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_free_stream_with_fv_elements(orc, N, nodes):
    m = box_mesh(2, N, deform="sinprod", rotate_seed=7)
    o = orc.Oracle(m, N, mu=0.01, nodes=nodes)
    U = _free_stream(o)
    for mask in (_checkerboard(m, 2), np.ones(m.n_elems)):
        o.set_fv_mask(mask)
        R = o.time_derivative(U)
        assert np.abs(R).max() < 2e-12 * N * N


@pytest.mark.parametrize("N,flux,nodes", [(2, 0, 0), (3, 1, 0), (4, 2, 0), (2, 0, 1), (3, 2, 1)])
def test_conservation_with_fv_elements(orc, N, flux, nodes):
    m = box_mesh(2, N, deform="sinprod", rotate_seed=13)
    o = orc.Oracle(m, N, mu=0.02, surf_flux=flux, nodes=nodes)
    U = random_state(m.n_elems, N, seed=3, **({} if nodes == 0 else dict(rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))))
    _, _, J = o.geometry()
    wq = _quad_weights(orc, N, nodes)
    rng = np.random.default_rng(5)
    for mask in (_checkerboard(m, 2), np.ones(m.n_elems), rng.integers(0, 2, m.n_elems)):
        o.set_fv_mask(mask)
        R = o.time_derivative(U).reshape(o.E, 5, -1)
        tot = np.einsum("evp,ep->v", R, J * wq)
        scale = np.einsum("evp,ep->v", np.abs(R), J * wq)
        assert (np.abs(tot) < 1e-13 * scale).all(), (mask, tot, scale)


@pytest.mark.parametrize("nodes", [0, 1])
def test_all_dg_mask_is_the_dg_operator(orc, nodes):
    N = 3
    m = box_mesh(2, N, deform="sinprod", rotate_seed=21)
    o = orc.Oracle(m, N, mu=0.01, nodes=nodes)
    U = random_state(m.n_elems, N, seed=4, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    R0 = o.time_derivative(U)
    o.set_fv_mask(np.zeros(m.n_elems))
    assert np.array_equal(o.time_derivative(U), R0)
    o.set_fv_mask(np.ones(m.n_elems))
    assert not np.allclose(o.time_derivative(U), R0)
    o.set_fv_mask(None)
    assert np.array_equal(o.time_derivative(U), R0)


@pytest.mark.parametrize("N,nodes", [(4, 0), (7, 0), (4, 1), (7, 1)])
def test_mixed_mesh_free_stream_rounding_does_not_grow(orc, N, nodes):
    """A free stream on a checkerboard of DG and FV elements, 100 LSERK4-5
    steps: the rounding-level departure stays bounded (a coupling of the DG
    side through the inverse means map of its interior sub-cells, instead of
    the means of its trace, lets it grow 1.8x (N = 4) to 14x (N = 7) every 25
    steps)."""
    K = 2
    m = box_mesh(K, 1, lo=0.0, hi=2 * np.pi)
    o = orc.Oracle(m, N, mu=1.0 / 1600, nodes=nodes)
    U = np.zeros(o.shape)
    u = np.array([0.1, 0.05, 0.02])
    U[:, 0] = 1.0
    U[:, 1:4] = u[None, :, None, None, None]
    U[:, 4] = 1.0 / GAMMA / (GAMMA - 1) + 0.5 * u @ u
    o.set_fv_mask(_checkerboard(m, K))
    U0, drift = U.copy(), []
    for blk in range(4):
        U = o.rk_steps(U, blk * 0.25, 0.01, 25)
        drift.append(np.abs(U - U0).max() / np.abs(U0).max())
    assert max(drift) < 1e-10 and drift[-1] < 3.0 * drift[0], drift


@pytest.mark.parametrize("N,nodes", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_mixed_faces_exact_for_a_linear_density(orc, N, nodes):
    """rho = 1 + 0.1 x with constant velocity and pressure, inviscid, on a
    Cartesian mesh of DG and FV elements (checkerboard in x and y, random
    element frames), central volume flux: every part of the scheme is exact
    for it -- the FV means and unlimited slopes, the DG side's trace means at
    the mixed faces (equal to the FV side's face values, so the LLF flux is the
    physical flux), the nodal form of the sub-face fluxes and the DG operator
    -- so R = -(u, u^2, u v, u w, |u|^2 u / 2) d rho/dx at every node of the
    elements clear of the periodic jump of rho at x = +-1."""
    Kx, Ky = 4, 2
    m = box_mesh(1, 1, dims=(Kx, Ky, 1), rotate_seed=5 + N)
    o = orc.Oracle(m, N, mu=0.0, nodes=nodes)
    o.set_vol_flux(1)
    e = np.arange(m.n_elems)
    ex, ey = e % Kx, (e // Kx) % Ky
    o.set_fv_mask((ex + ey) % 2)
    X = o.node_coords()
    u = np.array([0.3, 0.1, -0.2])
    rho = 1.0 + 0.1 * X[:, 0]
    U = np.zeros((m.n_elems, 5, X.shape[-1]))
    U[:, 0] = rho
    U[:, 1:4] = rho[:, None, :] * u[None, :, None]
    U[:, 4] = 1.0 / (GAMMA - 1) + 0.5 * rho * (u @ u)
    R = o.time_derivative(U.reshape(o.shape)).reshape(m.n_elems, 5, -1)
    ref = -0.1 * np.array([u[0], u[0] ** 2, u[0] * u[1], u[0] * u[2], 0.5 * (u @ u) * u[0]])
    inner = (ex == 1) | (ex == 2)
    err = np.abs(R[inner] - ref[None, :, None]).max()
    assert err < 1e-10, err   # rounding of O(1) fluxes over sub-cells of width 1/(2 (N+1))
    assert np.abs(R[~inner] - ref[None, :, None]).max() > 1e-3   # the jump is felt next to it


def _means_matrix(x, n):
    """V[a][j]: mean over equal sub-interval a of [-1, 1] of the Lagrange
    polynomial j on the nodes x (numpy power-basis fit and antiderivative)."""
    h = 2.0 / n
    V = np.zeros((n, n))
    for j in range(n):
        c = np.polynomial.polynomial.polyfit(x, np.eye(n)[j], n - 1)
        C = np.polynomial.polynomial.polyint(c)
        for a in range(n):
            lo, hi = -1.0 + a * h, -1.0 + (a + 1) * h
            V[a, j] = (np.polynomial.polynomial.polyval(hi, C) - np.polynomial.polynomial.polyval(lo, C)) / h
    return V


def _minmod(a, b):
    return np.where(a * b <= 0, 0.0, np.where(a > 0, np.minimum(a, b), np.maximum(a, b)))


def _muscl_llf_1d(qb, gb, dx, mu):
    """Semi-discrete MUSCL-minmod scheme for the 1-D Navier-Stokes equations on
    a periodic row of cells: qb[5][M] cell means (rho, rho u, 0, 0, E), gb the
    cell means of the gradients d(u, v, w, T)/dx; returns d qb / dt."""
    r = qb[0]
    u = qb[1] / r
    p = (GAMMA - 1) * (qb[4] - 0.5 * r * u * u)
    w = np.stack([r, u, p])
    sl = _minmod(np.roll(w, -1, 1) - w, w - np.roll(w, 1, 1))
    wl = w + 0.5 * sl                      # right face of each cell
    wr = np.roll(w - 0.5 * sl, -1, 1)      # left face of the next cell

    def cons_flux(wv):
        rr, uu, pp = wv
        E = pp / (GAMMA - 1) + 0.5 * rr * uu * uu
        q = np.stack([rr, rr * uu, 0 * rr, 0 * rr, E])
        f = np.stack([rr * uu, rr * uu * uu + pp, 0 * rr, 0 * rr, (E + pp) * uu])
        return q, f, np.abs(uu) + np.sqrt(GAMMA * pp / rr)

    qL, fL, sL = cons_flux(wl)
    qR, fR, sR = cons_flux(wr)
    F = 0.5 * (fL + fR) - 0.5 * np.maximum(sL, sR) * (qR - qL)
    # viscous flux of each cell from its mean state and mean gradients
    ux, vx, wx, Tx = gb
    lam = mu * GAMMA * RGAS / ((GAMMA - 1) * PR)
    txx, txy, txz = mu * (4.0 / 3.0) * ux, mu * vx, mu * wx
    fv = np.stack([0 * r, txx, txy, txz, txx * u + lam * Tx])
    F = F - 0.5 * (fv + np.roll(fv, -1, 1))
    return -(F - np.roll(F, 1, 1)) / dx


@pytest.mark.parametrize("N,mu,nodes", [(2, 0.0, 0), (3, 0.0, 0), (3, 0.02, 0), (5, 0.01, 0), (3, 0.0, 1),
                                        (4, 0.02, 1)])
def test_fv_matches_one_dimensional_muscl_llf(orc, N, mu, nodes):
    K, n = 3, N + 1
    m = box_mesh(K, 1)
    o = orc.Oracle(m, N, gamma=GAMMA, R=RGAS, Pr=PR, mu=mu, nodes=nodes)
    o.set_fv_mask(np.ones(m.n_elems))
    x, _ = _nodes(orc, N, nodes)
    rng = np.random.default_rng(17 + N)
    rho = rng.uniform(0.7, 1.3, (K, n))
    u = rng.uniform(-0.4, 0.4, (K, n))
    p = rng.uniform(0.6, 1.4, (K, n))
    line = np.stack([rho, rho * u, 0 * rho, 0 * rho, p / (GAMMA - 1) + 0.5 * rho * u * u])   # [5][ex][i]
    e = np.arange(m.n_elems)
    U = np.zeros(o.shape)
    U[...] = line[:, e % K].transpose(1, 0, 2)[:, :, None, None, :]
    Ut = o.time_derivative(U)
    # the same scheme in one dimension
    V = _means_matrix(x, n)
    qb = np.einsum("aj,vej->vea", V, line).reshape(5, K * n)
    G = o.lifting(U).reshape(m.n_elems, 4, 3, n, n, n)
    gx = G[:K, :, 0, 0, 0, :]                                     # d/dx along the first row of elements
    gb = np.einsum("aj,erj->rea", V, gx).reshape(4, K * n)
    Rb = _muscl_llf_1d(qb, gb, 2.0 / (K * n), mu).reshape(5, K, n)
    Rn = np.einsum("aj,vej->vea", np.linalg.inv(V), Rb)          # nodal values along x
    ref = Rn[:, e % K].transpose(1, 0, 2)[:, :, None, None, :] * np.ones(o.shape)
    assert np.abs(Ut - ref).max() < 1e-11 * np.abs(ref).max()


def _state_field(X):
    """A smooth field with a density and pressure jump across a tilted plane."""
    x, y, z = X
    s = np.where(0.6 * x + 0.3 * y - 0.2 * z > 0.05, 1.0, 0.0)
    rho = 1.0 + 0.2 * np.sin(np.pi * x) * np.cos(np.pi * y) + 0.3 * s
    u = np.stack([0.2 * np.cos(np.pi * z), -0.1 + 0.1 * np.sin(np.pi * x), 0.15 * np.sin(np.pi * y)])
    p = 1.0 + 0.1 * np.cos(np.pi * (x + z)) + 0.4 * s
    U = np.concatenate([rho[None], rho[None] * u, (p / (GAMMA - 1) + 0.5 * rho * (u * u).sum(0))[None]])
    return U


@pytest.mark.parametrize("N,fv,nodes", [(2, "all", 0), (3, "checker", 0), (4, "random", 0), (3, "random", 1)])
def test_fv_invariant_under_local_element_frames(orc, N, fv, nodes):
    """The same physical state on a Cartesian mesh with identity frames and with
    random element rotations (all face orientations): the residual at each
    physical node agrees."""
    K = 3
    m0, m1 = box_mesh(K, 1), box_mesh(K, 1, rotate_seed=31 + N)
    assert (m1.rot != m0.rot).any()
    mask = {"all": np.ones(m0.n_elems), "checker": _checkerboard(m0, K),
            "random": np.random.default_rng(3).integers(0, 2, m0.n_elems)}[fv]
    out = []
    for m in (m0, m1):
        o = orc.Oracle(m, N, gamma=GAMMA, R=RGAS, Pr=PR, mu=0.01, nodes=nodes)
        o.set_fv_mask(mask)
        X = o.node_coords()                                     # [E][3][P]
        U = np.stack([_state_field(X[e]) for e in range(o.E)])  # [E][5][P]
        R = o.time_derivative(U.reshape(o.shape)).reshape(o.E, 5, -1)
        key = np.round(X, 9)
        order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]), axis=-1)
        out.append(np.take_along_axis(R, order[:, None, :], axis=2))
    scale = np.abs(out[0]).max()
    assert np.abs(out[0] - out[1]).max() < 1e-11 * scale


def test_fv_mask_rejections(orc):
    m = box_mesh(2, 1)
    o = orc.Oracle(m, 2)
    with pytest.raises(ValueError):
        o.set_fv_mask(np.ones(m.n_elems + 1))
    o.set_fv_mask(np.ones(m.n_elems))
    U = _free_stream(o)
    with pytest.raises(ValueError):
        o.time_derivative_tl(U, U)
