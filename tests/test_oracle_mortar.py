"""Oracle pins for mortar (non-conforming) faces (GALAEXI Sec. 3.2.2, Algorithm 1;
Kopriva 1996): a periodic box whose selected cells are split 2:1, so that a
big face meets four small faces.  The big face's data are interpolated to the
four quadrants, the quadrant fluxes are projected back onto it.

Pins: the mesh generator reproduces box_mesh when nothing is split; free
stream and discrete conservation on split meshes (random element frames, all
surface fluxes); a linear density with constant velocity and pressure is
reproduced exactly next to mortar faces (interpolation of degree-1 data and the
projection of a linear flux are exact); the tangent-linear of R(U) through
mortar faces matches central differences."""
import numpy as np
import pytest

from workloads import box_mesh, random_state
from workloads.mesh import refined_box_mesh

GAMMA = 1.4


def _refine(K, cells):
    r = np.zeros(K ** 3, dtype=bool)
    r[list(cells)] = True
    return r


def test_generator_without_splits_is_box_mesh():
    for K, seed in ((1, 4), (2, 3), (3, 7)):
        m, b = refined_box_mesh(K, np.zeros(K ** 3, bool), rotate_seed=seed), box_mesh(K, 1, rotate_seed=seed)
        assert np.array_equal(m.face_nbr, b.face_nbr) and np.array_equal(m.xgeo, b.xgeo)
        assert m.mortars.shape == (0, 14)


def test_generator_mortar_table():
    K = 3
    m = refined_box_mesh(K, _refine(K, [0, 13]), rotate_seed=5)
    assert m.n_elems == 27 - 2 + 16
    assert m.mortars.shape == (12, 14)          # six unsplit neighbours of each split cell
    for i, r in enumerate(m.mortars):
        assert tuple(m.face_nbr[r[0], r[1]]) == (-1 - i, 0, 0) and m.size[r[0]] == 2
        for k in range(4):
            assert tuple(m.face_nbr[r[2 + 3 * k], r[3 + 3 * k]]) == (-1 - i, k, 0) and m.size[r[2 + 3 * k]] == 1
    # every element face is a conforming face, a big side or a quadrant
    assert (m.face_nbr[:, :, 0] < 0).sum() == 12 * 5


def _uniform(o, r=1.2, u=(0.3, -0.2, 0.45), p=0.9):
    u = np.array(u)
    U = np.zeros(o.shape)
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / (GAMMA - 1) + 0.5 * r * u @ u
    return U


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_free_stream_on_a_split_mesh(orc, N, nodes):
    K = 3
    m = refined_box_mesh(K, _refine(K, [0, 13]), rotate_seed=5)
    o = orc.Oracle(m, N, mu=0.01, nodes=nodes)
    U = _uniform(o)
    R = o.time_derivative(U)
    # rounding of O(1) fluxes through 1/(w_0 J) of the small elements
    _, Ja, J = o.geometry()
    x, w = (orc.basis(N) if nodes == 0 else orc.gauss_basis(N))[:2]
    scale = 2.0 / (w[0] * J.min())
    assert np.abs(R).max() < 2e-15 * scale * N ** 3, (np.abs(R).max(), scale)


@pytest.mark.parametrize("N,flux,nodes", [(1, 0, 0), (2, 0, 0), (3, 1, 0), (4, 2, 0), (3, 0, 0),
                                          (1, 0, 1), (2, 1, 1), (3, 0, 1), (4, 2, 1)])
def test_conservation_on_a_split_mesh(orc, N, flux, nodes):
    K = 3
    m = refined_box_mesh(K, _refine(K, [0, 13, 20]), rotate_seed=9)
    o = orc.Oracle(m, N, mu=0.02, surf_flux=flux, nodes=nodes)
    U = random_state(m.n_elems, N, seed=4, **(dict(rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05)) if nodes else {}))
    _, _, J = o.geometry()
    w = (orc.basis(N) if nodes == 0 else orc.gauss_basis(N))[1]
    wq = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    R = o.time_derivative(U).reshape(o.E, 5, -1)
    tot = np.einsum("evp,ep->v", R, J * wq)
    scale = np.einsum("evp,ep->v", np.abs(R), J * wq)
    assert (np.abs(tot) < 1e-13 * scale).all(), (tot, scale)


@pytest.mark.parametrize("N,seed,nodes", [(2, None, 0), (3, 11, 0), (4, 12, 0), (2, None, 1), (3, 11, 1), (4, 12, 1)])
def test_linear_density_exact_across_mortars(orc, N, seed, nodes):
    """rho = 1 + 0.1 x, constant velocity and pressure, inviscid, central
    volume flux on LGL nodes (the weak form on Gauss nodes takes the flux at
    the nodes): R = -(u, u^2, u v, u w, |u|^2 u / 2) d rho/dx exactly at
    every node of the elements clear of the periodic jump at x = +-1; the split
    cells sit in the middle of the box, so every mortar is among them."""
    K = 4
    cells = [1 + 4 * 1 + 16 * 1, 2 + 4 * 2 + 16 * 2, 1 + 4 * 2 + 16 * 3]
    m = refined_box_mesh(K, _refine(K, cells), rotate_seed=seed)
    o = orc.Oracle(m, N, mu=0.0, nodes=nodes)
    o.set_vol_flux(1)
    X = o.node_coords()
    u = np.array([0.3, 0.1, -0.2])
    rho = 1.0 + 0.1 * X[:, 0]
    U = np.zeros((m.n_elems, 5, X.shape[-1]))
    U[:, 0] = rho
    U[:, 1:4] = rho[:, None, :] * u[None, :, None]
    U[:, 4] = 1.0 / (GAMMA - 1) + 0.5 * rho * (u @ u)
    R = o.time_derivative(U.reshape(o.shape)).reshape(m.n_elems, 5, -1)
    ref = -0.1 * np.array([u[0], u[0] ** 2, u[0] * u[1], u[0] * u[2], 0.5 * (u @ u) * u[0]])
    xlo = m.origin[:, 0]
    inner = (xlo >= 2) & (xlo + m.size <= 6)   # elements within x in [-0.5, 0.5]
    assert inner.sum() > 0 and (m.face_nbr[inner, :, 0] < 0).any()
    err = np.abs(R[inner] - ref[None, :, None]).max()
    assert err < 1e-10, err


def test_tangent_linear_through_mortars(orc):
    """The dual-number path goes through the same mortar code: the
    tangent-linear of R(U) matches central differences."""
    N, K = 2, 2
    m = refined_box_mesh(K, _refine(K, [0]), rotate_seed=3)
    o = orc.Oracle(m, N, mu=0.02)
    U = random_state(m.n_elems, N, seed=5)
    dU = np.random.default_rng(6).normal(size=U.shape) * 1e-2
    _, dR = o.time_derivative_tl(U, dU)
    h = 1e-6
    fd = (o.time_derivative(U + h * dU) - o.time_derivative(U - h * dU)) / (2 * h)
    assert np.abs(dR - fd).max() < 1e-6 * np.abs(fd).max()


def test_mortar_rejections(orc):
    m = refined_box_mesh(2, _refine(2, [0]))
    o = orc.Oracle(m, 2)
    with pytest.raises(ValueError):
        o.set_fv_mask(np.ones(m.n_elems))
    bad = refined_box_mesh(2, _refine(2, [0]))
    bad.mortars = bad.mortars.copy()
    bad.mortars[0, 2] = bad.mortars[0, 5]       # a quadrant that does not name this mortar
    with pytest.raises(ValueError):
        orc.Oracle(bad, 2)
