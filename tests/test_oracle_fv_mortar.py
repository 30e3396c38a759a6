"""Oracle pins for FV sub-cell elements on 2:1 mortar meshes (GALAEXI Sec. 3.1
shock capturing with the mortars of Sec. 3.2.2, Algorithm 1).  The mortar maps
act on DG traces, so an element with a mortar face stays a DG element (a
reading: the paper does not treat FV sub-cells at mortars); FV elements
elsewhere meet DG or FV neighbours through conforming faces only.

Pins: a mask that flags an element with a mortar face is refused; an all-DG
mask is the DG operator bit for bit; free streams stay free streams and the
element integrals of R(U) vanish with FV elements next to elements that have
mortar faces (both node sets); the switching never flags an element with a
mortar face, flags others, and keeps the totals through steps."""
import numpy as np
import pytest

from workloads import random_state
from workloads.mesh import refined_box_mesh

GAMMA = 1.4


def _mesh(seed=3):
    r = np.zeros(27, dtype=bool)
    r[13] = True                     # the centre cell split: its six neighbours and its children have mortar faces
    return refined_box_mesh(3, r, rotate_seed=seed)


def _touching(m):
    return (m.face_nbr[:, :, 0] < 0).any(axis=1)


def _weights(orc, N, nodes):
    w = (orc.basis(N) if nodes == 0 else orc.gauss_basis(N))[1]
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)


def _fv_mask(m):
    """Every other element without a mortar face: FV elements next to DG
    elements that have mortar faces, and FV-FV faces."""
    free = np.where(~_touching(m))[0]
    mask = np.zeros(m.n_elems, dtype=np.int32)
    mask[free[::2]] = 1
    return mask


def test_mask_rule(orc):
    m = _mesh()
    o = orc.Oracle(m, 2, mu=0.01)
    bad = np.zeros(m.n_elems, dtype=np.int32)
    bad[np.where(_touching(m))[0][0]] = 1
    with pytest.raises(ValueError):
        o.set_fv_mask(bad)
    o.set_fv_mask(_fv_mask(m))
    assert o.fv_state()[0].sum() == _fv_mask(m).sum()


@pytest.mark.parametrize("nodes", [0, 1])
def test_all_dg_mask_is_the_dg_operator(orc, nodes):
    m = _mesh()
    N = 3
    U = random_state(m.n_elems, N, seed=4, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    o = orc.Oracle(m, N, mu=0.01, nodes=nodes)
    R0 = o.time_derivative(U)
    o.set_fv_mask(np.zeros(m.n_elems, dtype=np.int32))
    assert np.array_equal(o.time_derivative(U), R0)


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("N", [2, 3])
def test_free_stream_with_fv_elements_on_a_mortar_mesh(orc, N, nodes):
    m = _mesh(seed=5)
    o = orc.Oracle(m, N, mu=0.01, nodes=nodes)
    o.set_fv_mask(_fv_mask(m))
    U = np.zeros(o.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.1]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / (GAMMA - 1) + 0.5 * r * u @ u
    R = o.time_derivative(U)
    assert np.abs(R).max() < 1e-12 * np.abs(U).max(), np.abs(R).max()


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_conservation_with_fv_elements_on_a_mortar_mesh(orc, flux, nodes):
    m = _mesh(seed=6)
    N = 3
    o = orc.Oracle(m, N, mu=0.02, surf_flux=flux, nodes=nodes)
    o.set_fv_mask(_fv_mask(m))
    U = random_state(m.n_elems, N, seed=7, rho=(0.9, 1.1), vel=0.3, p=(0.9, 1.1))
    R = o.time_derivative(U).reshape(m.n_elems, 5, -1)
    J = o.geometry()[2]
    wq = _weights(orc, N, nodes)
    tot = np.einsum("evp,ep->v", R, J * wq)
    scale = np.einsum("evp,ep->v", np.abs(R), J * wq)
    assert (np.abs(tot) < 1e-13 * scale).all(), (tot, scale)


@pytest.mark.parametrize("nodes", [0, 1])
def test_switching_keeps_elements_with_mortar_faces_dg(orc, nodes):
    """A density and pressure jump across the mesh: the switching flags
    elements away from the mortars, never one with a mortar face, and the
    totals stay conserved through the steps."""
    m = _mesh(seed=8)
    N = 3
    o = orc.Oracle(m, N, mu=1e-3, nodes=nodes)
    X = o.node_coords()
    sel = X[:, 0] < X[:, 0].mean()
    U = np.zeros((m.n_elems, 5, X.shape[-1]))
    U[:, 0] = np.where(sel, 1.0, 0.5)
    U[:, 4] = np.where(sel, 1.0, 0.5) / (GAMMA - 1)
    U = U.reshape(o.shape)
    o.set_fv_switch(2, -2.0, -3.0)
    J = o.geometry()[2]
    wq = _weights(orc, N, nodes)
    tot0 = np.einsum("evp,ep->v", U.reshape(m.n_elems, 5, -1), J * wq)
    seen = np.zeros(m.n_elems, dtype=bool)
    for k in range(4):
        U = o.rk_steps(U, k * 1e-3, 1e-3, 1)
        assert np.isfinite(U).all()
        seen |= o.fv_state()[0] != 0
    assert seen.any() and not (seen & _touching(m)).any()
    tot = np.einsum("evp,ep->v", U.reshape(m.n_elems, 5, -1), J * wq)
    scale = np.einsum("evp,ep->", np.abs(U.reshape(m.n_elems, 5, -1)), J * wq)
    assert (np.abs(tot - tot0) < 1e-14 * scale).all(), (tot - tot0, scale)
