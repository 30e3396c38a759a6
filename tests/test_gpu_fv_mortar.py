"""FV sub-cell elements on 2:1 mortar meshes on the GPU, through the C ABI,
against the oracle: an element with a mortar face stays a DG element (the
mortar maps act on DG traces); FV elements elsewhere.  R(U) within 1e-12
relative per variable (both node sets, the three surface fluxes), RK steps
with automatic switching within 1e-10 with equal masks, and the refusal of a
mask that flags an element with a mortar face."""
import numpy as np
import pytest

from workloads import random_state
from workloads.mesh import refined_box_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAMMA = 1.4
_STATE = dict(rho=(0.9, 1.1), vel=0.3, p=(0.9, 1.1))


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _mesh(seed):
    r = np.zeros(27, dtype=bool)
    r[13] = True
    return refined_box_mesh(3, r, rotate_seed=seed)


def _touching(m):
    return (m.face_nbr[:, :, 0] < 0).any(axis=1)


def _fv_mask(m):
    free = np.where(~_touching(m))[0]
    mask = np.zeros(m.n_elems, dtype=np.int32)
    mask[free[::2]] = 1
    return mask


def _rel_err_per_var(got, ref):
    got = got.reshape(got.shape[0], 5, -1)
    ref = ref.reshape(ref.shape[0], 5, -1)
    return np.array([np.abs(got[:, v] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-300) for v in range(5)])


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("N,flux", [(2, 0), (3, 1), (3, 2), (4, 0)])
def test_fv_on_mortar_mesh_time_derivative_parity(orc, dg, N, flux, nodes):
    m = _mesh(300 + N)
    kw = dict(mu=0.02, surf_flux=flux, nodes=nodes)
    o, s = orc.Oracle(m, N, **kw), dg.Solver(m, N, **kw)
    mask = _fv_mask(m)
    o.set_fv_mask(mask)
    s.set_fv_mask(mask)
    U = random_state(m.n_elems, N, seed=310 + N, **_STATE)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < 1e-12).all(), err


@pytest.mark.parametrize("nodes", [0, 1])
def test_switching_on_mortar_mesh_rk_parity(orc, dg, nodes):
    """A density and pressure jump: the switching flags elements away from
    the mortars, none with a mortar face; the states after the steps and the
    masks equal the oracle's."""
    N = 3
    m = _mesh(320 + nodes)
    o = orc.Oracle(m, N, mu=1e-3, nodes=nodes)
    s = dg.Solver(m, N, mu=1e-3, nodes=nodes)
    X = o.node_coords()
    sel = X[:, 0] < X[:, 0].mean()
    U0 = np.zeros((m.n_elems, 5, X.shape[-1]))
    U0[:, 0] = np.where(sel, 1.0, 0.5)
    U0[:, 4] = np.where(sel, 1.0, 0.5) / (GAMMA - 1)
    U0 = U0.reshape(o.shape)
    o.set_fv_switch(2, -2.0, -3.0)
    s.set_fv_switch(dg.IND_RHOP, -2.0, -3.0)
    ref = U0.copy()
    seen = np.zeros(m.n_elems, dtype=bool)
    for k in range(4):
        ref = o.rk_steps(ref, k * 1e-3, 1e-3, 1)
        mk, margin = o.fv_state()
        assert margin > 1e-9, (k, margin)
        seen |= mk != 0
    assert seen.any() and not (seen & _touching(m)).any()
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 4)
    got = Ud.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-10
    assert np.array_equal(s.fv_mask().cpu().numpy(), o.fv_state()[0])


def test_mask_with_a_mortar_element_is_refused(dg):
    m = _mesh(330)
    s = dg.Solver(m, 2, mu=0.01)
    bad = np.zeros(m.n_elems, dtype=np.int32)
    bad[np.where(_touching(m))[0][-1]] = 1
    with pytest.raises(dg.DGError):
        s.set_fv_mask(bad)
    s.set_fv_mask(_fv_mask(m))
    assert np.array_equal(s.fv_mask().cpu().numpy(), _fv_mask(m))
