"""Seeded input generators shared by the oracle and the CUDA path: the mesh
format's connectivity and face-orientation codes against the sampled
geometry itself, the element frames, and the state and ensemble generators."""
import numpy as np
import pytest

from workloads import ROTATIONS, box_mesh, ensemble_members, random_state
from workloads.mesh import face_node_flip


def _face_samples(xgeo, e, f):
    """[3, n, n] coordinates of face f = 2d + s of element e, indexed (p, q)
    along the two other reference directions in increasing order."""
    d, s = divmod(f, 2)
    n = xgeo.shape[-1]
    a = 0 if s == 0 else n - 1
    x = xgeo[e]                                  # [c, k, j, i]
    if d == 0:
        return np.transpose(x[:, :, :, a], (0, 2, 1))    # (p, q) = (j, k)
    if d == 1:
        return np.transpose(x[:, :, a, :], (0, 2, 1))    # (p, q) = (i, k)
    return np.transpose(x[:, a, :, :], (0, 2, 1))        # (p, q) = (i, j)


def test_rotations_are_the_24_proper_ones():
    mats = {tuple(m.ravel()) for m in ROTATIONS}
    assert len(mats) == 24
    for m in ROTATIONS:
        assert round(np.linalg.det(m)) == 1
        assert (m.T @ m == np.eye(3, dtype=m.dtype)).all()


@pytest.mark.parametrize("ngeo,deform", [(1, None), (2, "sinprod"), (3, "sinprod")])
def test_face_codes_match_the_geometry(ngeo, deform):
    K, lo, hi = 3, 0.0, 2 * np.pi
    m = box_mesh(K, ngeo, lo=lo, hi=hi, deform=deform, rotate_seed=7)
    L = hi - lo
    for e in range(m.n_elems):
        for f in range(6):
            e2, f2, flip = (int(v) for v in m.face_nbr[e, f])
            back = m.face_nbr[e2, f2]
            assert back[0] == e and back[1] == f and (e2, f2) != (e, f)
            A, B = _face_samples(m.xgeo, e, f), _face_samples(m.xgeo, e2, f2)
            for p in range(ngeo + 1):
                for q in range(ngeo + 1):
                    p2, q2 = face_node_flip(flip, p, q, ngeo)
                    diff = A[:, p, q] - B[:, p2, q2]
                    # the same physical point, up to the periodic shift
                    assert np.abs(diff - L * np.round(diff / L)).max() < 1e-12


def test_all_orientations_occur_on_the_rotated_mesh():
    m = box_mesh(16, 1, rotate_seed=20260528)
    assert set(np.unique(m.face_nbr[:, :, 2])) == set(range(8))
    assert set(np.unique(m.rot)) == set(range(24))


def test_state_and_ensemble_generators():
    U = random_state(8, 3, seed=5)
    assert U.shape == (8, 5, 4, 4, 4)
    np.testing.assert_array_equal(U, random_state(8, 3, seed=5))
    r = U[:, 0]
    ke = 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / r
    p = 0.4 * (U[:, 4] - ke)
    assert r.min() > 0 and p.min() > 0
    runs = ensemble_members()
    assert runs == ensemble_members() and len(runs) == 64
    assert all(8 <= s["K"] <= 24 and 3 <= s["N"] <= 7 and 0.1 <= s["Ma"] <= 0.5 and 400 <= s["Re"] <= 1600
               for s in runs)
    assert len({s["N"] for s in runs}) == 5
