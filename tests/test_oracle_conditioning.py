"""Why the N = 8, 9 parity bars grow with kappa^3 (reading C17): the mesh is
given as equispaced samples of degree ngeo = N, and their interpolation to the
LGL nodes amplifies a change of the samples by kappa = max_i sum_j |V_ij| per
direction.  Moving every sample by one ulp (+-1 or 0, the same move at points
that elements share, so the mesh stays watertight) moves the oracle's own
R(U) by about 3e-15 kappa^3 relative: 9e-13 at N = 7, 3e-12 at N = 8 and
2e-11 at N = 9.  Two independent FP64 codes, which round the geometry
differently, cannot agree to 1e-12 there; the GPU bars of 1e-12 kappa^3/300
(x4.1 at N = 8, x18 at N = 9) are of the size of this spread."""
import numpy as np
import pytest

from workloads import box_mesh, random_state


def _kappa3(orc, N):
    x, _, _ = orc.basis(N)
    xe = np.linspace(-1.0, 1.0, N + 1)
    V = np.array([[np.prod([(xi - xe[m]) / (xe[j] - xe[m]) for m in range(N + 1) if m != j])
                   for j in range(N + 1)] for xi in x])
    return np.abs(V).sum(1).max() ** 3


def _ulp_move(xgeo):
    """+-1 ulp or no move per coordinate, a hash of the point's bits, so that
    the samples of a point shared by several elements move alike."""
    b = xgeo.view(np.uint64)
    out = xgeo.copy()
    with np.errstate(over="ignore"):
        for c in range(3):
            h = (b[:, 0] * np.uint64(0x9E3779B97F4A7C15) ^ b[:, 1] * np.uint64(0xC2B2AE3D27D4EB4F)
                 ^ b[:, 2] * np.uint64(0x165667B19E3779F9) ^ np.uint64(c + 1) * np.uint64(0x27D4EB2F165667C5))
            s = ((h >> np.uint64(33)) % np.uint64(3)).astype(np.int64) - 1
            v = out[:, c]
            out[:, c] = np.where(s > 0, np.nextafter(v, np.inf), np.where(s < 0, np.nextafter(v, -np.inf), v))
    return out


def test_geometry_rounding_spread_grows_with_kappa_cubed(orc):
    spread = {}
    for N in (5, 7, 8, 9):
        mesh = box_mesh(2, N, deform="sinprod", rotate_seed=1000 + N)
        moved = type(mesh)(**{**mesh.__dict__, "xgeo": _ulp_move(mesh.xgeo)})
        assert (np.abs(moved.xgeo - mesh.xgeo) <= np.spacing(np.abs(mesh.xgeo))).all()
        U = random_state(mesh.n_elems, N, seed=3 + N)
        R1 = orc.Oracle(mesh, N, mu=0.02).time_derivative(U).reshape(mesh.n_elems, 5, -1)
        R2 = orc.Oracle(moved, N, mu=0.02).time_derivative(U).reshape(mesh.n_elems, 5, -1)
        spread[N] = max(np.abs(R1[:, v] - R2[:, v]).max() / np.abs(R1[:, v]).max() for v in range(5))
        # the spread per unit of kappa^3 stays at a few 1e-15 from N = 5 to 9
        ratio = spread[N] / _kappa3(orc, N)
        assert 5e-16 < ratio < 2e-14, (N, spread[N], ratio)
    # a 1e-12 bar is within reach up to N = 7 and not beyond
    assert spread[5] < 1e-12 and spread[7] < 1e-12
    assert spread[8] > 1e-12 and spread[9] > 5e-12
