"""Pins of the oracle's modal troubled-cell indicator (Persson & Peraire
2006, the detector of the paper's FV sub-cell shock capturing, Sec. 3.1):
eta = energy share of the orthonormal Legendre modes of degree N in some
direction.  Fields built from numpy's Legendre polynomials (an independent
evaluation) with known coefficients fix the transform, the orthonormal
scaling and the choice of removed modes on both node sets."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from workloads import box_mesh


def _nodes(orc, N, gauss):
    if gauss:
        return npleg.leggauss(N + 1)[0]
    return orc.basis(N)[0]


def _lt(m, x):
    c = np.zeros(m + 1)
    c[m] = 1.0
    return np.sqrt((2 * m + 1) / 2.0) * npleg.legval(x, c)


def _field(x, coef):
    """sum_abc coef[c, b, a] Lt_a(x_i) Lt_b(x_j) Lt_c(x_k) at the nodes, [k][j][i]."""
    n = len(x)
    L = np.array([_lt(m, x) for m in range(n)])        # [m][i]
    return np.einsum("cba,ck,bj,ai->kji", coef, L, L, L).reshape(-1)


@pytest.mark.parametrize("gauss", [False, True])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9])
def test_single_modes(orc, N, gauss):
    x = _nodes(orc, N, gauss)
    n = N + 1
    modes = [(0, 0, 0), (N, 0, 0), (0, N, 0), (0, 0, N), (N - 1, N - 1, N - 1), (N, N, N), (1, 0, N - 1)]
    q = []
    for a, b, c in modes:
        coef = np.zeros((n, n, n))
        coef[c, b, a] = 1.0
        q.append(_field(x, coef))
    eta = orc.persson_field(N, x, np.array(q))
    for (a, b, c), e in zip(modes, eta):
        expect = 1.0 if max(a, b, c) == N else 0.0
        assert abs(e - expect) < 1e-12, (N, gauss, (a, b, c), e)


@pytest.mark.parametrize("gauss", [False, True])
@pytest.mark.parametrize("N", [2, 4, 7, 9])
def test_known_mixtures(orc, N, gauss):
    x = _nodes(orc, N, gauss)
    n = N + 1
    rng = np.random.default_rng(N + 10 * gauss)
    coefs = rng.normal(size=(6, n, n, n)) * np.logspace(0, -3, n)[None, :, None, None]
    q = np.array([_field(x, c) for c in coefs])
    eta = orc.persson_field(N, x, q)
    a, b, c = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    top = np.maximum(np.maximum(a, b), c) == N          # indexes [c, b, a] alike
    expect = np.array([(cf[top] ** 2).sum() / (cf ** 2).sum() for cf in coefs])
    np.testing.assert_allclose(eta, expect, rtol=1e-11)
    # the share is independent of the field's scale
    np.testing.assert_allclose(orc.persson_field(N, x, 3.5 * q), eta, rtol=1e-13)


def test_state_quantities(orc):
    """dg's quantities from a state: rho, p and rho p of U, at the nodes of
    the context (LGL and Gauss), equal the field form of the same values."""
    N = 4
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=3)
    n = N + 1
    rng = np.random.default_rng(0)
    for nodes in (0, 1):
        o = orc.Oracle(mesh, N, nodes=nodes)
        x = _nodes(orc, N, nodes == 1)
        rho = 1.0 + 0.2 * rng.random((mesh.n_elems, n, n, n))
        p = 0.8 + 0.3 * rng.random((mesh.n_elems, n, n, n))
        u = 0.1 * rng.normal(size=(3, mesh.n_elems, n, n, n))
        U = np.empty((mesh.n_elems, 5, n, n, n))
        U[:, 0] = rho
        for a in range(3):
            U[:, 1 + a] = rho * u[a]
        U[:, 4] = p / 0.4 + 0.5 * rho * (u ** 2).sum(0)
        for var, q in ((0, rho), (1, p), (2, rho * p)):
            got = o.persson(U, var)
            ref = orc.persson_field(N, x, q.reshape(mesh.n_elems, -1))
            np.testing.assert_allclose(got, ref, rtol=1e-10)


def test_discontinuity_is_marked(orc):
    """A jump inside the element puts orders of magnitude more energy in the
    top modes than a smooth field (the indicator's purpose)."""
    N = 5
    x = orc.basis(N)[0]
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    smooth = (1.0 + 0.1 * np.sin(X + 0.3 * Y) * np.cos(Z)).transpose(2, 1, 0).reshape(-1)
    jump = (1.0 + 0.5 * np.tanh(40.0 * (X - 0.1))).transpose(2, 1, 0).reshape(-1)
    e_s, e_j = orc.persson_field(N, x, np.array([smooth, jump]))
    assert e_j > 1e-3 and e_s < 1e-8 and e_j > 1e5 * e_s
