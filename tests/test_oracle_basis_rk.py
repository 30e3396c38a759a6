"""Oracle pins: LGL basis and the LSERK4-5 coefficients (GALAEXI Sec. 3.1)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ev(s):
    return eval(s, {"sqrt": math.sqrt})


def test_lgl_closed_forms(orc):
    g = json.load(open(os.path.join(GOLD, "lgl_closed_forms.json")))
    for N, ref in g["cases"].items():
        x, w, _ = orc.basis(int(N))
        np.testing.assert_allclose(x, [_ev(s) for s in ref["x"]], rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, [_ev(s) for s in ref["w"]], rtol=4e-16, atol=0)


@pytest.mark.parametrize("N", range(1, 10))
def test_sbp_and_exactness(orc, N):
    x, w, D = orc.basis(N)
    assert abs(w.sum() - 2.0) < 1e-14
    # summation-by-parts: W D + (W D)^T = diag(-1, 0, ..., 0, 1)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    assert np.abs(Q + Q.T - B).max() < 5e-14
    # D is exact on polynomials of degree <= N
    for k in range(N + 1):
        ref = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        assert np.abs(D @ x ** k - ref).max() < 1e-12 * max(1, k * k)
    # quadrature exact to degree 2N-1
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ x ** k - exact) < 1e-14
    # nodes are the roots of P_N' (interior)
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    assert np.abs(dP(x[1:-1])).max() < 1e-12 if N > 1 else True


def _butcher_from_2n(A, B):
    """Butcher tableau of a 2N-storage scheme G <- A_s G + dt R; U <- U + B_s G."""
    s = len(A)
    a = [[Fraction(0)] * s for _ in range(s)]
    b = [Fraction(0)] * s
    # coefficient of R_j in G_i:  g[i][j] = A_i g[i-1][j] (j<i), g[i][i] = 1
    g = [[Fraction(0)] * s for _ in range(s)]
    for i in range(s):
        for j in range(i):
            g[i][j] = A[i] * g[i - 1][j]
        g[i][i] = Fraction(1)
    # U_i = U_0 + sum_{k<i} B_k G_k  -> stage value used for R_i
    for i in range(s):
        for j in range(s):
            a[i][j] = sum((B[k] * g[k][j] for k in range(i)), Fraction(0))
    for j in range(s):
        b[j] = sum((B[k] * g[k][j] for k in range(s)), Fraction(0))
    return a, b


def test_lserk45_coefficients_and_order(orc):
    gold = json.load(open(os.path.join(GOLD, "lserk45_carpenter_kennedy.json")))
    A, B, Cc = orc.rk_coeffs()
    fA = [Fraction(s) for s in gold["A"]]
    fB = [Fraction(s) for s in gold["B"]]
    fC = [Fraction(s) for s in gold["c"]]
    np.testing.assert_allclose(A, [float(v) for v in fA], rtol=1e-16, atol=0)
    np.testing.assert_allclose(B, [float(v) for v in fB], rtol=1e-16, atol=0)
    np.testing.assert_allclose(Cc, [float(v) for v in fC], rtol=1e-16, atol=0)
    a, b = _butcher_from_2n(fA, fB)
    c = [sum(r, Fraction(0)) for r in a]
    for i in range(5):
        assert abs(float(c[i] - fC[i])) < 1e-15
    s = range(5)
    # the eight order conditions up to order 4
    conds = [
        (sum(b[i] for i in s), 1),
        (sum(b[i] * c[i] for i in s), Fraction(1, 2)),
        (sum(b[i] * c[i] ** 2 for i in s), Fraction(1, 3)),
        (sum(b[i] * a[i][j] * c[j] for i in s for j in s), Fraction(1, 6)),
        (sum(b[i] * c[i] ** 3 for i in s), Fraction(1, 4)),
        (sum(b[i] * c[i] * a[i][j] * c[j] for i in s for j in s), Fraction(1, 8)),
        (sum(b[i] * a[i][j] * c[j] ** 2 for i in s for j in s), Fraction(1, 12)),
        (sum(b[i] * a[i][j] * a[j][k] * c[k] for i in s for j in s for k in s), Fraction(1, 24)),
    ]
    for got, want in conds:
        assert abs(float(got - want)) < 1e-15
    # and it is not fifth order: one fifth-order condition fails
    assert abs(float(sum(b[i] * c[i] ** 4 for i in s) - Fraction(1, 5))) > 1e-6


def test_lserk_time_order_on_dg_system(orc):
    """Observed 4th-order convergence in dt of the oracle's LSERK loop."""
    from workloads import box_mesh, tgv_params
    prm = tgv_params(Ma=0.3, Re=100.0)
    m = box_mesh(2, 2, lo=0.0, hi=2 * np.pi)
    o = orc.Oracle(m, 2, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U0 = o.initial_state("tgv", prm["p0"])
    T = 0.2
    ref = o.rk_steps(U0, 0.0, T / 64, 64)
    errs = []
    for nst in (4, 8, 16):
        errs.append(np.abs(o.rk_steps(U0, 0.0, T / nst, nst) - ref).max())
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(eoc) > 3.6, (errs, eoc)


def test_rk414_coefficients_and_order(orc):
    """RK4-14 (Niegemann, Diehl & Busch 2012): the oracle's table equals the
    published sixteen digits; with those decimals taken exactly, the stage
    times are the row sums of the Butcher form, the eight conditions of order
    four hold to the rounding of the sixteenth digit, and a fifth-order
    condition fails."""
    gold = json.load(open(os.path.join(GOLD, "rk414_niegemann.json")))
    A, B, Cc = orc.rk14_coeffs()
    fA = [Fraction(s) for s in gold["A"]]
    fB = [Fraction(s) for s in gold["B"]]
    fC = [Fraction(s) for s in gold["c"]]
    np.testing.assert_allclose(A, [float(v) for v in fA], rtol=1e-16, atol=0)
    np.testing.assert_allclose(B, [float(v) for v in fB], rtol=1e-16, atol=0)
    np.testing.assert_allclose(Cc, [float(v) for v in fC], rtol=1e-16, atol=0)
    a, b = _butcher_from_2n(fA, fB)
    s = range(14)
    c = [sum(r, Fraction(0)) for r in a]
    for i in s:
        assert abs(float(c[i] - fC[i])) < 2e-15, i
    conds = [
        (sum(b[i] for i in s), 1),
        (sum(b[i] * c[i] for i in s), Fraction(1, 2)),
        (sum(b[i] * c[i] ** 2 for i in s), Fraction(1, 3)),
        (sum(b[i] * a[i][j] * c[j] for i in s for j in s), Fraction(1, 6)),
        (sum(b[i] * c[i] ** 3 for i in s), Fraction(1, 4)),
        (sum(b[i] * c[i] * a[i][j] * c[j] for i in s for j in s), Fraction(1, 8)),
        (sum(b[i] * a[i][j] * c[j] ** 2 for i in s for j in s), Fraction(1, 12)),
        (sum(b[i] * a[i][j] * a[j][k] * c[k] for i in s for j in s for k in s), Fraction(1, 24)),
    ]
    for got, want in conds:
        assert abs(float(got - want)) < 5e-15, float(got - want)
    assert abs(float(sum(b[i] * c[i] ** 4 for i in s) - Fraction(1, 5))) > 1e-6


def test_rk414_time_order_on_dg_system(orc):
    """Observed fourth-order convergence in dt of the oracle's RK4-14 loop, and
    agreement with RK4-5 to the schemes' truncation error."""
    from workloads import box_mesh, tgv_params
    prm = tgv_params(Ma=0.3, Re=100.0)
    m = box_mesh(2, 2, lo=0.0, hi=2 * np.pi)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    o = orc.Oracle(m, 2, rk=1, **kw)
    U0 = o.initial_state("tgv", prm["p0"])
    T = 0.4
    ref = o.rk_steps(U0, 0.0, T / 32, 32)
    errs = [np.abs(o.rk_steps(U0, 0.0, T / nst, nst) - ref).max() for nst in (2, 4, 8)]
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(eoc) > 3.5, (errs, eoc)
    ref45 = orc.Oracle(m, 2, **kw).rk_steps(U0, 0.0, T / 64, 64)
    assert np.abs(ref - ref45).max() < 1e-8 * np.abs(ref45).max()


def _butcher_float(A, B):
    s = len(A)
    alpha = np.zeros((s, s))
    for i in range(s):
        for j in range(i):
            alpha[i, j] = A[i] * alpha[i - 1, j]
        alpha[i, i] = 1.0
    a = np.zeros((s, s))
    for i in range(1, s):
        for j in range(i):
            a[i, j] = sum(B[k] * alpha[k, j] for k in range(j, i))
    b = np.array([sum(B[k] * alpha[k, j] for k in range(j, s)) for j in range(s)])
    return a, b


def _stable_dt(a, b, ev):
    """Largest dt with |R(dt lambda)| <= 1 on the spectrum ev (bisection),
    R(z) = 1 + z b^T (I - z A)^-1 1."""
    s = len(b)

    def ok(dt):
        for lam in ev:
            z = dt * lam
            if abs(1 + z * b @ np.linalg.solve(np.eye(s) - z * a, np.ones(s))) > 1 + 1e-12:
                return False
        return True
    lo, hi = 0.0, 8.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    return lo


@pytest.mark.parametrize("N", [5, 7])
def test_rk414_stability_per_stage_on_dg_spectrum(orc, N):
    """RK4-14 was optimised for the spectra of DG operators: on the 1-D upwind
    DG advection operator on Gauss nodes (8 periodic elements) its largest
    stable step is more than 14/5 x 1.2 times that of LSERK4-5, i.e. more than
    20 % more step per stage."""
    _, w, D, lm, lp = orc.gauss_basis(N)
    n, K = N + 1, 8
    A = np.zeros((n * K, n * K))
    for e in range(K):
        el = (e - 1) % K
        for i in range(n):
            for m in range(n):
                A[e * n + i, e * n + m] += w[m] / w[i] * D[m, i] - lp[i] / w[i] * lp[m]
                A[e * n + i, el * n + m] += lm[i] / w[i] * lp[m]
    ev = np.linalg.eigvals(A)
    a5, b5 = _butcher_float(*orc.rk_coeffs()[:2])
    a14, b14 = _butcher_float(*orc.rk14_coeffs()[:2])
    d5, d14 = _stable_dt(a5, b5, ev), _stable_dt(a14, b14, ev)
    assert (d14 / 14) / (d5 / 5) > 1.2, (d5, d14)
