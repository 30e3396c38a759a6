"""FP32-operator path (volume flux differencing, lifting and face fluxes in
FP32; state, metrics precomputation, stage update and reductions in FP64)
against the FP64 oracle.  The bars state the errors FP32 arithmetic allows;
they are not parity tolerances."""
import math

import numpy as np
import pytest

from workloads import box_mesh, random_state, tgv_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("N", [2, 3, 5, 7, 9])
def test_fp32_time_derivative_vs_oracle(orc, dg, N):
    K = 3 if N <= 4 else 2
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=400 + N)
    o = orc.Oracle(mesh, N, mu=0.02)
    s = dg.Solver(mesh, N, mu=0.02, precision=dg.FP32OP)
    U = random_state(mesh.n_elems, N, seed=500 + N)
    ref = o.time_derivative(U).reshape(mesh.n_elems, 5, -1)
    got = s.time_derivative(torch.from_numpy(U).cuda()).cpu().numpy().reshape(mesh.n_elems, 5, -1)
    for v in range(5):
        err = np.abs(got[:, v] - ref[:, v]).max() / np.abs(ref[:, v]).max()
        assert err < 2e-5, (v, err)


def test_fp32_tgv_rk_vs_oracle(orc, dg):
    prm = tgv_params(Ma=0.1, Re=1600.0)
    N = 3
    mesh = box_mesh(4, 1, lo=0.0, hi=2 * math.pi)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    o = orc.Oracle(mesh, N, **kw)
    s = dg.Solver(mesh, N, precision=dg.FP32OP, **kw)
    U0 = o.initial_state("tgv", prm["p0"])
    Ud = torch.from_numpy(U0).cuda()
    dt = s.max_dt(Ud)
    ref = o.rk_steps(U0, 0.0, dt, 10)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, dt, 10)
    got = Ud.cpu().numpy()
    # state: FP32 rounding of the stage updates relative to |U|
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-6
    # kinetic energy (the quantity the FP32 path is judged on)
    ek_ref, ek = o.integrals(ref)[5], s.integrals(Ud)[5]
    assert abs(ek - ek_ref) / ek_ref < 1e-6
    # mass stays conserved: FP32 flux rounding only
    I0 = o.integrals(U0)
    assert abs(s.integrals(Ud)[0] - I0[0]) / I0[0] < 1e-7


def test_fp32_free_stream(dg):
    N = 5
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=7)
    s = dg.Solver(mesh, N, mu=0.01, precision=dg.FP32OP)
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = s.time_derivative(torch.from_numpy(U).cuda()).cpu().numpy()
    # FP32 rounding of terms of size |D| |f . Ja| / J ~ 1e2
    assert np.abs(R).max() < 1e-3


@pytest.mark.parametrize("flux,nodes", [(0, 0), (1, 0), (2, 0), (0, 1), (2, 1)])
def test_fp32_pressure_offset_low_mach(orc, dg, flux, nodes):
    """The FP32 operator with the background pressure p_ref taken out of the
    momentum flux returns the same R(U) (the constant part has no discrete
    divergence), with momentum rounding errors set by p - p_ref instead of p:
    at Ma 0.1 (p0 = 71) at least five times smaller.  On Gauss nodes the FP32
    face values carry E - E_ref (prolonged from the FP64 difference)."""
    prm = tgv_params(Ma=0.1, Re=1600.0)
    N = 5
    mesh = box_mesh(3, N, lo=0.0, hi=2 * math.pi, deform="sinprod", amp=0.05, rotate_seed=31)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], surf_flux=flux, nodes=nodes)
    o = orc.Oracle(mesh, N, **kw)
    U0 = o.initial_state("tgv", prm["p0"])
    ref = o.time_derivative(U0).reshape(mesh.n_elems, 5, -1)
    errs = {}
    for p_ref in (0.0, prm["p0"]):
        s = dg.Solver(mesh, N, precision=dg.FP32OP, p_ref=p_ref, **kw)
        got = s.time_derivative(torch.from_numpy(U0).cuda()).cpu().numpy().reshape(mesh.n_elems, 5, -1)
        errs[p_ref] = [np.abs(got[:, v] - ref[:, v]).max() / np.abs(ref[:, v]).max() for v in range(5)]
        s.close()
    e0, e1 = errs[0.0], errs[prm["p0"]]
    # momentum: the offset removes the rounding of p0 from the pressure terms;
    # on Gauss nodes the face values are FP32 interpolations, whose rounding
    # enters the dissipation through the jumps (|lambda| ~ c = 10 at Ma 0.1)
    cap = 1e-4 if nodes == 0 else 3e-4
    for v in (1, 2, 3):
        assert e1[v] < 0.2 * e0[v] and e1[v] < cap, (v, e0, e1)
    # density and energy: unchanged by the offset (their relative errors are
    # large at low Mach numbers because R is O(Ma^2) smaller than its terms)
    for v in (0, 4):
        assert e1[v] < 1.5 * e0[v] + 1e-6, (v, e0, e1)


def test_fp32_conversions_match_hardware(dg):
    """The integer-bit FP64 -> FP32 narrowing equals the hardware
    round-to-nearest conversion (random mantissas never sit on an exact tie)
    over the normal FP32 range, flushes values below the smallest normal
    float to zero, and the widening back is exact."""
    rng = np.random.default_rng(11)
    m = rng.uniform(1.0, 2.0, 200000)
    ex = rng.integers(-126, 127, m.size)
    x = np.ldexp(m, ex) * rng.choice([-1.0, 1.0], m.size)
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.0, 1.5, np.nextafter(2.0, 1.0), 71.42857142857143,
                            np.ldexp(1.0, -126), np.ldexp(1.0, -127), np.ldexp(1.0, -140)]])
    xd = torch.from_numpy(x).cuda()
    f_op, f_hw, d_op, d_hw = [t.cpu().numpy() for t in dg.check_conversions(xd)]
    normal = np.abs(x) >= np.ldexp(1.0, -126)
    assert np.array_equal(f_op[normal].view(np.uint32), f_hw[normal].view(np.uint32))
    assert np.all(f_op[~normal] == 0.0)
    assert np.array_equal(d_op.view(np.uint64), d_hw.view(np.uint64))
    # the narrowing is a faithful rounding: within half an FP32 ulp
    rel = np.abs(f_op[normal].astype(np.float64) - x[normal]) / np.abs(x[normal])
    assert rel.max() <= 2.0 ** -24


def test_fp32_sutherland_vs_oracle(orc, dg):
    N = 5
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=41)
    kw = dict(mu=0.03, visc_law=1, T_ref=1.0, S_suth=0.4)
    o = orc.Oracle(mesh, N, **kw)
    s = dg.Solver(mesh, N, precision=dg.FP32OP, **kw)
    U = random_state(mesh.n_elems, N, seed=42)
    ref = o.time_derivative(U).reshape(mesh.n_elems, 5, -1)
    got = s.time_derivative(torch.from_numpy(U).cuda()).cpu().numpy().reshape(mesh.n_elems, 5, -1)
    for v in range(5):
        assert np.abs(got[:, v] - ref[:, v]).max() / np.abs(ref[:, v]).max() < 2e-5, v
