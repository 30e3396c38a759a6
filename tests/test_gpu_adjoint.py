"""Discrete adjoint: dot-product tests against the oracle's tangent-linear
(forward-mode dual numbers, an independent derivative of the oracle's R),
checkpointing invariance, and central finite differences through autograd."""
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,flux,law", [(2, 0, 0), (3, 0, 0), (3, 1, 0), (5, 0, 0), (3, 0, 1), (5, 1, 1),
                                        (3, 2, 0), (4, 2, 1)])
def test_vjp_dot_product_vs_oracle_tangent_linear(orc, dg, N, flux, law):
    """<(dR/dU)^T v, w> against <v, (dR/dU) w> of the oracle's tangent-linear,
    and v . dR/dmu; flux 2: Roe with the Harten-Hyman fix (differentiated on
    dual numbers, kinks by the value as in the oracle); law 1: Sutherland's
    viscosity (mu(T), T_ref 1, S 0.4), whose T-derivative enters through the
    state."""
    mesh = box_mesh(3 if N < 5 else 2, N, deform="sinprod", rotate_seed=600 + N)
    mu = 0.03
    kw = dict(mu=mu, surf_flux=flux, visc_law=law, T_ref=1.0, S_suth=0.4)
    o = orc.Oracle(mesh, N, **kw)
    s = dg.Solver(mesh, N, **kw)
    U = random_state(mesh.n_elems, N, seed=700 + N)
    rng = np.random.default_rng(800 + N)
    w = rng.normal(size=U.shape)
    v = rng.normal(size=U.shape)
    _, Jw = o.time_derivative_tl(U, w, 0.0)        # J w
    _, Rmu = o.time_derivative_tl(U, np.zeros_like(U), 1.0)   # dR/dmu
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    JTv = s.time_derivative_vjp(_cuda(U), _cuda(v), dJdmu=dmu).cpu().numpy()
    lhs, rhs = float((JTv * w).sum()), float((v * Jw).sum())
    scale = float(np.abs(JTv * w).sum())
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs)
    ref_mu = float((v * Rmu).sum())
    assert abs(dmu.item() - ref_mu) <= 1e-11 * float(np.abs(v * Rmu).sum()), (dmu.item(), ref_mu)


_GAUSS_STATE = dict(rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))


@pytest.mark.parametrize("N,flux,law", [(1, 0, 0), (2, 0, 0), (3, 0, 0), (3, 1, 0), (3, 2, 1), (4, 0, 1),
                                        (5, 1, 1), (7, 0, 0), (9, 2, 0)])
def test_vjp_gauss_nodes_vs_oracle_tangent_linear(orc, dg, N, flux, law):
    """Legendre-Gauss nodes (the weak form of Eqs. 2 and 3): the transposes of
    the face prolongation of the state and of the gradients, of the weak
    lifting and of the weak volume and surface terms, in the dot-product test
    against the oracle's tangent-linear of its Gauss-node operator."""
    mesh = box_mesh(3 if N < 5 else 2, N, deform="sinprod", rotate_seed=950 + N)
    kw = dict(mu=0.03, surf_flux=flux, visc_law=law, T_ref=1.0, S_suth=0.4)
    o = orc.Oracle(mesh, N, nodes=1, **kw)
    s = dg.Solver(mesh, N, nodes=dg.NODES_LG, **kw)
    U = random_state(mesh.n_elems, N, seed=960 + N, **_GAUSS_STATE)
    rng = np.random.default_rng(970 + N)
    w = rng.normal(size=U.shape)
    v = rng.normal(size=U.shape)
    _, Jw = o.time_derivative_tl(U, w, 0.0)
    _, Rmu = o.time_derivative_tl(U, np.zeros_like(U), 1.0)
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    JTv = s.time_derivative_vjp(_cuda(U), _cuda(v), dJdmu=dmu).cpu().numpy()
    lhs, rhs = float((JTv * w).sum()), float((v * Jw).sum())
    scale = float(np.abs(JTv * w).sum())
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs)
    ref_mu = float((v * Rmu).sum())
    assert abs(dmu.item() - ref_mu) <= 1e-11 * float(np.abs(v * Rmu).sum()), (dmu.item(), ref_mu)


def test_vjp_gauss_nodes_per_element(orc, dg):
    """Element by element on a small curved mesh: (dR/dU)^T v against the
    oracle's tangent-linear with directions supported on one element each
    (a dot product over the whole mesh could hide errors that cancel)."""
    N = 3
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=980)
    o = orc.Oracle(mesh, N, nodes=1, mu=0.03)
    s = dg.Solver(mesh, N, nodes=dg.NODES_LG, mu=0.03)
    U = random_state(mesh.n_elems, N, seed=981, **_GAUSS_STATE)
    rng = np.random.default_rng(982)
    v = rng.normal(size=U.shape)
    JTv = s.time_derivative_vjp(_cuda(U), _cuda(v)).cpu().numpy()
    for e in range(mesh.n_elems):
        w = np.zeros(U.shape)
        w[e] = rng.normal(size=U.shape[1:])
        _, Jw = o.time_derivative_tl(U, w, 0.0)
        lhs, rhs = float((JTv * w).sum()), float((v * Jw).sum())
        assert abs(lhs - rhs) <= 1e-11 * float(np.abs(JTv * w).sum()), (e, lhs, rhs)


def test_solve_adjoint_gauss_nodes_vs_oracle(orc, dg):
    """Adjoint of LSERK4-5 steps on Gauss nodes against the oracle's
    tangent-linear of the same steps, with d/dmu."""
    N = 3
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=990)
    o = orc.Oracle(mesh, N, nodes=1, mu=0.02)
    s = dg.Solver(mesh, N, nodes=dg.NODES_LG, mu=0.02)
    U0 = random_state(mesh.n_elems, N, seed=991, **_GAUSS_STATE)
    dt, nsteps = 2e-3, 4
    rng = np.random.default_rng(992)
    w = rng.normal(size=U0.shape)
    lam = rng.normal(size=U0.shape)
    _, dUT = o.rk_steps_tl(U0, w, 0.3, 0.0, dt, nsteps)
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam0, _ = s.adjoint_solve(_cuda(U0), _cuda(lam), 0.0, dt, nsteps, max_snapshots=2, dJdmu=dmu)
    lhs = float((lam0.cpu().numpy() * w).sum()) + 0.3 * dmu.item()
    rhs = float((lam * dUT).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)


def _mortar_mesh(N, seed):
    from workloads.mesh import refined_box_mesh
    K = 3 if N <= 7 else 2
    r = np.zeros(K ** 3, dtype=bool)
    r[[0, 13] if K == 3 else [0, 7]] = True
    return refined_box_mesh(K, r, rotate_seed=seed)


@pytest.mark.parametrize("N,flux,law,nodes", [(1, 0, 0, 0), (2, 0, 0, 0), (3, 1, 0, 0), (3, 2, 1, 0), (4, 0, 1, 0),
                                              (5, 1, 0, 0), (7, 0, 0, 0), (9, 2, 0, 0),
                                              (1, 0, 0, 1), (2, 1, 1, 1), (3, 0, 0, 1), (5, 2, 0, 1), (8, 0, 1, 1)])
def test_vjp_on_mortar_mesh_vs_oracle_tangent_linear(orc, dg, N, flux, law, nodes):
    """2:1 non-conforming meshes (Sec. 3.2.2, Algorithm 1): the transposes of
    the quadrant interpolation, of the flux projection and of the mortar
    sides' lifting states, in the same dot-product test; on Gauss nodes
    (nodes 1) the maps act on the face values."""
    mesh = _mortar_mesh(N, 900 + N)
    kw = dict(mu=0.03, surf_flux=flux, visc_law=law, T_ref=1.0, S_suth=0.4)
    o = orc.Oracle(mesh, N, nodes=nodes, **kw)
    s = dg.Solver(mesh, N, nodes=nodes, **kw)
    U = random_state(mesh.n_elems, N, seed=910 + N, **(_GAUSS_STATE if nodes else {}))
    rng = np.random.default_rng(920 + N)
    w = rng.normal(size=U.shape)
    v = rng.normal(size=U.shape)
    _, Jw = o.time_derivative_tl(U, w, 0.0)
    _, Rmu = o.time_derivative_tl(U, np.zeros_like(U), 1.0)
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    JTv = s.time_derivative_vjp(_cuda(U), _cuda(v), dJdmu=dmu).cpu().numpy()
    lhs, rhs = float((JTv * w).sum()), float((v * Jw).sum())
    scale = float(np.abs(JTv * w).sum())
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs)
    ref_mu = float((v * Rmu).sum())
    assert abs(dmu.item() - ref_mu) <= 1e-11 * float(np.abs(v * Rmu).sum()), (dmu.item(), ref_mu)


def test_vjp_on_mortar_mesh_per_entry(orc, dg):
    """Column by column on a small mortar mesh: (dR/dU)^T e_i against the
    oracle's tangent-linear rows, for seeds on the big face's and the small
    faces' nodes (a dot product alone could hide two errors that cancel)."""
    N = 2
    mesh = _mortar_mesh(N, 930)
    o = orc.Oracle(mesh, N, mu=0.03)
    s = dg.Solver(mesh, N, mu=0.03)
    U = random_state(mesh.n_elems, N, seed=931)
    rng = np.random.default_rng(932)
    n = N + 1
    # the refined cell 0's children and its neighbours through the mortars
    big = np.unique(mesh.mortars[:, 0])[:2]
    small = np.unique(mesh.mortars[:, 2])[:2]
    picks = [(int(e), c, int(rng.integers(0, n ** 3))) for e in list(big) + list(small) for c in (0, 4)]
    lam = np.zeros(U.shape)
    for e, c, node in picks:
        lam.reshape(mesh.n_elems, 5, -1)[e, c, node] = rng.normal()
    JTv = s.time_derivative_vjp(_cuda(U), _cuda(lam)).cpu().numpy()
    for trial in range(6):
        w = np.zeros(U.shape)
        e = int(rng.choice(np.concatenate([big, small])))
        w.reshape(mesh.n_elems, 5, -1)[e] = rng.normal(size=(5, n ** 3))
        _, Jw = o.time_derivative_tl(U, w, 0.0)
        lhs, rhs = float((JTv * w).sum()), float((lam * Jw).sum())
        assert abs(lhs - rhs) <= 1e-11 * max(float(np.abs(JTv * w).sum()), 1e-300), (trial, lhs, rhs)


def test_solve_adjoint_on_mortar_mesh_vs_oracle(orc, dg):
    """Adjoint of LSERK4-5 steps on a 2:1 mesh against the oracle's
    tangent-linear of the same steps, with d/dmu."""
    N = 3
    mesh = _mortar_mesh(N, 940)
    o = orc.Oracle(mesh, N, mu=0.02)
    s = dg.Solver(mesh, N, mu=0.02)
    U0 = random_state(mesh.n_elems, N, seed=941, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
    dt, nsteps = 2e-3, 4
    rng = np.random.default_rng(942)
    w = rng.normal(size=U0.shape)
    lam = rng.normal(size=U0.shape)
    _, dUT = o.rk_steps_tl(U0, w, 0.3, 0.0, dt, nsteps)
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam0, _ = s.adjoint_solve(_cuda(U0), _cuda(lam), 0.0, dt, nsteps, max_snapshots=2, dJdmu=dmu)
    lhs = float((lam0.cpu().numpy() * w).sum()) + 0.3 * dmu.item()
    rhs = float((lam * dUT).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)


@pytest.mark.parametrize("rk", [0, 1])
def test_step_and_solve_adjoint_vs_oracle(orc, dg, rk):
    """Adjoint of LSERK4-5 (rk 0) and RK4-14 (rk 1) steps against the oracle's
    tangent-linear of the same scheme."""
    prm = tgv_params(Ma=0.3, Re=400.0)
    N = 3
    mesh = box_mesh(3, 1, lo=0.0, hi=2 * math.pi, rotate_seed=5)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    o = orc.Oracle(mesh, N, rk=rk, **kw)
    s = dg.Solver(mesh, N, rk_scheme=rk, **kw)
    # a generic state near the Taylor-Green vortex: the vortex itself has w = 0
    # exactly, which puts |u . n| of the LLF speed at its kink on z-faces, where
    # the one-sided derivatives of the two codes may differ by rounding
    rng0 = np.random.default_rng(1)
    U0 = o.initial_state("tgv", prm["p0"]) * (1 + 0.01 * rng0.normal(size=(mesh.n_elems, 5, 4, 4, 4)))
    U0[:, 1:4] += 0.01 * rng0.normal(size=(mesh.n_elems, 3, 4, 4, 4))
    dt, nsteps = 0.02, 6
    rng = np.random.default_rng(2)
    w = rng.normal(size=U0.shape)
    lam = rng.normal(size=U0.shape)
    _, dUT = o.rk_steps_tl(U0, w, 0.4, 0.0, dt, nsteps)       # tangent of U_T for dU0 = w, dmu = 0.4
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam0, counts = s.adjoint_solve(_cuda(U0), _cuda(lam), 0.0, dt, nsteps, max_snapshots=3, dJdmu=dmu)
    lhs = float((lam0.cpu().numpy() * w).sum()) + 0.4 * dmu.item()
    rhs = float((lam * dUT).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)
    assert counts == dg.checkpoint_schedule(nsteps, 3) and counts[1] == nsteps
    # checkpointing does not change the result: all snapshots vs few vs one
    ref = None
    for snaps in (nsteps, 2, 1):
        dm = torch.zeros(1, dtype=torch.float64, device="cuda")
        l0, cnt = s.adjoint_solve(_cuda(U0), _cuda(lam), 0.0, dt, nsteps, max_snapshots=snaps, dJdmu=dm)
        assert cnt == dg.checkpoint_schedule(nsteps, snaps)
        cur = (l0.cpu().numpy(), dm.item())
        if ref is None:
            ref = cur
        else:
            np.testing.assert_array_equal(cur[0], ref[0])
            assert cur[1] == ref[1]
    np.testing.assert_array_equal(ref[0], lam0.cpu().numpy())


def test_autograd_gradient_vs_central_differences(dg):
    from paper_2605_28627_gb300.autograd import kinetic_energy, rk_solve
    prm = tgv_params(Ma=0.2, Re=800.0)
    N = 3
    mesh = box_mesh(3, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U0 = s.initial_state("tgv", prm["p0"])
    dt = s.max_dt(U0)
    nsteps = 20
    Ul = U0.clone().requires_grad_(True)
    mu = torch.tensor(prm["mu"], dtype=torch.float64, requires_grad=True)
    J = kinetic_energy(rk_solve(Ul, mu, s, 0.0, dt, nsteps, max_snapshots=4), s)
    J.backward()
    gU, gmu = Ul.grad.clone(), mu.grad.item()

    def Jof(U, m):
        with torch.no_grad():
            return kinetic_energy(rk_solve(U, torch.tensor(m, dtype=torch.float64), s, 0.0, dt, nsteps), s).item()

    gen = torch.Generator(device="cuda").manual_seed(3)
    # The vortex has symmetry planes on element faces, where the LLF speed
    # max(|u.n| + c) sits at its kinks; the adjoint takes the mean one-sided
    # derivative there, which is what central differences see.
    h = 1e-6 * U0.abs().max().item()
    gnorm = gU.norm().item()
    ghat = gU / gnorm
    # Four seeded random unit directions, whose directional derivatives are
    # typically ~1e-2 |g| or less (8640 unknowns), and four directions mixed
    # with the gradient so that |g.v| >= 1e-2 |g| for certain.  Every
    # direction with |g.v| >= 1e-2 |g| is held to the 1e-6 relative bar; the
    # others (where g.v is a difference of large cancelling terms) to
    # 1e-6 max(|g.v|, 1e-3 |g|), i.e. at most 1e-9 |g| absolute.
    dirs = []
    for _ in range(4):
        v = torch.randn(U0.shape, generator=gen, device="cuda", dtype=torch.float64)
        dirs.append(v / v.norm())
    for a in (0.05, 0.2, 0.5, 1.0):
        r = torch.randn(U0.shape, generator=gen, device="cuda", dtype=torch.float64)
        v = a * ghat + (1.0 - a) * r / r.norm()
        dirs.append(v / v.norm())
    strict = 0
    for v in dirs:
        fd = (Jof(U0 + h * v, prm["mu"]) - Jof(U0 - h * v, prm["mu"])) / (2 * h)
        ad = float((gU * v).sum())
        if abs(ad) >= 1e-2 * gnorm:
            strict += 1
            assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad, gnorm)
        else:
            assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-3 * gnorm), (fd, ad, gnorm)
    assert strict >= 4
    hm = 1e-7
    fd = (Jof(U0, prm["mu"] + hm) - Jof(U0, prm["mu"] - hm)) / (2 * hm)
    assert abs(fd - gmu) <= 1e-6 * abs(gmu), (fd, gmu)


def test_autograd_two_solves_with_different_viscosity(dg):
    """Two rk_solve calls on one solver with different mu in one graph: the
    second forward call changes the solver's mu before the first backward,
    which must still run its adjoint (and its forward recomputation) with the
    mu of its own forward call.  The gradients then equal those of the two
    calls taken one at a time, bit for bit, and the solver's mu is left as the
    last forward call set it."""
    from paper_2605_28627_gb300.autograd import kinetic_energy, rk_solve
    prm = tgv_params(Ma=0.2, Re=800.0)
    N = 3
    mesh = box_mesh(2, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U0 = s.initial_state("tgv", prm["p0"])
    dt = s.max_dt(U0)
    nsteps = 6
    mus = (prm["mu"], 8.0 * prm["mu"])
    single = []
    for m in mus:
        Ul = U0.clone().requires_grad_(True)
        mt = torch.tensor(m, dtype=torch.float64, requires_grad=True)
        kinetic_energy(rk_solve(Ul, mt, s, 0.0, dt, nsteps, max_snapshots=3), s).backward()
        single.append((Ul.grad.clone(), mt.grad.item()))
    # the viscosity matters: the two calls' gradients differ
    assert abs(single[0][1] - single[1][1]) > 1e-3 * abs(single[0][1])
    assert (single[0][0] - single[1][0]).abs().max().item() > 1e-6 * single[0][0].abs().max().item()
    Ul = U0.clone().requires_grad_(True)
    m1 = torch.tensor(mus[0], dtype=torch.float64, requires_grad=True)
    m2 = torch.tensor(mus[1], dtype=torch.float64, requires_grad=True)
    J = kinetic_energy(rk_solve(Ul, m1, s, 0.0, dt, nsteps, max_snapshots=3), s) + \
        kinetic_energy(rk_solve(Ul, m2, s, 0.0, dt, nsteps, max_snapshots=3), s)
    J.backward()
    assert m1.grad.item() == single[0][1]
    assert m2.grad.item() == single[1][1]
    assert torch.equal(Ul.grad, single[0][0] + single[1][0])
    assert s.mu == mus[1]
    s.close()


def test_adjoint_arrays_may_not_be_the_state(dg):
    prm = tgv_params(Ma=0.2, Re=800.0)
    mesh = box_mesh(2, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, 2, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U = s.initial_state("tgv", prm["p0"])
    lam = torch.ones_like(U)
    before = U.clone()
    with pytest.raises(dg.DGError):
        s.adjoint_step(U, lam, lam_n=U)
    with pytest.raises(dg.DGError):
        s.adjoint_solve(U, lam, 0.0, 1e-3, 3, lam0=U)
    torch.cuda.synchronize()
    assert torch.equal(U, before)
    lam0, counts = s.adjoint_solve(U, lam, 0.0, 1e-3, 3, max_snapshots=2)
    assert counts == dg.checkpoint_schedule(3, 2) and torch.isfinite(lam0).all()
    s.close()
