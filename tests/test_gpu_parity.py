"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bars: R(U) within 1e-12 relative (per variable, scaled by max |R|), ten
LSERK4-5 steps within 1e-10 relative (||dU||_inf / ||U||_inf), geometry
within 1e-13.  Meshes are curvilinear with randomly rotated element frames
(all eight face orientations occur) and sizes that leave a ragged last block.
"""
import math

import numpy as np
import pytest

from workloads import box_mesh, mms_params, random_state, tgv_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_R = 1e-12
RTOL_RK = 1e-10


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel_err_per_var(got, ref):
    got = got.reshape(got.shape[0], 5, -1)
    ref = ref.reshape(ref.shape[0], 5, -1)
    out = []
    for v in range(5):
        scale = max(np.abs(ref[:, v]).max(), 1e-300)
        out.append(np.abs(got[:, v] - ref[:, v]).max() / scale)
    return np.array(out)


def _geo_amp(orc, N, ngeo):
    """Growth of the rounding error of the geometry with the equispaced
    sample degree: the interpolation of the samples to the LGL nodes
    amplifies rounding by kappa = max_i sum_j |V_ij| per direction, kappa^3
    in 3D (kappa^3 = 291 at ngeo = 7, 1220 at 8, 5504 at 9).  The bars below
    hold as stated up to kappa^3 = 300 and grow in proportion beyond."""
    x, _, _ = orc.basis(N)
    xe = np.linspace(-1.0, 1.0, ngeo + 1)
    V = np.array([[np.prod([(xi - xe[m]) / (xe[j] - xe[m]) for m in range(ngeo + 1) if m != j])
                   for j in range(ngeo + 1)] for xi in x])
    return max(1.0, np.abs(V).sum(1).max() ** 3 / 300.0)


def _pair(orc, dg, mesh, N, **kw):
    o = orc.Oracle(mesh, N, **kw)
    kw2 = dict(kw)
    s = dg.Solver(mesh, N, **kw2)
    return o, s


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_geometry_parity(orc, dg, N):
    mesh = box_mesh(3 if N < 5 else 2, N, deform="sinprod", rotate_seed=100 + N)
    o, s = _pair(orc, dg, mesh, N)
    X, Ja, J = o.geometry()
    Jag, Jg = s.geometry()
    Xg = s.node_coords()
    amp = _geo_amp(orc, N, N)
    np.testing.assert_allclose(Xg.cpu().numpy(), X, rtol=0, atol=1e-14 * amp)
    np.testing.assert_allclose(Jg.cpu().numpy(), J, rtol=1e-12 * amp, atol=0)
    # the curl form differentiates products X_l dX_m: rounding scales with |X| |Ja|
    scale = np.abs(Ja).max() * max(1.0, np.abs(X).max())
    assert np.abs(Jag.cpu().numpy() - Ja).max() <= 1e-12 * amp * scale


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_time_derivative_parity_random_state(orc, dg, N, flux):
    K = 3 if N <= 4 else 2
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=200 + N)
    o, s = _pair(orc, dg, mesh, N, mu=0.02, surf_flux=flux)
    U = random_state(mesh.n_elems, N, seed=300 + N)
    ref = o.time_derivative(U, t=0.0)
    got = s.time_derivative(_cuda(U)).cpu().numpy()
    err = _rel_err_per_var(got, ref)
    assert (err < RTOL_R * _geo_amp(orc, N, N)).all(), err


def latency_kernels(N, n_elems, precision=0, nodes=0):
    """Whether the library runs this context with its latency kernels (FP64,
    LGL nodes, N <= 3, at most 16384 nodes): the rule of use_latency_kernels
    in the library."""
    return precision == 0 and nodes == 0 and N <= 3 and n_elems * (N + 1) ** 3 <= 16384


@pytest.mark.parametrize("N,K", [(1, 13), (2, 9), (3, 7)])
@pytest.mark.parametrize("flux", [0, 2])
def test_time_derivative_parity_above_latency_threshold(orc, dg, N, K, flux):
    """The one-thread-per-node kernels at N <= 3: meshes just above the node
    count below which the latency kernels take over (the small meshes of the
    other tests run those), with a ragged last block."""
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=230 + N)
    assert not latency_kernels(N, mesh.n_elems)
    o, s = _pair(orc, dg, mesh, N, mu=0.02, surf_flux=flux)
    U = random_state(mesh.n_elems, N, seed=330 + N)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U, t=0.0))
    assert (err < RTOL_R).all(), err
    if flux != 0:
        return
    # ten RK steps
    dt = 2e-4
    Ud = _cuda(U)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, dt, 10)
    ref = o.rk_steps(U, 0.0, dt, 10)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < RTOL_RK


@pytest.mark.parametrize("N", [1, 2, 3])
def test_latency_kernels_sutherland_and_mms(orc, dg, N):
    """The latency kernels (small meshes) with Sutherland's law and with the
    manufactured source, R(U) and RK steps against the oracle."""
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=240 + N)
    assert latency_kernels(N, mesh.n_elems)
    kw = dict(mu=0.03, visc_law=1, T_ref=1.0, S_suth=0.4)
    o, s = _pair(orc, dg, mesh, N, **kw)
    U = random_state(mesh.n_elems, N, seed=340 + N)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < RTOL_R).all(), err
    prm = mms_params()
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o, s = _pair(orc, dg, mesh, N, **kw)
    U = o.initial_state("mms", 0.1)
    Ud = _cuda(U)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.1, 1e-3, 10)
    ref = o.rk_steps(U, 0.1, 1e-3, 10)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < RTOL_RK


@pytest.mark.parametrize("N", [2, 3, 5])
def test_time_derivative_parity_mms_source(orc, dg, N):
    prm = mms_params()
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=20260528)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o, s = _pair(orc, dg, mesh, N, **kw)
    U = o.initial_state("mms", 0.37)
    # the built-in initial state matches the oracle's
    Ug = s.initial_state("mms", 0.37)
    np.testing.assert_allclose(Ug.cpu().numpy(), U, rtol=1e-14, atol=1e-14)
    ref = o.time_derivative(U, t=0.37)
    got = s.time_derivative(_cuda(U), t=0.37).cpu().numpy()
    # R of the exact solution is a small residual of large cancelling terms:
    # scale by the size of those terms, sum_m |2 D_im| |f . Ja| / J
    assert (np.abs(got - ref) < RTOL_R * _term_scale(orc, o, U, N)[None, :, None, None, None]).all()


def _term_scale(orc, o, U, N):
    """Per variable: max_i sum_m |2 D_im| x 3 max |f(q) . Ja^d| / min J, the size
    of the individual flux-differencing terms whose sum is R."""
    _, Ja, J = o.geometry()
    _, _, D = orc.basis(N)
    Uf = U.reshape(U.shape[0], 5, -1)
    r = Uf[:, 0]
    u = Uf[:, 1:4] / r[:, None]
    p = 0.4 * (Uf[:, 4] - 0.5 * r * (u ** 2).sum(1))
    out = np.zeros(5)
    for d in range(3):
        un = np.einsum("elp,elp->ep", u, Ja[:, d])
        f = [r * un] + [Uf[:, 1 + a] * un + p * Ja[:, d, a] for a in range(3)] + [(Uf[:, 4] + p) * un]
        for v in range(5):
            out[v] = max(out[v], np.abs(f[v]).max())
    return 3 * out * 2 * np.abs(D).sum(1).max() / J.min()


def test_free_stream_on_gpu(dg):
    N = 5
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=7)
    s = dg.Solver(mesh, N, mu=0.01)
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = s.time_derivative(_cuda(U)).cpu().numpy()
    assert np.abs(R).max() < 2e-12 * N * N


def test_tgv_config1_rk_parity(orc, dg):
    """Taylor-Green vortex, 4^3 Cartesian elements, N=3, Ma 0.1, Re 1600,
    LLF + BR1 + split form, ten LSERK4-5 steps at CFL 0.9."""
    prm = tgv_params(Ma=0.1, Re=1600.0)
    N = 3
    mesh = box_mesh(4, 1, lo=0.0, hi=2 * math.pi)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    o, s = _pair(orc, dg, mesh, N, **kw)
    U0 = o.initial_state("tgv", prm["p0"])
    Ug = s.initial_state("tgv", prm["p0"])
    np.testing.assert_allclose(Ug.cpu().numpy(), U0, rtol=1e-14, atol=1e-13)
    dt = s.max_dt(Ug, cfl=0.9, dfl=0.9)
    assert 1e-4 < dt < 1.0
    ref = o.rk_steps(U0, 0.0, dt, 10)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, dt, 10)
    got = Ud.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < RTOL_RK
    # integrals agree with the oracle's
    Ig, Io = s.integrals(Ud), o.integrals(ref)
    np.testing.assert_allclose(Ig, Io, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("N", [1, 4, 7, 9])
def test_mms_curved_rk_parity(orc, dg, N):
    prm = mms_params()
    mesh = box_mesh(3 if N < 7 else 2, N, deform="sinprod", rotate_seed=20260528)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    o, s = _pair(orc, dg, mesh, N, **kw)
    U0 = o.initial_state("mms", 0.0)
    ref = o.rk_steps(U0, 0.0, 1e-3, 10)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 4)
    s.rk_step(Ud, G, 4e-3, 1e-3, 6)        # a second graph, continued clock
    got = Ud.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < RTOL_RK


def test_advance_host_matches_device_path(dg):
    prm = tgv_params(Ma=0.2, Re=800.0)
    N = 4
    mesh = box_mesh(3, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U = s.initial_state("tgv", prm["p0"])
    host = U.cpu().numpy().copy()
    G = torch.empty_like(U)
    s.rk_step(U, G, 0.0, 2e-3, 3)
    s.advance_host(host, 0.0, 2e-3, 3)
    np.testing.assert_array_equal(host, U.cpu().numpy())


def test_conservation_full_size(orc, dg):
    """48^3 elements at N=7 (the large Taylor-Green launch configuration):
    discrete conservation of R(U) for a random state and after one RK step."""
    N, K = 7, 48
    mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, mu=1.0 / 1600)
    gen = torch.Generator(device="cuda").manual_seed(5)
    U = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    r = 1.0 + 0.1 * torch.rand(s.shape[0:1] + s.shape[2:], generator=gen, device="cuda", dtype=torch.float64)
    vel = 0.3 * (torch.rand((3,) + r.shape, generator=gen, device="cuda", dtype=torch.float64) - 0.5)
    p = 50.0 + torch.rand(r.shape, generator=gen, device="cuda", dtype=torch.float64)
    U[:, 0] = r
    for a in range(3):
        U[:, 1 + a] = r * vel[a]
    U[:, 4] = p / 0.4 + 0.5 * r * (vel ** 2).sum(0)
    R = s.time_derivative(U)
    _, J = s.geometry()
    x, w, _ = orc.basis(N)
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w).reshape(-1)).cuda()
    tot = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1), J * wq)
    scale = torch.einsum("evp,ep->v", R.reshape(s.E, 5, -1).abs(), J * wq)
    assert bool((tot.abs() <= 1e-12 * scale).all()), (tot, scale)
    I0 = s.integrals(U)
    G = torch.empty_like(U)
    s.rk_step(U, G, 0.0, 1e-4, 1)
    I1 = s.integrals(U)
    assert np.abs(I1[:5] - I0[:5]).max() <= 1e-12 * np.abs(I0[:5]).max()


def test_full_size_sampled_elements_against_oracle_patch(orc, dg):
    """At the full 48^3, N=7 size, R at sampled elements equals the oracle's
    R at the centre of a periodic 5^3 patch holding the same states: the
    operator reaches two elements out (face fluxes use the neighbours' lifted
    gradients, which use their neighbours' face states)."""
    N, K = 7, 48
    L = 2 * math.pi
    mesh = box_mesh(K, 1, lo=0.0, hi=L)
    mu = 1.0 / 1600
    s = dg.Solver(mesh, N, mu=mu)
    n = N + 1
    U = random_state(mesh.n_elems, N, seed=42, vel=0.3).reshape(K, K, K, 5, n, n, n)   # [ez, ey, ex, ...]
    R = s.time_derivative(_cuda(U.reshape(s.shape))).cpu().numpy().reshape(K, K, K, 5, n, n, n)
    patch_mesh = box_mesh(5, 1, lo=0.0, hi=1.0)
    xg_all = mesh.xgeo.reshape(K, K, K, 3, 2, 2, 2)
    rng = np.random.default_rng(9)
    for _ in range(3):
        cz, cy, cx = rng.integers(0, K, size=3)
        idx = [(np.arange(5) + c - 2) % K for c in (cz, cy, cx)]
        # the patch holds the same element geometry and states as the big mesh
        xg = np.ascontiguousarray(xg_all[np.ix_(idx[0], idx[1], idx[2])].reshape(125, 3, 2, 2, 2))
        o = orc.Oracle(type(patch_mesh)(**{**patch_mesh.__dict__, "xgeo": xg}), N, mu=mu)
        Up = U[np.ix_(idx[0], idx[1], idx[2])].reshape(125, 5, n, n, n)
        Rp = o.time_derivative(Up).reshape(5, 5, 5, 5, n, n, n)
        ref, got = Rp[2, 2, 2], R[cz, cy, cx]
        for v in range(5):
            assert np.abs(got[v] - ref[v]).max() <= RTOL_R * np.abs(ref[v]).max()


@pytest.mark.parametrize("N,flux", [(3, 0), (5, 2), (7, 1)])
def test_sutherland_parity(orc, dg, N, flux):
    """Sutherland's law at each node's temperature (viscous volume and face
    fluxes, dissipation diagnostic) against the oracle."""
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=600 + N)
    kw = dict(mu=0.03, surf_flux=flux, visc_law=1, T_ref=1.0, S_suth=110.4 / 273.15)
    o, s = _pair(orc, dg, mesh, N, **kw)
    U = random_state(mesh.n_elems, N, seed=700 + N)
    err = _rel_err_per_var(s.time_derivative(_cuda(U)).cpu().numpy(), o.time_derivative(U))
    assert (err < RTOL_R * _geo_amp(orc, N, N)).all(), err
    Ig, Io = s.integrals(_cuda(U)), o.integrals(U)
    assert abs(Ig[6] - Io[6]) <= 1e-12 * abs(Io[6])


@pytest.mark.parametrize("nodes", [0, 1])
def test_rk414_parity(orc, dg, nodes):
    """Ten RK4-14 steps (fourteen stages each) on the curved MMS mesh against
    the oracle's RK4-14, on both node sets."""
    prm = mms_params()
    N = 4
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=20260528)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1, nodes=nodes)
    o = orc.Oracle(mesh, N, rk=1, **kw)
    s = dg.Solver(mesh, N, rk_scheme=dg.RK414, **kw)
    U0 = o.initial_state("mms", 0.0)
    ref = o.rk_steps(U0, 0.0, 2e-3, 10)
    Ud = _cuda(U0)
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 2e-3, 3)
    s.rk_step(Ud, G, 6e-3, 2e-3, 7)
    assert np.abs(Ud.cpu().numpy() - ref).max() / np.abs(ref).max() < RTOL_RK
    # an ensemble whose members share RK4-14 steps with it
    ens = dg.Ensemble([s])
    ens.step([Ud], [G], [0.02], [2e-3])
    ens.close()
    assert torch.isfinite(Ud).all()


def test_init_rejects_inverted_element_on_gpu(dg):
    """A mirrored element (left-handed frame) has a negative Jacobian at its
    nodes: dg_init computes the geometry on the device and refuses the mesh."""
    m = box_mesh(2, 1, rotate_seed=3)
    inv = m.xgeo.copy()
    inv[0] = inv[0][:, :, :, ::-1]
    bad = type(m)(**{**m.__dict__, "xgeo": inv})
    with pytest.raises(dg.DGError) as err:
        dg.Solver(bad, 2)
    assert err.value.status == dg.DG_EMESH and "Jacobian" in str(err.value)
    # the library is still usable afterwards
    s = dg.Solver(m, 2)
    U = s.initial_state("tgv", 10.0)
    assert torch.isfinite(U).all()
    s.close()


@pytest.mark.parametrize("N", [3, 4, 7])
def test_inviscid_entropy_conservation_on_gpu(orc, dg, N):
    """Degenerate case mu = 0 (Euler) with the two-point flux on the faces:
    the GPU operator matches the oracle and conserves entropy discretely,
    sum w J w(U) . R(U) = 0 to round-off on the curved rotated mesh; with LLF
    faces entropy is dissipated (a property that holds at any size)."""
    mesh = box_mesh(2, N, deform="sinprod", rotate_seed=17)
    gamma = 1.4
    U = random_state(mesh.n_elems, N, seed=5)
    o = orc.Oracle(mesh, N, mu=0.0, surf_flux=dg.FLUX_EC)
    s = dg.Solver(mesh, N, mu=0.0, surf_flux=dg.FLUX_EC)
    R = s.time_derivative(_cuda(U)).cpu().numpy()
    assert (_rel_err_per_var(R, o.time_derivative(U)) < RTOL_R * _geo_amp(orc, N, N)).all()
    _, w, _ = orc.basis(N)
    wq = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    _, J = s.geometry()
    J = J.cpu().numpy().reshape(mesh.n_elems, -1)
    Uf = U.reshape(mesh.n_elems, 5, -1)
    r = Uf[:, 0]
    u = Uf[:, 1:4] / r[:, None]
    p = (gamma - 1) * (Uf[:, 4] - 0.5 * r * (u ** 2).sum(1))
    ent = np.log(p * r ** -gamma)
    W = np.concatenate([((gamma - ent) / (gamma - 1) - r * (u ** 2).sum(1) / (2 * p))[:, None],
                        r[:, None] * u / p[:, None], (-r / p)[:, None]], 1)
    R = R.reshape(mesh.n_elems, 5, -1)
    prod = np.einsum("evp,evp,ep->", W, R, J * wq)
    scale = np.einsum("evp,evp,ep->", np.abs(W), np.abs(R), J * wq)
    assert abs(prod) < 1e-13 * scale, (prod, scale)
    s2 = dg.Solver(mesh, N, mu=0.0, surf_flux=dg.FLUX_LLF)
    R2 = s2.time_derivative(_cuda(U)).cpu().numpy().reshape(mesh.n_elems, 5, -1)
    assert np.einsum("evp,evp,ep->", W, R2, J * wq) < -1e-6 * scale
    s.close()
    s2.close()


def test_non_finite_state_is_reported(dg):
    """A NaN planted (on the host) in one node of the state makes the FP64
    reductions report DG_ENONFINITE instead of returning numbers; the context
    stays usable for a clean state."""
    mesh = box_mesh(2, 1, lo=0.0, hi=2 * math.pi)
    prm = tgv_params()
    s = dg.Solver(mesh, 3, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    U = s.initial_state("tgv", prm["p0"])
    ok = s.integrals(U)
    assert np.isfinite(ok).all()
    bad = U.clone()
    bad.view(-1)[bad.numel() // 3] = float("nan")
    with pytest.raises(dg.DGError) as err:
        s.integrals(bad)
    assert err.value.status == dg.DG_ENONFINITE
    with pytest.raises(dg.DGError) as err:
        s.max_dt(bad)
    assert err.value.status == dg.DG_ENONFINITE
    np.testing.assert_array_equal(s.integrals(U), ok)
    s.close()


def test_bench_workload_properties(orc, dg):
    """The headline workload's own mesh and launch configuration (16^3 curved
    elements with seeded rotated frames, N=7, FP64): free-stream preservation
    (R of a uniform flow vanishes) and discrete conservation of R for a random
    state, properties that hold at any size; and after ten LSERK4-5 steps of
    the manufactured solution the state is finite and the density stays within
    the wave's bounds 2 -+ 0.1 (to 0.01)."""
    N, K = 7, 16
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=20260528)
    s = dg.Solver(mesh, N, mu=1e-3)
    U = np.zeros(s.shape)
    r, u, p = 1.2, np.array([0.3, -0.2, 0.45]), 0.9
    U[:, 0] = r
    U[:, 1:4] = (r * u)[None, :, None, None, None]
    U[:, 4] = p / 0.4 + 0.5 * r * u @ u
    R = s.time_derivative(_cuda(U)).cpu().numpy()
    # relative to the flux-differencing terms that cancel (the bar of the
    # manufactured-solution parity test; they grow as 1/h with the mesh)
    Ja, J = (a.cpu().numpy() for a in s.geometry())
    _, _, D = orc.basis(N)
    un = np.einsum("l,edlp->edp", u, Ja)
    fmax = max(np.abs(r * un).max(), np.abs(r * u[0] * un + p * Ja[:, :, 0]).max(),
               np.abs(r * u[1] * un + p * Ja[:, :, 1]).max(), np.abs(r * u[2] * un + p * Ja[:, :, 2]).max(),
               np.abs((U[0, 4, 0, 0, 0] + p) * un).max())
    term = 3 * fmax * 2 * np.abs(D).sum(1).max() / J.min()
    assert np.abs(R).max() < RTOL_R * term, (np.abs(R).max(), term)
    Ur = random_state(mesh.n_elems, N, seed=77)
    R = s.time_derivative(_cuda(Ur)).reshape(s.E, 5, -1)
    _, J = s.geometry()
    _, w, _ = orc.basis(N)
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w).reshape(-1)).cuda()
    tot = torch.einsum("evp,ep->v", R, J * wq)
    scale = torch.einsum("evp,ep->v", R.abs(), J * wq)
    assert bool((tot.abs() <= 1e-12 * scale).all()), (tot, scale)
    s.close()
    prm = mms_params()
    sm = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS)
    Um = sm.initial_state("mms", 0.0)
    G = torch.empty_like(Um)
    sm.rk_step(Um, G, 0.0, 1e-3, 10)
    rho = Um[:, 0]
    assert bool(torch.isfinite(Um).all()) and float(rho.min()) > 1.89 and float(rho.max()) < 2.11
    sm.close()


@pytest.mark.parametrize("N", [2, 5])
def test_max_dt_matches_the_stated_formula(orc, dg, N):
    """dg_max_dt on LGL nodes against the step it states (Sec. 3.1, CFL and
    viscous limits): dt = min(cfl h / max sum_d lambda_d, dfl h^2 / max
    mu_eff sum_d |Ja^d|^2 / J^2), h = 2/(2N+1), lambda_d = (|u . Ja^d| +
    c |Ja^d|)/J, mu_eff = max(4/3, gamma/Pr) mu / rho, evaluated here from the
    oracle's geometry and the state; both limits take their turn."""
    gamma, Pr, mu = 1.4, 0.72, 0.05
    mesh = box_mesh(3, N, deform="sinprod", rotate_seed=41)
    o, s = _pair(orc, dg, mesh, N, gamma=gamma, Pr=Pr, mu=mu)
    U = random_state(mesh.n_elems, N, seed=8)
    _, Ja, J = o.geometry()
    q = U.reshape(mesh.n_elems, 5, -1)
    rho = q[:, 0]
    u = q[:, 1:4] / rho[:, None]
    p = (gamma - 1) * (q[:, 4] - 0.5 * rho * (u ** 2).sum(1))
    c = np.sqrt(gamma * p / rho)
    lam = sum((np.abs(np.einsum("elp,elp->ep", u, Ja[:, d])) + c * np.linalg.norm(Ja[:, d], axis=1)) / J
              for d in range(3))
    visc = max(4.0 / 3.0, gamma / Pr) * mu / rho * sum((Ja[:, d] ** 2).sum(1) for d in range(3)) / J ** 2
    h = 2.0 / (2 * N + 1)
    Ud = _cuda(U)
    limits = set()
    for cfl, dfl in ((0.9, 5.0), (0.9, 1e-3)):
        conv, vis = cfl * h / lam.max(), dfl * h * h / visc.max()
        limits.add(conv < vis)
        ref = min(conv, vis)
        got = s.max_dt(Ud, cfl=cfl, dfl=dfl)
        assert abs(got - ref) <= 1e-11 * ref, (got, ref)
    assert limits == {True, False}
    s.close()


@pytest.mark.parametrize("N", [2, 3, 4, 7])
def test_state_at_an_odd_offset_gives_the_same_result(dg, N):
    """The volume kernel stages each element's state by a bulk copy, which
    needs 16-byte aligned addresses: a caller's state that starts 8 bytes off
    (a view one double into a buffer) goes through the unaligned head and tail
    path, and R(U) and RK steps equal those of an aligned copy bit for bit.
    Odd (N+1)^3 (N = 2, 4) also puts every other element at an odd offset.
    Meshes above the latency-kernel size (those have no bulk copies)."""
    K = 10 if N <= 3 else (6 if N <= 4 else 3)
    mesh = box_mesh(K, N, deform="sinprod", rotate_seed=50 + N)
    s = dg.Solver(mesh, N, mu=0.02)
    U = _cuda(random_state(mesh.n_elems, N, seed=90 + N))
    buf = torch.zeros(U.numel() + 1, dtype=torch.float64, device="cuda")
    V = buf[1:].view(U.shape)
    V.copy_(U)
    assert V.data_ptr() % 16 == 8
    assert torch.equal(s.time_derivative(V), s.time_derivative(U))
    G1, G2 = torch.empty_like(U), torch.zeros_like(buf)[1:].view(U.shape)
    s.rk_step(U, G1, 0.0, 1e-4, 2)
    s.rk_step(V, G2, 0.0, 1e-4, 2)
    assert torch.equal(U, V)
