"""Batched ensemble: every member advanced by the tile-table kernels against
the oracle's LSERK4-5 steps at the FP64 bar, and against the single-context
path bit for bit (the ensemble kernels run the same per-element arithmetic;
small FP64 runs alone take the latency kernels, which agree to rounding)."""
import math
import os

import numpy as np
import pytest

from workloads import box_mesh, tgv_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MEMBERS = [dict(K=2, N=2, Ma=0.1, Re=400.0), dict(K=3, N=3, Ma=0.3, Re=1600.0), dict(K=2, N=3, Ma=0.5, Re=800.0),
           dict(K=2, N=5, Ma=0.2, Re=1000.0), dict(K=1, N=7, Ma=0.4, Re=600.0), dict(K=3, N=1, Ma=0.2, Re=900.0)]


@pytest.fixture(scope="module")
def dg():
    import paper_2605_28627_gb300 as m
    m.load()
    return m


def _make(dg, spec, precision):
    prm = tgv_params(Ma=spec["Ma"], Re=spec["Re"])
    mesh = box_mesh(spec["K"], 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, spec["N"], gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], precision=precision)
    U = s.initial_state("tgv", prm["p0"])
    dt = s.max_dt(U, cfl=0.9, dfl=0.9)
    return s, U, dt


@pytest.mark.parametrize("choice,grid,rk", [(0, 3, 0), (1, 5, 0), (0, 3, 1)])
def test_ensemble_tile_tables_vs_oracle(orc, dg, tmp_path, choice, grid, rk):
    """FP64 members of mixed N (1, 2, 3, 5, 7) on small meshes, advanced three
    steps by the persistent tile-table kernels -- forced through the tuning
    cache: the default (choice 0) or doubled (choice 1) element tile and a
    grid of a few blocks, so that every block walks many tiles of several
    members -- against the oracle's steps of each member (LSERK4-5, or RK4-14
    for all members): max |U - U_oracle| / max |U_oracle| <= 1e-10."""
    gpu = torch.cuda.get_device_name()
    Ns = sorted({m["N"] for m in MEMBERS})
    (tmp_path / "tune.txt").write_text("".join("%s|N=%d|fp64\t%d\t%d\t%d\t%d\n" % (gpu, N, choice, grid, grid, grid)
                                                for N in Ns))
    runs, orcs, U0s = [], [], []
    for m in MEMBERS:
        prm = tgv_params(Ma=m["Ma"], Re=m["Re"])
        mesh = box_mesh(m["K"], 1, lo=0.0, hi=2 * math.pi, rotate_seed=m["K"] + m["N"])
        kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
        o = orc.Oracle(mesh, m["N"], rk=rk, **kw)
        U0 = o.initial_state("tgv", prm["p0"])
        s = dg.Solver(mesh, m["N"], rk_scheme=rk, **kw)
        dt = s.max_dt(torch.from_numpy(U0).cuda(), cfl=0.9, dfl=0.9)
        runs.append((s, dt))
        orcs.append(o)
        U0s.append(U0)
    ens = dg.Ensemble([r[0] for r in runs], tune_cache_path=str(tmp_path / "tune.txt"))
    Us = [torch.from_numpy(U0).cuda() for U0 in U0s]
    Gs = [torch.empty_like(U) for U in Us]
    t0 = [0.02 * i for i in range(len(runs))]
    dts = [r[1] for r in runs]
    ens.step(Us, Gs, t0, dts, nsteps=3)
    torch.cuda.synchronize()
    plan = ens.plan()
    assert len(plan["groups"]) == len(Ns)
    for g in plan["groups"]:
        assert g["mode"] == "tile table" and g["cached"], g
        assert 1 <= g["volume_grid"] <= grid and g["element_tiles"] >= g["volume_grid"]
    for o, U0, U, t, dt in zip(orcs, U0s, Us, t0, dts):
        ref = o.rk_steps(U0, t, dt, 3)
        err = np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-10, (o.N, err)
    ens.close()
    for r in runs:
        r[0].close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ensemble_matches_single_runs_bitwise(dg, tmp_path, precision):
    runs = [_make(dg, m, precision) for m in MEMBERS]
    cache = str(tmp_path / "tune.txt")
    ens = dg.Ensemble([r[0] for r in runs], tune_cache_path=cache)
    Us = [r[1].clone() for r in runs]
    Gs = [torch.empty_like(U) for U in Us]
    t0 = [0.01 * i for i in range(len(runs))]
    dts = [r[2] for r in runs]
    ens.step(Us, Gs, t0, dts, nsteps=2)
    ens.step(Us, Gs, [t + 2 * d for t, d in zip(t0, dts)], dts, nsteps=1)
    torch.cuda.synchronize()
    for (s, U0, dt), U, t in zip(runs, Us, t0):
        ref = U0.clone()
        G = torch.empty_like(ref)
        s.rk_step(ref, G, t, dt, 3)
        torch.cuda.synchronize()
        if precision == 0 and s.N <= 3 and s.E * s.P <= 16384:
            # a small FP64 run alone takes the latency kernels, whose sums are
            # grouped by direction: the same to rounding, not bit for bit
            assert ((U - ref).abs().max() / ref.abs().max()).item() < 1e-13
        else:
            assert torch.equal(U, ref)
    plan = ens.plan()
    assert plan is not None and len(plan["groups"]) == len({m["N"] for m in MEMBERS})
    assert os.path.exists(cache)
    ens.close()
    # a second ensemble reads the tuned plan from the cache
    ens2 = dg.Ensemble([r[0] for r in runs], tune_cache_path=cache)
    ens2.step(Us, Gs, t0, dts, nsteps=1)
    assert all(g["cached"] for g in ens2.plan()["groups"])
    ens2.close()
    for r in runs:
        r[0].close()


def test_damaged_tuning_cache_is_retuned(dg, tmp_path):
    """Cache lines no tuning run writes (an unknown tile choice, a zero grid)
    are ignored: those groups are tuned again and the results do not change."""
    runs = [_make(dg, m, 0) for m in MEMBERS[:3]]     # N = 2 and N = 3
    cache = tmp_path / "tune.txt"
    dts = [r[2] for r in runs]
    t0 = [0.0] * len(runs)
    ens = dg.Ensemble([r[0] for r in runs], tune_cache_path=str(cache))
    Us = [r[1].clone() for r in runs]
    Gs = [torch.empty_like(U) for U in Us]
    ens.step(Us, Gs, t0, dts, nsteps=1)
    ens.close()
    lines = cache.read_text().splitlines()
    assert len(lines) == 2
    damaged = []
    for i, line in enumerate(lines):
        f = line.split("\t")
        if i == 0:
            f[1] = "7"
        else:
            f[1], f[2] = "0", "0"
        damaged.append("\t".join(f))
    cache.write_text("\n".join(damaged) + "\n")
    ens2 = dg.Ensemble([r[0] for r in runs], tune_cache_path=str(cache))
    Us2 = [r[1].clone() for r in runs]
    Gs2 = [torch.empty_like(U) for U in Us2]
    ens2.step(Us2, Gs2, t0, dts, nsteps=1)
    torch.cuda.synchronize()
    assert not any(g["cached"] for g in ens2.plan()["groups"])
    ens2.close()
    for U, U2 in zip(Us, Us2):
        assert torch.equal(U, U2)
    for r in runs:
        r[0].close()


def test_repeated_members_and_states_are_rejected(dg):
    runs = [_make(dg, m, 0) for m in MEMBERS[:2]]
    with pytest.raises(dg.DGError):
        dg.Ensemble([runs[0][0], runs[1][0], runs[0][0]])
    ens = dg.Ensemble([r[0] for r in runs])
    Us = [r[1].clone() for r in runs]
    Gs = [torch.empty_like(U) for U in Us]
    dts = [r[2] for r in runs]
    before = [U.clone() for U in Us]
    with pytest.raises(dg.DGError):            # a member's register is its own state
        ens.step(Us, [Us[0], Gs[1]], [0.0, 0.0], dts, nsteps=1)
    torch.cuda.synchronize()
    assert all(torch.equal(U, B) for U, B in zip(Us, before))
    ens.step(Us, Gs, [0.0, 0.0], dts, nsteps=1)     # the ensemble stays usable
    ens.close()
    for r in runs:
        r[0].close()


def test_mixed_time_schemes_are_rejected(dg):
    m = MEMBERS[0]
    prm = tgv_params(Ma=m["Ma"], Re=m["Re"])
    mesh = box_mesh(m["K"], 1, lo=0.0, hi=2 * math.pi)
    kw = dict(gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    a = dg.Solver(mesh, m["N"], rk_scheme=dg.RK45, **kw)
    b = dg.Solver(mesh, m["N"], rk_scheme=dg.RK414, **kw)
    with pytest.raises(dg.DGError):
        dg.Ensemble([a, b])
    dg.Ensemble([b]).close()      # one scheme, RK4-14: accepted


def test_members_outside_the_tile_tables_run_as_single_units(orc, dg):
    """An ensemble of a conforming LGL member, a Gauss-node member, a 2:1
    mortar mesh and a member with FV elements (mask set before creation):
    the last three run as single-member units of the graph; every member
    matches the oracle after three steps (1e-10)."""
    from workloads import random_state
    from workloads.mesh import refined_box_mesh
    ref2 = np.zeros(8, dtype=bool)
    ref2[0] = True
    specs = [dict(mesh=box_mesh(3, 1, rotate_seed=1), N=3, kw={}),
             dict(mesh=box_mesh(3, 1, rotate_seed=2), N=3, kw=dict(nodes=1)),
             dict(mesh=refined_box_mesh(2, ref2, rotate_seed=3), N=2, kw={}),
             dict(mesh=box_mesh(2, 1, rotate_seed=4), N=4, kw={}, fv=True)]
    runs, orcs, U0s = [], [], []
    for i, sp in enumerate(specs):
        o = orc.Oracle(sp["mesh"], sp["N"], mu=0.01, **sp["kw"])
        s = dg.Solver(sp["mesh"], sp["N"], mu=0.01, **sp["kw"])
        if sp.get("fv"):
            mask = (np.arange(sp["mesh"].n_elems) % 2).astype(np.int32)
            o.set_fv_mask(mask)
            s.set_fv_mask(mask)
        U0s.append(random_state(sp["mesh"].n_elems, sp["N"], seed=20 + i, rho=(0.95, 1.05), vel=0.2,
                                p=(0.95, 1.05)))
        runs.append(s)
        orcs.append(o)
    ens = dg.Ensemble(runs)
    Us = [torch.from_numpy(U).cuda() for U in U0s]
    Gs = [torch.empty_like(U) for U in Us]
    ens.step(Us, Gs, [0.0] * 4, [1e-3] * 4, nsteps=3)
    torch.cuda.synchronize()
    modes = [g["mode"] for g in ens.plan()["groups"]]
    assert sum(m.startswith("per-member launches (Gauss") for m in modes) >= 2, modes
    for o, U0, U in zip(orcs, U0s, Us):
        ref = o.rk_steps(U0, 0.0, 1e-3, 3)
        err = np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-10, (o.N, err)
    ens.close()
