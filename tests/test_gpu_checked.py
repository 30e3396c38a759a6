"""The checked build (-DDG_BOUNDS_CHECK: every index read from a connectivity
table is bounds-checked inside the kernels; a violation would be recorded and
reported as DG_ECUDA) on one- and two-element meshes, where every face of an
element meets the element itself or its single neighbour, and on a small 2:1
mesh with mortar faces: the operator, RK
steps, diagnostics, the Gauss-node operator, the adjoint and the ensemble (its
persistent tile-table kernels) run without a report -- neither an index out of
range nor a bulk-copy wait that gave up -- and match the oracle and the normal
build.  Runs in a child
process (the checked library is loaded instead of the normal one)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, math, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle
import paper_2605_28627_gb300 as dg
from workloads import box_mesh, random_state, tgv_params
assert dg.CHECKED and dg.LIB_PATH.endswith("libdgsem_checked.so")
out = {}
for name, dims, N in (("one", (1, 1, 1), 3), ("two", (2, 1, 1), 4), ("two_rot", (1, 2, 1), 5)):
    mesh = box_mesh(1, N, deform="sinprod", rotate_seed=11 + N, dims=dims)
    U = random_state(mesh.n_elems, N, seed=N)
    o = oracle.Oracle(mesh, N, mu=0.02)
    s = dg.Solver(mesh, N, mu=0.02)
    Ud = torch.from_numpy(U).cuda()
    R = s.time_derivative(Ud).cpu().numpy()
    Ro = o.time_derivative(U)
    err_r = float(np.abs(R - Ro).max() / np.abs(Ro).max())
    G = torch.empty_like(Ud)
    s.rk_step(Ud, G, 0.0, 1e-3, 3)
    Uo = o.rk_steps(U, 0.0, 1e-3, 3)
    err_rk = float(np.abs(Ud.cpu().numpy() - Uo).max() / np.abs(Uo).max())
    I = s.integrals(Ud)
    lam = torch.from_numpy(random_state(mesh.n_elems, N, seed=50 + N)).cuda()
    vj = s.time_derivative_vjp(Ud, lam)
    lam0, counts = s.adjoint_solve(Ud, lam, 0.0, 1e-3, 3, max_snapshots=2)
    sg = dg.Solver(mesh, N, mu=0.02, nodes=dg.NODES_LG)
    Ug = torch.from_numpy(random_state(mesh.n_elems, N, seed=7, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))).cuda()
    Rg = sg.time_derivative(Ug)
    vg = sg.time_derivative_vjp(Ug, lam)               # the Gauss-node adjoint kernels
    out[name] = dict(err_r=err_r, err_rk=err_rk, finite=bool(torch.isfinite(vj).all() and torch.isfinite(lam0).all()
                     and torch.isfinite(Rg).all() and np.isfinite(I).all() and torch.isfinite(vg).all()))
# a 2:1 mesh: every mortar table entry and the mortar neighbour states checked
from workloads.mesh import refined_box_mesh
ref = np.zeros(8, dtype=bool); ref[0] = True
mesh = refined_box_mesh(2, ref, rotate_seed=5)
U = random_state(mesh.n_elems, 3, seed=12)
o = oracle.Oracle(mesh, 3, mu=0.02)
s = dg.Solver(mesh, 3, mu=0.02)
Ud = torch.from_numpy(U).cuda()
Ro = o.time_derivative(U)
err_r = float(np.abs(s.time_derivative(Ud).cpu().numpy() - Ro).max() / np.abs(Ro).max())
G = torch.empty_like(Ud)
s.rk_step(Ud, G, 0.0, 1e-3, 3)
Uo = o.rk_steps(U, 0.0, 1e-3, 3)
lam = torch.from_numpy(random_state(mesh.n_elems, 3, seed=14)).cuda()
vj = s.time_derivative_vjp(Ud, lam)                 # the mortar kernels of the adjoint
lam0, _ = s.adjoint_solve(Ud, lam, 0.0, 1e-3, 2, max_snapshots=2)
out["mortar"] = dict(err_r=err_r, err_rk=float(np.abs(Ud.cpu().numpy() - Uo).max() / np.abs(Uo).max()),
                     finite=bool(torch.isfinite(vj).all() and torch.isfinite(lam0).all()))
# the same mesh on Gauss nodes (mortar maps on the face values)
Ug = random_state(mesh.n_elems, 3, seed=13, rho=(0.95, 1.05), vel=0.2, p=(0.95, 1.05))
og = oracle.Oracle(mesh, 3, mu=0.02, nodes=1)
sg = dg.Solver(mesh, 3, mu=0.02, nodes=dg.NODES_LG)
Rgo = og.time_derivative(Ug)
vgm = sg.time_derivative_vjp(torch.from_numpy(Ug).cuda(), lam)   # mortar adjoint on the face values
out["mortar_gauss"] = dict(err_r=float(np.abs(sg.time_derivative(torch.from_numpy(Ug).cuda()).cpu().numpy() - Rgo).max()
                                       / np.abs(Rgo).max()), err_rk=0.0, finite=bool(torch.isfinite(vgm).all()))
prm = tgv_params(Ma=0.2, Re=800.0)
runs = []
for dims, N in (((1, 1, 1), 3), ((2, 1, 1), 3), ((1, 1, 2), 2)):
    mesh = box_mesh(1, 1, lo=0.0, hi=2 * math.pi, dims=dims)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"])
    runs.append((s, s.initial_state("tgv", prm["p0"])))
# the tile-table kernels, forced through the tuning cache with one block, so
# that it walks every tile of a group (a persistent loop re-arms the volume
# body's bulk-copy barriers once per tile)
import tempfile
gpu = torch.cuda.get_device_name()
cache = tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False)
cache.write("".join("%s|N=%d|fp64\t0\t1\t1\t1\n" % (gpu, N) for N in (2, 3)))
cache.close()
ens = dg.Ensemble([r[0] for r in runs], tune_cache_path=cache.name)
Us = [r[1].clone() for r in runs]
Gs = [torch.empty_like(U) for U in Us]
ens.step(Us, Gs, [0.0] * 3, [1e-3] * 3, nsteps=2)
out["ensemble_tile_tables"] = all(g["mode"] == "tile table" for g in ens.plan()["groups"])
refs = []
for s, U0 in runs:
    ref = U0.clone(); G = torch.empty_like(ref); s.rk_step(ref, G, 0.0, 1e-3, 2); refs.append(ref)
torch.cuda.synchronize()
# the single runs of these tiny FP64 meshes take the latency kernels: equal to rounding
out["ensemble_bitwise"] = all(float((a - b).abs().max() / b.abs().max()) < 1e-13 for a, b in zip(Us, refs))
print(json.dumps(out))
'''


def test_checked_build_on_one_and_two_element_meshes():
    env = dict(os.environ, DGSEM_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for name in ("one", "two", "two_rot", "mortar", "mortar_gauss"):
        assert res[name]["err_r"] < 1e-12, res
        assert res[name]["err_rk"] < 1e-10, res
        assert res[name]["finite"], res
    assert res["ensemble_bitwise"], res   # to rounding: see the child's note
    assert res["ensemble_tile_tables"], res
