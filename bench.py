"""Throughput of the DGSEM hot path: one step = one LSERK4-5 step (five stages
of lifting, face fluxes, split-form volume integral, surface integral,
Jacobian and stage update) of the density-wave manufactured solution on the
16^3-element curvilinear mesh with randomly rotated element frames.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--order 7] [--impl reference]

Prints one JSON line (rank 0).  Metric: DOF*stage/s = (nodes x 5 stages x K)
/ time; PID = 1 / that, in ns.  `--impl reference` times the plain CPU oracle
on the same workload (one R(U) evaluation of an 8^3-element sample per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF·stage/s (1/PID) of R(U)+RK at N=3..7 on 1 GB300 vs fp64 plain; % roofline"
UNIT = "DOF*stage/s"
K_ELEMS = 16
MMS_SEED = 20260528
DT = 1e-3


def workload_name(N):
    return ("MMS density wave rho=2+0.1sin(pi(x+y+z-t)), u=(1,1,1), p=1 on [-1,1]^3, %d^3 curvilinear hexes "
            "(x_i += 0.1 prod sin(pi x_j)), seeded rotated element frames, N=%d LGL, LLF + BR1 + "
            "Chandrashekar split form, LSERK4-5, dt=1e-3" % (K_ELEMS, N))


def build_mesh(N):
    from workloads import box_mesh
    return box_mesh(K_ELEMS, N, deform="sinprod", rotate_seed=MMS_SEED)


# DRAM bytes (read + write) per launch of the volume kernel on this workload,
# the median over the launches of one ncu capture of the current kernels
# (profiles/volume_traffic_N7_mms16.txt); absent = not captured.
MEASURED_TRAFFIC = {(7, "fp64"): 670.667520e6 + 217.116672e6, (7, "fp32op"): 406.712064e6 + 143.888640e6}
# The other orders of the sweep, DRAM read + write per launch (medians, MB) from one capture of
# the volume kernels of `--sweep 1,2,3,4,5,6,8,9`; up to N = 4 the working set stays in the
# 129 MB L2 between launches, so DRAM sees less than the kernel's algorithmic bytes.
for _N, _f64, _f32 in ((1, 11.0, 7.1), (2, 34.7, 22.7), (3, 79.7, 52.3), (4, 165.9, 102.6), (5, 302.5, 203.7),
                       (6, 499.7, 344.3), (8, 1084.3, 800.5), (9, 1765.2, 1067.8)):
    MEASURED_TRAFFIC[(_N, "fp64")] = _f64 * 1e6
    MEASURED_TRAFFIC[(_N, "fp32op")] = _f32 * 1e6


# ---------------------------------------------------------------------------
# Algorithmic FP64 operation count of the volume kernel per node and stage
# (FMA = 2 flops; a divide, square root or logarithm counts as 1).  The
# two-point flux with symmetric reuse is evaluated 3(n-1)/2 times per node.
PAIR_FLOPS = 97.0                      # Chandrashekar flux + metric average + both accumulations


def volume_flops_per_dof(N):
    n = N + 1
    pair = PAIR_FLOPS
    diag = 3 * 2.0 * 5                 # D_ii terms folded into the accumulators
    visc = 20.0 + 3 * 26.0 + 12 * n * 2.0
    prim = 13.0
    surf = (6.0 / n) * 25.0
    epi = 5 * 6.0
    return 1.5 * (n - 1) * pair + diag + visc + prim + surf + epi


# Algorithmic FP64 count of the lifting kernel per node and stage: the
# primitives (a reciprocal, velocities, pressure, temperature: 14), the face
# jumps at the 6 n^2 face points of an element (the neighbour's primitives and
# four scaled differences: 22 per point, 6/n per node), the line derivatives of
# four fields in three directions (12 n FMAs), the metric products (12
# components of three terms, 5 each) and the 1/J scaling (12).
def lift_flops_per_dof(N):
    n = N + 1
    return 14.0 + 22.0 * 6.0 / n + 24.0 * n + 60.0 + 12.0


# Algorithmic FP64 count of the LLF face kernel per face point and stage: both
# sides' primitives (24), the two Euler fluxes in n (28), sound speeds and the
# wave-speed bound (19), the dissipative combination (20), the two viscous
# fluxes in n (92) and the BR1 average times sJ (17).  3 (N+1)^2 face points
# per element: 3/(N+1) per node.
FACE_POINT_FLOPS = 24.0 + 28.0 + 19.0 + 20.0 + 92.0 + 17.0


def face_flops_per_dof(N):
    return FACE_POINT_FLOPS * 3.0 / (N + 1)


def step_flops_per_dof(N):
    return lift_flops_per_dof(N) + face_flops_per_dof(N) + volume_flops_per_dof(N)


# ---------------------------------------------------------------------------
# Algorithmic DRAM bytes per node and stage of the FP32-operator volume kernel
# (HBM-bound): FP64 state U and register G read and written (160 B), FP32
# metric terms J a^d and 1/J (40 B), FP32 lifted gradients (48 B), the
# manufactured source's phases (16 B, FP64) and the six faces' FP32 fluxes
# F* (6 (N+1)^2 points x 20 B per element = 120/(N+1) B per node).
def fp32_volume_bytes_per_dof(N, mms=True):
    return 160.0 + 40.0 + 48.0 + (16.0 if mms else 0.0) + 120.0 / (N + 1)


def hbm_peak_gbs():
    """(GB/s, source): the measured copy bandwidth if the file is
    present, else the recipe's fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 copy measurement)"


def host_cpu():
    """(usable cores, CPU model) of this host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip().lower() in ("model name", "cpu model") and v.strip():
                    model = v.strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    import platform
    return cores, (model or "unknown") + " (%s)" % platform.machine()


# Algorithmic FP64 operations per node of one VJP (dR/dU)^T v in the adjoint
# volume kernel (same counting: FMA = 2, divide/log = 1), counted from the
# formulas it evaluates: per unique pair 214 (the two log means with their
# partial derivatives 2 x 35, the reverse sweep of the two-point flux 118, the
# metric average 6, the pair's two adjoint seeds 15, the partner's share 5),
# 1.5 (n-1) pairs per node; per node the primitives and reciprocals (19),
# -lambda/J (5), the viscous-flux adjoint in three directions (90 each) with
# its D^T line sums (8 n) and the primitive adjoint (25).
ADJ_PAIR_FLOPS = 214.0


def adjoint_volume_flops_per_dof(N):
    n = N + 1
    return 1.5 * (n - 1) * ADJ_PAIR_FLOPS + 19.0 + 5.0 + 3 * 90.0 + 3 * 8.0 * n + 25.0


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(N, n_evals=2):
    """The plain oracle on the same workload, single-threaded and with its
    element and face loops on all host cores (OpenMP build, bit-identical
    results): DOF*stage/s of R(U) of the whole mesh for each."""
    import oracle
    from workloads import mms_params
    prm = mms_params()
    mesh = build_mesh(N)
    dof = mesh.n_elems * (N + 1) ** 3
    cores, model = host_cpu()
    out = {}
    for name, par in (("single", False), ("all_cores", True)):
        o = oracle.Oracle(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1,
                          parallel=par)
        threads = oracle.set_threads(cores) if par else 1
        U = o.initial_state("mms", 0.0)
        reps = n_evals if not par else max(n_evals, 4)
        if par:
            o.time_derivative(U, t=0.0)                   # starts the thread pool
        t0 = time.perf_counter()
        for _ in range(reps):
            o.time_derivative(U, t=0.0)
        dt = (time.perf_counter() - t0) / reps
        out[name] = {"value": dof / dt, "threads": threads, "s_per_eval": dt, "evals": reps}
        del o
    return out, cores, model


def run_reference(args, world, rank):
    """The plain oracle on the host: each step is one R(U) of a bounded
    sample of the workload -- the same mesh family (deformation, seeded
    rotations, MMS state, N) at 8^3 elements -- on all host cores (its
    element and face loops split by OpenMP, bit-identical to the serial
    oracle), so that K steps stay within a few minutes; DOF*stage/s does not
    depend on the mesh size.  The single-threaded rate of the same sample is
    reported beside it."""
    if rank != 0:
        return 0
    N = args.order
    import oracle
    from workloads import box_mesh, mms_params
    prm = mms_params()
    mesh = box_mesh(8, N, deform="sinprod", rotate_seed=MMS_SEED)
    dof = mesh.n_elems * (N + 1) ** 3
    cores, model = host_cpu()
    rates = {}
    for name, par in (("all_cores", True), ("single", False)):
        o = oracle.Oracle(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1,
                          parallel=par)
        threads = oracle.set_threads(cores) if par else 1
        U = o.initial_state("mms", 0.0)
        steps = args.steps if par else max(2, args.steps // 10)
        for _ in range(args.warmup if par else 1):
            o.time_derivative(U, t=0.0)
        t0 = time.perf_counter()
        for _ in range(steps):
            o.time_derivative(U, t=0.0)
        el = time.perf_counter() - t0
        rates[name] = (dof * steps / el, el, steps, threads)
        del o
    val, el, steps, threads = rates["all_cores"]
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(N), "elements": K_ELEMS ** 3, "N": N,
                   "dof": K_ELEMS ** 3 * (N + 1) ** 3, "sample_elements": mesh.n_elems, "pid_ns": 1e9 / val},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": model,
                         "pid_ns_times_cores": 1e9 * threads / val,
                         "single_core_value": rates["single"][0],
                         "sample": "each step = one R(U) evaluation (one RK stage) by the plain C++ oracle (-O3, "
                                   "element and face loops on %d OpenMP threads, bit-identical to the serial "
                                   "oracle) of an 8^3-element sample of the workload's mesh family (same N, "
                                   "deformation, seeded rotations and MMS state), %d nodes; single_core_value: "
                                   "the same sample single-threaded (%d evaluations)"
                                   % (threads, dof, rates["single"][2])},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def tgv_large(nsteps, local):
    """Large Taylor-Green vortex: 48^3 Cartesian elements, N=7 (56.6 M nodes),
    Ma 0.1, Re 1600, LSERK4-5 at CFL 0.9 (dt from the initial state), run once
    with the FP64 operator and twice with the FP32 operator (without and with
    the background pressure p0 taken out of the momentum flux).  Reports PID
    of each and the error of the kinetic-energy dissipation rate
    eps = -dE_k/dt (central differences of the per-step E_k):
    max_t |eps_32 - eps_64| / max_t |eps_64|."""
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import box_mesh, tgv_params
    K, N = 48, 7
    prm = tgv_params(Ma=0.1, Re=1600.0)
    mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
    dofs = mesh.n_elems * (N + 1) ** 3
    out, hist, dt = {}, {}, None
    runs = (("fp64", dg.FP64, 0.0), ("fp32op", dg.FP32OP, 0.0), ("fp32op_pref", dg.FP32OP, prm["p0"]))
    for name, prec, p_ref in runs:
        s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], precision=prec,
                      device=local, p_ref=p_ref)
        st = torch.cuda.Stream(device="cuda:%d" % local)
        U = s.initial_state("tgv", prm["p0"], stream=st)
        G = torch.empty_like(U)
        if dt is None:
            dt = s.max_dt(U, cfl=0.9, dfl=0.9, stream=st)
        ek = [s.integrals(U, stream=st)[5]]
        ms_tot = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(nsteps):
            e0.record(st)
            s.rk_step(U, G, k * dt, dt, 1, stream=st)
            e1.record(st)
            e1.synchronize()
            # the first step also captures the step graph: not timed
            if k > 0 or nsteps == 1:
                ms_tot += e0.elapsed_time(e1)
            ek.append(s.integrals(U, stream=st)[5])
        hist[name] = np.array(ek)
        timed = max(nsteps - 1, 1)
        rate = dofs * 5 * timed / (ms_tot * 1e-3)
        out[name] = {"dof_stage_per_s": rate, "pid_ns": 1e9 / rate, "ms_per_step": ms_tot / timed,
                     "ek_final": float(ek[-1])}
        del U, G
        s.close()
        torch.cuda.empty_cache()
    eps = {k: -(v[2:] - v[:-2]) / (2 * dt) for k, v in hist.items()}
    line = {"experiment": "Taylor-Green vortex 48^3 elements, N=7, Ma 0.1, Re 1600, %d LSERK4-5 steps" % nsteps,
            "dof": dofs, "dt": dt, "p_ref_of_fp32op_pref": prm["p0"],
            "eps_fp64_first_last": [float(eps["fp64"][0]), float(eps["fp64"][-1])]}
    for name, _, _ in runs:
        line[name] = out[name]
        if name == "fp64":
            continue
        line[name]["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out[name]["ms_per_step"]
        line[name]["dissipation_rate_rel_err"] = float(np.abs(eps[name] - eps["fp64"]).max() /
                                                       np.abs(eps["fp64"]).max())
        line[name]["ek_rel_diff_final"] = abs(out[name]["ek_final"] - out["fp64"]["ek_final"]) / out["fp64"]["ek_final"]
    return line


def tgv_shock(t_end, local, every=20, thr=(-1.9, -2.4), variants=""):
    """Compressible Taylor-Green vortex of Sec. 4.2: Ma 1.25, Re 1600, 16^3
    Cartesian elements on [0, 2 pi]^3, N = 3, Sutherland viscosity (T_ref = T0,
    S = 110.4 K / 273.15 K T0), LSERK4-5 at CFL 0.9 (dt from the state every
    `every` steps), to t_end.  Variants: Gauss nodes with automatic DG/FV
    switching (the paper's setup), LGL split form with and without switching,
    Gauss nodes without it.  Switching on rho p, log10 thresholds thr (upper,
    lower).  Reports E_k and eps_S at
    every unit of time, the FV fraction, the time of the eps_S peak, and the
    PID of the timed RK calls (indicator and switch included); a run whose
    state becomes non-finite records the time."""
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import box_mesh, tgv_params
    K, N = 16, 3
    prm = tgv_params(Ma=1.25, Re=1600.0)
    mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
    dofs = mesh.n_elems * (N + 1) ** 3
    runs = (("gauss_fv_switch", dg.NODES_LG, True), ("lgl_split_fv_switch", dg.NODES_LGL, True),
            ("lgl_split_dg", dg.NODES_LGL, False), ("gauss_dg", dg.NODES_LG, False))
    line = {"experiment": "compressible Taylor-Green vortex, Ma 1.25, Re 1600, 16^3 elements, N=3, Sutherland, "
                          "to t=%g" % t_end, "dof": dofs, "switch": {"var": "rho p", "log10_upper": thr[0],
                                                                     "log10_lower": thr[1]}}
    for name, nodes, sw in runs:
        if variants and name not in variants.split(","):
            continue
        s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], nodes=nodes,
                      visc_law=dg.VISC_SUTHERLAND, T_ref=prm["T0"], S_suth=110.4 / 273.15 * prm["T0"],
                      device=local)
        st = torch.cuda.Stream(device="cuda:%d" % local)
        U = s.initial_state("tgv", prm["p0"], stream=st)
        G = torch.empty_like(U)
        if sw:
            s.set_fv_switch(dg.IND_RHOP, thr[0], thr[1], stream=st)
        t, steps, ms_tot, failed = 0.0, 0, 0.0, None
        hist = {"t": [], "ek": [], "eps_s": [], "fv_fraction": []}
        next_rec = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        first = True
        fv_chunks = []
        while t < t_end - 1e-12:
            try:
                if t >= next_rec - 1e-12:
                    I = s.integrals(U, stream=st)
                    hist["t"].append(round(t, 4))
                    hist["ek"].append(float(I[5]))
                    hist["eps_s"].append(float(I[6]))
                    hist["fv_fraction"].append(float(s.fv_mask(stream=st).sum().item()) / mesh.n_elems)
                    next_rec += 1.0
                dt = min(s.max_dt(U, cfl=0.9, dfl=0.9, stream=st), t_end - t)
            except dg.DGError:
                failed = t
                break
            e0.record(st)
            s.rk_step(U, G, t, dt, every, stream=st)
            e1.record(st)
            e1.synchronize()
            if not first:             # the first call captures the graph
                ms_tot += e0.elapsed_time(e1)
                steps += every
            first = False
            t += every * dt
            if sw:   # the mask of the chunk's last stage
                fv_chunks.append(float(s.fv_mask(stream=st).sum().item()) / mesh.n_elems)
        res = {"steps_timed": steps, "t_reached": round(t, 4), "nonfinite_at_t": failed}
        if fv_chunks:
            res.update({"fv_fraction_max_over_chunks": max(fv_chunks),
                        "fv_fraction_mean_over_chunks": float(np.mean(fv_chunks))})
        if steps:
            rate = dofs * 5 * steps / (ms_tot * 1e-3)
            res.update({"dof_stage_per_s": rate, "pid_ns": 1e9 / rate})
        if hist["eps_s"]:
            k = int(np.argmax(hist["eps_s"]))
            res.update({"eps_s_peak": hist["eps_s"][k], "t_eps_s_peak": hist["t"][k],
                        "fv_fraction_max": max(hist["fv_fraction"])})
        res["history"] = hist
        line[name] = res
        del U, G
        s.close()
        torch.cuda.empty_cache()
    return line


def run_tgv_shock(args, local):
    thr = tuple(float(v) for v in args.tgv_shock_thr.split(","))
    print(json.dumps(tgv_shock(args.tgv_shock_t, local, thr=thr, variants=args.tgv_shock_variants)))
    return 0


def run_tgv_large(args, local):
    print(json.dumps(tgv_large(args.tgv_steps, local)))
    return 0


def ensemble_study(k_lo, k_hi, nsteps, local, cache_dir=None):
    """Batched ensemble: 64 uneven Taylor-Green runs (seed 20260529: K ~
    U{k_lo..k_hi} elements per direction, N ~ U{3..7}, Ma ~ U[0.1, 0.5], Re ~
    U[400, 1600]), each with its own CFL-0.9 time step, FP32 operator with FP64
    state, nsteps steps in one graph launch of the autotuned ensemble kernels.
    Compared with the same 64 runs advanced one after the other by the
    single-context path (each run's step graph launched back to back on one
    stream, the gaps between runs included), in FP64 and in FP32-operator
    precision."""
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import box_mesh, ensemble_members, tgv_params
    specs = ensemble_members(64, 20260529, k_lo, k_hi)
    dev = "cuda:%d" % local
    st = torch.cuda.Stream(device=dev)

    def member(spec, precision):
        prm = tgv_params(Ma=spec["Ma"], Re=spec["Re"])
        mesh = box_mesh(spec["K"], 1, lo=0.0, hi=2 * math.pi)
        s = dg.Solver(mesh, spec["N"], gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"],
                      precision=precision, device=local)
        U = s.initial_state("tgv", prm["p0"], stream=st)
        dt = s.max_dt(U, cfl=0.9, dfl=0.9, stream=st)
        return s, U, dt

    dofs = [sp["K"] ** 3 * (sp["N"] + 1) ** 3 for sp in specs]
    total = sum(dofs)
    runs = [member(sp, dg.FP32OP) for sp in specs]
    # the tuned plan depends on the member sizes: one cache file per size range
    cache = None
    if cache_dir and os.path.isdir(cache_dir):
        name = "ensemble_tune.txt" if (k_lo, k_hi) == (8, 24) else "ensemble_tune_K%d-%d.txt" % (k_lo, k_hi)
        cache = os.path.join(cache_dir, name)
    ens = dg.Ensemble([r[0] for r in runs], tune_cache_path=cache)
    Us = [r[1] for r in runs]
    Gs = [torch.empty_like(U) for U in Us]
    dts = [r[2] for r in runs]
    t0 = time.perf_counter()
    ens.step(Us, Gs, [0.0] * 64, dts, nsteps=1, stream=st)       # tunes, captures
    st.synchronize()
    tune_s = time.perf_counter() - t0
    ens.step(Us, Gs, dts, dts, nsteps=nsteps, stream=st)         # warm-up of the timed graph
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tt = [(1 + nsteps) * d for d in dts]
    e0.record(st)
    ens.step(Us, Gs, tt, dts, nsteps=nsteps, stream=st)
    e1.record(st)
    e1.synchronize()
    ms_ens = e0.elapsed_time(e1)
    ek_ens = [r[0].integrals(U, stream=st)[5] for r, U in zip(runs, Us)]
    plan = ens.plan()
    ens.close()
    for r in runs:
        r[0].close()
    del runs, Us, Gs
    torch.cuda.empty_cache()

    def sequential(precision):
        # the same 1 + 2 nsteps steps as the ensemble members took; the timed
        # part launches the 64 runs' step graphs back to back on one stream
        mem = [member(sp, precision) for sp in specs]
        Gq = [torch.empty_like(U) for _, U, _ in mem]
        for (s, U, dt), G in zip(mem, Gq):
            s.rk_step(U, G, 0.0, dt, 1, stream=st)
            s.rk_step(U, G, dt, dt, nsteps, stream=st)            # warm-up + graph capture
        st.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for (s, U, dt), G in zip(mem, Gq):
            s.rk_step(U, G, (1 + nsteps) * dt, dt, nsteps, stream=st)
        b.record(st)
        b.synchronize()
        ek = [s.integrals(U, stream=st)[5] for s, U, _ in mem]
        for s, _, _ in mem:
            s.close()
        del mem, Gq
        torch.cuda.empty_cache()
        return a.elapsed_time(b), ek

    ms_seq64, ek64 = sequential(dg.FP64)
    ms_seq32, ek32 = sequential(dg.FP32OP)
    ek_err = [abs(a - b) / abs(b) for a, b in zip(ek_ens, ek64)]
    rate = total * 5 * nsteps / (ms_ens * 1e-3)
    return {"experiment": "ensemble of 64 uneven Taylor-Green runs (seed 20260529, K^3 elements, K in %d..%d), "
                          "FP32 operator / FP64 state, %d LSERK4-5 steps in one graph launch" % (k_lo, k_hi, nsteps),
            "members": 64, "total_dof": total, "value": rate, "unit": UNIT, "pid_ns": 1e9 / rate,
            "ms_per_step": ms_ens / nsteps,
            "sequential_fp64_ms_per_step": ms_seq64 / nsteps, "sequential_fp32op_ms_per_step": ms_seq32 / nsteps,
            "speedup_vs_sequential_fp64": ms_seq64 / ms_ens, "speedup_vs_sequential_fp32op": ms_seq32 / ms_ens,
            "sequential_timing": "the 64 step graphs launched back to back on one stream, gaps included",
            "first_step_with_tuning_s": tune_s,
            "ek_rel_err_vs_fp64_max": max(ek_err), "ek_rel_err_vs_fp64_median": float(np.median(ek_err)),
            "ek_rel_diff_ensemble_vs_sequential_fp32op_max": max(abs(a - b) / abs(b) for a, b in zip(ek_ens, ek32)),
            "steps_compared": 1 + 2 * nsteps, "plan": plan}


def run_ensemble(args, local):
    k_lo, k_hi = (int(v) for v in args.ens_K.split(","))
    print(json.dumps(ensemble_study(k_lo, k_hi, args.ens_steps, local,
                                    os.path.join(ROOT, "paper_2605_28627_gb300", "_build"))))
    return 0


def fv50_rate(dg, N, dev, prm, dg_rate, steps=5):
    """The headline workload with half of its elements in the FV sub-cell
    representation (checkerboard, as the paper forces it for its DG/FV PID
    runs): LSERK4-5 steps as one graph launch after 3 warm-up steps, CUDA
    events; per-stage kernel times (the FV kernels are inside 'volume')."""
    import torch
    mesh = build_mesh(N)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                  device=dev)
    K = K_ELEMS
    e = torch.arange(mesh.n_elems, device="cuda:%d" % dev)
    st = torch.cuda.Stream(device="cuda:%d" % dev)
    with torch.cuda.stream(st):
        U = s.initial_state("mms", 0.0, stream=st)
        G = torch.empty_like(U)
    s.set_fv_mask(((e % K) + (e // K) % K + e // (K * K)) % 2, stream=st)
    s.rk_step(U, G, 0.0, DT, 3, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.rk_step(U, G, 3 * DT, DT, steps, stream=st)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    dofs = mesh.n_elems * (N + 1) ** 3
    rate = dofs * 5 * steps / (ms * 1e-3)
    ms3 = s.profile_stages(U, G, DT, reps=5, stream=st)
    finite = bool(torch.isfinite(U).all().item())
    s.close()
    return {"workload": workload_name(N) + ", 50 % FV sub-cell elements (checkerboard)", "value": rate,
            "unit": UNIT, "pid_ns": 1e9 / rate, "ms_per_step": ms / steps, "vs_all_dg": rate / dg_rate,
            "stage_ms": {"lift": ms3[0], "face": ms3[1], "volume_dg_and_fv": ms3[2]}, "state_finite": finite}


def mortar_rate(dg, N, dev, prm, dg_rate, K=12, steps=5):
    """A non-conforming 2:1 mesh: a periodic K^3 box (rotated element frames)
    whose cells with three even indices are split into eight, so that every
    split cell meets its six neighbours through mortars (Algorithm 1); MMS
    LSERK4-5 steps as one graph launch after 3 warm-up steps, CUDA events."""
    import numpy as np
    import torch
    from workloads.mesh import refined_box_mesh
    i = np.arange(K ** 3)
    mesh = refined_box_mesh(K, (i % 2 == 0) & ((i // K) % 2 == 0) & ((i // (K * K)) % 2 == 0), rotate_seed=3)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                  device=dev)
    st = torch.cuda.Stream(device="cuda:%d" % dev)
    with torch.cuda.stream(st):
        U = s.initial_state("mms", 0.0, stream=st)
        G = torch.empty_like(U)
    dt = min(DT, s.max_dt(U, cfl=0.9, dfl=0.9, stream=st))
    s.rk_step(U, G, 0.0, dt, 3, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.rk_step(U, G, 3 * dt, dt, steps, stream=st)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    dofs = mesh.n_elems * (N + 1) ** 3
    rate = dofs * 5 * steps / (ms * 1e-3)
    ms3 = s.profile_stages(U, G, dt, reps=5, stream=st)
    finite = bool(torch.isfinite(U).all().item())
    s.close()
    # the same steps with the FP32 operator
    s32 = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                    device=dev, precision=dg.FP32OP)
    with torch.cuda.stream(st):
        U32 = s32.initial_state("mms", 0.0, stream=st)
    s32.rk_step(U32, G, 0.0, dt, 3, stream=st)
    e0.record(st)
    s32.rk_step(U32, G, 3 * dt, dt, steps, stream=st)
    e1.record(st)
    e1.synchronize()
    rate32 = dofs * 5 * steps / (e0.elapsed_time(e1) * 1e-3)
    s32.close()
    # and on Legendre-Gauss nodes (weak form, mortar maps on the face values)
    slg = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                    device=dev, nodes=dg.NODES_LG)
    with torch.cuda.stream(st):
        Ulg = slg.initial_state("mms", 0.0, stream=st)
    dtl = min(DT, slg.max_dt(Ulg, cfl=0.9, dfl=0.9, stream=st))
    slg.rk_step(Ulg, G, 0.0, dtl, 3, stream=st)
    e0.record(st)
    slg.rk_step(Ulg, G, 3 * dtl, dtl, steps, stream=st)
    e1.record(st)
    e1.synchronize()
    rate_lg = dofs * 5 * steps / (e0.elapsed_time(e1) * 1e-3)
    finite_lg = bool(torch.isfinite(Ulg).all().item())
    slg.close()
    return {"workload": "MMS density wave, periodic %d^3 box with 1/8 of its cells split 2:1 (%d elements, %d "
                        "mortars), N=%d, rotated element frames" % (K, mesh.n_elems, len(mesh.mortars), N),
            "value": rate, "unit": UNIT, "pid_ns": 1e9 / rate, "ms_per_step": ms / steps,
            "vs_headline": rate / dg_rate,
            "stage_ms": {"lift_with_mortar_states": ms3[0], "face_with_mortar_fluxes": ms3[1], "volume": ms3[2]},
            "state_finite": finite,
            "fp32_operator": {"value": rate32, "pid_ns": 1e9 / rate32, "speedup_vs_fp64": rate32 / rate},
            "gauss_nodes": {"value": rate_lg, "pid_ns": 1e9 / rate_lg, "state_finite": finite_lg}}


def run_adj_vjp(args, local):
    """Cost of one VJP (dR/dU)^T lambda against one R(U) on the same state,
    per node set and mesh: a periodic 16^3 box (Taylor-Green state, Ma 0.2)
    and the 2:1 mortar mesh of the mortar leg (12^3 box, cells with three even
    indices split, MMS state), LGL and Gauss nodes, FP64; CUDA events on one
    stream, 20 calls each after 3 warm-up pairs."""
    import numpy as np
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import box_mesh, mms_params, tgv_params
    from workloads.mesh import refined_box_mesh
    torch.cuda.set_device(local)
    K = 12
    i = np.arange(K ** 3)
    split = (i % 2 == 0) & ((i // K) % 2 == 0) & ((i // (K * K)) % 2 == 0)
    st = torch.cuda.Stream(device="cuda:%d" % local)
    out = []
    for N in [int(x) for x in args.adj_vjp_orders.split(",")]:
        for mesh_name in ("box16", "mortar12"):
            for nodes in (dg.NODES_LGL, dg.NODES_LG):
                if mesh_name == "box16":
                    prm = tgv_params(Ma=0.2, Re=800.0)
                    mesh = box_mesh(16, 1, lo=0.0, hi=2 * math.pi)
                else:
                    prm = mms_params()
                    mesh = refined_box_mesh(K, split, rotate_seed=3)
                s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], nodes=nodes,
                              device=local)
                with torch.cuda.stream(st):
                    U = (s.initial_state("tgv", prm["p0"], stream=st) if mesh_name == "box16"
                         else s.initial_state("mms", 0.0, stream=st))
                    lam = torch.empty_like(U).normal_(generator=torch.Generator(device="cuda:%d" % local)
                                                      .manual_seed(7))
                    vj = torch.empty_like(U)
                    Rt = torch.empty_like(U)
                for _ in range(3):
                    s.time_derivative_vjp(U, lam, out=vj, stream=st)
                    s.time_derivative(U, Rt, stream=st)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                reps = 20
                ev[0].record(st)
                for _ in range(reps):
                    s.time_derivative_vjp(U, lam, out=vj, stream=st)
                ev[1].record(st)
                for _ in range(reps):
                    s.time_derivative(U, Rt, stream=st)
                ev[2].record(st)
                ev[2].synchronize()
                ms_vjp = ev[0].elapsed_time(ev[1]) / reps
                ms_r = ev[1].elapsed_time(ev[2]) / reps
                dof = mesh.n_elems * (N + 1) ** 3
                out.append({"N": N, "mesh": mesh_name, "nodes": "gauss" if nodes == dg.NODES_LG else "lgl",
                            "elements": mesh.n_elems, "dof": dof, "ms_R": round(ms_r, 4), "ms_vjp": round(ms_vjp, 4),
                            "vjp_over_R": round(ms_vjp / ms_r, 3), "ns_per_dof_vjp": round(ms_vjp * 1e6 / dof, 3),
                            "finite": bool(torch.isfinite(vj).all().item())})
                s.close()
    print(json.dumps({"adjoint_vjp_cost": out}))
    return 0


def run_mortar_fv(args, local):
    """FV sub-cell elements on the 2:1 mortar mesh of the mortar leg (12^3 box,
    cells with three even indices split): every other element without a
    mortar face is an FV element (the elements with one stay DG); MMS
    LSERK4-5 steps as one graph launch after 3 warm-up steps, CUDA events,
    against the same steps all DG.  FP64, LGL and Gauss nodes."""
    import numpy as np
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import mms_params
    from workloads.mesh import refined_box_mesh
    torch.cuda.set_device(local)
    prm = mms_params()
    K = 12
    i = np.arange(K ** 3)
    mesh = refined_box_mesh(K, (i % 2 == 0) & ((i // K) % 2 == 0) & ((i // (K * K)) % 2 == 0), rotate_seed=3)
    touching = (mesh.face_nbr[:, :, 0] < 0).any(axis=1)
    mask = np.zeros(mesh.n_elems, dtype=np.int32)
    mask[np.where(~touching)[0][::2]] = 1
    st = torch.cuda.Stream(device="cuda:%d" % local)
    out = []
    for N in [int(x) for x in args.mortar_fv_orders.split(",")]:
        for nodes in (dg.NODES_LGL, dg.NODES_LG):
            row = {"N": N, "nodes": "gauss" if nodes == dg.NODES_LG else "lgl", "elements": mesh.n_elems,
                   "fv_elements": int(mask.sum()), "elements_with_mortar_faces": int(touching.sum())}
            for label, use in (("all_dg", False), ("fv", True)):
                s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"],
                              source=dg.SOURCE_MMS, nodes=nodes, device=local)
                if use:
                    s.set_fv_mask(mask, stream=st)
                with torch.cuda.stream(st):
                    U = s.initial_state("mms", 0.0, stream=st)
                    G = torch.empty_like(U)
                dt = min(DT, s.max_dt(U, cfl=0.9, dfl=0.9, stream=st))
                s.rk_step(U, G, 0.0, dt, 3, stream=st)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                s.rk_step(U, G, 3 * dt, dt, args.steps, stream=st)
                e1.record(st)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                dof = mesh.n_elems * (N + 1) ** 3
                row[label + "_pid_ns"] = round(ms * 1e6 / (dof * 5 * args.steps), 3)
                row[label + "_finite"] = bool(torch.isfinite(U).all().item())
                s.close()
            row["fv_over_all_dg"] = round(row["fv_pid_ns"] / row["all_dg_pid_ns"], 3)
            out.append(row)
    print(json.dumps({"mortar_fv": out}))
    return 0


def run_mortar(args, local):
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import mms_params
    torch.cuda.set_device(local)
    prm = mms_params()
    ms, _ = sweep_rate(dg, args.order, local, prm)
    dg_rate = K_ELEMS ** 3 * (args.order + 1) ** 3 * 5 / (ms * 1e-3)
    print(json.dumps({"mortar": mortar_rate(dg, args.order, local, prm, dg_rate, steps=args.steps)}))
    return 0


def small_tgv_rate(dg, local, reps=20):
    """The small Taylor-Green case (4^3 Cartesian elements of [0, 2pi]^3, N=3,
    4096 nodes, Ma 0.1, Re 1600, LLF + BR1 + split form, dt at CFL 0.9): ten
    LSERK4-5 steps as one graph launch, timed with CUDA events; the median of
    `reps` launches.  At 4096 nodes this is launch- and latency-bound, so it is
    reported as microseconds per stage, not against a roofline."""
    import torch
    from workloads import box_mesh, tgv_params
    prm = tgv_params(Ma=0.1, Re=1600.0)
    mesh = box_mesh(4, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, 3, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], device=local)
    st = torch.cuda.Stream(device="cuda:%d" % local)
    with torch.cuda.stream(st):
        U = s.initial_state("tgv", prm["p0"], stream=st)
        G = torch.empty_like(U)
    dt = s.max_dt(U, cfl=0.9, dfl=0.9, stream=st)
    for i in range(3):
        s.rk_step(U, G, i * dt, dt, 10, stream=st)
    times = []
    for i in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.rk_step(U, G, (3 + i) * dt, dt, 10, stream=st)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    s.close()
    return {"workload": "Taylor-Green vortex, 4^3 Cartesian elements, N=3 (4096 nodes), Ma 0.1, Re 1600, "
                        "10 LSERK4-5 steps per graph launch", "us_per_stage": ms * 1e3 / 50,
            "us_per_step": ms * 1e3 / 10, "kernel_launches_per_stage": 3,
            "dof_stage_per_s": 4096 * 50 / (ms * 1e-3)}


def run_pid(args, local):
    """Free-stream PID runs in the setups of the paper's performance section:
    16.78 M DOF at N=3 (64^3 Cartesian elements; the paper's node-level PID
    comparison, run there on Gauss nodes) and N=9 at 20^3 elements (8.0 M DOF,
    the per-GPU load of the paper's weak-scaling runs of the split-form LGL
    operator), 10 steps each: LGL split form and Gauss nodes (standard weak
    form), each in FP64 and with the FP32 operator, each FP64 case also with RK4-14
    (PID counts stages, so it is per stage), and every case with half of the
    elements in the FV sub-cell representation (checkerboard, as the paper's
    DG/FV runs force it; its Table 4 runs are on Gauss nodes).  Uniform flow
    rho = 1, u = (0.1, 0.05, 0.02), p = 1/gamma, mu = 1/1600; every kernel
    does its full work on it.  Reports DOF*stage/s, PID and the free-stream
    preservation error max|U - U0| / max|U0| after the steps."""
    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import box_mesh
    cases = (("N3_64cubed", 3, 64, dg.NODES_LGL), ("N3_64cubed_gauss", 3, 64, dg.NODES_LG),
             ("N9_20cubed", 9, 20, dg.NODES_LGL), ("N9_20cubed_gauss", 9, 20, dg.NODES_LG))
    if args.pid_cases:
        keep = args.pid_cases.split(",")
        cases = tuple(c for c in cases if c[0] in keep)
    if args.pid_K:   # smaller meshes of the same cases (for profiler captures)
        cases = tuple(("N%d_%dcubed%s" % (N, args.pid_K, "_gauss" if nd == dg.NODES_LG else ""), N, args.pid_K, nd)
                      for _, N, _, nd in cases)
    gamma, nsteps = 1.4, args.pid_steps
    out = {}
    for name, N, K, nodes in cases:
        mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
        dofs = mesh.n_elems * (N + 1) ** 3
        res = {"N": N, "elements": mesh.n_elems, "dof": dofs,
               "nodes": "Legendre-Gauss, standard weak form" if nodes == dg.NODES_LG else "LGL, split form"}
        precs = [("fp64", dg.FP64, dg.RK45, False), ("fp64_rk414", dg.FP64, dg.RK414, False)]
        precs.append(("fp32op", dg.FP32OP, dg.RK45, False))
        precs.append(("fp64_fv50", dg.FP64, dg.RK45, True))
        if args.pid_variants:
            precs = [p for p in precs if p[0] in args.pid_variants.split(",")]
        for prec_name, prec, rk, fv in precs:
            s = dg.Solver(mesh, N, gamma=gamma, R=1.0, Pr=0.72, mu=1.0 / 1600.0, precision=prec, device=local,
                          nodes=nodes, rk_scheme=rk)
            if fv:   # half of the elements in the FV representation, checkerboard (the paper's forcing)
                e = torch.arange(mesh.n_elems, device="cuda:%d" % local)
                s.set_fv_mask(((e % K) + (e // K) % K + e // (K * K)) % 2)
            stages = 14 if rk == dg.RK414 else 5
            st = torch.cuda.Stream(device="cuda:%d" % local)
            with torch.cuda.stream(st):
                U = torch.zeros(s.shape, dtype=torch.float64, device="cuda:%d" % local)
                u = (0.1, 0.05, 0.02)
                U[:, 0] = 1.0
                for a in range(3):
                    U[:, 1 + a] = u[a]
                U[:, 4] = 1.0 / gamma / (gamma - 1.0) + 0.5 * sum(c * c for c in u)
                U0 = U.clone()
                G = torch.empty_like(U)
            dt = s.max_dt(U, cfl=0.9, dfl=0.9, stream=st)
            for i in range(3):
                s.rk_step(U, G, i * dt, dt, 1, stream=st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.rk_step(U, G, 3 * dt, dt, nsteps, stream=st)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            rate = dofs * stages * nsteps / (ms * 1e-3)
            drift = float((U - U0).abs().max() / U0.abs().max())
            res[prec_name] = {"dof_stage_per_s": rate, "pid_ns": 1e9 / rate, "ms_per_step": ms / nsteps,
                              "freestream_drift": drift}
            if fv:
                res[prec_name]["fv_elements"] = "50 %, checkerboard"
            del U, U0, G
            s.close()
            torch.cuda.empty_cache()
        out[name] = res
    line = {"experiment": "free-stream PID, %d steps after 3 warm-up steps, one graph launch" % nsteps,
            "cases": out,
            "paper_context": {"pid_ns_full_dg_N3_16.78M_dof_per_MI300A_gauss_nodes": 3.56864,
                              "pid_ns_50pct_fv_N3_16.78M_dof_per_MI300A_gauss_nodes": 8.35923,
                              "weak_scaling_N9_dof_per_gpu_range": [1.024e6, 8.192e6]}}
    print(json.dumps(line))
    return 0


def run_adjoint(args, local):
    """Discrete adjoint: 16^3 Cartesian elements, N=5 (884,736 nodes), Taylor-
    Green vortex at Ma 0.2, Re 800, FP64, 200 LSERK4-5 steps at CFL 0.9.
    J = volume-integrated kinetic energy at t_end; dJ/dU0 and dJ/dmu through
    torch.autograd (binomial checkpointing, <= 16 stored states), checked
    against central differences on 32 seeded unit directions (h = 1e-6
    max|U0|) and for mu (h = 1e-7)."""
    import torch
    import paper_2605_28627_gb300 as dg
    from paper_2605_28627_gb300.autograd import kinetic_energy, rk_solve
    from workloads import box_mesh, tgv_params
    K, N, nsteps, ndir = 16, 5, args.adj_steps, args.adj_dirs
    prm = tgv_params(Ma=0.2, Re=800.0)
    mesh = box_mesh(K, 1, lo=0.0, hi=2 * math.pi)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], device=local)
    U0 = s.initial_state("tgv", prm["p0"])
    dt = s.max_dt(U0, cfl=0.9, dfl=0.9)
    mu0 = prm["mu"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ul = U0.clone().requires_grad_(True)
    mu = torch.tensor(mu0, dtype=torch.float64, requires_grad=True)
    UT = rk_solve(Ul, mu, s, 0.0, dt, nsteps, max_snapshots=16)
    J = kinetic_energy(UT, s)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    gU, gmu = Ul.grad, mu.grad.item()
    # revolve counts of the same schedule
    lamT = torch.empty_like(U0)
    s.kinetic_energy(UT.detach(), grad=lamT)
    _, counts = s.adjoint_solve(U0, lamT, 0.0, dt, nsteps, max_snapshots=16)
    # one VJP of R (volume, face, gather and lifting adjoint kernels), CUDA
    # events on its stream, against the forward R(U) on the same state
    st = torch.cuda.Stream(device="cuda:%d" % local)
    with torch.cuda.stream(st):
        vj = torch.empty_like(U0)
        Rt = torch.empty_like(U0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(3):
        s.time_derivative_vjp(U0, lamT, out=vj, stream=st)
        s.time_derivative(U0, Rt, stream=st)
    reps = 20
    ev[0].record(st)
    for _ in range(reps):
        s.time_derivative_vjp(U0, lamT, out=vj, stream=st)
    ev[1].record(st)
    for _ in range(reps):
        s.time_derivative(U0, Rt, stream=st)
    ev[2].record(st)
    ev[2].synchronize()
    ms_vjp = ev[0].elapsed_time(ev[1]) / reps
    ms_fwd = ev[1].elapsed_time(ev[2]) / reps
    fp64_peak, _ = dg.probe_peaks(local)
    dof = s.E * (N + 1) ** 3
    adj_flops = adjoint_volume_flops_per_dof(N) * dof
    adj_roof = {"bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak,
                "achieved_lower_bound": adj_flops / (ms_vjp * 1e-3) / 1e12,
                "frac_lower_bound": adj_flops / (ms_vjp * 1e-3) / 1e12 / fp64_peak,
                "algorithmic_flops_per_dof": adjoint_volume_flops_per_dof(N),
                "note": "the adjoint volume kernel's algorithmic FP64 count over the time of the whole VJP call "
                        "(volume, face, gather and lifting adjoint kernels): a lower bound of the volume "
                        "kernel's own fraction; its share of the VJP time is in the ncu launch list"}

    def Jof(U, m):
        with torch.no_grad():
            return kinetic_energy(rk_solve(U, torch.tensor(m, dtype=torch.float64), s, 0.0, dt, nsteps), s).item()

    gen = torch.Generator(device="cuda:%d" % local).manual_seed(20260605)
    # central differences at two step sizes: the vortex's initial state sits on
    # kinks of the LLF speed (continuous across faces, w = 0), which gives the
    # differences an O(h) error on top of the O(h^2) truncation
    hmax = U0.abs().max().item()
    gnorm = gU.norm().item()
    ghat = gU / gnorm
    errs, errs_small, errs_norm = [], [], []
    # the steepest direction, seeded random unit directions (|g.v| ~ |g| / 1900
    # for 3.5 M unknowns: their relative error measures the rounding of J, not
    # the gradient), and eight directions mixed with the gradient, whose
    # |g.v| >= 1e-2 |g| puts them under the 1e-6 relative bar
    dirs = [gU / gnorm]
    for _ in range(ndir):
        v = torch.randn(U0.shape, generator=gen, device=U0.device, dtype=torch.float64)
        dirs.append(v / v.norm())
    for a in (0.02, 0.05, 0.1, 0.2, 0.35, 0.5, 0.7, 0.9):
        r = torch.randn(U0.shape, generator=gen, device=U0.device, dtype=torch.float64)
        v = a * ghat + (1.0 - a) * r / r.norm()
        dirs.append(v / v.norm())
    steep = None
    strict = []
    for q, v in enumerate(dirs):
        ad = float((gU * v).sum())
        for hh, out in ((1e-6 * hmax, errs), (1e-7 * hmax, errs_small)):
            fd = (Jof(U0 + hh * v, mu0) - Jof(U0 - hh * v, mu0)) / (2 * hh)
            if q == 0:
                if out is errs:
                    steep = abs(fd - ad) / abs(ad)
                continue
            if out is errs and abs(ad) >= 1e-2 * gnorm:
                strict.append(abs(fd - ad) / abs(ad))
            if q > ndir:
                continue
            out.append(abs(fd - ad) / max(abs(ad), 1e-300))
            if out is errs:
                errs_norm.append(abs(fd - ad) / gnorm)
    hm = 1e-7
    fdm = (Jof(U0, mu0 + hm) - Jof(U0, mu0 - hm)) / (2 * hm)
    line = {"experiment": "discrete adjoint, Taylor-Green vortex 16^3 elements, N=5, Ma 0.2, Re 800, FP64, %d LSERK4-5 "
                          "steps, J = volume-integrated kinetic energy at t_end" % nsteps,
            "dof": s.E * (N + 1) ** 3, "dt": dt, "J": J.item(), "dJ_dmu": gmu, "dJ_dmu_fd": fdm,
            "dJ_dmu_rel_err": abs(fdm - gmu) / abs(gmu),
            "directions": ndir, "grad_norm": gnorm,
            "dJ_dU0_fd_err_over_grad_norm_max_h1e-6": max(errs_norm),
            "steepest_direction_fd_rel_err_h1e-6": steep,
            "directions_with_g_dot_v_ge_1e-2_g": len(strict),
            "dJ_dU0_fd_rel_err_max_where_g_dot_v_ge_1e-2_g": max(strict) if strict else None,
            "random_directions_below_1e-2_g_excluded_from_the_relative_bar": ndir - sum(
                1 for v in dirs[1:ndir + 1] if abs(float((gU * v).sum())) >= 1e-2 * gnorm),
            "dJ_dU0_fd_rel_err_max_h1e-6": max(errs),
            "dJ_dU0_fd_rel_err_median_h1e-6": float(np.median(errs)),
            "dJ_dU0_fd_rel_err_max_h1e-7": max(errs_small),
            "dJ_dU0_fd_rel_err_median_h1e-7": float(np.median(errs_small)),
            "forward_s": t_fwd, "adjoint_s": t_adj, "adjoint_over_forward": t_adj / t_fwd,
            "vjp_ms": ms_vjp, "time_derivative_ms": ms_fwd, "vjp_over_time_derivative": ms_vjp / ms_fwd,
            "roofline": adj_roof,
            "snapshots": 16, "recomputed_forward_steps": counts[0], "adjoint_steps": counts[1]}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--order", type=int, default=7)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", default="1,2,3,4,5,6,7,8,9", help="extra orders timed for the per-N table ('' = none)")
    ap.add_argument("--tgv-large", action="store_true", help="run the 48^3, N=7 FP64-vs-FP32 Taylor-Green study")
    ap.add_argument("--tgv-steps", type=int, default=200)
    ap.add_argument("--ensemble", action="store_true", help="run the 64-member batched ensemble study")
    ap.add_argument("--ens-steps", type=int, default=10)
    ap.add_argument("--ens-K", default="8,24", help="range of elements per direction of the ensemble members")
    ap.add_argument("--adjoint", action="store_true", help="run the 16^3, N=5 discrete-adjoint study")
    ap.add_argument("--pid", action="store_true", help="run the free-stream PID study (N=3 at 64^3, N=9 at 20^3)")
    ap.add_argument("--pid-steps", type=int, default=10)
    ap.add_argument("--pid-cases", default="", help="comma list of PID case names ('' = all)")
    ap.add_argument("--pid-K", type=int, default=0, help="elements per direction instead of the cases' own")
    ap.add_argument("--pid-variants", default="", help="comma list of PID variants (fp64, fp64_rk414, fp32op, "
                    "fp64_fv50; '' = all)")
    ap.add_argument("--no-extra-legs", dest="extra_legs", action="store_false",
                    help="skip the 48^3 Taylor-Green and ensemble legs of the default line")
    ap.add_argument("--tgv-leg-steps", type=int, default=6, help="steps of the 48^3 leg of the default line")
    ap.add_argument("--mortar", action="store_true", help="run the 2:1 non-conforming mesh leg alone")
    ap.add_argument("--mortar-fv", action="store_true", help="FV elements on the 2:1 mortar mesh against all DG")
    ap.add_argument("--mortar-fv-orders", default="3,7", help="orders of the --mortar-fv study")
    ap.add_argument("--tgv-shock", action="store_true",
                    help="run the Ma 1.25 Taylor-Green study with automatic DG/FV switching")
    ap.add_argument("--tgv-shock-t", type=float, default=20.0)
    ap.add_argument("--tgv-shock-thr", default="-3.0,-3.5", help="log10 switching thresholds: upper,lower")
    ap.add_argument("--tgv-shock-variants", default="", help="comma list of the study's variants ('' = all)")
    ap.add_argument("--adj-vjp", action="store_true", help="time one VJP against one R(U) per node set and mesh")
    ap.add_argument("--adj-vjp-orders", default="3,5", help="orders of the --adj-vjp study")
    ap.add_argument("--adj-steps", type=int, default=200)
    ap.add_argument("--adj-dirs", type=int, default=32)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args.gpus)
    if args.tgv_large:
        return run_tgv_large(args, local) if rank == 0 else 0
    if args.ensemble:
        return run_ensemble(args, local) if rank == 0 else 0
    if args.pid:
        return run_pid(args, local) if rank == 0 else 0
    if args.adjoint:
        return run_adjoint(args, local) if rank == 0 else 0
    if args.adj_vjp:
        return run_adj_vjp(args, local) if rank == 0 else 0
    if args.mortar:
        return run_mortar(args, local) if rank == 0 else 0
    if args.mortar_fv:
        return run_mortar_fv(args, local) if rank == 0 else 0
    if args.tgv_shock:
        return run_tgv_shock(args, local) if rank == 0 else 0
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_2605_28627_gb300 as dg
    from workloads import mms_params

    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    N = args.order
    prm = mms_params()
    mesh = build_mesh(N)
    solver = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                       device=local)
    dof = solver.E * (N + 1) ** 3
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        U = solver.initial_state("mms", 0.0, stream=stream)
        G = torch.empty_like(U)
        U0 = U.clone()
    stream.synchronize()

    # warm-up (also captures the one-step graph)
    t = 0.0
    for _ in range(args.warmup):
        solver.rk_step(U, G, t, DT, 1, stream=stream)
        t += DT
    stream.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.rk_step(U, G, t, DT, 1, stream=stream)
        t += DT
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    value = world * dof * 5 * args.steps / (ms_total * 1e-3)
    launches_per_step = 5 * 3 + 1 + 1   # stages x (lift, face, volume) + clock advance + clock set
    gpu_launches = launches_per_step * args.steps

    # per-kernel times on the same stream, same inputs
    ms3 = solver.profile_stages(U, G, DT, reps=10, stream=stream)
    fp64_peak, fp32_peak = dg.probe_peaks(local)
    vol_flops = volume_flops_per_dof(N) * dof
    achieved = vol_flops / (ms3[2] * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": MEASURED_TRAFFIC.get((N, "fp64")),
                "kernel": "k_volume2<%d> (split-form volume + surface + Jacobian + LSERK update)" % N,
                "peak_source": "measured FP64 DFMA chain throughput on this GPU (dg_probe_peaks)",
                "stage_ms": {"lift": ms3[0], "face": ms3[1], "volume": ms3[2]}}
    # the whole stage (lifting, face fluxes, volume) by the same count
    stage_tf = step_flops_per_dof(N) * dof / (sum(ms3) * 1e-3) / 1e12
    roofline["stage"] = {
        "achieved": stage_tf, "frac": stage_tf / fp64_peak,
        "algorithmic_flops_per_dof": {"lift": lift_flops_per_dof(N), "face": face_flops_per_dof(N),
                                      "volume": volume_flops_per_dof(N)},
        "kernel_frac": {"lift": lift_flops_per_dof(N) * dof / (ms3[0] * 1e-3) / 1e12 / fp64_peak,
                        "face": face_flops_per_dof(N) * dof / (ms3[1] * 1e-3) / 1e12 / fp64_peak,
                        "volume": achieved / fp64_peak}}

    # end to end through the C ABI with host buffers (pinned)
    host = U0.cpu().pin_memory()
    solver.advance_host(host, 0.0, DT, 1, stream=stream)      # allocate the context's buffers
    torch.cuda.synchronize()
    nb = host.numel() * 8
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.advance_host(host, 0.0, DT, 1, stream=stream)
    el = time.perf_counter() - t0
    el = max_over_ranks(el, world)
    e2e = {"value": world * dof * 5 * args.steps / el, "unit": UNIT, "h2d_bytes_per_step": nb,
           "d2h_bytes_per_step": nb}

    hbm_peak, hbm_src = hbm_peak_gbs()
    fp32 = fp32_operator_rate(dg, N, local, prm, U0, args.steps, value / world, hbm_peak, hbm_src) \
        if rank == 0 else None
    tgv_small = small_tgv_rate(dg, local) if rank == 0 else None
    indicator = indicator_rate(solver, U, stream, fp64_peak) if rank == 0 else None
    fv50 = fv50_rate(dg, N, local, prm, value / world) if rank == 0 else None
    mortar = mortar_rate(dg, N, local, prm, value / world) if rank == 0 else None

    sweep = {}
    if args.sweep and rank == 0:
        for Ns in [int(v) for v in args.sweep.split(",") if v]:
            dofs = K_ELEMS ** 3 * (Ns + 1) ** 3
            if Ns == N:
                sweep[str(Ns)] = {"dof_stage_per_s": value / world, "pid_ns": 1e9 * world / value,
                                  "volume_ms": ms3[2], "volume_roofline_frac": roofline["frac"]}
            else:
                ms, ms3n = sweep_rate(dg, Ns, local, prm)
                # roofline of the volume kernel at this N: algorithmic FP64 flops / its event time
                ach = volume_flops_per_dof(Ns) * dofs / (ms3n[2] * 1e-3) / 1e12
                sweep[str(Ns)] = {"dof_stage_per_s": dofs * 5 / (ms * 1e-3), "pid_ns": ms * 1e6 / (dofs * 5),
                                  "volume_ms": ms3n[2], "volume_roofline_frac": ach / fp64_peak}
            sweep[str(Ns)]["volume_traffic"] = MEASURED_TRAFFIC.get((Ns, "fp64"))
            sweep[str(Ns)]["fp32op_volume_traffic"] = MEASURED_TRAFFIC.get((Ns, "fp32op"))
            # the FP32-operator path on the same mesh and state, and its
            # deviation from the FP64 path after the same 8 steps
            states = []
            sweep_rate(dg, Ns, local, prm, keep_state=states)
            ms32, _ = sweep_rate(dg, Ns, local, prm, precision=dg.FP32OP, keep_state=states)
            sweep[str(Ns)]["fp32op_dof_stage_per_s"] = dofs * 5 / (ms32 * 1e-3)
            sweep[str(Ns)]["fp32op_speedup"] = sweep[str(Ns)]["pid_ns"] / (ms32 * 1e6 / (dofs * 5))
            torch.cuda.synchronize()
            sweep[str(Ns)]["fp32op_max_rel_state_diff"] = float((states[1] - states[0]).abs().max() /
                                                                states[0].abs().max())
            del states

    # the larger workloads, each a few steps (their own studies run them longer)
    extra = {}
    if rank == 0 and args.extra_legs:
        for key, fn in (("tgv_large", lambda: tgv_large(args.tgv_leg_steps, local)),
                        ("ensemble", lambda: ensemble_study(8, 24, 10, local)),
                        ("ensemble_small_members", lambda: ensemble_study(2, 6, 10, local))):
            try:
                extra[key] = fn()
            except Exception as exc:          # a failed leg must not cost the headline line
                extra[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rates, cores, model = cpu_oracle_rate(N, n_evals=2)
        a, s1 = rates["all_cores"], rates["single"]
        cpu = {"value": a["value"], "unit": UNIT, "cores": a["threads"], "kind": "oracle", "cpu": model,
               "pid_ns_times_cores": 1e9 * a["threads"] / a["value"], "single_core_value": s1["value"],
               "sample": "R(U) (one RK stage) of the whole %d^3, N=%d mesh by the plain C++ oracle (-O3): %d "
                         "evaluations with its element and face loops on %d OpenMP threads (%.2f s each; "
                         "bit-identical to the serial oracle), and %d single-threaded (%.1f s each) for "
                         "single_core_value" % (K_ELEMS, N, a["evals"], a["threads"], a["s_per_eval"],
                                                s1["evals"], s1["s_per_eval"])}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(N), "elements": solver.E, "N": N, "dof": dof,
                       "pid_ns": 1e9 * world / value, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2: %.0f MB of state, metrics, gradients and face data touched "
                             "per stage" % working_set_mb(solver)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clk, "sweep": sweep, "fp32_operator": fp32, "tgv_small": tgv_small, "indicator": indicator,
            "fv50": fv50, "mortar": mortar,
            "peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
        }
        line.update(extra)
        print(json.dumps(line))
    solver.close()
    return 0


def fp32_operator_rate(dg, N, dev, prm, U0, steps, fp64_rate, hbm_peak, hbm_src):
    """The FP32-operator path on the same workload: throughput, speedup over
    the FP64 path, its deviation from the FP64 path after warm-up + steps, and
    the HBM roofline of its volume kernel (algorithmic bytes / event time)."""
    import torch
    mesh = build_mesh(N)
    results = {}
    ms3 = None
    for name, prec in (("fp64", dg.FP64), ("fp32op", dg.FP32OP)):
        s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                      precision=prec, device=dev)
        st = torch.cuda.Stream(device="cuda:%d" % dev)
        with torch.cuda.stream(st):
            U = U0.clone()
            G = torch.empty_like(U)
        st.synchronize()
        for i in range(3):
            s.rk_step(U, G, i * DT, DT, 1, stream=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(steps):
            s.rk_step(U, G, (3 + i) * DT, DT, 1, stream=st)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        results[name] = (U, s.integrals(U, stream=st), ms)
        if prec == dg.FP32OP:
            with torch.cuda.stream(st):
                Up, Gp = U.clone(), torch.empty_like(U)
            ms3 = s.profile_stages(Up, Gp, DT, reps=10, stream=st)
            del Up, Gp
        s.close()
    dofs = mesh.n_elems * (N + 1) ** 3
    U64, I64, ms64 = results["fp64"]
    U32, I32, ms32 = results["fp32op"]
    rate = dofs * 5 / (ms32 * 1e-3)
    vb = fp32_volume_bytes_per_dof(N) * dofs
    ach = vb / (ms3[2] * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": MEASURED_TRAFFIC.get((N, "fp32op")),
            "kernel": "k_volume2<%d, float> (FP32 split-form volume + surface + Jacobian, FP64 LSERK update)" % N,
            "algorithmic_bytes_per_dof": fp32_volume_bytes_per_dof(N), "peak_source": hbm_src,
            "stage_ms": {"lift": ms3[0], "face": ms3[1], "volume": ms3[2]}}
    return {"value": rate, "unit": UNIT, "pid_ns": 1e9 / rate, "speedup_vs_fp64": ms64 / ms32,
            "steps_compared": 3 + steps,
            "max_rel_state_diff_vs_fp64": float((U32 - U64).abs().max() / U64.abs().max()),
            "ek_rel_diff_vs_fp64": float(abs(I32[5] - I64[5]) / abs(I64[5])),
            "roofline": roof,
            "note": "same workload and steps as the headline; operator arithmetic FP32; state, LSERK register "
                    "update, U update and reductions FP64"}


def indicator_flops_per_dof(N):
    """Algorithmic FP64 operations per node of the Persson indicator (FMA = 2,
    divide = 1): p and rho p from the state (11), the modal transform in three
    directions (2 (N+1) each), the mode's square and its share of the two
    element sums (4)."""
    return 6.0 * (N + 1) + 15.0


def indicator_rate(solver, U, stream, fp64_peak, reps=20):
    """The Persson troubled-cell indicator (rho p) on the headline state: CUDA
    events around `reps` launches.  It reads 40 B and does 6 (N+1) + 15 FP64
    operations per node, so it is bound by the FP64 pipe, not by HBM."""
    import torch
    for _ in range(3):
        solver.indicator(U, log10_threshold=-4.0, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        eta, flag = solver.indicator(U, log10_threshold=-4.0, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    fl = indicator_flops_per_dof(solver.N) * solver.E * solver.P
    tf = fl / (ms * 1e-3) / 1e12
    return {"kernel": "k_indicator<%d> (Persson modal indicator of rho p, FP64)" % solver.N, "ms": ms,
            "elements_flagged_at_log10_eta_gt_-4": int(flag.sum().item()), "max_eta": float(eta.max().item()),
            "dram_gbs_algorithmic": solver.E * (40.0 * solver.P + 12.0) / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf / fp64_peak,
                         "algorithmic_flops_per_dof": indicator_flops_per_dof(solver.N),
                         "peak_source": "measured FP64 DFMA chain throughput on this GPU (dg_probe_peaks)"}}


def working_set_mb(s):
    P, NN, E = s.P, s.n * s.n, s.E
    F = 3 * E
    doubles = E * P * (5 + 5 + 10 + 12 + 2) + F * NN * (4 + 5)
    return doubles * 8 / 1e6


def sweep_rate(dg, N, dev, prm, steps=5, precision=None, keep_state=None):
    """ms per step of the MMS workload at order N (warm-up 3 steps, then
    `steps`), and the per-stage kernel times; with keep_state (a list) the
    final state is appended to it instead of profiling the stages."""
    import torch
    mesh = build_mesh(N)
    s = dg.Solver(mesh, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=dg.SOURCE_MMS,
                  device=dev, precision=dg.FP64 if precision is None else precision)
    st = torch.cuda.Stream(device="cuda:%d" % dev)
    with torch.cuda.stream(st):
        U = s.initial_state("mms", 0.0, stream=st)
        G = torch.empty_like(U)
    # the workload's dt = 1e-3 exceeds the CFL-0.9 step of the 16^3 mesh at
    # N = 8, 9 (7.6e-4 at N = 9): there the CFL step, as in a real run
    dt = min(DT, s.max_dt(U, cfl=0.9, dfl=0.9, stream=st))
    for i in range(3):
        s.rk_step(U, G, i * dt, dt, 1, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(steps):
        s.rk_step(U, G, (3 + i) * dt, dt, 1, stream=st)
    e1.record(st)
    e1.synchronize()
    ms3 = s.profile_stages(U, G, dt, reps=10, stream=st) if keep_state is None else None
    s.close()
    if keep_state is not None:
        keep_state.append(U)
    return e0.elapsed_time(e1) / steps, ms3


if __name__ == "__main__":
    sys.exit(main())
