"""Seeded nodal states and the parameter sets of the synthetic workloads.

Random states are drawn per node (no node positions are needed), in primitive
variables inside a physically admissible range, and returned as conserved
variables ``U[e, v, k, j, i]`` (v: rho, rho*u, rho*v, rho*w, rho*E).
"""
from __future__ import annotations

import numpy as np


def random_state(n_elems: int, N: int, seed: int, gamma: float = 1.4,
                 rho=(0.8, 1.2), vel=0.5, p=(0.8, 1.2), smooth_base: float = 0.0):
    """Random admissible conserved state, shape [E, 5, N+1, N+1, N+1]."""
    rng = np.random.default_rng(seed)
    n = N + 1
    shp = (n_elems, n, n, n)
    r = rng.uniform(rho[0], rho[1], size=shp)
    u = rng.uniform(-vel, vel, size=(3,) + shp)
    pr = rng.uniform(p[0], p[1], size=shp)
    U = np.empty((n_elems, 5, n, n, n))
    U[:, 0] = r
    for a in range(3):
        U[:, 1 + a] = r * u[a]
    U[:, 4] = pr / (gamma - 1.0) + 0.5 * r * (u ** 2).sum(0)
    return U


def tgv_params(Ma: float = 0.1, Re: float = 1600.0, gamma: float = 1.4, Pr: float = 0.72):
    """Taylor-Green vortex in units rho0 = U0 = L = R = 1.

    p0 = 1/(gamma Ma^2) gives the background Mach number Ma, T0 = p0/rho0 and
    mu = rho0 U0 L / Re = 1/Re."""
    p0 = 1.0 / (gamma * Ma * Ma)
    return dict(gamma=gamma, R=1.0, Pr=Pr, mu=1.0 / Re, p0=p0, T0=p0, Ma=Ma, Re=Re)


def mms_params(gamma: float = 1.4, Pr: float = 0.72, mu: float = 0.001):
    """Density-wave manufactured solution rho = 2 + 0.1 sin(pi (x+y+z-t)),
    u = (1,1,1), p = 1 on [-1,1]^3 with the gas constants of the workload."""
    return dict(gamma=gamma, R=1.0, Pr=Pr, mu=mu, amp=0.1)


def ensemble_members(count: int = 64, seed: int = 20260529, k_lo: int = 8, k_hi: int = 24):
    """Uneven Taylor-Green runs: K ~ U{k_lo..k_hi} (K^3 elements; 8..24 by
    default), N ~ U{3..7}, Ma ~ U[0.1, 0.5], Re ~ U[400, 1600]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        K = int(rng.integers(k_lo, k_hi + 1))
        N = int(rng.integers(3, 8))
        Ma = float(rng.uniform(0.1, 0.5))
        Re = float(rng.uniform(400.0, 1600.0))
        out.append(dict(K=K, N=N, Ma=Ma, Re=Re))
    return out
