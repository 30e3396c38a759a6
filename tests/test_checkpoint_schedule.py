"""Binomial checkpointing schedule of the adjoint solve (host logic, no GPU):
the counts of the schedule dg_adjoint_solve runs, against a brute-force
minimum over every split and against Griewank's closed form."""
import time
from functools import lru_cache
from math import comb

import pytest

import paper_2605_28627_gb300 as dg


@lru_cache(maxsize=None)
def _fewest_forward_steps(n, free):
    """Least forward steps that reverse n steps when the state at the start
    is stored and `free` more states may be stored: try every position of the
    next stored state (reverse the right part with one state less, then the
    left part); with none free, every step is recomputed from the start."""
    if n <= 1:
        return 0
    if free == 0:
        return n * (n - 1) // 2
    return min(m + _fewest_forward_steps(n - m, free - 1) + _fewest_forward_steps(m, free) for m in range(1, n))


def _griewank(n, s):
    """t(n, s) = r n - C(s + r, s + 1), r the least with C(s + r, s) >= n
    (Griewank 1992), s stored states including the initial one."""
    if n <= 1:
        return 0
    r = 0
    while comb(s + r, s) < n:
        r += 1
    return r * n - comb(s + r, s + 1)


def test_schedule_is_the_brute_force_minimum():
    for snaps in range(1, 9):
        for n in range(0, 61):
            fwd, adj = dg.checkpoint_schedule(n, snaps)
            assert adj == n
            assert fwd == _fewest_forward_steps(n, max(min(snaps, n) - 1, 0)), (n, snaps, fwd)


@pytest.mark.parametrize("n,snaps", [(200, 16), (1000, 4), (5000, 2), (12345, 30), (100000, 16), (4096, 4096)])
def test_schedule_matches_closed_form(n, snaps):
    fwd, adj = dg.checkpoint_schedule(n, snaps)
    assert adj == n
    assert fwd == _griewank(n, min(snaps, n))


def test_all_states_stored_needs_no_recomputation_beyond_one_sweep():
    # n states for n steps: each step advanced once to store the next state
    for n in (1, 2, 7, 64):
        assert dg.checkpoint_schedule(n, n) == (n - 1, n)
        assert dg.checkpoint_schedule(n, 10 * n) == (n - 1, n)


def test_long_horizons_run_without_deep_recursion():
    t0 = time.perf_counter()
    fwd, adj = dg.checkpoint_schedule(1_000_000, 200_000)
    assert adj == 1_000_000 and fwd == _griewank(1_000_000, 200_000)
    assert time.perf_counter() - t0 < 30


def test_bad_arguments():
    for args in ((-1, 4), (10, 0), (10, -3)):
        with pytest.raises(dg.DGError):
            dg.checkpoint_schedule(*args)
