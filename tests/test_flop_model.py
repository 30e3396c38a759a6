"""The algorithmic FP64 count behind the volume kernel's roofline figure
(bench.py: FMA = 2 flops, a divide, square root or logarithm = 1) against the
plain oracle's own work, counted by the oracle's operation-counting scalar:
the model charges no more per pair, or per node, than the oracle spends."""
import numpy as np
import pytest

import bench
from workloads import box_mesh, mms_params


def test_pair_count_is_not_above_the_oracle(orc):
    """One unique pair of the split-form sum (Sec. 3.1): one two-point flux
    in the averaged metric direction, added with +-2 D into both nodes.  The
    oracle counts the flux itself (from the primitive states on: beta, two
    logarithmic means, averages, flux); its metric average 1/2 (Ja_i + Ja_m)
    is taken in plain double (3 additions, 3 multiplications) and its
    accumulation is 2 D f per component and node (a multiplication and an
    addition, five components, two nodes)."""
    rng = np.random.default_rng(3)
    worst = None
    for _ in range(200):
        r = rng.uniform(0.8, 1.2, 2)
        u = rng.uniform(-0.5, 0.5, (2, 3))
        p = rng.uniform(0.8, 1.2, 2)
        q = [np.r_[r[k], r[k] * u[k], p[k] / 0.4 + 0.5 * r[k] * (u[k] ** 2).sum()] for k in range(2)]
        if rng.random() < 0.5:                       # nearby states: the series branch of the log mean
            q[1] = q[0] * (1 + 1e-4 * rng.normal(size=5))
        ops = orc.count_ec_flux_ops(q[0], q[1], rng.normal(size=3))
        flux = sum(ops.values())
        worst = flux if worst is None else min(worst, flux)
    oracle_pair = worst + 6 + 2 * 5 * 2
    assert bench.PAIR_FLOPS <= oracle_pair, (bench.PAIR_FLOPS, oracle_pair)


@pytest.mark.parametrize("N", [1, 3, 5, 7, 9])
def test_volume_model_is_below_the_oracle_operator(orc, N):
    """Per node and stage, the volume-kernel model stays below what the oracle
    spends on the whole R(U) of the bench workload's mesh family."""
    prm = mms_params()
    m = box_mesh(2, N, deform="sinprod", rotate_seed=20260528)
    o = orc.Oracle(m, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    U = o.initial_state("mms", 0.0)
    per_node = sum(o.count_ops(U).values()) / (o.E * o.P)
    assert bench.volume_flops_per_dof(N) < per_node
    # counting does not change the result
    Ut = o.time_derivative(U)
    assert np.isfinite(Ut).all()


@pytest.mark.parametrize("N", [1, 3, 5, 7, 9])
def test_stage_model_is_below_the_oracle_operator(orc, N):
    """Lifting + face + volume models together (the whole-stage roofline of
    the bench line) stay below the oracle's count for the whole R(U)."""
    prm = mms_params()
    m = box_mesh(2, N, deform="sinprod", rotate_seed=20260528)
    o = orc.Oracle(m, N, gamma=prm["gamma"], R=prm["R"], Pr=prm["Pr"], mu=prm["mu"], source=1)
    U = o.initial_state("mms", 0.0)
    per_node = sum(o.count_ops(U).values()) / (o.E * o.P)
    assert bench.step_flops_per_dof(N) < per_node, (bench.step_flops_per_dof(N), per_node)
