"""Batched systems (many independent drums in one context, one launch per step for all of
them) against the same systems run one at a time: the FP64 batch reproduces the oracle
run of each instance bit for bit, the mixed batch reproduces the single-system mixed path
bit for bit, and instances never interact even when they occupy the same space."""
import numpy as np
import pytest

import workloads
from gpu_helpers import make_gpu, make_oracle
from paper_2106_09576_gb300.dem import DemError

pytestmark = pytest.mark.gpu


def small_batch(precision, seed=77, n_instances=6):
    b = workloads.batched_drums(n_instances=n_instances, n_lo=200, n_hi=1500, seed=seed, precision=precision,
                                dt=1e-5)
    return b


def instance_slice(state, I):
    lo, hi = I["first"], I["first"] + I["n"]
    return [np.asarray(a)[lo:hi] for a in state]


def test_fp64_batch_equals_oracle_per_instance():
    b = small_batch("fp64")
    g = make_gpu(b, "fp64")
    g.step(1500)
    st = g.state()
    assert g.stats()["rebuilds"] > 1
    for k in (0, 3, 5):
        wk = workloads.instance_workload(b, k)
        o = make_oracle(wk)
        o.step(1500)
        for a, r in zip(instance_slice(st, b.cfg["instances"][k]), o.state()):
            assert np.array_equal(a, np.asarray(r)), k


def test_mixed_batch_equals_single_system_mixed_runs():
    b = small_batch("mixed", seed=91)
    g = make_gpu(b, "mixed")
    g.step(1200)
    st = g.state()
    for k, I in enumerate(b.cfg["instances"]):
        gk = make_gpu(workloads.instance_workload(b, k), "mixed")
        gk.step(1200)
        for a, r in zip(instance_slice(st, I), gk.state()):
            assert np.array_equal(a, np.asarray(r)), k
        gk.close()


def test_instances_never_interact_even_in_the_same_place():
    b = small_batch("mixed", seed=5, n_instances=1)
    one = workloads.instance_workload(b, 0)
    n = one.n
    # two copies of the same drum at the same coordinates, as a batch of two
    I0 = dict(b.cfg["instances"][0])
    I1 = dict(I0, first=n)
    cfg = dict(b.cfg, instances=[I0, I1], n_instances=2)
    two = workloads.Workload("twin", cfg, [], np.vstack([b.x, b.x]), np.vstack([b.v, b.v]),
                             np.vstack([b.w, b.w]), np.concatenate([b.radius, b.radius]))
    g2 = make_gpu(two, "mixed")
    g1 = make_gpu(one, "mixed")
    g2.step(800)
    g1.step(800)
    s2, s1 = g2.state(), g1.state()
    for a, r in zip(s2, s1):
        a = np.asarray(a)
        assert np.array_equal(a[:n], np.asarray(r)) and np.array_equal(a[n:], np.asarray(r))


def test_batch_argument_and_state_errors():
    b = small_batch("mixed", seed=3, n_instances=2)
    insts = b.cfg["instances"]
    cfg = dict(b.cfg)
    cfg.pop("instances")                      # the context is a batch, but no tables yet
    g = make_gpu(workloads.Workload("b", cfg, [], b.x, b.v, b.w, b.radius), "mixed")
    with pytest.raises(DemError, match="ERR_STATE"):
        g.step(1)
    with pytest.raises(DemError, match="ERR_ARG"):
        g.set_instances([dict(insts[0], first=5), insts[1]])        # must start at 0
    with pytest.raises(DemError, match="ERR_ARG"):
        g.set_instances([insts[0], dict(insts[1], first=b.n + 1)])  # beyond n
    with pytest.raises(DemError, match="ERR_STATE"):
        g.set_walls(insts[0]["walls"])                              # walls are per instance
    g.set_instances(insts)
    g.step(2)
    single = make_gpu(workloads.instance_workload(b, 0), "mixed")
    with pytest.raises(DemError, match="ERR_STATE"):
        single.set_instances(insts)
