"""ER sampling on the device (tusq_plan with device_sampling = 1): the draws
of every channel of every shot are made by a CUDA kernel and tallied on the
host by hash with exact word-list comparison; the plan must be bit-exact
against the oracle's independent implementation, and identical to the host
planner's, on the same circuits as the host planner's parity test."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W
from tests.test_plan_parity import CASES

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,maker,shots", CASES, ids=[c[0] for c in CASES])
def test_device_sampled_plan_bit_exact_vs_oracle(name, maker, shots):
    circ = maker()
    for prune, seed in [(False, 17), (True, 5)]:
        ref = oracle.plan(circ, shots, seed, commute_mode=2, prune=prune)
        pl = T.plan(circ, shots, seed, prune=prune, device_sampling=True)
        raw, raw_count = pl.tally(0)
        assert raw == ref.raw
        assert np.array_equal(raw_count, ref.raw_count)
        keys, key_count = pl.tally(1)
        assert keys == ref.keys and np.array_equal(key_count, ref.key_count)
        inst, counts, weights, lcp = pl.instances()
        assert inst == ref.inst
        assert np.array_equal(counts, ref.inst_count)
        assert np.array_equal(weights, ref.weights)
        assert np.array_equal(lcp, ref.lcp)


def test_device_and_host_sampling_agree_at_full_size():
    # the 28-qubit QAOA workload: 1e6 shots x 308 channels
    circ = W.WORKLOADS["qaoa_28q"]()
    a = T.plan(circ, 1_000_000, 0)
    b = T.plan(circ, 1_000_000, 0, device_sampling=True)
    ra, ca = a.tally(0)
    rb, cb = b.tally(0)
    assert ra == rb and np.array_equal(ca, cb)
    ia, na, wa, la = a.instances()
    ib, nb, wb, lb = b.instances()
    assert ia == ib and np.array_equal(wa, wb) and np.array_equal(la, lb)


def test_device_sampling_edge_cases():
    # no channels at all: one (ideal) instance; zero shots: rejected like the host path
    c = W.random_layers(4, 3, 1, 0.0, 0.0)
    pl = T.plan(c, 1000, 0, device_sampling=True)
    assert pl.stats()["n_instances"] == 1
    with pytest.raises(T.TusqError):
        T.plan(W.random_layers(4, 3, 1, 1e-2, 1e-2), 0, 0, device_sampling=True)
