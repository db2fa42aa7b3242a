"""Non-invertible operations (mid-circuit RESET / MEASURE) and DFTT+Caching
(Sec. III-B2).

Each such gate is unravelled into its two Kraus branches K_m (reset:
|0><m|, measurement: |m><m|); every kept ECM instance becomes 2^R leaves,
one per branch record, whose unnormalised states carry the branch
probabilities, so the weighted sum of |psi_leaf|^2 is the exact output.

Pins on the oracle: its density-matrix simulator against a numpy one built
from full Kraus operators; exact enumeration of every ER and every branch
record against the density matrix; closed forms for one qubit; trace
preservation.  Then the planner bit-exact against the oracle, and the device
program (interpreted on the host) against the oracle for every traversal,
cache capacity and drift-check setting, plus the operation counts of
DFTT+Caching as the capacity grows."""
import itertools

import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W
from tests import bruteforce as BF
from tests.test_schedule_emulated import emu_run


def _tiny_mixed():
    c = W.Circuit(3)
    c.add(W.H, 0, channel=W.depolarizing_1q(0.2))
    c.add(W.CX, 0, 1, channel=W.depolarizing_2q(0.15))
    c.add(W.MEASURE, 0, channel=W.measurement_flip(0.1))
    c.add(W.RY, 2, params=(0.7,), channel=W.depolarizing_1q(0.1))
    c.add(W.CX, 1, 2)
    c.add(W.RESET, 1, channel=W.depolarizing_1q(0.1))
    c.add(W.H, 1)
    c.add(W.CZ, 1, 2, channel=W.depolarizing_2q(0.1))
    return c


CIRCUITS = [
    ("repetition_reset", lambda: W.repetition_memory(3, 2, 1, 2e-2, 3e-2, 2e-2), 4000),
    ("repetition_measure", lambda: W.repetition_memory(3, 3, 5, 1e-2, 2e-2, 1e-2, kind=W.MEASURE), 3000),
    ("mcm_brickwork", lambda: W.mcm_brickwork(6, 8, 3, 2, 2, 1e-2, 3e-2), 3000),
    ("tiny_mixed", _tiny_mixed, 3000),
]


# ------------------------------------------------------------------ oracle pins

@pytest.mark.parametrize("maker", [
    _tiny_mixed,
    lambda: W.repetition_memory(2, 2, 3, 5e-2, 5e-2, 5e-2),
    lambda: W.mcm_brickwork(4, 4, 2, 2, 1, 3e-2, 5e-2, kind=W.MEASURE),
])
def test_dm_matches_numpy_kraus_density_matrix(maker):
    c = maker()
    np.testing.assert_allclose(oracle.dm_run(c), BF.dm_bruteforce(c), atol=1e-13)


def test_exact_enumeration_of_ers_and_branches_equals_dm():
    # every ER with its exact probability, times every branch record of the
    # two non-invertible gates, simulated independently
    c = _tiny_mixed()
    c.channels[-1] = None              # 2048 ERs x 4 branch records
    outs = [(j, c.gates[j][1]) for j in range(c.n_gates) if c.gates[j][0] in W.NONINVERTIBLE]
    total = np.zeros(1 << c.n_qubits)
    for prob, ev in BF.enumerate_ers(c):
        for rec in itertools.product((0, 1), repeat=len(outs)):
            evs = sorted(ev + [(j, q, W.OUTCOME1) for (j, q), m in zip(outs, rec) if m])
            total += oracle.simulate(c, evs, weight=prob)[0]
            if prob > 0.01:
                psi = BF.state_of_instance(c, evs)
                np.testing.assert_allclose(oracle.simulate(c, evs)[0], np.abs(psi) ** 2, atol=1e-14)
    np.testing.assert_allclose(total, oracle.dm_run(c), atol=1e-12)


def test_one_qubit_closed_forms():
    theta = 1.1
    c = W.Circuit(1)
    c.add(W.H, 0)
    c.add(W.RESET, 0)
    p, pl = oracle.run(c, 100, 0, prune=False)
    np.testing.assert_allclose(p, [1.0, 0.0], atol=1e-15)
    assert len(pl.inst) == 2           # one instance, two Kraus branches
    c = W.Circuit(1)
    c.add(W.H, 0)
    c.add(W.MEASURE, 0)
    c.add(W.H, 0)
    np.testing.assert_allclose(oracle.run(c, 100, 0, prune=False)[0], [0.5, 0.5], atol=1e-15)
    c = W.Circuit(1)
    c.add(W.RX, 0, params=(theta,))
    c.add(W.MEASURE, 0)
    c.add(W.RX, 0, params=(theta,))
    want = [np.cos(theta / 2) ** 4 + np.sin(theta / 2) ** 4, 2 * (np.cos(theta / 2) * np.sin(theta / 2)) ** 2]
    np.testing.assert_allclose(oracle.run(c, 100, 0, prune=False)[0], want, atol=1e-15)


@pytest.mark.parametrize("name,maker,shots", CIRCUITS, ids=[c[0] for c in CIRCUITS])
def test_expansion_bookkeeping_and_trace(name, maker, shots):
    c = maker()
    outs = {(j, c.gates[j][1]) for j in range(c.n_gates) if c.gates[j][0] in W.NONINVERTIBLE}
    p, pl = oracle.run(c, shots, 2, prune=False)
    assert len(pl.inst) % (1 << len(outs)) == 0
    for ev in pl.inst:
        assert all((s, q) in outs for s, q, code in ev if code == W.OUTCOME1)
    assert abs(p.sum() - 1.0) < 1e-12      # the Kraus sums preserve the trace


# -------------------------------------------------------------- library planner

@pytest.mark.parametrize("name,maker,shots", CIRCUITS, ids=[c[0] for c in CIRCUITS])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_planner_bit_exact_vs_oracle(name, maker, shots, mode):
    c = maker()
    for prune, seed in [(False, 4), (True, 9)]:
        ref = oracle.plan(c, shots, seed, commute_mode=mode, prune=prune)
        pl = T.plan(c, shots, seed, commute_mode=mode, prune=prune)
        inst, counts, weights, lcp = pl.instances()
        assert inst == ref.inst
        assert np.array_equal(counts, ref.inst_count)
        assert np.array_equal(weights, ref.weights) and np.array_equal(lcp, ref.lcp)
        st = pl.stats()
        R = sum(g[0] in W.NONINVERTIBLE for g in c.gates)
        assert st["n_noninvertible"] == R and st["n_instances"] == st["n_ecm_instances"] << R


def test_plan_rejects_too_many_branches():
    c = W.Circuit(2)
    c.add(W.H, 0, channel=W.depolarizing_1q(0.1))
    for _ in range(25):
        c.add(W.RESET, 1)
    with pytest.raises(T.TusqError):
        T.plan(c, 100, 0)
    with pytest.raises(ValueError):
        oracle.plan(c, 100, 0)


def test_plan_from_instances_outcome_events():
    c = W.Circuit(2)
    c.add(W.H, 0)
    c.add(W.RESET, 0)
    c.add(W.CX, 0, 1)
    inst = [[(1, 0, 1), (1, 0, W.OUTCOME1)], [(1, 0, W.OUTCOME1)], []]
    pl = T.tusq_plan_from_instances(T.circuit_from(c), inst, [0.25, 0.25, 0.5])
    assert pl.stats()["n_instances"] == 3
    for bad in ([(2, 0, W.OUTCOME1)], [(1, 1, W.OUTCOME1)], [(1, 0, W.OUTCOME1), (1, 0, 1)]):
        with pytest.raises(T.TusqError):
            T.tusq_plan_from_instances(T.circuit_from(c), [bad], [1.0])


# ------------------------------------------------- device program, host-interpreted

SETTINGS = [
    (T.DFTT, -1.0, 0),          # uncompute, no drift checks: the cache is the only saved state
    (T.DFTT, 1e-6, 1),          # drift checks with branch snapshots
    (T.DFTT_SNAPSHOT, -1.0, 2),
    (T.FROM_SCRATCH, -1.0, 0),
]


@pytest.mark.parametrize("name,maker,shots", CIRCUITS, ids=[c[0] for c in CIRCUITS])
@pytest.mark.parametrize("traversal,tol,nsnap", SETTINGS)
@pytest.mark.parametrize("cache", [0, 1, 2, -1])
def test_device_program_vs_oracle(name, maker, shots, traversal, tol, nsnap, cache):
    c = maker()
    ref, _ = oracle.run(c, shots, 3)
    pl = T.plan(c, shots, 3)
    sb = (nsnap * 16 << c.n_qubits) or 16
    got, info = emu_run(pl, precision=T.C128, traversal=traversal, drift_tol=tol, snapshot_bytes=sb,
                        cache_states=cache)
    assert np.abs(got - ref).max() < 1e-12
    got64, _ = emu_run(pl, precision=T.C64, traversal=traversal, drift_tol=tol, snapshot_bytes=sb,
                       cache_states=cache, max_window=3)
    assert np.abs(got64 - ref).max() < 1e-7


@pytest.mark.parametrize("name,maker,shots", CIRCUITS[:3], ids=[c[0] for c in CIRCUITS[:3]])
def test_caching_operation_counts(name, maker, shots):
    # Sec. III-B2: a larger cache never costs more gate applications; with no
    # cache every crossing re-derives from |0..0>; with one the cached
    # pre-layer states serve some of the returns
    c = maker()
    pl = T.plan(c, shots, 3)
    st = pl.stats()
    apps = []
    for K in range(0, st["n_noninv_layers"] + 2):
        cs = T.tusq_compile_stats(pl, T.run_opts(traversal=T.DFTT, drift_tol=-1.0, cache_states=K))
        apps.append(cs["gate_apps"])
        if K == 0:
            assert cs["cache_restores"] == 0 and cs["rederives"] > 0
        else:
            assert cs["cache_restores"] > 0
    assert all(a >= b for a, b in zip(apps, apps[1:]))
    assert apps[0] <= st["scratch_gate_apps"]
    assert apps[-1] < apps[0]


@pytest.mark.parametrize("name,maker,shots", CIRCUITS, ids=[c[0] for c in CIRCUITS])
def test_from_scratch_counts_match_plan(name, maker, shots):
    # every leaf from |0..0>: N_l x G gate applications and the plan's Pauli
    # count (the Kraus-branch choices select a gate's matrix, they are not
    # Pauli applications)
    pl = T.plan(maker(), shots, 3)
    st = pl.stats()
    cs = T.tusq_compile_stats(pl, T.run_opts(traversal=T.FROM_SCRATCH))
    assert cs["gate_apps"] == st["scratch_gate_apps"]
    assert cs["pauli_apps"] == st["scratch_pauli_apps"]
