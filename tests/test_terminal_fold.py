"""Readout fold of the Paulis left after the last gate (terminal_fold).

The output is the computational-basis distribution |psi_x|^2 (Sec. II), so a
Z that survives commutation to slot G changes nothing and a Y there acts like
an X.  The fold drops the first and turns the second into an X before the
re-tally, so instances that differ only there merge.  Pins on the oracle:
hand cases with known instance sets, losslessness of the unpruned output
(a property of the mathematics, not of the code), and the count bookkeeping;
then the planner bit-exact against the oracle and the device program
(interpreted on the host) against the oracle with the fold on."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W
from tests.test_plan_parity import CASES
from tests.test_schedule_emulated import emu_run


def _one_qubit(codes, probs, kind=W.H, params=()):
    c = W.Circuit(1)
    c.add(kind, 0, params=params, channel=(codes, probs))
    return c


def test_terminal_z_merges_into_the_ideal_instance():
    # H then a Z-only channel: the Z sits at slot G = 1 in every noisy shot
    c = _one_qubit((3,), (0.3,))
    plain = oracle.plan(c, 10_000, 4, prune=False)
    # keys in DFS order: the empty (ideal) key sorts after every event
    assert plain.keys == [((1, 0, 3),), ()]
    fold = oracle.plan(c, 10_000, 4, prune=False, terminal_fold=True)
    assert fold.keys == [()]
    assert int(fold.key_count[0]) == 10_000
    assert fold.weights.tolist() == [1.0]


def test_terminal_y_becomes_x():
    c = _one_qubit((1, 2, 3), (0.1, 0.2, 0.3), kind=W.RY, params=(0.7,))
    plain = oracle.plan(c, 20_000, 9, prune=False)
    fold = oracle.plan(c, 20_000, 9, prune=False, terminal_fold=True)
    assert plain.keys == [((1, 0, 1),), ((1, 0, 2),), ((1, 0, 3),), ()]
    assert fold.keys == [((1, 0, 1),), ()]
    pc = dict(zip(plain.keys, plain.key_count.tolist()))
    fc = dict(zip(fold.keys, fold.key_count.tolist()))
    # I + Z merge, X + Y merge
    assert fc[()] == pc[()] + pc[((1, 0, 3),)]
    assert fc[((1, 0, 1),)] == pc[((1, 0, 1),)] + pc[((1, 0, 2),)]


def test_events_before_the_last_slot_are_untouched():
    # a Z before a non-commuting gate stays where commutation left it
    c = W.Circuit(1)
    c.add(W.H, 0, channel=((3,), (0.5,)))
    c.add(W.RX, 0, params=(0.3,))
    fold = oracle.plan(c, 4000, 1, prune=False, terminal_fold=True)
    assert fold.keys == [((1, 0, 3),), ()]


@pytest.mark.parametrize("maker,shots,seed", [
    (lambda: W.random_layers(5, 10, 2, 2e-2, 5e-2), 4000, 3),
    (lambda: W.qaoa_3regular(6, 2, 1, 2e-2, 4e-2), 4000, 5),
    (lambda: W.random_mixed(4, 40, 9, 3e-2, 5e-2), 3000, 7),
])
def test_fold_is_lossless_without_pruning(maker, shots, seed):
    circ = maker()
    ref, pl = oracle.run(circ, shots, seed, prune=False)
    got, fl = oracle.run(circ, shots, seed, prune=False, terminal_fold=True)
    assert len(fl.keys) <= len(pl.keys)
    assert int(fl.key_count.sum()) == int(pl.key_count.sum()) == shots
    assert all(ev[0] < circ.n_gates or ev[2] == 1 for k in fl.keys for ev in k)
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("name,maker,shots", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_planner_fold_bit_exact_vs_oracle(name, maker, shots, mode):
    circ = maker()
    for prune, seed in [(False, 11), (True, 2)]:
        ref = oracle.plan(circ, shots, seed, commute_mode=mode, prune=prune, terminal_fold=True)
        pl = T.plan(circ, shots, seed, commute_mode=mode, prune=prune, terminal_fold=True)
        keys, key_count = pl.tally(1)
        assert keys == ref.keys and np.array_equal(key_count, ref.key_count)
        inst, counts, weights, lcp = pl.instances()
        assert inst == ref.inst
        assert np.array_equal(weights, ref.weights) and np.array_equal(lcp, ref.lcp)


@pytest.mark.parametrize("prune", [False, True])
def test_device_program_with_fold_vs_oracle(prune):
    circ = W.qaoa_3regular(8, 2, 3, 1e-2, 3e-2)
    ref, _ = oracle.run(circ, 8000, 4, prune=prune, terminal_fold=True)
    got, info = emu_run(T.plan(circ, 8000, 4, prune=prune, terminal_fold=True), precision=T.C128,
                        traversal=T.DFTT_SNAPSHOT)
    assert np.abs(got - ref).max() < 1e-12
