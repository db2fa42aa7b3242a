"""The library's host planner (ER sampling, tally, commutation, pruning, DFS
order) is bit-exact against the oracle's independent implementation."""
import ctypes
import re
import os

import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    ("random_layers_6q", lambda: W.random_layers(6, 20, 0, 1e-3, 1e-2), 10_000),
    ("random_layers_noisy", lambda: W.random_layers(5, 12, 3, 2e-2, 5e-2), 5_000),
    ("mixed_all_kinds", lambda: W.random_mixed(5, 60, 7, 2e-2, 4e-2), 4_000),
    ("mixed_all_kinds_b", lambda: W.random_mixed(7, 90, 11, 1e-2, 3e-2), 4_000),
    ("brickwork_10q", lambda: W.brickwork(10, 8, 1, 1e-3, 1e-2), 20_000),
    ("qaoa_12q", lambda: W.qaoa_3regular(12, 2, 5, 5e-3, 2e-2), 20_000),
    ("ghz_8q", lambda: W.ghz(8, 2e-2, 3e-2), 3_000),
    ("twirl", lambda: _twirl_circuit(), 3_000),
]


def _twirl_circuit():
    c = W.Circuit(3)
    c.add(W.H, 0, channel=W.pauli_twirled_decoherence(1.0, 8.0, 5.0))
    c.add(W.CX, 0, 1, channel=W.depolarizing_2q(0.05))
    c.add(W.RY, 2, params=(0.4,), channel=W.measurement_flip(0.07))
    c.add(W.CZ, 1, 2, channel=W.depolarizing_2q(0.04))
    c.add(W.T, 2, channel=W.depolarizing_1q(0.05))
    c.add(W.RZZ, 0, 2, params=(1.1,), channel=W.depolarizing_2q(0.03))
    return c


@pytest.mark.parametrize("name,maker,shots", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_plan_bit_exact_vs_oracle(name, maker, shots, mode):
    circ = maker()
    seed = 17
    for prune, alpha, beta in [(False, 0.01, 100), (True, 0.01, 100), (True, 0.05, 7)]:
        ref = oracle.plan(circ, shots, seed, commute_mode=mode, prune=prune, alpha=alpha, beta=beta)
        pl = T.plan(circ, shots, seed, commute_mode=mode, prune=prune, alpha=alpha, beta=beta)
        raw, raw_count = pl.tally(0)
        assert raw == ref.raw
        assert np.array_equal(raw_count, ref.raw_count)
        keys, key_count = pl.tally(1)
        assert keys == ref.keys
        assert np.array_equal(key_count, ref.key_count)
        inst, counts, weights, lcp = pl.instances()
        assert inst == ref.inst
        assert np.array_equal(counts, ref.inst_count)
        assert np.array_equal(weights, ref.weights)           # bit-exact FP64
        assert np.array_equal(lcp, ref.lcp)
        st = pl.stats()
        assert st["n_raw_unique"] == len(ref.raw)
        assert st["n_commuted_unique"] == len(ref.keys)
        assert st["n_instances"] == len(ref.inst)
        if prune:
            assert st["n_significant"] == ref.n_sig
            assert st["n_picked"] == ref.n_pick
            assert st["n_insignificant"] == ref.n_insig


def test_plan_independent_of_threads():
    circ = W.random_layers(6, 20, 0)
    a = T.plan(circ, 50_000, 3, n_threads=1)
    b = T.plan(circ, 50_000, 3, n_threads=7)
    assert a.instances()[0] == b.instances()[0]
    assert np.array_equal(a.instances()[2], b.instances()[2])
    assert a.tally(0) [0] == b.tally(0)[0]


def test_plan_stats_tree_identities():
    # T_dftt = 2|E| - G (the last path is not uncomputed) and T_naive = N_l G
    # (Sec. III-B1); |E| = G + sum of (G - t_i) over branch slots.
    circ = W.random_layers(6, 20, 0)
    pl = T.plan(circ, 10_000, 0, prune=False)
    st = pl.stats()
    inst, counts, w, lcp = pl.instances()
    G = circ.n_gates
    assert st["tree_gate_edges"] == G + sum(G - int(t) for t in lcp)
    assert st["dftt_gate_apps"] == 2 * st["tree_gate_edges"] - G
    assert st["scratch_gate_apps"] == len(inst) * G
    assert st["scratch_pauli_apps"] == sum(len(e) for e in inst)
    assert abs(w.sum() - 1.0) < 1e-12 and int(counts.sum()) == 10_000


def test_plan_rejects_bad_input():
    with pytest.raises(T.TusqError):
        T.Circuit(0)
    c = T.Circuit(2)
    with pytest.raises(T.TusqError):
        c.add_gate(W.CX, 0, 0)
    with pytest.raises(T.TusqError):
        c.add_gate(W.RX, 0, -1, ())
    with pytest.raises(T.TusqError):
        c.add_gate(W.U1Q, 0, -1, (1, 0, 1, 0, 0, 0, 1, 0))          # not unitary
    j = c.add_gate(W.H, 0)
    with pytest.raises(T.TusqError):
        c.set_channel(j, [4], [0.1])                                # 2q code on a 1q gate
    with pytest.raises(T.TusqError):
        c.set_channel(j, [1, 2], [0.7, 0.6])                        # sums above 1
    with pytest.raises(T.TusqError):
        T.tusq_plan(c, 0, 0)


def test_plan_from_instances():
    circ = T.circuit_from(W.ghz(3, 0.1, 0.1))
    with pytest.raises(T.TusqError):
        T.tusq_plan_from_instances(circ, [((0, 5, 1),)], [1.0])            # qubit out of range
    with pytest.raises(T.TusqError):
        T.tusq_plan_from_instances(circ, [((1, 0, 1), (0, 1, 1))], [1.0])  # unsorted
    with pytest.raises(T.TusqError):
        T.tusq_plan_from_instances(circ, [(), ()], [0.5, 0.5])             # duplicates
    # a valid list comes back in DFS order with its branch slots
    pl = T.tusq_plan_from_instances(circ, [(), ((1, 0, 3),), ((0, 2, 1), (2, 1, 2))], [0.5, 0.3, 0.2])
    inst, counts, w, lcp = pl.instances()
    assert inst == [((0, 2, 1), (2, 1, 2)), ((1, 0, 3),), ()]
    assert list(w) == [0.2, 0.3, 0.5]
    assert list(lcp) == [0, 1]


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "tusq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tusq_\w+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    names = _header_symbols()
    assert "tusq_plan" in names and "tusq_exec_launch" in names
    L = ctypes.CDLL(T.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(T.EXPORTS) == names


def test_host_side_option_checks():
    # checks that run before any CUDA call: a batch's tc_mode out of range,
    # and the serving loop's job-state query without a server
    pl = T.plan(W.brickwork(6, 2, 0, 1e-3, 1e-2), 100, 0)
    for bad in (-1, 4):
        with pytest.raises(T.TusqError) as e:
            T.Batch([pl], [0x1000], T.run_opts(precision=T.C64, tc_mode=bad))
        assert e.value.code == T.TUSQ_EINVAL
    st = ctypes.c_int(-1)
    assert T.lib.tusq_job_state(None, 1, ctypes.byref(st)) == T.TUSQ_EINVAL
    assert st.value == -1
