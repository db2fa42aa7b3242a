"""GPU parity at full size, in the launch configuration the benchmark times
(complex64 state, default 13-qubit pass window).

28-qubit QAOA (random 3-regular graph, 4 layers, 2q depolarizing 5e-3, 1q
5e-4, 1e6 shots, alpha 0.01, beta 100 -> 101 kept instances).  The oracle
costs about a minute per instance at this size, so the comparison over all
2^28 outcomes runs on an instance subset planned by the oracle: the first
eight leaves in DFS order plus the ideal instance (the last leaf), with
their weights.  As one plan of nine leaves it has branch nodes at several
depths, so it exercises branch snapshots, restores fused into the next
pass's tile loads, the leaf pass that skips its write, and -- in the
uncompute traversal -- the drift check at every return (Sec. III-B).  Both
the snapshot traversal and the paper's uncompute traversal are compared
element by element (max-abs 1e-5, total variation 1e-4).  The whole
101-leaf traversal is checked against properties that hold at any size.

20-qubit brickwork, depth 40 (Haar SU(2) on every qubit and CZ on
alternating neighbour pairs, 1180 gates), 1q/2q depolarizing 1e-3/1e-2, 1e6
shots, pruned: the whole 101-leaf plan against the oracle, in complex64
(1e-5 / 1e-4; SIMT and the two split tensor-core modes) and in the
complex128 mode (1e-12 / 1e-10).

The largest state the serving mix admits (30 qubits, 8 GiB) is checked
against a closed form: a GHZ circuit under Pauli noise, whose every instance
is the ideal GHZ distribution XOR-shifted by the X part of its Pauli frame
propagated to the end (Sec. II mixture view; Clifford conjugation of
Paulis).
"""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu

MAX_ABS, TV = 1e-5, 1e-4
MAX_ABS_C128, TV_C128 = 1e-12, 1e-10


def _torch():
    import torch
    return torch


def _run(plan, **opts):
    torch = _torch()
    probs, info = T.run_torch(plan, T.run_opts(**opts))
    torch.cuda.synchronize()
    return probs, info


def _events(inst):
    return [[tuple(int(v) for v in e) for e in ev] for ev in inst]


def _compare(probs, ref, max_abs, tv, what):
    torch = _torch()
    d = (probs - torch.from_numpy(ref).to(probs.device)).abs()
    m, s = float(d.max()), float(d.sum())
    assert m <= max_abs, f"{what}: max-abs {m:.3e} > {max_abs}"
    assert s <= tv, f"{what}: TV {s:.3e} > {tv}"
    return m, s


@pytest.fixture(scope="module")
def qaoa28_subset():
    circ = W.WORKLOADS["qaoa_28q"]()
    opl = oracle.plan(circ, 1_000_000, 0)
    assert len(opl.inst) == 101 and len(opl.inst[-1]) == 0
    idx = list(range(8)) + [len(opl.inst) - 1]
    subset = [list(opl.inst[i]) for i in idx]
    weights = np.array([opl.weights[i] for i in idx])
    ref = oracle.run_instances(circ, subset, weights)
    pl = T.tusq_plan_from_instances(T.circuit_from(circ), _events(subset), weights)
    return circ, pl, ref, float(weights.sum())


def test_qaoa28_nine_leaves_snapshot_traversal_matches_oracle(qaoa28_subset):
    circ, pl, ref, wsum = qaoa28_subset
    probs, info = _run(pl, precision=T.C64, traversal=T.DFTT_SNAPSHOT)
    _compare(probs, ref, MAX_ABS, TV, "28q nine leaves, snapshot traversal")
    assert info["leaf_passes"] == 9 and info["unrecovered"] == 0
    # every return to a branch node below the root is a snapshot restore
    assert info["restores"] > 0
    del probs
    _torch().cuda.empty_cache()


def test_qaoa28_nine_leaves_uncompute_traversal_matches_oracle(qaoa28_subset):
    circ, pl, ref, wsum = qaoa28_subset
    probs, info = _run(pl, precision=T.C64, traversal=T.DFTT, drift_tol=1e-6)
    _compare(probs, ref, MAX_ABS, TV, "28q nine leaves, uncompute traversal")
    # a drift check after every uncompute back to a branch node; complex64
    # uncompute at 28 qubits drifts above 1e-6 at some nodes, which restore
    # their snapshot, so none is left unrecovered
    assert info["leaf_passes"] == 9 and info["checks"] > 0
    assert info["unrecovered"] == 0
    del probs
    _torch().cuda.empty_cache()


def test_qaoa28_full_traversal_properties():
    torch = _torch()
    circ = W.WORKLOADS["qaoa_28q"]()
    pl = T.plan(circ, 1_000_000, 0)
    wsum = float(np.sum(pl.instances()[2]))
    outs = {}
    for name, trav in (("snapshot", T.DFTT_SNAPSHOT), ("dftt", T.DFTT), ("scratch", T.FROM_SCRATCH)):
        probs, info = _run(pl, precision=T.C64, traversal=trav)
        assert info["unrecovered"] == 0
        # |sum p - sum w| is bounded by the total-variation error of p
        assert abs(float(probs.sum()) - wsum) <= TV, (name, float(probs.sum()))
        assert float(probs.min()) >= 0.0
        outs[name] = probs
    for name in ("dftt", "scratch"):
        d = (outs[name] - outs["snapshot"]).abs()
        assert float(d.max()) <= MAX_ABS, (name, float(d.max()))
        assert float(d.sum()) <= TV, (name, float(d.sum()))
    del outs
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def brickwork20():
    circ = W.WORKLOADS["brickwork_20q"]()
    assert circ.n_qubits == 20 and circ.n_gates == 1180
    opl = oracle.plan(circ, 1_000_000, 0)
    ref = oracle.run_instances(circ, opl.inst, opl.weights)
    return circ, opl, ref


def test_brickwork20_depth40_plan_is_the_oracles(brickwork20):
    circ, opl, ref = brickwork20
    pl = T.plan(circ, 1_000_000, 0)
    inst, counts, weights, lcp = pl.instances()
    assert len(inst) == len(opl.inst) == 101
    assert [tuple(ev) for ev in inst] == [tuple(tuple(int(v) for v in e) for e in ev) for ev in opl.inst]
    assert np.array_equal(counts, opl.inst_count)
    assert np.array_equal(weights, opl.weights)
    assert np.array_equal(lcp, opl.lcp)


@pytest.mark.parametrize("trav", [T.DFTT_SNAPSHOT, T.DFTT])
def test_brickwork20_depth40_all_leaves_c64(brickwork20, trav):
    circ, opl, ref = brickwork20
    pl = T.tusq_plan_from_instances(T.circuit_from(circ), _events(opl.inst), opl.weights)
    probs, info = _run(pl, precision=T.C64, traversal=trav)
    _compare(probs, ref, MAX_ABS, TV, f"20q brickwork depth 40, complex64, traversal {trav}")
    assert info["leaf_passes"] == 101 and info["unrecovered"] == 0


@pytest.mark.parametrize("tc_mode", [T.TC_TF32X3, T.TC_BF16X3])
def test_brickwork20_depth40_all_leaves_tensor_cores(brickwork20, tc_mode):
    # the single-qubit layers of most register stages as 32x32 matrices on
    # the tensor cores (split TF32 or BF16 products, FP32 accumulation, the
    # norm of each unitary stage's vectors restored): same tolerance as the
    # SIMT path
    circ, opl, ref = brickwork20
    pl = T.tusq_plan_from_instances(T.circuit_from(circ), _events(opl.inst), opl.weights)
    probs, info = _run(pl, precision=T.C64, traversal=T.DFTT_SNAPSHOT, tc_mode=tc_mode)
    _compare(probs, ref, MAX_ABS, TV, f"20q brickwork depth 40, tensor cores mode {tc_mode}")
    assert info["dense_ops"] > 0 and info["leaf_passes"] == 101


def test_brickwork20_depth40_all_leaves_c128(brickwork20):
    circ, opl, ref = brickwork20
    pl = T.tusq_plan_from_instances(T.circuit_from(circ), _events(opl.inst), opl.weights)
    probs, info = _run(pl, precision=T.C128, traversal=T.DFTT_SNAPSHOT)
    _compare(probs, ref, MAX_ABS_C128, TV_C128, "20q brickwork depth 40, complex128")
    assert info["leaf_passes"] == 101 and info["unrecovered"] == 0


def _frame_xmask(circ, events):
    """X part of the Pauli frame of `events` after the circuit's H / CX gates
    (Clifford conjugation: H swaps x and z; CX copies x of the control to
    the target and z of the target to the control)."""
    x = [0] * circ.n_qubits
    z = [0] * circ.n_qubits
    for j in range(circ.n_gates + 1):
        for (s, q, p) in events:
            if s == j:
                x[q] ^= p in (1, 2)
                z[q] ^= p in (2, 3)
        if j == circ.n_gates:
            break
        kind, a, b, _ = circ.gates[j]
        if kind == W.H:
            x[a], z[a] = z[a], x[a]
        elif kind == W.CX:
            x[b] ^= x[a]
            z[a] ^= z[b]
    return sum(bit << q for q, bit in enumerate(x))


def test_ghz30_closed_form_at_maximum_state_size():
    torch = _torch()
    n = 30
    circ = W.ghz(n, p1=2e-3, p2=2e-2)
    opl = oracle.plan(circ, 20_000, 3)
    idx, val = [], []
    for ev, w in zip(opl.inst, opl.weights):
        m = _frame_xmask(circ, [tuple(int(v) for v in e) for e in ev])
        idx += [m, m ^ ((1 << n) - 1)]
        val += [0.5 * w, 0.5 * w]
    pl = T.tusq_plan_from_instances(T.circuit_from(circ), _events(opl.inst), np.asarray(opl.weights))
    probs, info = _run(pl, precision=T.C64, traversal=T.DFTT, snapshot_bytes=2 * (8 << n))
    want = torch.zeros_like(probs)
    want.index_put_((torch.tensor(idx, device=probs.device),),
                    torch.tensor(val, dtype=torch.float64, device=probs.device), accumulate=True)
    d = (probs - want).abs()
    assert float(d.max()) <= MAX_ABS, float(d.max())
    assert float(d.sum()) <= TV, float(d.sum())
    assert info["unrecovered"] == 0
    del probs, want, d
    torch.cuda.empty_cache()
