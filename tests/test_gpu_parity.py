"""GPU parity: the CUDA DFTT engine (through the C ABI) against the CPU
oracle, element by element, on the same seeded inputs.

Tolerances: complex128 mode max-abs 1e-12 per outcome (total variation
1e-10: thousands of uncompute passes leave ~1e-14 per outcome, summed over
up to 2^11 outcomes here); complex64 mode max-abs 1e-5 and total variation
1e-4 (FP32 state with FP64 leaf accumulation)."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu

TOL = {T.C128: (1e-12, 1e-10), T.C64: (1e-5, 1e-4)}
TRAVERSALS = [T.DFTT, T.FROM_SCRATCH, T.DFTT_SNAPSHOT]


def gpu_run(plan, **opts):
    import torch
    probs, info = T.run_torch(plan, T.run_opts(**opts))
    torch.cuda.synchronize()
    return probs.cpu().numpy(), info


def assert_close(got, ref, precision, what=""):
    ma, tv = TOL[precision]
    d = np.abs(got - ref)
    assert d.max() <= ma, f"{what}: max-abs {d.max():.3e} > {ma}"
    assert d.sum() <= tv, f"{what}: TV {d.sum():.3e} > {tv}"


@pytest.mark.parametrize("precision", [T.C128, T.C64])
@pytest.mark.parametrize("traversal", TRAVERSALS)
@pytest.mark.parametrize("prune", [True, False])
def test_random_layers_6q_matches_oracle(precision, traversal, prune):
    circ = W.random_layers(6, 20, 0, 1e-3, 1e-2)
    ref, _ = oracle.run(circ, 10_000, 0, prune=prune)
    pl = T.plan(circ, 10_000, 0, prune=prune)
    got, info = gpu_run(pl, precision=precision, traversal=traversal)
    assert_close(got, ref, precision, f"trav {traversal}")
    assert info["unrecovered"] == 0


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (8, 4), (11, 5)])
@pytest.mark.parametrize("window", [0, 4, 6])
@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_every_gate_kind_many_tiles(n, seed, window, precision):
    # all 16 gate kinds; small windows force many tiles and many passes, and
    # n below the window exercises the single-tile path
    circ = W.random_mixed(n, 40, seed, p1=3e-2, p2=6e-2)
    ref, _ = oracle.run(circ, 3000, seed, prune=False)
    pl = T.plan(circ, 3000, seed, prune=False)
    for trav in TRAVERSALS:
        got, info = gpu_run(pl, precision=precision, traversal=trav, max_window=window)
        assert_close(got, ref, precision, f"n {n} window {window} trav {trav}")


@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_brickwork_and_qaoa_multi_tile(precision):
    for circ, shots in [(W.brickwork(16, 12, 2, 2e-3, 2e-2), 20_000),
                        (W.qaoa_3regular(18, 3, 4, 1e-3, 1e-2), 20_000)]:
        ref, _ = oracle.run(circ, shots, 1)
        pl = T.plan(circ, shots, 1)
        for trav in TRAVERSALS:
            got, _ = gpu_run(pl, precision=precision, traversal=trav)
            assert_close(got, ref, precision, f"{circ.name} trav {trav}")


def test_degenerate_circuits():
    # no gates at all; noiseless circuit (a single instance); one qubit
    c0 = W.Circuit(3)
    pl = T.plan(c0, 100, 0)
    got, _ = gpu_run(pl, precision=T.C128)
    want = np.zeros(8)
    want[0] = 1
    assert_close(got, want, T.C128)
    c1 = W.random_layers(7, 6, 1, 0.0, 0.0)
    ref, _ = oracle.run(c1, 1000, 0)
    got, info = gpu_run(T.plan(c1, 1000, 0), precision=T.C128)
    assert_close(got, ref, T.C128)
    assert info["leaf_passes"] == 1
    c2 = W.Circuit(1)
    c2.add(W.H, 0, channel=W.depolarizing_1q(0.3))
    c2.add(W.RZ, 0, params=(0.3,), channel=W.depolarizing_1q(0.3))
    c2.add(W.H, 0, channel=W.depolarizing_1q(0.3))
    ref, _ = oracle.run(c2, 5000, 2, prune=False)
    for trav in TRAVERSALS:
        got, _ = gpu_run(T.plan(c2, 5000, 2, prune=False), precision=T.C128, traversal=trav)
        assert_close(got, ref, T.C128)


@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_dftt_counts_match_plan(precision):
    # with no root resets and no leaf peek, DFTT applies exactly 2|E| - G
    # gates (Sec. III-B1) and the plan's Pauli count; from scratch N_l * G
    circ = W.random_layers(6, 20, 0)
    pl = T.plan(circ, 10_000, 0, prune=False)
    st = pl.stats()
    _, info = gpu_run(pl, precision=precision, traversal=T.DFTT, root_reset=0, leaf_peek=0)
    assert info["gate_apps"] == st["dftt_gate_apps"]
    assert info["pauli_apps"] == st["dftt_pauli_apps"]
    _, info = gpu_run(pl, precision=precision, traversal=T.FROM_SCRATCH)
    assert info["gate_apps"] == st["scratch_gate_apps"]
    assert info["pauli_apps"] == st["scratch_pauli_apps"]


@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_drift_path_forced(precision):
    # tolerance 0: every check after an uncompute restores the branch node
    # from its snapshot; the answer is unchanged
    circ = W.brickwork(12, 10, 3, 2e-3, 2e-2)
    ref, _ = oracle.run(circ, 20_000, 5)
    pl = T.plan(circ, 20_000, 5)
    got, info = gpu_run(pl, precision=precision, traversal=T.DFTT, drift_tol=0.0)
    assert info["checks"] > 0
    assert info["restores"] == info["checks"]
    assert info["unrecovered"] == 0
    assert_close(got, ref, precision)


def test_drift_path_record_bias_and_no_snapshot():
    import torch
    circ = W.brickwork(10, 8, 3, 2e-3, 2e-2)
    pl = T.plan(circ, 20_000, 5)
    ref, _ = oracle.run(circ, 20_000, 5)
    # a host-side bias on the recorded norms forces every check to fail
    ex = T.Exec(pl, T.run_opts(precision=T.C64, traversal=T.DFTT))
    ex.set_record_bias(1e-3)
    probs = torch.empty(1 << 10, dtype=torch.float64, device="cuda")
    ex.launch(probs.data_ptr())
    info = ex.finish()
    assert info["restores"] == info["checks"] > 0
    assert_close(probs.cpu().numpy(), ref, T.C64)
    # with no snapshot budget a failed check cannot be repaired: EDRIFT
    ex = T.Exec(pl, T.run_opts(precision=T.C64, traversal=T.DFTT, snapshot_bytes=1))
    ex.set_record_bias(1e-3)
    ex.launch(probs.data_ptr())
    with pytest.raises(T.TusqError) as e:
        ex.finish()
    assert e.value.code == T.TUSQ_EDRIFT


def test_c64_vs_c128_brickwork():
    # the complex64 engine against the complex128 engine and the oracle
    circ = W.brickwork(20, 10, 0, 1e-3, 1e-2)
    pl = T.plan(circ, 100_000, 0)
    a, _ = gpu_run(pl, precision=T.C64, traversal=T.DFTT_SNAPSHOT)
    b, _ = gpu_run(pl, precision=T.C128, traversal=T.DFTT_SNAPSHOT)
    assert_close(a, b, T.C64)
    # the oracle plans its own instances (no oracle input from the library)
    opl = oracle.plan(circ, 100_000, 0)
    inst = [[tuple(int(v) for v in e) for e in ev] for ev in opl.inst[:4]]
    w = np.asarray(opl.weights[:4])
    ref = oracle.run_instances(circ, inst, w)
    sub = T.tusq_plan_from_instances(T.circuit_from(circ), inst, w)
    got, _ = gpu_run(sub, precision=T.C128)
    assert_close(got, ref, T.C128)



@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_graph_replay_equals_direct_launches(precision):
    # use_graph: the first launch captures the traversal into a CUDA graph on a
    # side stream, later launches replay it; a new output buffer re-captures
    import torch
    circ = W.brickwork(12, 10, 3, 2e-3, 2e-2)
    pl = T.plan(circ, 20_000, 2)
    ref, _ = oracle.run(circ, 20_000, 2)
    side = torch.cuda.Stream()
    direct = torch.empty(1 << 12, dtype=torch.float64, device="cuda")
    ex0 = T.Exec(pl, T.run_opts(precision=precision, traversal=T.DFTT), side.cuda_stream)
    ex0.launch(direct.data_ptr(), side.cuda_stream)
    ex0.finish()
    ex = T.Exec(pl, T.run_opts(precision=precision, traversal=T.DFTT, use_graph=1), side.cuda_stream)
    outs = [torch.full((1 << 12,), -1.0, dtype=torch.float64, device="cuda") for _ in range(2)]
    for o in (outs[0], outs[0], outs[1], outs[0]):
        ex.launch(o.data_ptr(), side.cuda_stream)
        info = ex.finish()
        assert info["unrecovered"] == 0
    for o in outs:
        assert torch.equal(o, direct)
    assert_close(direct.cpu().numpy(), ref, precision, "graph replay")


@pytest.mark.parametrize("precision", [T.C128, T.C64])
@pytest.mark.parametrize("prune", [True, False])
def test_terminal_fold_matches_oracle(precision, prune):
    # readout fold on: Z at slot G dropped, Y there turned into X; the kept
    # instances and their weights are the oracle's, and without pruning the
    # output equals the unfolded one
    circ = W.qaoa_3regular(12, 2, 5, 5e-3, 2e-2)
    ref, _ = oracle.run(circ, 20_000, 3, prune=prune, terminal_fold=True)
    got, info = gpu_run(T.plan(circ, 20_000, 3, prune=prune, terminal_fold=True), precision=precision,
                        traversal=T.DFTT_SNAPSHOT)
    assert_close(got, ref, precision, "fold")
    if not prune:
        plain, _ = gpu_run(T.plan(circ, 20_000, 3, prune=False), precision=precision, traversal=T.DFTT_SNAPSHOT)
        assert_close(got, plain, precision, "fold vs plain")
