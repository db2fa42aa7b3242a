"""Parallel-subtree DFTT on one GPU (run option `subtrees`, Sec. III-B):
the DFS order cut into k chunks traversed concurrently on k streams, the
chunks' FP64 outputs summed in a fixed order.  The result must match the
oracle and the single traversal within the parity tolerances, for every
traversal, with CUDA-graph replay, with mid-circuit resets, and when k
exceeds the number of leaves."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

TOL = {T.C128: (1e-12, 1e-10), T.C64: (1e-5, 1e-4)}


def close(got, ref, precision, what=""):
    ma, tv = TOL[precision]
    d = np.abs(got - ref)
    assert d.max() <= ma and d.sum() <= tv, (what, d.max(), d.sum())


def test_option_range_checked_on_the_host():
    pl = T.plan(W.random_layers(4, 3, 1, 1e-2, 1e-2), 1000, 0)
    T.tusq_compile_stats(pl, T.run_opts(subtrees=16))
    T.tusq_compile_stats(pl, T.run_opts(subtrees=-1))
    for bad in (17, -2):
        with pytest.raises(T.TusqError):
            T.tusq_compile_stats(pl, T.run_opts(subtrees=bad))


@pytest.mark.parametrize("maker,shots", [
    (lambda: W.brickwork(8, 10, 3, 5e-3, 3e-2), 20_000),
    (lambda: W.repetition_memory(3, 2, 1, 2e-2, 3e-2, 2e-2), 4000),
])
@pytest.mark.parametrize("k", [2, 5])
def test_chunk_programs_sum_to_the_oracle(maker, shots, k):
    # the host side of the subtree cut: each chunk's device program
    # (interpreted on the host) starts from |0..0>, and the chunks' outputs
    # add up to the whole distribution
    from tests.test_schedule_emulated import emu_run
    c = maker()
    ref, _ = oracle.run(c, shots, 3)
    pl = T.plan(c, shots, 3)
    total = np.zeros(1 << c.n_qubits)
    for r in range(k):
        got, _ = emu_run(pl.shard(r, k), precision=T.C128, traversal=T.DFTT, drift_tol=-1.0)
        total += got
    assert np.abs(total - ref).max() < 1e-12


def _gpu(plan, **kw):
    import torch
    probs, info = T.run_torch(plan, T.run_opts(**kw))
    torch.cuda.synchronize()
    return probs.cpu().numpy(), info


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [T.C128, T.C64])
@pytest.mark.parametrize("traversal", [T.DFTT, T.DFTT_SNAPSHOT, T.FROM_SCRATCH])
def test_matches_oracle_and_single_traversal(precision, traversal):
    c = W.brickwork(14, 12, 3, 2e-3, 2e-2)
    ref, _ = oracle.run(c, 50_000, 1)
    pl = T.plan(c, 50_000, 1)
    single, info1 = _gpu(pl, precision=precision, traversal=traversal)
    for k in (2, 3, 4):
        got, info = _gpu(pl, precision=precision, traversal=traversal, subtrees=k)
        close(got, ref, precision, f"k {k}")
        close(got, single, precision, f"k {k} vs single")
        assert info["leaf_passes"] == info1["leaf_passes"] and info["unrecovered"] == 0


@pytest.mark.gpu
def test_more_chunks_than_leaves_and_resets():
    c = W.repetition_memory(3, 2, 1, 2e-2, 3e-2, 2e-2)
    ref, _ = oracle.run(c, 4000, 3)
    got, _ = _gpu(T.plan(c, 4000, 3), precision=T.C128, traversal=T.DFTT, drift_tol=-1.0, subtrees=5)
    close(got, ref, T.C128)
    tiny = W.Circuit(2)
    tiny.add(W.H, 0, channel=((3,), (0.5,)))
    tiny.add(W.RX, 0, params=(0.4,))
    pl = T.plan(tiny, 1000, 0, prune=False)
    assert pl.stats()["n_instances"] == 2
    ref, _ = oracle.run(tiny, 1000, 0, prune=False)
    got, _ = _gpu(pl, precision=T.C128, subtrees=8)
    close(got, ref, T.C128)


@pytest.mark.gpu
def test_graph_replay_with_subtrees():
    import torch
    c = W.qaoa_3regular(14, 2, 4, 2e-3, 1e-2)
    pl = T.plan(c, 50_000, 2)
    side = torch.cuda.Stream()
    direct = torch.empty(1 << 14, dtype=torch.float64, device="cuda")
    ex0 = T.Exec(pl, T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT, subtrees=3), side.cuda_stream)
    ex0.launch(direct.data_ptr(), side.cuda_stream)
    ex0.finish()
    ex = T.Exec(pl, T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT, subtrees=3, use_graph=1),
                side.cuda_stream)
    out = torch.full((1 << 14,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ex.launch(out.data_ptr(), side.cuda_stream)
        ex.finish()
        assert torch.equal(out, direct)
    ref, _ = oracle.run(c, 50_000, 2)
    close(direct.cpu().numpy(), ref, T.C64)


@pytest.mark.gpu
@pytest.mark.parametrize("k", [8, 16])
def test_six_qubit_configuration_with_many_chunks(k):
    # the 6-qubit benchmark configuration (complex128, uncompute traversal
    # with drift checks) as 8 and 16 concurrent chunks, graph-replayed
    import torch
    c = W.random_layers(6, 20, 0, 1e-3, 1e-2)
    ref, _ = oracle.run(c, 10_000, 0)
    pl = T.plan(c, 10_000, 0)
    side = torch.cuda.Stream()
    out = torch.empty(1 << 6, dtype=torch.float64, device="cuda")
    ex = T.Exec(pl, T.run_opts(precision=T.C128, traversal=T.DFTT, subtrees=k, use_graph=1), side.cuda_stream)
    for _ in range(2):
        ex.launch(out.data_ptr(), side.cuda_stream)
        info = ex.finish()
        assert info["unrecovered"] == 0
        close(out.cpu().numpy(), ref, T.C128, f"k {k}")


@pytest.mark.gpu
@pytest.mark.parametrize("n", [6, 12, 18])
def test_automatic_chunk_count(n):
    c = W.brickwork(n, 8, n, 2e-3, 2e-2)
    ref, _ = oracle.run(c, 20_000, 4)
    pl = T.plan(c, 20_000, 4)
    for precision in (T.C128, T.C64):
        got, info = _gpu(pl, precision=precision, traversal=T.DFTT_SNAPSHOT, subtrees=-1)
        close(got, ref, precision, f"n {n}")
        # the rule: chunks until the passes in flight offer about twice the
        # CTA slots, at most 16 -- a 6-qubit pass is one tile (16 chunks), a
        # 23-qubit complex64 pass already has 1024 tiles (one chunk)
        if n == 6:
            assert info["chunks"] == 16, info["chunks"]
        if n == 18:
            # 32 complex64 tiles of 2^13 (2 CTAs per SM) or 64 complex128 tiles
            # of 2^12 (1 CTA per SM) against 148 SMs
            assert info["chunks"] == (16 if precision == T.C64 else 5), (precision, info["chunks"])


@pytest.mark.gpu
def test_automatic_chunk_count_one_chunk_at_23_qubits():
    # a 23-qubit complex64 pass has 1024 tiles, more than twice the CTA
    # slots: the automatic rule keeps one traversal
    import torch
    c = W.brickwork(23, 2, 3, 0.0, 0.0)
    pl = T.tusq_plan_from_instances(T.circuit_from(c), [[], [(0, 0, 1)]], np.array([0.5, 0.5]))
    got, info = _gpu(pl, precision=T.C64, traversal=T.DFTT_SNAPSHOT, subtrees=-1)
    assert info["chunks"] == 1
    assert abs(float(np.sum(got)) - 1.0) < 1e-5
