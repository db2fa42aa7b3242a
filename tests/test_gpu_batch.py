"""Batched jobs (one persistent launch, state in shared memory) against the
oracle and against the per-job engine; CUDA-graph replay; autotuner."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu

TOL = {T.C128: (1e-12, 1e-10), T.C64: (1e-5, 1e-4)}


def _jobs():
    return [
        (W.random_layers(6, 20, 0, 1e-3, 1e-2), 10_000, 0),
        (W.brickwork(9, 12, 1, 2e-3, 2e-2), 20_000, 1),
        (W.qaoa_3regular(10, 2, 2, 1e-3, 1e-2), 20_000, 2),
        (W.random_mixed(7, 60, 3, 1e-2, 3e-2), 5_000, 3),
        (W.brickwork(12, 20, 4, 1e-3, 1e-2), 50_000, 4),
        (W.qaoa_3regular(12, 3, 5, 1e-3, 1e-2), 50_000, 5),
        (W.random_layers(5, 3, 6, 0.0, 0.0), 100, 6),
    ]


def _close(a, b, precision, what=""):
    ma, tv = TOL[precision]
    d = np.abs(a - b)
    assert d.max() <= ma and d.sum() <= tv, (what, d.max(), d.sum())


@pytest.mark.parametrize("precision", [T.C128, T.C64])
@pytest.mark.parametrize("traversal", [T.DFTT, T.DFTT_SNAPSHOT, T.FROM_SCRATCH])
def test_batch_matches_oracle(precision, traversal):
    import torch
    jobs = _jobs()
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    b = T.Batch(plans, [o.data_ptr() for o in outs], T.run_opts(precision=precision, traversal=traversal))
    b.launch()
    info = b.finish()
    assert info["unrecovered"] == 0
    for (c, s, seed), o in zip(jobs, outs):
        ref, _ = oracle.run(c, s, seed)
        _close(o.cpu().numpy(), ref, precision, c.name)


def test_batch_graph_replay_and_forced_drift():
    import torch
    jobs = _jobs()
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = T.Batch(plans, [o.data_ptr() for o in outs], T.run_opts(precision=T.C128, drift_tol=0.0),
                    use_graph=True, stream=stream.cuda_stream)
        first = None
        for _ in range(3):
            for o in outs:
                o.fill_(7.0)
            b.launch(stream.cuda_stream)
            info = b.finish()
            cur = [o.cpu().numpy() for o in outs]
            if first is None:
                first = cur
            for a, c in zip(first, cur):
                assert np.array_equal(a, c)        # replays are bit-identical
    # tolerance 0: every check whose drift is not exactly zero restores
    assert info["checks"] > 0 and 0 < info["restores"] <= info["checks"]
    for (c, s, seed), o in zip(jobs, first):
        ref, _ = oracle.run(c, s, seed)
        _close(o, ref, T.C128, c.name)


def test_batch_equals_single_job_engine():
    import torch
    jobs = _jobs()
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    opts = T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT)
    b = T.Batch(plans, [o.data_ptr() for o in outs], opts)
    b.launch()
    b.finish()
    for p, o in zip(plans, outs):
        single, _ = T.run_torch(p, opts)
        _close(o.cpu().numpy(), single.cpu().numpy(), T.C64)


def test_batch_autotune_and_size_limits():
    import torch
    jobs = _jobs()
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    best, ms = T.tusq_batch_autotune(plans, [o.data_ptr() for o in outs], T.run_opts(precision=T.C64))
    assert ms > 0 and best.traversal in (T.DFTT, T.FROM_SCRATCH, T.DFTT_SNAPSHOT) and best.schedule in (0, 1)
    assert best.group_ctas in (0, 4, 8, 16)
    # group jobs go up to 22 qubits; a 23-qubit job is refused before any allocation
    big = T.plan(W.brickwork(23, 1, 0, 0.0, 0.0), 10, 0)
    with pytest.raises(T.TusqError):
        T.Batch([big], [0x1000], T.run_opts(precision=T.C64))


def _mixed_jobs():
    # single-CTA jobs and group jobs (14-18 qubits: 2-32 tiles of 2^13
    # amplitudes, groups of 2-16 CTAs, state in global memory) in one launch
    return [
        (W.brickwork(14, 8, 11, 2e-3, 2e-2), 5_000, 11),
        (W.qaoa_3regular(16, 2, 12, 1e-3, 1e-2), 5_000, 12),
        (W.random_layers(6, 20, 13, 1e-3, 1e-2), 5_000, 13),
        (W.brickwork(18, 6, 14, 2e-3, 2e-2), 3_000, 14),
        (W.brickwork(12, 10, 15, 1e-3, 1e-2), 10_000, 15),
        (W.qaoa_3regular(14, 3, 16, 1e-3, 1e-2), 10_000, 16),
    ]


@pytest.fixture(scope="module")
def mixed_refs():
    jobs = _mixed_jobs()
    return jobs, [oracle.run(c, s, seed)[0] for c, s, seed in jobs]


@pytest.mark.parametrize("precision", [T.C64, T.C128])
@pytest.mark.parametrize("traversal", [T.DFTT, T.DFTT_SNAPSHOT])
def test_group_jobs_match_oracle(mixed_refs, precision, traversal):
    import torch
    jobs, refs = mixed_refs
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    b = T.Batch(plans, [o.data_ptr() for o in outs], T.run_opts(precision=precision, traversal=traversal))
    assert b.group_jobs() == sum(1 for c, _, _ in jobs if c.n_qubits > (12 if precision == T.C128 else 13))
    b.launch()
    info = b.finish()
    assert info["unrecovered"] == 0
    for (c, s, seed), o, ref in zip(jobs, outs, refs):
        _close(o.cpu().numpy(), ref, precision, c.name)


def test_group_jobs_graph_replay_and_bounded_barrier():
    # replayed from a CUDA graph: the same result every time; then the test
    # hook makes every group barrier wait for one member too many -- a
    # dependency that never resolves -- so the bounded waits run out and the
    # batch reports TUSQ_ETIMEOUT; with the hook off it runs normally again
    import torch
    jobs = _mixed_jobs()
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = T.Batch(plans, [o.data_ptr() for o in outs], T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT),
                    use_graph=True, stream=stream.cuda_stream)
        first = None
        for _ in range(3):
            b.launch(stream.cuda_stream)
            b.finish()
            now = [o.cpu().numpy() for o in outs]
            if first is None:
                first = now
            for a_, c_ in zip(first, now):
                assert np.array_equal(a_, c_)
        b.set_stall_test(True)
        b.launch(stream.cuda_stream)
        with pytest.raises(T.TusqError) as e:
            b.finish()
        assert e.value.code == T.TUSQ_ETIMEOUT
        b.set_stall_test(False)
        b.launch(stream.cuda_stream)
        b.finish()
        for a_, o in zip(first, outs):
            assert np.array_equal(a_, o.cpu().numpy())


# tensor-core dense ops in the batch: 13-qubit single-CTA jobs (the whole
# state is the tile) and group jobs (13-qubit tiles in global memory), held to
# the split modes' complex64 bound against the oracle
TC_BOUND = (1e-5, 1e-4)


@pytest.fixture(scope="module")
def tc_refs():
    jobs = [(W.brickwork(13, 10, 21, 1e-3, 1e-2), 5_000, 21),
            (W.brickwork(15, 8, 22, 1e-3, 1e-2), 5_000, 22),
            (W.qaoa_3regular(12, 2, 23, 1e-3, 1e-2), 5_000, 23),
            (W.brickwork(16, 6, 24, 2e-3, 2e-2), 3_000, 24),
            (W.brickwork(9, 12, 25, 1e-3, 1e-2), 5_000, 25)]
    return jobs, [oracle.run(c, s, seed)[0] for c, s, seed in jobs]


@pytest.mark.parametrize("mode", [T.TC_BF16X3, T.TC_TF32X3])
def test_batch_dense_stages_match_oracle(tc_refs, mode):
    import torch
    jobs, refs = tc_refs
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    b = T.Batch(plans, [o.data_ptr() for o in outs],
                T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT, tc_mode=mode))
    assert b.group_jobs() == 2
    b.launch()
    info = b.finish()
    assert info["dense_ops"] > 0 and info["unrecovered"] == 0
    for (c, s, seed), o, ref in zip(jobs, outs, refs):
        d = np.abs(o.cpu().numpy() - ref)
        assert d.max() <= TC_BOUND[0] and d.sum() <= TC_BOUND[1], (mode, c.name, d.max(), d.sum())
