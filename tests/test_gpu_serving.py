"""Serving loop: continuous batching of jobs under an HBM budget.  Each
job's result is the same alone and in the mix; oversize jobs are refused at
admission; latencies are reported."""
import numpy as np
import pytest

import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu


def _jobs():
    return [(W.brickwork(14, 10, j, 2e-3, 2e-2), 20_000, j) if j % 2 else
            (W.qaoa_3regular(16, 2, j, 1e-3, 1e-2), 20_000, j) for j in range(10)]


@pytest.mark.parametrize("precision", [T.C64, T.C128])
def test_results_alone_equal_results_in_the_mix(precision):
    import torch
    opts = T.run_opts(precision=precision, traversal=T.DFTT_SNAPSHOT)
    jobs = _jobs()
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    alone = []
    for p in plans:
        out, _ = T.run_torch(p, opts)
        alone.append(out.cpu().numpy())
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    # a budget that fits only a few jobs at a time: later ones wait for slots
    fp = (16 if precision == T.C128 else 8) << 16
    srv = T.Server(hbm_budget_bytes=4 * 9 * fp + (8 << 20), n_streams=4)
    ids = [srv.submit(p, o.data_ptr(), opts) for p, o in zip(plans, outs)]
    srv.drain()
    for i, (jid, o, a) in enumerate(zip(ids, outs, alone)):
        done, lat = srv.poll(jid)
        assert done and lat > 0
        assert np.array_equal(o.cpu().numpy(), a), i       # same kernels, same order: bit-identical


def test_admission_refuses_oversize_job():
    import torch
    p = T.plan(W.brickwork(20, 2, 0, 1e-3, 1e-2), 1000, 0)
    o = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    srv = T.Server(hbm_budget_bytes=1 << 20, n_streams=2)
    with pytest.raises(T.TusqError) as e:
        srv.submit(p, o.data_ptr())
    assert e.value.code == T.TUSQ_ENOMEM_ADMIT


def test_admitted_jobs_overlap_on_the_device():
    # a job admitted while another runs executes concurrently with it: their
    # traversals' device intervals (CUDA events on their streams) overlap.
    # 16-qubit passes have 8 tiles each, so one job leaves most of the GPU
    # idle for the other.  The short job is submitted once the long one is
    # running (about 6600 passes, ~0.5 s on the device), so the outcome does
    # not depend on how fast the host compiles.
    import time
    import torch
    opts = T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT)
    long_plan = T.plan(W.brickwork(16, 30, 0, 2e-3, 2e-2), 50_000, 0, beta=1000)
    short_plan = T.plan(W.brickwork(16, 30, 1, 2e-3, 2e-2), 50_000, 1)
    outs = [torch.empty(1 << 16, dtype=torch.float64, device="cuda") for _ in range(2)]
    srv = T.Server(hbm_budget_bytes=1 << 34, n_streams=2)
    a = srv.submit(long_plan, outs[0].data_ptr(), opts)
    seen = set()
    t0 = time.monotonic()
    while srv.state(a) != T.JOB_RUNNING:
        seen.add(srv.state(a))
        assert srv.state(a) != T.JOB_DONE and time.monotonic() - t0 < 120
        time.sleep(0.001)
    assert seen <= {T.JOB_COMPILING, T.JOB_READY}
    b = srv.submit(short_plan, outs[1].data_ptr(), opts)
    srv.drain()
    assert srv.state(a) == T.JOB_DONE and srv.state(b) == T.JOB_DONE
    with pytest.raises(T.TusqError) as e:
        srv.state(b + 1000)
    assert e.value.code == T.TUSQ_ENOTFOUND
    (a0, a1), (b0, b1) = srv.device_interval(a), srv.device_interval(b)
    assert 0 <= a0 < a1 and 0 <= b0 < b1 and a0 < b0
    overlap = min(a1, b1) - max(a0, b0)
    assert overlap > 0.5 * (b1 - b0), ((a0, a1), (b0, b1))
    # each job's result is the one it gets alone
    for pl, o in ((long_plan, outs[0]), (short_plan, outs[1])):
        alone, _ = T.run_torch(pl, opts)
        assert np.array_equal(o.cpu().numpy(), alone.cpu().numpy())
