"""GPU parity for mid-circuit RESET / MEASURE and DFTT+Caching (Sec. III-B2):
the CUDA engine (through the C ABI) against the oracle on the same plans,
for every traversal, cache capacity and drift-check setting; the batched
launch on the same circuits; graph replay; the uncompute traversal without
drift checks (leaf pass that skips its write)."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W
from tests.test_noninvertible import CIRCUITS, SETTINGS

pytestmark = pytest.mark.gpu

TOL = {T.C128: (1e-12, 1e-10), T.C64: (1e-5, 1e-4)}


def gpu_run(plan, **opts):
    import torch
    probs, info = T.run_torch(plan, T.run_opts(**opts))
    torch.cuda.synchronize()
    return probs.cpu().numpy(), info


def close(got, ref, precision, what=""):
    ma, tv = TOL[precision]
    d = np.abs(got - ref)
    assert d.max() <= ma and d.sum() <= tv, (what, d.max(), d.sum())


@pytest.mark.parametrize("name,maker,shots", CIRCUITS, ids=[c[0] for c in CIRCUITS])
@pytest.mark.parametrize("traversal,tol,nsnap", SETTINGS)
@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_matches_oracle(name, maker, shots, traversal, tol, nsnap, precision):
    c = maker()
    ref, _ = oracle.run(c, shots, 3)
    pl = T.plan(c, shots, 3)
    amp = 16 if precision == T.C128 else 8
    sb = (nsnap * amp << c.n_qubits) or amp
    for cache in (0, 1, -1):
        got, info = gpu_run(pl, precision=precision, traversal=traversal, drift_tol=tol, snapshot_bytes=sb,
                            cache_states=cache)
        close(got, ref, precision, f"cache {cache}")
        assert info["unrecovered"] == 0


@pytest.mark.parametrize("precision", [T.C128, T.C64])
@pytest.mark.parametrize("traversal", [T.DFTT, T.DFTT_SNAPSHOT])
def test_many_tiles(precision, traversal):
    # 12 qubits with 6-qubit windows: 64 tiles per pass and many passes
    c = W.mcm_brickwork(12, 10, 3, 2, 7, 2e-3, 1e-2)
    ref, _ = oracle.run(c, 20_000, 1)
    pl = T.plan(c, 20_000, 1)
    for cache in (0, 2):
        got, info = gpu_run(pl, precision=precision, traversal=traversal, drift_tol=-1.0, max_window=6,
                            cache_states=cache)
        close(got, ref, precision, f"cache {cache}")


def test_graph_replay_equals_direct():
    import torch
    c = W.repetition_memory(4, 2, 2, 1e-2, 2e-2, 1e-2)
    pl = T.plan(c, 20_000, 2)
    kw = dict(precision=T.C128, traversal=T.DFTT, drift_tol=-1.0, cache_states=1)
    side = torch.cuda.Stream()
    direct = torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda")
    ex0 = T.Exec(pl, T.run_opts(**kw), side.cuda_stream)
    ex0.launch(direct.data_ptr(), side.cuda_stream)
    ex0.finish()
    ex = T.Exec(pl, T.run_opts(use_graph=1, **kw), side.cuda_stream)
    out = torch.full((1 << c.n_qubits,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ex.launch(out.data_ptr(), side.cuda_stream)
        ex.finish()
        assert torch.equal(out, direct)
    ref, _ = oracle.run(c, 20_000, 2)
    close(direct.cpu().numpy(), ref, T.C128)


@pytest.mark.parametrize("traversal", [T.DFTT, T.DFTT_SNAPSHOT, T.FROM_SCRATCH])
def test_batch_matches_oracle(traversal):
    import torch
    # the batched launch takes jobs of 4..12 qubits (complex128)
    jobs = [(c, shots, 3) for c, shots in ((maker(), shots) for _, maker, shots in CIRCUITS) if c.n_qubits >= 4]
    plans = [T.plan(c, s, seed) for c, s, seed in jobs]
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c, _, _ in jobs]
    b = T.Batch(plans, [o.data_ptr() for o in outs],
                T.run_opts(precision=T.C128, traversal=traversal, drift_tol=-1.0, cache_states=1))
    b.launch()
    b.finish()
    for (c, s, seed), o in zip(jobs, outs):
        ref, _ = oracle.run(c, s, seed)
        close(o.cpu().numpy(), ref, T.C128, c.name)


@pytest.mark.parametrize("window", [0, 4])
def test_uncompute_without_drift_checks(window):
    # a plain circuit: the leaf pass that skips its write, with no branch
    # stack.  Complex128 only: in complex64 the thousands of unchecked
    # uncompute passes lose ~0.1% of the norm (measured: TV 1.2e-3 on this
    # circuit), which is what the drift checks are there to catch
    c = W.random_layers(8, 20, 0, 1e-2, 3e-2)
    ref, _ = oracle.run(c, 10_000, 3)
    got, _ = gpu_run(T.plan(c, 10_000, 3), precision=T.C128, traversal=T.DFTT, drift_tol=-1.0,
                     max_window=window)
    close(got, ref, T.C128)
