"""The allocation-free entry point (tusq_run_noalloc) through the C ABI.

It serves callers that cannot call cudaMalloc (an application whose device
memory is owned by its own pool allocator, a plugin host that only lends
out its own buffers): all scratch lives in the library's static device
array.  Its output must equal the allocating entry point's (tusq_run) on
the same plan, within the parity tolerances, on two calls in a row (the
array keeps the previous call's contents, so the second call checks that
everything that must start at zero is cleared).  This file is collected
last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu

TOL = {T.C128: (1e-12, 1e-10), T.C64: (1e-5, 1e-4)}


def _close(a, b, precision):
    ma, tv = TOL[precision]
    d = np.abs(a - b)
    assert d.max() <= ma and d.sum() <= tv, (d.max(), d.sum())


@pytest.mark.parametrize("precision,traversal", [(T.C128, T.DFTT), (T.C64, T.DFTT_SNAPSHOT),
                                                 (T.C64, T.DFTT), (T.C128, T.FROM_SCRATCH)])
def test_noalloc_matches_tusq_run_twice(precision, traversal):
    import torch
    circ = W.brickwork(16, 10, 3, 2e-3, 2e-2)
    plan = T.plan(circ, 50_000, 7)
    opts = T.run_opts(precision=precision, traversal=traversal)
    ref = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
    T.tusq_run(plan, ref.data_ptr(), opts, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(123.0)                        # stale output must not leak through
        info = T.tusq_run_noalloc(plan, out.data_ptr(), opts, torch.cuda.current_stream().cuda_stream)
        assert info["unrecovered"] == 0
        _close(out.cpu().numpy(), ref_h, precision)


def test_noalloc_rejects_states_beyond_the_scratch():
    import torch
    circ = W.brickwork(22, 1, 0, 0.0, 0.0)      # 2^22 complex64 = 32 MiB: more than half the scratch
    plan = T.plan(circ, 10, 0)
    out = torch.empty(1 << 22, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TusqError) as e:
        T.tusq_run_noalloc(plan, out.data_ptr(), T.run_opts(precision=T.C64))
    assert e.value.code == T.TUSQ_EINVAL
    assert "static scratch" in str(e.value)


@pytest.mark.parametrize("traversal", [T.DFTT, T.DFTT_SNAPSHOT])
def test_noalloc_with_mid_circuit_resets(traversal):
    # non-invertible gates: the allocation-free path keeps no cache and
    # re-derives across a reset from the saved states it has, or from |0..0>
    import torch
    circ = W.mcm_brickwork(10, 8, 2, 1, 7, 2e-3, 1e-2)     # 404 leaves, ~5 MB device program
    plan = T.plan(circ, 20_000, 1)
    opts = T.run_opts(precision=T.C128, traversal=traversal, drift_tol=-1.0)
    ref = torch.empty(1 << 10, dtype=torch.float64, device="cuda")
    T.tusq_run(plan, ref.data_ptr(), opts, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out = torch.empty_like(ref)
    T.tusq_run_noalloc(plan, out.data_ptr(), opts, torch.cuda.current_stream().cuda_stream)
    _close(out.cpu().numpy(), ref.cpu().numpy(), T.C128)
