"""Streamed traversal (tusq_run_streamed) of a wide, unpruned instance tree:
the DFS order cut into chunks whose device programs are compiled on host
threads ahead of the GPU (Sec. III-B subtree cut), all chunks adding into one
output.  Lossless tree: the result is the tally-weighted mixture of every
distinct instance, which the oracle computes from its own plan, instance by
instance from |0..0>."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wide():
    circ = W.random_layers(10, 20, 4, 1e-3, 1e-2)
    ref, opl = oracle.run(circ, 40_000, 4, prune=False)
    pl = T.plan(circ, 40_000, 4, prune=False)
    assert pl.stats()["n_instances"] == len(opl.inst) >= 10_000
    return circ, pl, ref


@pytest.mark.parametrize("precision,tol", [(T.C64, (1e-5, 1e-4)), (T.C128, (1e-12, 1e-10))])
def test_streamed_chunks_match_oracle(wide, precision, tol):
    import torch
    circ, pl, ref = wide
    probs = torch.empty(1 << circ.n_qubits, dtype=torch.float64, device="cuda")
    info = T.tusq_run_streamed(pl, probs.data_ptr(), 1024,
                               T.run_opts(precision=precision, traversal=T.DFTT_SNAPSHOT), compile_threads=4,
                               stream=torch.cuda.current_stream().cuda_stream)
    d = np.abs(probs.cpu().numpy() - ref)
    assert d.max() <= tol[0] and d.sum() <= tol[1], (d.max(), d.sum())
    assert info["leaf_passes"] == pl.stats()["n_instances"] and info["unrecovered"] == 0


def test_streamed_equals_one_traversal_up_to_rounding(wide):
    import torch
    circ, pl, ref = wide
    st = torch.cuda.current_stream().cuda_stream
    one, _ = T.run_torch(pl, T.run_opts(precision=T.C128, traversal=T.DFTT_SNAPSHOT))
    probs = torch.empty_like(one)
    T.tusq_run_streamed(pl, probs.data_ptr(), 3000, T.run_opts(precision=T.C128, traversal=T.DFTT),
                        compile_threads=2, stream=st)
    assert float((probs - one).abs().max()) <= 1e-12
