"""GPU shot sampling (tusq_sample, through the C ABI) against the oracle's
sampler, bit for bit: both draw shot s from Philox4x64-10 at counter
(s, 0, 0, 0), key (seed, 3), and land it by the inverse transform on
integer cumulative weights floor(p 2^56), so the counts must be identical
whatever order the device sums the weights in."""
import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

pytestmark = pytest.mark.gpu


def _gpu_counts(p, shots, seed):
    import torch
    probs = torch.from_numpy(np.ascontiguousarray(p, dtype=np.float64)).cuda()
    counts = T.sample_torch(probs, shots, seed)
    torch.cuda.synchronize()
    return counts.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("n", [0, 1, 3, 12, 13, 17])
def test_counts_match_oracle_on_random_distributions(n):
    # sizes below, at and across the 4096-outcome scan chunk, plus a ragged
    # tail of zeros and a negative rounding residue
    rng = np.random.default_rng(n)
    p = rng.dirichlet(np.ones(1 << n) * 0.3)
    if n >= 3:
        p[rng.integers(0, 1 << n, max(1, (1 << n) // 8))] = 0.0
        p[-1] = -1e-18
    for shots, seed in [(1, 0), (10_000, 1), (200_003, 7)]:
        got = _gpu_counts(p, shots, seed)
        want = oracle.sample(p, shots, seed)
        np.testing.assert_array_equal(got, want)


def test_counts_match_oracle_on_an_engine_output():
    circ = W.qaoa_3regular(16, 3, 4, 1e-3, 1e-2)
    probs, _ = T.run_torch(T.plan(circ, 20_000, 1), T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT))
    import torch
    torch.cuda.synchronize()
    counts = T.sample_torch(probs, 1_000_000, 42)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64),
                                  oracle.sample(probs.cpu().numpy(), 1_000_000, 42))


def test_point_mass_zero_shots_and_empty_distribution():
    p = np.zeros(1 << 10)
    p[777] = 0.5
    got = _gpu_counts(p, 5000, 3)
    assert got[777] == 5000 and got.sum() == 5000
    assert _gpu_counts(p, 0, 3).sum() == 0
    with pytest.raises(T.TusqError):
        _gpu_counts(np.zeros(8), 10, 0)
