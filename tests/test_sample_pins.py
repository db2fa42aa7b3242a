"""Pins of the oracle's shot sampler (shots drawn from the output
distribution; the paper samples each kept instance's state vector s_i times,
Sec. III-A1).  The draws come from Philox4x64-10 at counter (s, 0, 0, 0),
key (seed, 3); the pins check the sampler against numpy's independent
Philox on distributions whose inverse transform has a closed form, and
against the multinomial law."""
import numpy as np
import pytest
import scipy.stats

import oracle
from tests.test_oracle_pins import _numpy_philox


def _draws(seed, shots):
    return [_numpy_philox([s, 0, 0, 0], [seed, 3])[0] for s in range(shots)]


def test_draw_definition():
    for seed, s in [(0, 0), (1, 7), (2 ** 40, 12345)]:
        assert oracle.draw_sample(seed, s) == _numpy_philox([s, 0, 0, 0], [seed, 3])[0]


@pytest.mark.parametrize("k", [1, 2, 5])
def test_uniform_lands_on_the_top_bits_of_each_draw(k):
    # equal weights 2^-k: the cumulative weights are multiples of 2^(56-k), so
    # a shot lands on the outcome given by the top k bits of its draw
    shots, seed = 3000, 11
    counts = oracle.sample(np.full(1 << k, 2.0 ** -k), shots, seed)
    want = np.bincount([r >> (64 - k) for r in _draws(seed, shots)], minlength=1 << k)
    np.testing.assert_array_equal(counts, want)


def test_two_point_split_at_a_dyadic_cut():
    # p = (1/4, 3/4): outcome 0 iff the draw is below 2^62
    shots, seed = 2000, 5
    counts = oracle.sample(np.array([0.25, 0.75]), shots, seed)
    low = sum(r < (1 << 62) for r in _draws(seed, shots))
    assert counts[0] == low and counts[1] == shots - low


def test_point_mass_and_zero_outcomes():
    p = np.zeros(64)
    p[37] = 1.0
    counts = oracle.sample(p, 500, 2)
    assert counts[37] == 500 and counts.sum() == 500
    # outcomes of probability 0 are never drawn; negative entries count as 0
    q = np.zeros(16)
    q[[1, 4, 9]] = [0.2, 0.3, 0.5]
    q[3] = -1e-9
    c = oracle.sample(q, 4000, 3)
    assert c.sum() == 4000 and set(np.nonzero(c)[0]) <= {1, 4, 9}


def test_counts_follow_the_multinomial_law():
    rng = np.random.default_rng(4)
    p = rng.dirichlet(np.ones(32))
    shots = 200_000
    counts = oracle.sample(p, shots, 9)
    assert counts.sum() == shots
    chi2 = ((counts - shots * p) ** 2 / (shots * p)).sum()
    assert scipy.stats.chi2.sf(chi2, 31) > 1e-4


def test_unnormalised_input_is_sampled_in_proportion():
    # a distribution off by a rounding-size factor samples like the normalised one
    rng = np.random.default_rng(6)
    p = rng.dirichlet(np.ones(8))
    a = oracle.sample(p, 50_000, 1)
    b = oracle.sample(p * (1 + 1e-12), 50_000, 1)
    assert np.abs(a.astype(np.int64) - b.astype(np.int64)).sum() <= 4


def test_empty_distribution_is_an_error():
    with pytest.raises(ValueError):
        oracle.sample(np.zeros(4), 10, 0)
