"""The oracle's posterior probabilities of contrasts (§3.1: means of indicators
of conjunctions of linear inequalities in beta_g) against hand counts, a
closed-form normal probability and the inclusion-exclusion rule the paper uses
for disjunctions."""
import numpy as np
from scipy import stats

import oracle


def test_hand_counted_trace():
    beta = np.array([[[1.0, 2.0], [0.0, -1.0]],
                     [[-3.0, 1.0], [2.0, 2.0]],
                     [[0.5, 0.5], [1.0, -2.0]]])          # M=3, G=2, L=2
    props = [[([1.0, 1.0], 0.0)],                          # b1 + b2 > 0
             [([1.0, 0.0], 0.0), ([0.0, 1.0], 0.0)],       # b1 > 0 and b2 > 0
             [([1.0, -1.0], 1.5)]]                         # b1 - b2 > 1.5
    p = oracle.contrast_probs(beta, props)
    # gene 0: sums 3, -2, 1 -> 2/3; both positive: it 1, 3 -> 2/3; b1-b2: -1, -4, 0 -> 0
    # gene 1: sums -1, 4, -1 -> 1/3; both positive: it 2 -> 1/3; b1-b2: 1, 0, 3 -> 1/3
    np.testing.assert_allclose(p, [[2 / 3, 2 / 3, 0.0], [1 / 3, 1 / 3, 1 / 3]])


def test_normal_closed_form():
    rng = np.random.default_rng(5)
    M, G = 200000, 3
    m = np.array([[0.3, -0.1], [0.0, 0.0], [-1.0, 0.4]])
    sd = np.array([0.5, 0.8])
    beta = m[None] + sd * rng.normal(size=(M, G, 2))
    p = oracle.contrast_probs(beta, [[([1.0, 1.0], 0.2)]])[:, 0]
    want = stats.norm.sf((0.2 - m.sum(1)) / np.hypot(*sd))
    se = np.sqrt(want * (1 - want) / M)
    assert np.all(np.abs(p - want) < 5 * se), (p, want)


def test_disjunction_by_inclusion_exclusion():
    rng = np.random.default_rng(6)
    beta = rng.normal(size=(5000, 4, 3))
    A = [([1.0, 0.0, 1.0], 0.1)]
    B = [([0.0, 2.0, -1.0], -0.3)]
    p = oracle.contrast_probs(beta, [A, B, A + B])
    s = beta @ np.array([1.0, 0.0, 1.0]) > 0.1
    t = beta @ np.array([0.0, 2.0, -1.0]) > -0.3
    np.testing.assert_allclose(p[:, 0] + p[:, 1] - p[:, 2], (s | t).mean(0), atol=1e-12)
