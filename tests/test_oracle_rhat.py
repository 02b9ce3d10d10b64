"""The oracle's Gelman-Rubin factor (§3.1, from running means and mean squares)
against its definition from the stored draws (between-chain variance of the
chain means and mean within-chain sample variance), a hand-worked case, and its
behaviour for well-mixed and separated chains."""
import numpy as np

import oracle


def test_equals_definition_from_draws():
    rng = np.random.default_rng(3)
    C, M = 5, 400
    x = rng.normal(size=(C, M, 7)) + rng.normal(0, 0.3, size=(C, 1, 7))
    got = oracle.rhat(x.mean(1), (x ** 2).mean(1), M)
    B = M * x.mean(1).var(0, ddof=1)
    W = x.var(1, ddof=1).mean(0)
    want = np.sqrt(((M - 1) / M * W + B / M) / W)
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_hand_worked():
    # two chains of M = 3 draws: (0, 1, 2) and (2, 3, 4): means 1, 3; S^2 = 1, 1;
    # B = 3/1 * ((1-2)^2 + (3-2)^2) = 6, W = 1, Rhat = sqrt(1 + (6 - 1)/3)
    means = np.array([1.0, 3.0])
    msqs = np.array([5 / 3, 29 / 3])
    np.testing.assert_allclose(oracle.rhat(means, msqs, 3), np.sqrt(1 + 5 / 3), rtol=1e-14)


def test_mixed_and_separated_chains():
    rng = np.random.default_rng(4)
    C, M = 4, 2000
    x = rng.normal(size=(C, M, 500))
    r = oracle.rhat(x.mean(1), (x ** 2).mean(1), M)
    assert np.all(np.abs(r - 1) < 0.01)
    y = x + np.arange(C)[:, None, None]
    assert np.all(oracle.rhat(y.mean(1), (y ** 2).mean(1), M) > 1.5)
    assert np.isnan(oracle.rhat(np.ones(3), np.ones(3), 10))
