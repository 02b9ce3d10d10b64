"""Pins for the oracle of the learned proposal (oracle/proposal.py)."""
import numpy as np
import pytest
from scipy import stats

from oracle import proposal as P
from paper_1606_06659_gb300.synthetic import paper_design


def _batch(L=5, B=7, seed=0):
    rng = np.random.default_rng(seed)
    n_in, n_out = P.n_features(L), P.n_outputs(L)
    p = P.init_params(n_in, n_out, hidden=16, seed=seed)
    p = {k: v + rng.normal(0, 0.05, v.shape) for k, v in p.items()}
    f = rng.normal(0, 1, (B, n_in))
    beta = rng.normal(0, 1, (B, L))
    return p, f, beta


def test_nll_is_multivariate_normal_density():
    rng = np.random.default_rng(1)
    L = 5
    out = rng.normal(0, 0.5, (6, P.n_outputs(L)))
    beta = rng.normal(0, 1, (6, L))
    mu, C = P.unpack(out, L)
    for b in range(6):
        assert np.allclose(np.tril(C[b]), C[b]) and np.all(np.diag(C[b]) > 0)
        want = -stats.multivariate_normal(mu[b], C[b] @ C[b].T).logpdf(beta[b])
        assert P.nll(out[b:b + 1], beta[b:b + 1], L)[0] + 0.5 * L * np.log(2 * np.pi) == \
            pytest.approx(want, rel=1e-10)


def test_gelu_gradient_finite_difference():
    x = np.linspace(-4, 4, 101)
    h = 1e-6
    assert np.allclose(P.gelu_grad(x), (P.gelu(x + h) - P.gelu(x - h)) / (2 * h), atol=1e-8)


def test_parameter_gradients_finite_difference():
    p, f, beta = _batch()
    L = beta.shape[1]
    _, g = P.loss_and_grads(p, f, beta, L)
    rng = np.random.default_rng(2)
    for name, val in p.items():
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in val.shape)
            h = 1e-6
            q1 = {k: v.copy() for k, v in p.items()}
            q2 = {k: v.copy() for k, v in p.items()}
            q1[name][idx] += h
            q2[name][idx] -= h
            fd = (P.loss_and_grads(q1, f, beta, L)[0] - P.loss_and_grads(q2, f, beta, L)[0]) / (2 * h)
            assert g[name][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (name, idx)


def test_mh_ratio_equals_joint_density_ratio():
    """The move keeps h + eps + X beta, so the Poisson likelihood must cancel:
    the oracle's ratio equals the full joint density ratio computed from scipy."""
    rng = np.random.default_rng(3)
    X = paper_design(4)
    N, L = X.shape
    G = 5
    h = rng.normal(0, 0.1, N)
    y = rng.poisson(20, (G, N))
    eps = rng.normal(0, 0.3, (G, N))
    beta = rng.normal(0, 0.5, (G, L))
    beta_new = beta + rng.normal(0, 0.2, (G, L))
    gam = rng.uniform(0.05, 0.5, G)
    theta, sigma2 = rng.normal(0, 1, L), rng.uniform(0.1, 1, L)
    out = rng.normal(0, 0.3, (G, P.n_outputs(L)))
    got = P.mh_log_ratio(eps, beta, beta_new, gam, theta, sigma2, X, out)
    eps_new = eps - (beta_new - beta) @ X.T
    mu, C = P.unpack(out, L)
    for g in range(G):
        def joint(e, b):
            lam = np.exp(h + e + X @ b)
            return (stats.poisson.logpmf(y[g], lam).sum()
                    + stats.norm.logpdf(e, 0, np.sqrt(gam[g])).sum()
                    + stats.norm.logpdf(b, theta, np.sqrt(sigma2)).sum())
        q = stats.multivariate_normal(mu[g], C[g] @ C[g].T)
        want = (joint(eps_new[g], beta_new[g]) - joint(eps[g], beta[g])
                + q.logpdf(beta[g]) - q.logpdf(beta_new[g]))
        assert got[g] == pytest.approx(want, rel=1e-8, abs=1e-8)


def test_features_invariant_under_the_move():
    rng = np.random.default_rng(4)
    X = paper_design(4)
    N, L = X.shape
    eps = rng.normal(0, 0.3, (3, N))
    beta = rng.normal(0, 0.5, (3, L))
    beta_new = beta + rng.normal(0, 0.2, (3, L))
    eps_new = eps - (beta_new - beta) @ X.T
    y = rng.poisson(10, (3, N))
    args = (np.array([0.1, 0.2, 0.3]), np.zeros(L), np.ones(L), y, X)
    a = P.features(eps, beta, *args)
    b = P.features(eps_new, beta_new, *args)
    assert a.shape == (3, P.n_features(L))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
