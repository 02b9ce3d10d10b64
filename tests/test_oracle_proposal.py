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
        q = stats.multivariate_t(mu[g], C[g] @ C[g].T, df=P.T_DOF)
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


def test_move_keeps_the_exact_conditional_of_beta():
    """Given eta (and gamma, theta, sigma^2) the conditional of beta is Gaussian
    with precision X^T X / gamma + diag(1/sigma^2) and mean that precision's
    inverse times (X^T (eta - h) / gamma + theta / sigma^2).  Rows drawn from it
    and moved with a deliberately poor proposal must still follow it: the mean
    and the covariance of the moved rows are checked, and the rate must be
    neither 0 nor 1 so that both branches run.  A sign error in either prior term
    or in the proposal ratio shifts the moved rows."""
    rng = np.random.default_rng(11)
    X = paper_design(2)[:, :3]
    N, L = X.shape
    gam, theta, sigma2 = 0.2, np.array([1.0, -0.5, 0.3]), np.array([0.5, 0.2, 0.8])
    lin = rng.normal(0.0, 1.0, N)                       # eta - h, held fixed
    prec = X.T @ X / gam + np.diag(1.0 / sigma2)
    cov = np.linalg.inv(prec)
    mean = cov @ (X.T @ lin / gam + theta / sigma2)
    G = 200000
    beta = rng.multivariate_normal(mean, cov, G)
    eps = lin[None, :] - beta @ X.T
    Lc = 1.3 * np.linalg.cholesky(cov)                      # too wide
    out = np.zeros((G, P.n_outputs(L)))
    out[:, :L] = mean + 0.4 * np.sqrt(np.diag(cov))          # biased
    out[:, L:2 * L] = np.log(np.diag(Lc))
    out[:, 2 * L:] = Lc[np.tril_indices(L, -1)]             # row order
    xi = rng.normal(size=(G, L))
    log_u = np.log(rng.uniform(size=G))
    chi2 = rng.chisquare(P.T_DOF, size=G)
    e2, b2, acc, la = P.mh_move(eps, beta, np.full(G, gam), theta, sigma2, X, out, xi, log_u,
                                chi2)
    np.testing.assert_allclose(e2 + b2 @ X.T, lin[None, :].repeat(G, 0), atol=1e-10)
    rate = acc.mean()
    assert 0.2 < rate < 0.95, rate
    se = np.sqrt(np.diag(cov) / G)
    assert np.all(np.abs(b2.mean(0) - mean) < 5 * se), (b2.mean(0) - mean) / se
    c2 = np.cov(b2.T)
    # standard error of a sample covariance entry: sqrt((s_ii s_jj + s_ij^2) / G)
    sec = np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov ** 2) / G)
    assert np.all(np.abs(c2 - cov) < 5 * sec), (c2 - cov) / sec


def test_move_with_a_proposal_at_the_current_point_accepts_by_the_uniform():
    """If mu + s C xi reproduces the current beta, the ratio is zero: the move
    accepts exactly when log u < 0 and leaves eps unchanged."""
    rng = np.random.default_rng(12)
    X = paper_design(2)
    N, L = X.shape
    G = 4
    beta = rng.normal(0, 0.5, (G, L))
    eps = rng.normal(0, 0.3, (G, N))
    out = rng.normal(0, 0.3, (G, P.n_outputs(L)))
    mu, C = P.unpack(out, L)
    chi2 = np.array([2.0, 8.0, 11.0, 30.0])
    xi = np.linalg.solve(C, (beta - mu)[..., None])[..., 0] / np.sqrt(P.T_DOF / chi2)[:, None]
    e2, b2, acc, la = P.mh_move(eps, beta, np.full(G, 0.3), np.zeros(L), np.ones(L), X, out, xi,
                                np.array([-1e-9, -1e-9, 1e-9, 1e-9]), chi2)
    np.testing.assert_allclose(la, 0.0, atol=1e-9)
    assert list(acc) == [True, True, False, False]
    np.testing.assert_allclose(e2, eps, atol=1e-12)
    np.testing.assert_allclose(b2, beta, atol=1e-12)


def test_block_conditional_is_the_joint_density_at_fixed_log_rates():
    """Along any change of beta_g that keeps eta_g (eps moving by -X d), the
    joint log density (scipy Poisson and Normal terms of the model) changes
    exactly as the log density of the Gaussian block conditional: the closed
    form's precision and mean are those of the model."""
    rng = np.random.default_rng(21)
    X = paper_design(4)
    N, L = X.shape
    G = 6
    h = rng.normal(0, 0.1, N)
    y = rng.poisson(30, (G, N))
    eps = rng.normal(0, 0.4, (G, N))
    beta = rng.normal(0, 0.6, (G, L))
    gam = rng.uniform(0.05, 0.8, G)
    theta, sigma2 = rng.normal(0, 1, L), rng.uniform(0.05, 2, L)
    mean, cov = P.block_conditional(eps, beta, gam, theta, sigma2, X)
    for g in range(G):
        def joint(e, b):
            lam = np.exp(h + e + X @ b)
            return (stats.poisson.logpmf(y[g], lam).sum()
                    + stats.norm.logpdf(e, 0, np.sqrt(gam[g])).sum()
                    + stats.norm.logpdf(b, theta, np.sqrt(sigma2)).sum())
        q = stats.multivariate_normal(mean[g], cov[g])
        for _ in range(3):
            b2 = beta[g] + rng.normal(0, 0.3, L)
            e2 = eps[g] - X @ (b2 - beta[g])
            want = joint(e2, b2) - joint(eps[g], beta[g])
            assert q.logpdf(b2) - q.logpdf(beta[g]) == pytest.approx(want, rel=1e-9, abs=1e-9)


def test_block_step_draws_the_conditional_and_keeps_log_rates():
    """block_step's draws have the block conditional's mean and covariance (5
    standard errors, 2e5 rows of one gene) and keep h + eps + X beta."""
    rng = np.random.default_rng(22)
    X = paper_design(4)
    N, L = X.shape
    G = 200000
    eps0 = np.tile(rng.normal(0, 0.3, N), (G, 1))
    beta0 = np.tile(rng.normal(0, 0.5, L), (G, 1))
    gam = np.full(G, 0.15)
    theta, sigma2 = rng.normal(0, 1, L), rng.uniform(0.1, 1, L)
    e2, b2 = P.block_step(eps0, beta0, gam, theta, sigma2, X, rng.normal(size=(G, L)))
    np.testing.assert_allclose(e2 + b2 @ X.T, eps0 + beta0 @ X.T, atol=1e-10)
    mean, cov = P.block_conditional(eps0[:1], beta0[:1], gam[:1], theta, sigma2, X)
    mean, cov = mean[0], cov[0]
    se = np.sqrt(np.diag(cov) / G)
    assert np.all(np.abs(b2.mean(0) - mean) < 5 * se)
    sec = np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov ** 2) / G)
    assert np.all(np.abs(np.cov(b2.T) - cov) < 5 * sec)


@pytest.mark.parametrize("mutant", ["no_prior_precision", "gamma_squared", "theta_sign"])
def test_block_conditional_pin_catches_planted_mistakes(mutant):
    """Planted mistakes in the block conditional (the prior's precision dropped,
    gamma squared, the prior mean's sign flipped) break the joint-density pin."""
    rng = np.random.default_rng(23)
    X = paper_design(4)
    N, L = X.shape
    h = rng.normal(0, 0.1, N)
    y = rng.poisson(30, N)
    eps, beta = rng.normal(0, 0.4, N), rng.normal(0, 0.6, L)
    gam, theta, sigma2 = 0.3, rng.normal(0, 1, L), rng.uniform(0.05, 2, L)
    lin = eps + X @ beta
    prec = X.T @ X / (gam ** 2 if mutant == "gamma_squared" else gam)
    if mutant != "no_prior_precision":
        prec = prec + np.diag(1.0 / sigma2)
    sgn = -1.0 if mutant == "theta_sign" else 1.0
    cov = np.linalg.inv(prec)
    mean = cov @ (X.T @ lin / gam + sgn * theta / sigma2)
    q = stats.multivariate_normal(mean, cov)

    def joint(e, b):
        return (stats.poisson.logpmf(y, np.exp(h + e + X @ b)).sum()
                + stats.norm.logpdf(e, 0, np.sqrt(gam)).sum()
                + stats.norm.logpdf(b, theta, np.sqrt(sigma2)).sum())
    bad = 0
    for _ in range(5):
        b2 = beta + rng.normal(0, 0.3, L)
        e2 = eps - X @ (b2 - beta)
        want = joint(e2, b2) - joint(eps, beta)
        bad += abs(q.logpdf(b2) - q.logpdf(beta) - want) > 1e-6
    assert bad >= 4
