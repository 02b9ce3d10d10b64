"""Pins for the oracle's full conditionals and Gibbs steps (Algorithm 1).

Every target density here is assembled from scipy.stats densities of the
model's own terms in Figure 3 (Poisson likelihood, Normal, Inverse-Gamma,
Gamma and Uniform priors), normalised by quadrature, and compared with draws
from the oracle's steps by Kolmogorov-Smirnov tests.  The slice-sampled steps
are started from exact draws of their conditional, so one transition must
leave that distribution unchanged.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from tests._quad import GridDist, bracket, ks_pvalue, vectorized

P_MIN = 1e-4


def two_group_X(N):
    return np.stack([np.ones(N), np.array([1.0] * (N // 2) + [-1.0] * (N - N // 2))], 1)


def make_chain(G, N=4, L=2, y_row=None, seed=3, priors=None, **kw):
    X = two_group_X(N) if L == 2 else np.ones((N, 1))
    h = np.linspace(-0.1, 0.1, N)
    y = np.tile(np.asarray(y_row if y_row is not None else np.arange(N) * 3 + 2, np.int32), (G, 1))
    pri = priors or {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(L, 10.0), "s": np.full(L, 10.0)}
    ch = oracle.Chain(y, X, h, pri, seed=seed, **kw)
    return ch


# ---------------------------------------------------------------- density values
def test_density_differences_match_model_terms():
    rng = np.random.default_rng(0)
    ch = make_chain(3, N=4, L=2, y_row=[0, 5, 40, 1])
    ch.set_state(eps=rng.normal(0, 0.3, (3, 4)), beta=rng.normal(1, 0.5, (3, 2)),
                 gam=[0.2, 0.5, 1.5], phi=[4.0, 0.3, 1.0, -0.5, 0.8, 0.09])
    X, h, y = ch.X, ch.h, ch.y

    def eps_model(g, n, x):
        lam = np.exp(h[n] + x + X[n] @ ch.beta[g])
        return stats.poisson.logpmf(y[g, n], lam) + stats.norm.logpdf(x, 0, np.sqrt(ch.gam[g]))

    def beta_model(g, l, b):
        bb = ch.beta[g].copy(); bb[l] = b
        lam = np.exp(h + ch.eps[g] + X @ bb)
        return (stats.poisson.logpmf(y[g], lam).sum()
                + stats.norm.logpdf(b, ch.phi[2 + l], np.sqrt(ch.phi[4 + l])))

    def nu_model(nu):
        return stats.invgamma.logpdf(ch.gam, nu / 2, scale=nu * ch.phi[1] / 2).sum()

    for g in range(3):
        for n in range(4):
            d_or = ch.logf_eps(g, n, 0.7) - ch.logf_eps(g, n, -0.4)
            d_mo = eps_model(g, n, 0.7) - eps_model(g, n, -0.4)
            assert d_or == pytest.approx(d_mo, rel=1e-10, abs=1e-10)
        for l in range(2):
            d_or = ch.logf_beta(g, l, 1.3) - ch.logf_beta(g, l, 0.2)
            d_mo = beta_model(g, l, 1.3) - beta_model(g, l, 0.2)
            assert d_or == pytest.approx(d_mo, rel=1e-10, abs=1e-10)
    d_or = ch.logf_nu(6.5) - ch.logf_nu(2.25)
    assert d_or == pytest.approx(nu_model(6.5) - nu_model(2.25), rel=1e-10, abs=1e-10)
    assert ch.logf_nu(0.0) == -np.inf and ch.logf_nu(10.0) == -np.inf
    assert ch.logf_nu(-1.0) == -np.inf and np.isfinite(ch.logf_nu(9.999))


# ---------------------------------------------------------------- conjugate steps
def test_gamma_step_matches_posterior():
    G, N = 8000, 4
    ch = make_chain(G, N=N)
    eps_row = np.array([0.3, -0.8, 0.1, 0.5])
    nu, tau = 3.0, 0.2
    ch.set_state(eps=np.tile(eps_row, (G, 1)), phi=[nu, tau, 0, 0, 1, 1])
    ch.step_gamma(1)

    @vectorized
    def logpost(gv):
        gv = np.asarray(gv, float)
        out = stats.invgamma.logpdf(gv, nu / 2, scale=nu * tau / 2)
        for e in eps_row:
            out = out + stats.norm.logpdf(e, 0, np.sqrt(np.maximum(gv, 1e-300)))
        return np.where(gv > 0, out, -np.inf)

    lo, hi = bracket(logpost, 0.3, 0.05, lo_bound=1e-9, drop=40)
    dist = GridDist(logpost, lo, hi)
    assert ks_pvalue(ch.gam, dist) > P_MIN


def test_tau_step_matches_posterior():
    G = 8
    pri = {"a": 2.0, "b": 3.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.full(2, 10.0)}
    ch = make_chain(G, priors=pri)
    gam = np.array([0.1, 0.3, 0.25, 0.7, 0.05, 0.2, 0.4, 0.15])
    nu = 2.5
    draws = []
    for it in range(1, 5001):
        ch.set_state(gam=gam, phi=[nu, 1.0, 0, 0, 1, 1])
        ch.step_tau(it)
        draws.append(ch.phi[1])

    @vectorized
    def logpost(t):
        t = np.asarray(t, float)
        out = stats.gamma.logpdf(t, 2.0, scale=1 / 3.0)
        for gv in gam:
            out = out + stats.invgamma.logpdf(gv, nu / 2, scale=nu * np.maximum(t, 1e-300) / 2)
        return np.where(t > 0, out, -np.inf)

    lo, hi = bracket(logpost, 0.2, 0.02, lo_bound=1e-9)
    assert ks_pvalue(draws, GridDist(logpost, lo, hi)) > P_MIN


def test_theta_step_matches_posterior():
    G = 12
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.array([0.5, 2.0]), "s": np.full(2, 10.0)}
    ch = make_chain(G, priors=pri)
    rng = np.random.default_rng(1)
    beta = np.stack([rng.normal(1.0, 0.6, G), rng.normal(-0.3, 0.4, G)], 1)
    sig2 = np.array([0.36, 0.16])
    draws = []
    for it in range(1, 4001):
        ch.set_state(beta=beta, phi=[3.0, 1.0, 0.0, 0.0, *sig2])
        ch.step_theta(it)
        draws.append(ch.phi[2:4].copy())
    draws = np.array(draws)
    for l in range(2):
        @vectorized
        def logpost(t, l=l):
            t = np.asarray(t, float)
            out = stats.norm.logpdf(t, 0, pri["c"][l])
            for bv in beta[:, l]:
                out = out + stats.norm.logpdf(bv, t, np.sqrt(sig2[l]))
            return out
        lo, hi = bracket(logpost, beta[:, l].mean(), 0.05)
        assert ks_pvalue(draws[:, l], GridDist(logpost, lo, hi)) > P_MIN


def test_sigma_step_matches_posterior_with_truncation():
    """sigma_l ~ Uniform(0, s_l); s_1 is set close to the spread of the beta so
    that the truncation is active.  Draws of sqrt(sigma^2) are compared with the
    posterior of sigma itself, which pins the shape (G-1)/2 and the Jacobian.
    When every rejection attempt fails the previous value is kept, a kernel that
    also leaves the conditional unchanged, so the chain is started from exact
    draws and one transition must keep their distribution."""
    G = 9
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.array([0.5, 3.0])}
    ch = make_chain(G, priors=pri)
    rng = np.random.default_rng(2)
    beta = np.stack([rng.normal(0.2, 0.45, G), rng.normal(1.0, 0.8, G)], 1)
    theta = np.array([0.1, 1.2])
    dists = []
    for l in range(2):
        s = pri["s"][l]

        @vectorized
        def logpost(sd, l=l, s=s):
            sd = np.asarray(sd, float)
            out = stats.uniform.logpdf(sd, 0, s)
            for bv in beta[:, l]:
                out = out + stats.norm.logpdf(bv, theta[l], np.maximum(sd, 1e-300))
            return np.where((sd > 0) & (sd < s), out, -np.inf)

        dists.append(GridDist(logpost, 1e-6, s))
    n = 4000
    start = np.stack([dists[0].sample(n, rng), dists[1].sample(n, rng)], 1)
    draws = []
    for it in range(1, n + 1):
        ch.set_state(beta=beta, phi=[3.0, 1.0, *theta, *(start[it - 1] ** 2)])
        ch.step_sigma(it)
        draws.append(np.sqrt(ch.phi[4:6]))
    draws = np.array(draws)
    assert np.all(draws[:, 0] < 0.5) and np.all(draws[:, 1] < 3.0)
    assert ch.counters_dict()["trunc_caps"] < 0.05 * n
    for l in range(2):
        assert ks_pvalue(draws[:, l], dists[l]) > P_MIN


# ---------------------------------------------------------------- slice-sampled steps
def test_eps_step_preserves_conditional():
    G, N = 20000, 2
    ch = make_chain(G, N=N, L=1, y_row=[0, 37])
    beta0, gam0 = np.array([1.5]), 0.4
    ch.set_state(beta=np.tile(beta0, (G, 1)), gam=np.full(G, gam0))
    rng = np.random.default_rng(4)
    dists = []
    start = np.zeros((G, N))
    for n in range(N):
        @vectorized
        def logpost(x, n=n):
            x = np.asarray(x, float)
            lam = np.exp(ch.h[n] + x + ch.X[n] @ beta0)
            return stats.poisson.logpmf(ch.y[0, n], lam) + stats.norm.logpdf(x, 0, np.sqrt(gam0))
        lo, hi = bracket(logpost, 0.0, 0.05)
        d = GridDist(logpost, lo, hi)
        dists.append(d)
        start[:, n] = d.sample(G, rng)
    ch.set_state(eps=start)
    ch.step_eps(1)
    for n in range(N):
        assert ks_pvalue(ch.eps[:, n], dists[n]) > P_MIN
    moved = np.mean(ch.eps != start)
    assert moved > 0.99
    # two transitions from a point far out reach the conditional too
    ch.set_state(eps=np.full((G, N), 3.0))
    for it in (2, 3, 4, 5, 6, 7, 8, 9):
        ch.step_eps(it)
    for n in range(N):
        assert ks_pvalue(ch.eps[:, n], dists[n]) > P_MIN


@pytest.mark.parametrize("l", [0, 1])
def test_beta_step_preserves_conditional(l):
    G, N = 20000, 4
    ch = make_chain(G, N=N, L=2, y_row=[3, 9, 0, 22])
    rng = np.random.default_rng(5 + l)
    eps_row = np.array([0.2, -0.1, 0.4, -0.3])
    beta_row = np.array([1.2, -0.4])
    phi = [3.0, 1.0, 0.8, 0.1, 0.5, 0.3]
    ch.set_state(eps=np.tile(eps_row, (G, 1)), beta=np.tile(beta_row, (G, 1)), phi=phi)

    @vectorized
    def logpost(b):
        b = np.asarray(b, float)[..., None]
        bb = np.where(np.arange(2) == l, b, beta_row)
        lam = np.exp(ch.h + eps_row + bb @ ch.X.T)
        out = stats.poisson.logpmf(ch.y[0], lam).sum(-1)
        return out + stats.norm.logpdf(b[..., 0], phi[2 + l], np.sqrt(phi[4 + l]))

    lo, hi = bracket(logpost, beta_row[l], 0.05)
    dist = GridDist(logpost, lo, hi)
    start = np.tile(beta_row, (G, 1))
    start[:, l] = dist.sample(G, rng)
    ch.set_state(beta=start)
    ch.step_beta_l(1, l)
    assert ks_pvalue(ch.beta[:, l], dist) > P_MIN
    other = 1 - l
    assert np.array_equal(ch.beta[:, other], start[:, other])


def test_nu_step_preserves_conditional():
    G = 15
    ch = make_chain(G)
    rng = np.random.default_rng(6)
    gam = 1.0 / rng.gamma(2.0, 1 / (2.0 * 0.3), G)
    tau, d = 0.3, 10.0
    ch.set_state(gam=gam)

    @vectorized
    def logpost(nu):
        nu = np.asarray(nu, float)
        out = np.zeros_like(nu)
        for gv in gam:
            out = out + stats.invgamma.logpdf(gv, np.maximum(nu, 1e-300) / 2,
                                              scale=np.maximum(nu, 1e-300) * tau / 2)
        return np.where((nu > 0) & (nu < d), out + stats.uniform.logpdf(nu, 0, d), -np.inf)

    dist = GridDist(logpost, 1e-6, d - 1e-9)
    x0 = dist.sample(4000, rng)
    draws = []
    for it, x in enumerate(x0, start=1):
        ch.set_state(phi=[x, tau, 0, 0, 1, 1])
        ch.step_nu(it)
        draws.append(ch.phi[0])
    assert ks_pvalue(draws, dist) > P_MIN
    assert np.all((np.array(draws) > 0) & (np.array(draws) < d))


# ---------------------------------------------------------------- sweep order
def test_sweep_order_does_not_change_draws():
    """beta's conditional involves neither nu nor tau and theirs involve no beta
    (Figure 3), so drawing beta right after gamma (as the GPU sweep does) must give
    the same numbers as the order of Algorithm 1."""
    rng = np.random.default_rng(7)
    G, N = 50, 4
    y = rng.poisson(20, (G, N)).astype(np.int32)
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.full(2, 10.0)}
    a = oracle.Chain(y, two_group_X(N), np.zeros(N), pri, seed=11).init_default()
    b = oracle.Chain(y, two_group_X(N), np.zeros(N), pri, seed=11).init_default()
    for it in range(1, 6):
        a.sweep()
        b.step_eps(it); b.step_gamma(it); b.step_beta(it)
        b.step_nu(it); b.step_tau(it); b.step_theta(it); b.step_sigma(it)
        for k, v in a.get_state().items():
            assert np.array_equal(v, b.get_state()[k]), k
