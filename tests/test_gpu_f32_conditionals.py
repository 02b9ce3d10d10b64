"""One FP32 transition from exact draws keeps each full conditional (§4.1,
Algorithm 1 steps 1, 2, 5 with Algorithm 2) on the GPU.

The FP32 form's draws differ from the oracle's by design (FP32 arithmetic, FP32
uniforms), so it is pinned the way the oracle itself is: 1e5 replicas of one
gene (identical counts) start from exact draws of a conditional, obtained by
inverting its quadrature CDF, and one sweep must leave that conditional
unchanged (Kolmogorov-Smirnov test).  The target densities are assembled from
scipy.stats densities of the model's terms, not from any sampler.  A variable
that must stay put while another is tested is given a slice width of 1e-30:
its slice update then moves it by less than 1e-27, far below what the test can
see, and every other update of the sweep is the product's own."""
import numpy as np
import pytest
from scipy import stats

import paper_1606_06659_gb300 as fbs
from tests._quad import GridDist, bracket, ks_pvalue, vectorized

pytestmark = pytest.mark.gpu

P_MIN = 1e-4
G = 100000
FROZEN = 1e-30


def _sampler(N, L, y_row, seed):
    X = (np.stack([np.ones(N), np.array([1.0] * (N // 2) + [-1.0] * (N - N // 2))], 1)
         if L == 2 else np.ones((N, 1)))
    h = np.linspace(-0.1, 0.1, N)
    y = np.tile(np.asarray(y_row, np.int32), (G, 1))
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(L, 10.0), "s": np.full(L, 10.0)}
    s = fbs.Sampler(y, X, h, pri, seed=seed, precision=fbs.FBS_F32)
    return s, X, h, y[0]


def test_f32_eps_transition_keeps_its_conditional():
    N = 2
    s, X, h, y = _sampler(N, 1, [0, 37], seed=41)
    beta0, gam0 = np.array([1.5]), 0.4
    rng = np.random.default_rng(41)
    dists, start = [], np.zeros((G, N))
    for n in range(N):
        @vectorized
        def logpost(x, n=n):
            x = np.asarray(x, float)
            lam = np.exp(h[n] + x + X[n] @ beta0)
            return stats.poisson.logpmf(y[n], lam) + stats.norm.logpdf(x, 0, np.sqrt(gam0))
        lo, hi = bracket(logpost, 0.0, 0.05)
        dists.append(GridDist(logpost, lo, hi))
        start[:, n] = dists[-1].sample(G, rng)
    s.set_state(it=0, eps=start, beta=np.tile(beta0, (G, 1)), gam=np.full(G, gam0),
                phi=[3.0, 1.0, 1.5, 0.25])
    s.run(1, burnin=0)
    s.sync()
    eps = s.get_state()["eps"]
    assert np.mean(eps != start.astype(np.float32)) > 0.99
    for n in range(N):
        assert ks_pvalue(eps[:, n], dists[n]) > P_MIN, n


@pytest.mark.parametrize("l", [0, 1])
def test_f32_beta_transition_keeps_its_conditional(l):
    """Column 0 (all ones: one value class) and column 1 (+/-1: two classes);
    eps and the other column are held."""
    N = 4
    s, X, h, y = _sampler(N, 2, [3, 9, 0, 22], seed=51 + l)
    eps_row = np.array([0.2, -0.1, 0.4, -0.3])
    beta_row = np.array([1.2, -0.4])
    phi = [3.0, 1.0, 0.8, 0.1, 0.5, 0.3]

    @vectorized
    def logpost(b):
        b = np.asarray(b, float)[..., None]
        bb = np.where(np.arange(2) == l, b, beta_row)
        lam = np.exp(h + eps_row + bb @ X.T)
        out = stats.poisson.logpmf(y, lam).sum(-1)
        return out + stats.norm.logpdf(b[..., 0], phi[2 + l], np.sqrt(phi[4 + l]))

    lo, hi = bracket(logpost, beta_row[l], 0.05)
    dist = GridDist(logpost, lo, hi)
    rng = np.random.default_rng(61 + l)
    start = np.tile(beta_row, (G, 1))
    start[:, l] = dist.sample(G, rng)
    w_beta = np.ones((G, 2))
    w_beta[:, 1 - l] = FROZEN
    s.set_state(it=0, eps=np.tile(eps_row, (G, 1)), beta=start, gam=np.full(G, 0.3), phi=phi,
                w_eps=np.full((G, N), FROZEN), w_beta=w_beta)
    s.run(1, burnin=0)
    s.sync()
    st = s.get_state()
    assert np.max(np.abs(st["eps"] - eps_row.astype(np.float32))) < 1e-6
    assert np.max(np.abs(st["beta"][:, 1 - l] - beta_row[1 - l])) < 1e-6
    assert np.mean(st["beta"][:, l] != start[:, l].astype(np.float32)) > 0.99
    assert ks_pvalue(st["beta"][:, l], dist) > P_MIN


def test_f32_beta_transition_many_rows():
    """A design with 12 distinct rows, more than the 8 row patterns whose rate
    sums the FP32 beta columns keep in registers, so the update sums the rates
    sample by sample: column 1 (three value classes) keeps its conditional;
    eps and columns 0 and 2 are held."""
    N, L, l = 12, 3, 1
    a_vals, b_vals = np.array([-1.0, 1.0, 2.0]), np.array([-1.0, 0.0, 1.0, 2.0])
    X = np.stack([np.ones(N), a_vals[np.arange(N) % 3], b_vals[np.arange(N) // 3]], 1)
    assert len({tuple(r) for r in X}) == 12
    h = np.linspace(-0.1, 0.1, N)
    y_row = np.array([3, 9, 0, 22, 5, 1, 14, 7, 2, 30, 6, 11], np.int32)
    y = np.tile(y_row, (G, 1))
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(L, 10.0), "s": np.full(L, 10.0)}
    s = fbs.Sampler(y, X, h, pri, seed=81, precision=fbs.FBS_F32)
    eps_row = np.linspace(-0.3, 0.3, N)
    beta_row = np.array([1.2, -0.3, 0.2])
    phi = [3.0, 1.0, 0.8, 0.1, 0.0, 0.5, 0.3, 0.4]

    @vectorized
    def logpost(b):
        b = np.asarray(b, float)[..., None]
        bb = np.where(np.arange(L) == l, b, beta_row)
        lam = np.exp(h + eps_row + bb @ X.T)
        out = stats.poisson.logpmf(y_row, lam).sum(-1)
        return out + stats.norm.logpdf(b[..., 0], phi[2 + l], np.sqrt(phi[2 + L + l]))

    lo, hi = bracket(logpost, beta_row[l], 0.05)
    dist = GridDist(logpost, lo, hi)
    rng = np.random.default_rng(91)
    start = np.tile(beta_row, (G, 1))
    start[:, l] = dist.sample(G, rng)
    w_beta = np.full((G, L), FROZEN)
    w_beta[:, l] = 1.0
    s.set_state(it=0, eps=np.tile(eps_row, (G, 1)), beta=start, gam=np.full(G, 0.3), phi=phi,
                w_eps=np.full((G, N), FROZEN), w_beta=w_beta)
    s.run(1, burnin=0)
    s.sync()
    st = s.get_state()
    assert np.max(np.abs(st["eps"] - eps_row.astype(np.float32))) < 1e-6
    for k in (0, 2):
        assert np.max(np.abs(st["beta"][:, k] - beta_row[k])) < 1e-6
    assert np.mean(st["beta"][:, l] != start[:, l].astype(np.float32)) > 0.99
    assert ks_pvalue(st["beta"][:, l], dist) > P_MIN
    s.close()


def test_f32_gamma_draw_is_its_inverse_gamma():
    """With eps held, gamma_g after one sweep is a draw from Inverse-Gamma((N +
    nu)/2, (sum_n eps_gn^2 + nu tau)/2) (step 2); tested against scipy's CDF."""
    N = 4
    s, X, h, y = _sampler(N, 2, [3, 9, 0, 22], seed=71)
    eps_row = np.array([0.2, -0.1, 0.4, -0.3])
    nu, tau = 3.0, 0.5
    s.set_state(it=0, eps=np.tile(eps_row, (G, 1)), beta=np.tile([1.2, -0.4], (G, 1)),
                gam=np.full(G, 0.3), phi=[nu, tau, 0.8, 0.1, 0.5, 0.3],
                w_eps=np.full((G, N), FROZEN))
    s.run(1, burnin=0)
    s.sync()
    gam = s.get_state()["gam"]
    e32 = eps_row.astype(np.float32).astype(np.float64)
    law = stats.invgamma(0.5 * (N + nu), scale=0.5 * (np.sum(e32 ** 2) + nu * tau))
    assert stats.kstest(gam, law.cdf).pvalue > P_MIN
    assert s.counters()["gamma_caps"] == 0
