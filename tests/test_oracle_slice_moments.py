"""Pins for Algorithm 2 on textbook targets, the width tuning, Welford moments,
the default starting values, the integer count sums and the ESS estimator."""
import numpy as np
import pytest
from scipy import stats

import oracle


@pytest.mark.parametrize("w", [0.05, 1.0, 40.0])
def test_slice_normal_target(w):
    rng = np.random.default_rng(1)
    x0 = rng.normal(2.0, 1.5, 40000)            # exact draws of Normal(2, 1.5^2)
    out, ev = oracle.slice_textbook(0, 2.0, 2.25, x0, w=w, K=100, shrink_max=100, seed=3)
    assert stats.kstest(out, stats.norm(2.0, 1.5).cdf).pvalue > 1e-4
    # stepping out grows the interval by w per evaluation (bounded by K = 100) and
    # shrinkage roughly halves it per rejection: evaluations per update stay small
    bound = {0.05: 110, 1.0: 12, 40.0: 12}[w]
    assert out.size <= ev < bound * out.size


def test_slice_gamma_target_and_far_start():
    rng = np.random.default_rng(2)
    x0 = rng.gamma(3.0, 1.0, 40000)
    out, _ = oracle.slice_textbook(1, 3.0, 1.0, x0, w=1.0, seed=4)
    assert np.all(out > 0)
    assert stats.kstest(out, stats.gamma(3.0).cdf).pvalue > 1e-4
    # repeated transitions from one far point converge to the target
    x = np.full(40000, 25.0)
    for it in range(1, 30):
        x, _ = oracle.slice_textbook(1, 3.0, 1.0, x, w=1.0, seed=5, it=it)
    assert stats.kstest(x, stats.gamma(3.0).cdf).pvalue > 1e-4


def test_slice_stepping_out_bound_and_cap():
    x0 = np.zeros(1000)
    # no stepping out at all (K = 0) is still a valid update
    out, _ = oracle.slice_textbook(0, 0.0, 1.0, np.random.default_rng(3).normal(size=20000),
                                   w=1.0, K=0, seed=6)
    assert stats.kstest(out, "norm").pvalue > 1e-4
    # no shrinkage proposals allowed: every update keeps its start and counts a cap
    out, ev = oracle.slice_textbook(0, 0.0, 1.0, x0 + 0.5, w=1.0, K=3, shrink_max=0, seed=7)
    assert np.array_equal(out, x0 + 0.5)


def _two_group_X(N):
    return np.stack([np.ones(N), np.array([1.0] * (N // 2) + [-1.0] * (N - N // 2))], 1)


def _small_chain(G=40, N=4, burnin=30, seed=2):
    rng = np.random.default_rng(8)
    y = rng.poisson(rng.gamma(2.0, 10.0, (G, 1)) * np.ones((1, N))).astype(np.int32)
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.full(2, 10.0)}
    return oracle.Chain(y, _two_group_X(N), np.zeros(N), pri, seed=seed, burnin=burnin,
                        tune_start=10).init_default()


def test_width_tuning_is_weighted_mean_of_moves():
    """Algorithm 2 step 7: after M_C the width is the mean of |x(m+1) - x(m)| with
    weights m = 1..it; before M_C it stays at w0; after burn-in it is frozen."""
    ch = _small_chain()
    traj = [ch.get_state()]
    for _ in range(40):
        ch.sweep()
        traj.append(ch.get_state())
    for it in range(1, 41):
        st = traj[it]
        moves = np.stack([np.abs(traj[m]["beta"] - traj[m - 1]["beta"])
                          for m in range(1, min(it, 30) + 1)])
        if it <= 10:
            assert np.all(st["w_beta"] == 1.0)
        else:
            k = min(it, 30)
            want = np.average(moves[:k], axis=0, weights=np.arange(1, k + 1))
            np.testing.assert_allclose(st["w_beta"], want, rtol=1e-12)
    nu_moves = np.array([abs(traj[m]["phi"][0] - traj[m - 1]["phi"][0]) for m in range(1, 31)])
    assert traj[40]["w_nu"][0] == pytest.approx(
        np.average(nu_moves, weights=np.arange(1, 31)), rel=1e-12)


def test_welford_moments_equal_two_pass_means():
    ch = _small_chain(burnin=5)
    tr = ch.run(45, thin=1, trace_cap=1000, trace_beta=True)
    assert tr["phi"].shape[0] == 40 and ch.moments.count == 40
    m = ch.moments_dict()
    np.testing.assert_allclose(m["mean_phi"], tr["phi"].mean(0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m["msq_phi"], (tr["phi"] ** 2).mean(0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m["mean_beta"], tr["beta"].mean(0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m["msq_beta"], (tr["beta"] ** 2).mean(0), rtol=1e-12, atol=1e-14)


def test_thinning_picks_every_thin_th_post_burnin_draw():
    a = _small_chain(burnin=4)
    b = _small_chain(burnin=4)
    tr = a.run(24, thin=5, trace_cap=100)
    rows = []
    for it in range(1, 25):
        b.sweep()
        if it > 4 and (it - 4) % 5 == 0:
            rows.append(b.phi.copy())
    np.testing.assert_array_equal(tr["phi"], np.array(rows))


def test_default_start_is_least_squares_fit():
    ch = _small_chain()
    r = np.log(ch.y + 1.0) - ch.h[None, :]
    want = np.linalg.lstsq(ch.X, r.T, rcond=None)[0].T
    np.testing.assert_allclose(ch.beta, want, rtol=1e-10, atol=1e-12)
    assert np.all(ch.eps == 0) and np.all(ch.gam == 1)
    np.testing.assert_allclose(ch.phi[2:4], want.mean(0), rtol=1e-12)
    np.testing.assert_allclose(ch.phi[4:6], np.clip(want.var(0), 1e-6, 25.0), rtol=1e-10)
    assert ch.phi[0] == 3.0 and ch.phi[1] == 1.0


def test_singular_design_is_rejected():
    y = np.ones((3, 4), np.int32)
    X = np.stack([np.ones(4), np.ones(4)], 1)
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.full(2, 10.0)}
    with pytest.raises(ValueError):
        oracle.Chain(y, X, np.zeros(4), pri).init_default()


def test_count_sums_exact():
    rng = np.random.default_rng(9)
    y = rng.integers(0, 2 ** 31 - 1, (50, 16), dtype=np.int64).astype(np.int32)
    from paper_1606_06659_gb300.synthetic import paper_design
    X = paper_design(4)
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(5, 10.0), "s": np.full(5, 10.0)}
    ch = oracle.Chain(y, X, np.zeros(16), pri)
    want = y.astype(np.int64) @ X.astype(np.int64)
    assert np.array_equal(ch.count_sums(), want)


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_ar1_closed_form(rho):
    rng = np.random.default_rng(10)
    n = 20000
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - rho ** 2)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    want = n * (1 - rho) / (1 + rho)
    assert oracle.ess(x) == pytest.approx(want, rel=0.15)


def test_ess_constant_series():
    assert oracle.ess(np.ones(100)) == 100.0
