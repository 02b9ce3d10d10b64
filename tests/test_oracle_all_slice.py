"""Pins for the all-slice variant of the oracle: gamma_g, tau and sigma_l
slice-sampled (Algorithm 2) from their full conditionals instead of drawn
exactly, as Section 4.2 does for every non-normal conditional.

Each target is assembled from scipy.stats densities of the model's own terms
(Figure 3) and normalised by quadrature.  The chains start from exact draws of
the target, so a few slice transitions must leave its distribution unchanged;
a wrong exponent, rate or truncation in the slice densities moves the draws
toward another law and fails the Kolmogorov-Smirnov test."""
import numpy as np
from scipy import stats

from tests._quad import GridDist, bracket, ks_pvalue, vectorized
from tests.test_oracle_conditionals import P_MIN, make_chain

N_TRANSITIONS = 3


def test_gamma_slice_step_matches_posterior():
    G, N = 8000, 4
    ch = make_chain(G, N=N, all_slice=True)
    eps_row = np.array([0.3, -0.8, 0.1, 0.5])
    nu, tau = 3.0, 0.2

    @vectorized
    def logpost(gv):
        gv = np.asarray(gv, float)
        out = stats.invgamma.logpdf(gv, nu / 2, scale=nu * tau / 2)
        for e in eps_row:
            out = out + stats.norm.logpdf(e, 0, np.sqrt(np.maximum(gv, 1e-300)))
        return np.where(gv > 0, out, -np.inf)

    lo, hi = bracket(logpost, 0.3, 0.05, lo_bound=1e-9, drop=40)
    dist = GridDist(logpost, lo, hi)
    start = dist.sample(G, np.random.default_rng(5))
    ch.set_state(eps=np.tile(eps_row, (G, 1)), gam=start, phi=[nu, tau, 0, 0, 1, 1])
    for it in range(1, N_TRANSITIONS + 1):
        ch.step_gamma(it)
    c = ch.counters_dict()
    assert c["gamma_caps"] == 0 and c["evals_gam"] >= 3 * G * N_TRANSITIONS
    assert not np.array_equal(ch.gam, start)
    assert ks_pvalue(ch.gam, dist) > P_MIN


def test_tau_slice_step_matches_posterior():
    G = 8
    pri = {"a": 2.0, "b": 3.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.full(2, 10.0)}
    ch = make_chain(G, priors=pri, all_slice=True)
    gam = np.array([0.1, 0.3, 0.25, 0.7, 0.05, 0.2, 0.4, 0.15])
    nu = 2.5

    @vectorized
    def logpost(t):
        t = np.asarray(t, float)
        out = stats.gamma.logpdf(t, 2.0, scale=1 / 3.0)
        for gv in gam:
            out = out + stats.invgamma.logpdf(gv, nu / 2, scale=nu * np.maximum(t, 1e-300) / 2)
        return np.where(t > 0, out, -np.inf)

    lo, hi = bracket(logpost, 0.2, 0.02, lo_bound=1e-9)
    dist = GridDist(logpost, lo, hi)
    n = 3000
    start = dist.sample(n, np.random.default_rng(6))
    draws = []
    for i in range(n):
        ch.set_state(gam=gam, phi=[nu, start[i], 0, 0, 1, 1])
        for k in range(N_TRANSITIONS):
            ch.step_tau(N_TRANSITIONS * i + k + 1)
        draws.append(ch.phi[1])
    assert ch.counters_dict()["gamma_caps"] == 0
    assert ks_pvalue(draws, dist) > P_MIN


def test_sigma_slice_step_matches_posterior_with_truncation():
    """The slice variable is sigma_l on (0, s_l); s_1 sits inside the spread of
    the beta so that the bound is active."""
    G = 9
    pri = {"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(2, 10.0), "s": np.array([0.5, 3.0])}
    ch = make_chain(G, priors=pri, all_slice=True)
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
    n = 3000
    start = np.stack([dists[0].sample(n, rng), dists[1].sample(n, rng)], 1)
    draws = []
    for i in range(n):
        ch.set_state(beta=beta, phi=[3.0, 1.0, *theta, *(start[i] ** 2)])
        for k in range(N_TRANSITIONS):
            ch.step_sigma(N_TRANSITIONS * i + k + 1)
        draws.append(np.sqrt(ch.phi[4:6]))
    draws = np.array(draws)
    assert np.all(draws[:, 0] < 0.5) and np.all(draws[:, 1] < 3.0)
    c = ch.counters_dict()
    assert c["trunc_caps"] == 0 and c["evals_hyp"] >= 3 * 2 * n * N_TRANSITIONS
    for l in range(2):
        assert ks_pvalue(draws[:, l], dists[l]) > P_MIN


def test_all_slice_widths_tune_and_conjugate_streams_idle():
    """During burn-in every new slice variable tunes its own width (Algorithm 2
    step 7); the exact gamma and truncated draws are never called."""
    ch = make_chain(500, N=4, all_slice=True, burnin=20)
    ch.init_default()
    for _ in range(20):
        ch.sweep()
    st = ch.get_state()
    assert np.all(st["waux_gam"] > 0) and np.all(st["waux_hyp"] > 0)
    assert np.all(st["w_gam"] != 1.0) and np.all(st["w_hyp"] != 1.0)
    assert np.all(st["w_gam"] > 0) and np.all(np.isfinite(st["w_hyp"]))
    c = ch.counters_dict()
    assert c["gamma_caps"] == 0 and c["trunc_caps"] == 0
    assert c["evals_gam"] >= 3 * 500 * 20 and c["evals_hyp"] >= 3 * 3 * 20
    plain = make_chain(500, N=4, burnin=20).init_default()
    for _ in range(20):
        plain.sweep()
    pc = plain.counters_dict()
    assert pc["evals_gam"] == 0 and pc["evals_hyp"] == 0
    assert np.all(plain.get_state()["w_gam"] == 1.0)


def _chain_phi(args):
    all_slice, seed, n_iter, burnin = args
    import oracle as orc
    from paper_1606_06659_gb300 import synthetic as syn
    d = syn.make_config(0, G=300)
    ch = orc.Chain(d["y"], d["X"], d["h"], d["priors"], seed=seed, burnin=burnin,
                   tune_start=burnin // 2, all_slice=all_slice).init_default()
    return ch.run(n_iter, thin=1, trace_cap=n_iter)["phi"]


def test_all_slice_sweeps_target_the_exact_draw_posterior():
    """Whole sweeps: 8 chains of the all-slice sampler and 8 of the exact-draw
    sampler (N = 4, G = 300) give the same posterior means of every
    hyperparameter, within 4.5 standard errors of the difference of the chain
    means."""
    import multiprocessing as mp
    jobs = [(a, 100 + 10 * c + a, 3000, 600) for a in (False, True) for c in range(8)]
    with mp.get_context("spawn").Pool(8) as pool:
        res = pool.map(_chain_phi, jobs)
    means = np.array([r.mean(0) for r in res])
    exact, sliced = means[:8], means[8:]
    se = np.sqrt(exact.var(0, ddof=1) / 8 + sliced.var(0, ddof=1) / 8)
    z = (sliced.mean(0) - exact.mean(0)) / se
    assert np.all(np.abs(z) < 4.5), z
