"""Posterior probabilities of contrasts (§3.1) on the GPU: counts of the
iterations whose beta_g satisfies each proposition, against the oracle's
probabilities from its own chain (FP64, same random numbers) and against the
FP32 chain's own beta trace."""
import numpy as np
import pytest

import oracle
import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import make_pair, small_data

pytestmark = pytest.mark.gpu

# config 1's heterosis-type statement (beta_2 + beta_4 > 0 and beta_3 + beta_4 > 0),
# a single contrast with a threshold, and a three-term conjunction
PROPS5 = [[([0, 1, 0, 1, 0], 0.0), ([0, 0, 1, 1, 0], 0.0)],
          [([1, 0, 0, 0, 0], 4.0)],
          [([0, 1, 0, 0, 0], -0.1), ([0, 0, 0, 0, 1], 0.05), ([0, 1, -1, 0, 0], 0.0)]]
PROPS2 = [[([0, 1], 0.0)], [([1, 0], 3.0), ([0, 1], -0.2)]]


def test_fp64_counts_match_oracle_chain():
    """Both chains run on their own from the same start (the free-running
    parity case); the device probabilities equal the oracle's fractions over its
    post-burn-in draws, except where an oracle draw lies within 1e-9 of a
    threshold (none is expected)."""
    d = small_data(1, G=1537)
    g, o = make_pair(d)
    o.init_default()
    burnin, n_it = 15, 45
    o.set_opts(burnin=burnin, tune_start=burnin // 2)
    g.set_contrasts(PROPS5)
    draws = []
    for it in range(1, n_it + 1):
        g.run(1, burnin=burnin, thin=1)
        o.sweep()
        if it > burnin:
            draws.append(o.get_state()["beta"].copy())
    p, m = g.contrast_probs()
    assert m == n_it - burnin
    want = oracle.contrast_probs(np.array(draws), PROPS5)
    assert p.shape == want.shape == (1537, 3)
    np.testing.assert_array_equal(p, want)
    assert 0.0 < want.mean() < 1.0


def test_fp32_counts_match_own_trace_and_mid_run_start():
    """FP32 form (learned proposal off): the probabilities equal the fractions
    of the chain's own beta trace (thin 1) evaluated in FP32; propositions set
    after some post-burn-in iterations count only the iterations that follow."""
    d = synthetic.make_config(0, G=777)
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=9, precision=fbs.FBS_F32,
                    trace_cap=100, trace_beta=1)
    s.run(30, burnin=20, thin=1)            # 10 post-burn-in rows before counting
    s.set_contrasts(PROPS2)
    s.run(60, burnin=20, thin=1)
    p, m = s.contrast_probs()
    assert m == 60
    tr = s.trace(beta=True)["beta"]
    assert tr.shape[0] == 70
    want = oracle.contrast_probs(tr[10:], PROPS2, dtype=np.float32)
    np.testing.assert_array_equal(p, want)
    s.set_contrasts([])
    with pytest.raises(fbs.FbsError):
        s.contrast_probs()
    s.close()


def test_contrast_arguments_are_checked():
    d = synthetic.make_config(0, G=100)
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=1)
    with pytest.raises(fbs.FbsError):
        s.set_contrasts([[([1, 0], 0.0)]] * (fbs.FBS_MAX_CONTRASTS + 1))
    with pytest.raises(fbs.FbsError):
        s.set_contrasts([[([1, 0], 0.0)] * (fbs.FBS_MAX_CONTRAST_TERMS + 1)])
    with pytest.raises(fbs.FbsError):
        s.set_contrasts([[([np.nan, 0], 0.0)]])
    with pytest.raises(fbs.FbsError):
        s.set_contrasts([[]])
    s.close()


def test_rhat_matches_oracle_chains():
    """Four FP64 chains (chain numbers 0..3) and the oracle's four chains on the
    same random numbers: the device Gelman-Rubin factors equal the oracle's
    formula applied to the oracle chains' moments; FP32 chains: the device
    factors equal the formula applied to their own moments."""
    d = small_data(0, G=900)
    burnin, n_it = 10, 40
    gs, os_ = [], []
    for c in range(4):
        g, o = make_pair(d, chain=c)
        o.init_default()
        o.set_opts(burnin=burnin, tune_start=burnin // 2)
        g.run(n_it, burnin=burnin, thin=1)
        for _ in range(n_it):
            o.sweep()
        gs.append(g)
        os_.append(o.moments_dict())
    r = fbs.rhat(gs, eps=True)
    M = n_it - burnin
    for key, k in (("phi", "phi"), ("beta", "beta"), ("gam", "gam"), ("eps", "eps")):
        want = oracle.rhat([m["mean_" + k] for m in os_], [m["msq_" + k] for m in os_], M)
        np.testing.assert_allclose(r[key], want, rtol=1e-8, atol=1e-10, err_msg=key)
    assert np.nanmax(r["phi"]) > 1.0
    fs = []
    for c in range(3):
        s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=4, chain=c,
                        precision=fbs.FBS_F32)
        s.run(n_it, burnin=burnin)
        fs.append(s)
    r32 = fbs.rhat(fs)
    ms = [s.moments() for s in fs]
    # W = msq - mean^2 cancels where the within-chain variance is small against
    # the mean square (R-hat in the hundreds), and the device sums the chains in
    # another order than numpy: agreement to 1e-9 relative
    for k in ("phi", "beta", "gam"):
        want = oracle.rhat([m["mean_" + k] for m in ms], [m["msq_" + k] for m in ms], M)
        np.testing.assert_allclose(r32[k], want, rtol=1e-9, atol=1e-12, err_msg=k)
    fs[2].run(1, burnin=burnin)
    with pytest.raises(fbs.FbsError):
        fbs.rhat(fs)                       # unequal draw counts
    with pytest.raises(fbs.FbsError):
        fbs.rhat([gs[0], fs[0]])           # mixed precision
    for s in gs + fs:
        s.close()
