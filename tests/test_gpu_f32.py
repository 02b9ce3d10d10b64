"""The FP32 form of the sweep (log densities in FP32 relative to the start
point, Kahan-compensated FP32 moments, FP64 reductions and hyperparameters):
deterministic properties here, posterior agreement with the FP64 oracle in
test_gpu_posterior.py."""
import numpy as np
import pytest

import oracle
import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import STATE_KEYS, close

pytestmark = pytest.mark.gpu


def _f32(d, seed=3, **kw):
    return fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed, precision=fbs.FBS_F32, **kw)


def test_f32_start_is_oracle_start_rounded():
    d = synthetic.make_config(1, G=2001)
    g = _f32(d)
    o = oracle.Chain(d["y"], d["X"], d["h"], d["priors"]).init_default()
    gs, os_ = g.get_state(), o.get_state()
    for k in ("eps", "beta", "gam", "w_eps", "w_beta"):
        assert close(gs[k], np.float32(os_[k]).astype(np.float64), 0, 0).all(), k
    assert close(gs["phi"], os_["phi"], 1e-6, 1e-9).all()
    assert np.array_equal(g.count_sums(), o.count_sums())


def test_f32_kahan_moments_equal_two_pass_means():
    d = synthetic.make_config(0, G=700)
    g = _f32(d, trace_cap=3000, trace_beta=1)
    g.run(3200, burnin=200, thin=1)
    tr = g.trace(beta=True)
    m = g.moments()
    assert m["count"] == 3000 and tr["beta"].shape[0] == 3000
    # the trace holds the FP32 draws exactly; the compensated FP32 running mean
    # must match their FP64 two-pass mean to a few FP32 ulps, not 3000 of them
    np.testing.assert_allclose(m["mean_beta"], tr["beta"].mean(0), rtol=3e-7, atol=3e-7)
    np.testing.assert_allclose(m["msq_beta"], (tr["beta"] ** 2).mean(0), rtol=3e-7, atol=3e-7)
    np.testing.assert_allclose(m["mean_phi"], tr["phi"].mean(0), rtol=1e-12, atol=1e-14)


def test_f32_graph_segments_equal_direct_launches():
    d = synthetic.make_config(0, G=1500)
    a = _f32(d, seed=5, graph_segment=7)
    b = _f32(d, seed=5, graph_segment=1000)
    a.run(23, burnin=10, thin=2)
    b.run(23, burnin=10, thin=2)
    sa, sb = a.get_state(), b.get_state()
    for k in STATE_KEYS:
        assert np.array_equal(sa[k], sb[k]), k
    assert a.counters() == b.counters()


def test_f32_resume_equals_one_run():
    d = synthetic.make_config(1, G=900)
    a, b = _f32(d, seed=9), _f32(d, seed=9)
    a.run(25, burnin=10, thin=1)
    b.run(11, burnin=10, thin=1)
    b.run(14, burnin=10, thin=1)
    sa, sb = a.get_state(), b.get_state()
    for k in STATE_KEYS:
        assert np.array_equal(sa[k], sb[k]), k
    ma, mb = a.moments(), b.moments()
    for k in ma:
        assert np.array_equal(np.asarray(ma[k]), np.asarray(mb[k])), k


def test_f32_set_state_round_trip_and_moves():
    d = synthetic.make_config(0, G=300)
    g = _f32(d)
    st = g.get_state()
    g.set_state(it=0, **{k: st[k] for k in STATE_KEYS})
    st2 = g.get_state()
    for k in STATE_KEYS:
        assert np.array_equal(st[k], st2[k]), k
    g.run(5, burnin=0)
    g.sync()
    assert not np.array_equal(g.get_state()["eps"], st["eps"])
    c = g.counters()
    assert c["sweeps"] == 5 and c["evals_eps"] > 0 and c["nonfinite"] == 0
