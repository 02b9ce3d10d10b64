"""Posterior summaries (§3.1) and the failure paths of the C ABI on the GPU.

fbs_estimates is compared with the summaries of the oracle chain that the FP64
GPU chain reproduces step by step.  The failure conditions are created on the
host, never by a GPU fault: a shrinkage bound of 0 (Algorithm 2's shrinkage
loop has no bound of its own), non-finite starting states set through
fbs_set_state, and a poll bound of 0 for the tensor-core waits of the learned
proposal's network pass, which makes the pass give up at its first wait while
the copy it waited for is still drained before the block exits."""
import numpy as np
import pytest

import oracle
import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import close, make_pair, small_data

pytestmark = pytest.mark.gpu


def _oracle_summaries(m, z):
    sd = np.sqrt(np.maximum(m["msq"] - m["mean"] ** 2, 0.0))
    return m["mean"], sd, m["mean"] - z * sd, m["mean"] + z * sd


def test_estimates_match_oracle_summaries():
    """A free-running FP64 chain equals the oracle chain, so its posterior means,
    sds sqrt(msq - mean^2) and intervals mean -/+ z sd equal those of the oracle's
    running moments (1e-9 relative; sd of nearly constant parameters to 1e-6 of
    the mean's size)."""
    d = small_data(0, G=1500)
    g, o = make_pair(d, seed=99, trace_cap=20)
    o.init_default()
    burnin = 10
    o.set_opts(burnin=burnin, tune_start=burnin // 2)
    for _ in range(30):
        g.run(1, burnin=burnin, thin=1)
        o.sweep()
    z = 1.644853626951473
    e = g.estimates(z=z, eps=True, trace_rows=50)
    om = o.moments_dict()
    assert e["count"] == 20 == om["count"]
    for v in ("eps", "beta", "gam", "phi"):
        mean, sd, lo, hi = _oracle_summaries({"mean": om["mean_" + v], "msq": om["msq_" + v]}, z)
        assert close(e["mean_" + v], mean, 1e-9, 1e-12).all(), v
        scale = np.abs(mean) + 1.0
        assert (np.abs(e["sd_" + v] - sd) <= 1e-6 * scale).all(), v
        assert (np.abs(e["lo_" + v] - lo) <= 1e-5 * scale).all(), v
        assert (np.abs(e["hi_" + v] - hi) <= 1e-5 * scale).all(), v
        assert np.all(e["sd_" + v] >= 0) and np.all(e["lo_" + v] <= e["hi_" + v])
    tr = g.trace()["phi"]
    assert np.array_equal(e["trace_phi"], tr) and len(tr) == 20
    assert e["counters"] == g.counters() and e["counters"]["sweeps"] == 30
    assert e["mh_tried"] == 0


@pytest.mark.parametrize("precision", [fbs.FBS_F64, fbs.FBS_F32])
def test_estimates_pool_chains_as_section_3_1(precision):
    """Pooled over chains, the mean is the mean of the chain means and the mean
    square the mean of the chain mean squares (§3.1); computed here from each
    chain's own running moments."""
    d = small_data(0, G=700)
    chains = [fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=5 + c, precision=precision)
              for c in range(3)]
    for c in chains:
        c.run(40, burnin=20)
    e = fbs.estimates(chains, z=2.0)
    ms = [c.moments() for c in chains]
    for v in ("beta", "gam", "phi"):
        mean = np.mean([m["mean_" + v] for m in ms], 0)
        msq = np.mean([m["msq_" + v] for m in ms], 0)
        sd = np.sqrt(np.maximum(msq - mean ** 2, 0.0))
        tol = 1e-12 if precision == fbs.FBS_F64 else 1e-6
        assert np.allclose(e["mean_" + v], mean, rtol=tol, atol=tol), v
        assert np.allclose(e["sd_" + v], sd, rtol=1e-5, atol=1e-5 * np.abs(mean).max()), v
        assert np.allclose(e["hi_" + v] - e["lo_" + v], 4.0 * e["sd_" + v], rtol=1e-12, atol=1e-12)
    assert e["count"] == 20
    assert e["counters"]["sweeps"] == 120
    with pytest.raises(fbs.FbsError) as err:
        chains[0].run(1, burnin=20)
        fbs.estimates(chains)  # the chains now hold different numbers of draws
    assert err.value.code == fbs.FBS_E_ARG
    for c in chains:
        c.close()


@pytest.mark.parametrize("precision", [fbs.FBS_F64, fbs.FBS_F32])
def test_slice_cap_is_counted_and_reported(precision):
    """shrink_max = 0: every slice update ends without a shrinkage proposal and
    keeps its value; each is counted (one per eps_gn, beta_gl and nu per sweep,
    as the oracle counts them) and fbs_sync returns FBS_E_SLICE_CAP."""
    d = small_data(0, G=600)
    N, L, G = 4, 2, 600
    g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=3, precision=precision,
                    shrink_max=0)
    st0 = g.get_state()
    g.run(3, burnin=0)
    with pytest.raises(fbs.FbsError) as e:
        g.sync()
    assert e.value.code == fbs.FBS_E_SLICE_CAP and "shrinkage" in str(e.value)
    c = g.counters()
    assert c["slice_caps"] == 3 * (N * G + L * G + 1) and c["nonfinite"] == 0
    st = g.get_state()
    assert np.array_equal(st["eps"], st0["eps"]) and np.array_equal(st["beta"], st0["beta"])
    assert st["phi"][0] == st0["phi"][0]  # nu is a slice variable too
    assert not np.array_equal(st["gam"], st0["gam"])  # the exact draws still move
    if precision == fbs.FBS_F64:
        o = oracle.Chain(d["y"], d["X"], d["h"], d["priors"], seed=3, shrink_max=0)
        o.init_default()
        o.set_opts(burnin=0, tune_start=0)
        for _ in range(3):
            o.sweep()
        assert o.counters_dict()["slice_caps"] == c["slice_caps"]
        assert o.counters_dict()["evals_eps"] == c["evals_eps"]
    g.close()


def test_nonfinite_start_is_reported_fp32():
    """The FP32 form needs every log-rate below 88 (FP32 exp range); a state set
    from outside with a larger one starts a slice update at a non-finite density,
    which is counted and turned into FBS_E_NONFINITE by fbs_sync."""
    d = small_data(0, G=500)
    g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=4, precision=fbs.FBS_F32)
    st = g.get_state()
    eps = st["eps"].copy()
    eps[17, 2] = 120.0
    g.set_state(it=0, eps=eps)
    g.run(2, burnin=0)
    with pytest.raises(fbs.FbsError) as e:
        g.sync()
    assert e.value.code == fbs.FBS_E_NONFINITE
    assert g.counters()["nonfinite"] >= 1
    g.close()


def test_nonfinite_start_is_reported_fp64_and_batch():
    d = small_data(0, G=500)
    g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=4)
    st = g.get_state()
    eps = st["eps"].copy()
    eps[3, 1] = np.nan
    g.set_state(it=0, eps=eps)
    g.run(1, burnin=0)
    with pytest.raises(fbs.FbsError) as e:
        g.sync()
    assert e.value.code == fbs.FBS_E_NONFINITE and g.counters()["nonfinite"] >= 1
    g.close()
    b = fbs.BatchSampler([d, small_data(0, G=300, seed=8)], seeds=[1, 2])
    v = b.chain(1)
    s1 = v.get_state()
    beta = s1["beta"].copy()
    beta[5, 0] = np.inf
    v.set_state(it=0, beta=beta)
    b.run(2, burnin=0)
    with pytest.raises(fbs.FbsError) as e:
        b.sync()
    assert e.value.code == fbs.FBS_E_NONFINITE
    assert b.chain(0).counters()["nonfinite"] == 0 and v.counters()["nonfinite"] >= 1
    b.close()


def test_tensor_core_wait_that_gives_up_is_reported():
    """With a poll bound of 0 every network pass gives up at its first wait (for
    the weight image): the block drains the copy, frees its tensor memory, its
    genes skip the network's move, and fbs_sync returns FBS_E_CUDA naming the
    wait.  The chain itself stays finite and the prior-centred moves go on."""
    d = synthetic.make_config(1, G=1000)
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=12, precision=fbs.FBS_F32)
    t = d["truth"]
    s.set_state(it=0, eps=t["eps"], beta=t["beta"], gam=t["gam"], phi=t["phi"])
    s.proposal_collect(30, burnin=30, thin=1)
    s.proposal_train(epochs=5, batch=2048, lr=2e-3, seed=12)
    s.proposal_calibrate(20, burnin=100, min_accept=0.0)
    kinds = s.proposal_kinds()
    n_net = int((kinds == 1).sum())
    assert n_net > 0
    s.sync()
    s.run(10, burnin=100)
    s.sync()
    before = s.proposal_stats()
    assert before["tried"] == 10 * before["mh_genes"]
    s.proposal_wait_limit(0)
    s.run(5, burnin=100)
    with pytest.raises(fbs.FbsError) as e:
        s.sync()
    assert e.value.code == fbs.FBS_E_CUDA and "tensor-core wait" in str(e.value)
    after = s.proposal_stats()
    # only the genes on the prior-centred proposal moved in those 5 sweeps
    assert after["tried"] - before["tried"] == 5 * (before["mh_genes"] - n_net)
    st = s.get_state()
    assert all(np.isfinite(st[k]).all() for k in ("eps", "beta", "gam", "phi"))
    assert s.counters()["sweeps"] == 30 + 20 + 10 + 5
    s.close()


def test_training_wait_that_gives_up_is_reported():
    """With a poll bound of 0 the training kernel gives up at its first wait (for
    the weight image): every block drains the copy and frees its tensor memory,
    the Adam update skips the step, and fbs_proposal_train returns FBS_E_CUDA
    naming the wait with the parameters as they were (back in raw coordinates).
    With the default bound restored the same call trains."""
    d = synthetic.make_config(1, G=1000)
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=13, precision=fbs.FBS_F32)
    t = d["truth"]
    s.set_state(it=0, eps=t["eps"], beta=t["beta"], gam=t["gam"], phi=t["phi"])
    s.proposal_collect(20, burnin=20, thin=1)
    s.proposal_train(epochs=1, batch=2048, lr=2e-3, seed=13)
    before = s.proposal_params()
    s.proposal_wait_limit(0)
    with pytest.raises(fbs.FbsError) as e:
        s.proposal_train(epochs=2, batch=2048, lr=2e-3, seed=13)
    assert e.value.code == fbs.FBS_E_CUDA and "tensor-core wait" in str(e.value)
    assert np.allclose(s.proposal_params(), before, rtol=1e-5, atol=1e-6)
    s.proposal_wait_limit(1 << 24)
    loss = s.proposal_train(epochs=2, batch=2048, lr=2e-3, seed=13)
    assert np.isfinite(loss)
    after = s.proposal_params()
    assert np.all(np.isfinite(after)) and not np.allclose(after, before)
    s.close()
