"""Batched sweeps: datasets of different N, G and L swept together in one set of
launches.  A batch must give, for every dataset, exactly what a single-chain
FP32 sampler with the same seed and chain number gives (same kernels, same
per-dataset reduction order)."""
import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import STATE_KEYS

pytestmark = pytest.mark.gpu


def _sets():
    rng = np.random.default_rng(5)
    shapes = [(4, 700, 2), (16, 1500, 5), (7, 257, 2), (32, 999, 5), (12, 2, 5), (5, 130, 2)]
    out = []
    for i, (N, G, L) in enumerate(shapes):
        if L == 5:
            reps = N // 4
            X = synthetic.paper_design(reps)
            X = X[:N] if X.shape[0] >= N else X
            N = X.shape[0]
            theta, sigma = (4.0, 0, 0, 0, 0), (2.0, 0.5, 0.3, 0.2, 0.2)
        else:
            X = synthetic.two_group_design(N)
            theta, sigma = (3.0, 0.0), (1.5, 0.3)
        d = synthetic.simulate(X, theta, sigma, 0.1, 3.0, G, seed=None, rng=rng)
        d["priors"] = synthetic.default_priors(X.shape[1])
        out.append(d)
    return out


def test_batch_equals_single_chains():
    sets = _sets()
    seeds = [11 + i for i in range(len(sets))]
    chains = [i % 3 for i in range(len(sets))]
    b = fbs.BatchSampler(sets, seeds=seeds, chains=chains, trace_cap=20)
    b.run(230, burnin=100, thin=5)  # two graph segments and 30 direct sweeps
    b.sync()
    for i, d in enumerate(sets):
        s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seeds[i], chain=chains[i],
                        precision=fbs.FBS_F32, trace_cap=20)
        s.run(230, burnin=100, thin=5)
        v = b.chain(i)
        sv, ss = v.get_state(), s.get_state()
        for k in STATE_KEYS:
            assert np.array_equal(sv[k], ss[k]), (i, k)
        mv, ms = v.moments(), s.moments()
        for k in mv:
            assert np.array_equal(np.asarray(mv[k]), np.asarray(ms[k])), (i, k)
        assert np.array_equal(v.trace()["phi"], s.trace()["phi"])
        assert v.counters() == s.counters()
        assert np.array_equal(v.count_sums(), s.count_sums())


def test_batch_schedules_and_autotune():
    sets = _sets()
    b = fbs.BatchSampler(sets)
    eb, gb, ms = b.autotune(sweeps=3, burnin=1000)
    assert eb in (128, 256) and gb in (32, 64, 128) and ms > 0
    b.run(150, burnin=1000)
    b.sync()
    for eb, gb in ((128, 32), (256, 64)):
        b.set_schedule(eb, gb)
        b.run(120, burnin=1000)
        b.sync()
    for i, d in enumerate(sets):
        c = b.chain(i).counters()
        assert c["sweeps"] == 3 * 6 + 6 + 150 + 240 and c["nonfinite"] == 0
        st = b.chain(i).get_state()
        assert np.all(np.isfinite(st["beta"])) and np.all(st["gam"] > 0)


def test_batch_view_cannot_run_and_bad_schedule():
    b = fbs.BatchSampler(_sets()[:2])
    with pytest.raises(fbs.FbsError):
        b.chain(0).run(1)
    with pytest.raises(fbs.FbsError) as e:
        b.set_schedule(100, 32)
    assert e.value.code == fbs.FBS_E_ARG
    assert b.lib.fbs_batch_chain(b.b, 7) is None
