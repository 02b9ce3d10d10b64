"""The persistent sweep (fbs_options.persistent): a segment of sweeps in one
cooperative launch of resident blocks with grid barriers, every step of
Algorithm 1 inside, must give exactly the chain of the graph of separate
launches (same device functions, Philox counters and reduction order): state,
widths, running moments, thinned trace and counters bit-identical, across
segment boundaries, burn-in and odd sizes."""
import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import STATE_KEYS

pytestmark = pytest.mark.gpu


def _run(d, persistent, n_iter, burnin, thin, seed=17, chain=2, **kw):
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed, chain=chain,
                    precision=fbs.FBS_F32, persistent=persistent, trace_cap=200, trace_beta=1,
                    **kw)
    s.run(n_iter, burnin=burnin, thin=thin)
    s.run(37, burnin=burnin, thin=thin)  # a second call continues the chain
    s.sync()
    out = (s.get_state(), s.moments(), s.trace(beta=True), s.counters())
    s.close()
    return out


@pytest.mark.parametrize("cfg,G,seg", [(1, 5000, 100), (0, 3001, 100), (1, 1537, 64)])
def test_persistent_equals_graph_path(cfg, G, seg):
    d = synthetic.make_config(cfg, G=G)
    a = _run(d, 0, 230, burnin=120, thin=5, graph_segment=seg)
    b = _run(d, 1, 230, burnin=120, thin=5, graph_segment=seg)
    (sa, ma, ta, ca), (sb, mb, tb, cb) = a, b
    for k in STATE_KEYS:
        assert np.array_equal(sa[k], sb[k]), k
    for k in ma:
        assert np.array_equal(np.asarray(ma[k]), np.asarray(mb[k])), k
    assert np.array_equal(ta["phi"], tb["phi"]) and np.array_equal(ta["beta"], tb["beta"])
    assert ca == cb and ca["sweeps"] == 267
    assert not np.array_equal(sa["eps"], 0.0)


def test_persistent_edge_sizes():
    for N, G, L in [(64, 130, 1), (5, 2, 2), (12, 257, 2)]:
        X = synthetic.two_group_design(N) if L == 2 else np.ones((N, 1))
        d = synthetic.simulate(X, (2.0, 0.5)[:L], (1.0, 0.3)[:L], 0.2, 5.0, G, seed=N + G)
        d["priors"] = synthetic.default_priors(L)
        a = _run(d, 0, 120, burnin=60, thin=3)
        b = _run(d, 1, 120, burnin=60, thin=3)
        for k in STATE_KEYS:
            assert np.array_equal(a[0][k], b[0][k]), (N, G, L, k)
        assert a[3] == b[3]
