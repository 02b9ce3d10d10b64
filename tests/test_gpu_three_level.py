"""The three-level model (Section 2.3) over a batch of datasets on the GPU
against the oracle's three-level model.

The batch runs the FP32 form, whose slice updates draw different random
numbers than the FP64 oracle, so the chains are compared two ways:
* step by step: after every GPU sweep, the oracle's tau, theta and sigma^2
  steps of each dataset are applied to the GPU's own new gamma, beta and nu
  with the GPU's previous phi_k and psi (same Philox numbers), and the oracle's
  psi step to the GPU's new phi_k; the results must equal the GPU's (tau,
  theta, sigma^2 to the FP32 partial sums' rounding, psi to 1e-12);
* in distribution: posterior means and mean squares of psi and of every phi_k
  from 16 GPU batches and 16 oracle chains agree within 4 MCSE."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic

pytestmark = pytest.mark.gpu

E = np.array([4.0, 1.0])
A_B, B_B = 2.0, 1.0


def _sets(K=4, G=(600, 350, 901, 128)):
    out = []
    for k in range(K):
        X = synthetic.two_group_design(4 + 2 * k)
        theta = (2.5 + 0.5 * k, 0.3 * (k - 1.5))
        d = synthetic.simulate(X, theta, (1.2, 0.3), 0.1 * (1 + k), 3.0, G[k], seed=700 + k)
        d["priors"] = synthetic.default_priors(2, a=1.5 + 0.5 * k, c=2.0)
        d["priors"]["c"] = np.array([2.0, 0.6])
        d["seed"], d["chain"] = 31 + k, k
        out.append(d)
    return out


def _batch(sets, psi0=None, **kw):
    b = fbs.BatchSampler(sets, seeds=[d["seed"] for d in sets],
                         chains=[d["chain"] for d in sets], **kw)
    b.three_level(E, A_B, B_B, seed=909, psi0=psi0)
    return b


def test_three_level_steps_match_oracle():
    sets = _sets()
    burnin = 4
    b = _batch(sets, psi0=[0.8, 2.0, -0.1])
    L = 2
    for m in range(1, 9):
        before = [v.get_state() for v in b.views]
        psi_before = b.top_level()["psi"]
        b.run(1, burnin=burnin, thin=1)
        b.sync()
        after = [v.get_state() for v in b.views]
        psi_after = b.top_level()["psi"]
        phis = []
        for k, d in enumerate(sets):
            assert after[k]["it"] == m
            ch = oracle.Chain(d["y"], d["X"], d["h"], d["priors"], seed=d["seed"],
                              chain=d["chain"], burnin=burnin, tune_start=burnin // 2)
            ch.set_top_level(psi_before[0], psi_before[1:])
            phi0 = before[k]["phi"].copy()
            phi0[0] = after[k]["phi"][0]     # nu of this sweep, from the GPU
            ch.set_state(beta=after[k]["beta"], gam=after[k]["gam"], phi=phi0)
            ch.step_tau(m)
            ch.step_theta(m)
            ch.step_sigma(m)
            got, want = after[k]["phi"], ch.phi
            np.testing.assert_allclose(got[1], want[1], rtol=1e-6, err_msg=f"tau, sweep {m}")
            np.testing.assert_allclose(got[2:2 + L], want[2:2 + L], rtol=1e-6, atol=1e-7,
                                       err_msg=f"theta, sweep {m}")
            np.testing.assert_allclose(got[2 + L:], want[2 + L:], rtol=1e-5,
                                       err_msg=f"sigma^2, sweep {m}")
            phis.append(got)
        t = oracle.ThreeLevel(sets, E, A_B, B_B, psi_seed=909, psi0=psi_before)
        for k, ch in enumerate(t.chains):
            ch.phi[...] = phis[k]
        t.step_psi(m)
        np.testing.assert_allclose(psi_after, t.psi, rtol=1e-12, err_msg=f"psi, sweep {m}")
    top = b.top_level()
    assert top["count"] == 8 - burnin and top["gamma_caps"] == 0


def test_three_level_graph_equals_direct_and_off_equals_plain():
    sets = _sets()
    a = _batch(sets, graph_segment=7, trace_cap=10)
    c = _batch(sets, graph_segment=1000, trace_cap=10)
    a.run(23, burnin=10, thin=2)
    c.run(23, burnin=10, thin=2)
    ta, tc = a.top_level(), c.top_level()
    for k in ("psi", "mean", "msq", "trace"):
        assert np.array_equal(ta[k], tc[k]), k
    assert ta["count"] == 13 and ta["trace"].shape == (6, 3)
    for va, vc in zip(a.views, c.views):
        assert np.array_equal(va.get_state()["phi"], vc.get_state()["phi"])
    # switched off, the batch is K independent datasets again
    p = fbs.BatchSampler(sets, seeds=[d["seed"] for d in sets], chains=[d["chain"] for d in sets])
    q = _batch(sets)
    q.three_level(None, 0, 0, 0)
    p.run(30, burnin=10)
    q.run(30, burnin=10)
    for vp, vq in zip(p.views, q.views):
        sp, sq = vp.get_state(), vq.get_state()
        for k in ("eps", "beta", "gam", "phi"):
            assert np.array_equal(sp[k], sq[k]), k
    with pytest.raises(fbs.FbsError):
        q.top_level()


def test_three_level_argument_checks():
    sets = _sets()
    b = fbs.BatchSampler(sets)
    for e, ab, bb, psi0 in ((np.array([1.0, 0.0]), 1, 1, None), (E, 0.0, 1, None),
                            (E, 1, np.inf, None), (E, 1, 1, [0.0, 0, 0]),
                            (E, 1, 1, [1.0, np.nan, 0])):
        with pytest.raises(fbs.FbsError) as ex:
            b.three_level(e, ab, bb, seed=1, psi0=psi0)
        assert ex.value.code == fbs.FBS_E_ARG
    mixed = sets[:2] + [synthetic.make_config(1, G=300)]
    mixed[2]["priors"] = synthetic.default_priors(5)
    m = fbs.BatchSampler(mixed)
    with pytest.raises(fbs.FbsError) as ex:
        m.three_level(np.ones(2), 1, 1, seed=1)
    assert ex.value.code == fbs.FBS_E_ARG


# ------------------------------------------------------------------ in distribution
N_CHAINS = 16


def _oracle_three_level(args):
    c, iters, burnin, thin = args
    import oracle as orc
    sets = _sets(K=3, G=(300, 200, 250))
    for k, d in enumerate(sets):
        d["seed"], d["chain"] = 5000 + 10 * c + k, c
    t = orc.ThreeLevel(sets, E, A_B, B_B, psi_seed=777 + c, burnin=burnin).init_default()
    tr = t.run(iters, thin=thin)
    return tr["psi"], tr["phi"]


def _chain_stats(traces):
    m1 = np.stack([t.mean(0) for t in traces])
    m2 = np.stack([(t ** 2).mean(0) for t in traces])
    k = len(traces)
    return (m1.mean(0), m1.std(0, ddof=1) / np.sqrt(k), m2.mean(0), m2.std(0, ddof=1) / np.sqrt(k))


@pytest.mark.slow
def test_three_level_posterior_matches_oracle():
    orc_iters, orc_burn, gpu_iters, gpu_burn = 3000, 1000, 12000, 2000
    ctx = mp.get_context("spawn")
    with ctx.Pool(N_CHAINS) as pool:
        res = pool.map(_oracle_three_level, [(c, orc_iters, orc_burn, 2)
                                             for c in range(N_CHAINS)])
    o_psi = _chain_stats([r[0] for r in res])
    o_phi = _chain_stats([r[1] for r in res])
    g_psi, g_phi = [], []
    for c in range(N_CHAINS):
        sets = _sets(K=3, G=(300, 200, 250))
        rows = (gpu_iters - gpu_burn) // 5
        b = fbs.BatchSampler(sets, seeds=[9000 + 10 * c + k for k in range(3)],
                             chains=[c] * 3, trace_cap=rows)
        b.three_level(E, A_B, B_B, seed=4242 + c)
        b.run(gpu_iters, burnin=gpu_burn, thin=5)
        b.sync()
        top = b.top_level()
        assert top["trace"].shape[0] == rows and top["gamma_caps"] == 0
        g_psi.append(top["trace"])
        g_phi.append(np.stack([v.trace()["phi"] for v in b.views], 1))
        for v in b.views:
            cnt = v.counters()
            assert cnt["slice_caps"] == 0 and cnt["nonfinite"] == 0
        b.close()
    g_psi, g_phi = _chain_stats(g_psi), _chain_stats(g_phi)
    for name, g, o in (("psi", g_psi, o_psi), ("phi", g_phi, o_phi)):
        for j in (0, 2):
            z = np.abs(g[j] - o[j]) / np.hypot(g[j + 1], o[j + 1])
            assert np.all(z < 4.0), (name, "m1" if j == 0 else "m2", z)
