"""Long-run agreement of the GPU chains (FP64 and FP32 forms) with the FP64
oracle: posterior means and mean squares of every hyperparameter and of the
beta_gl must agree within 4 Monte Carlo standard errors.

Different chains give different draws, so the comparison is statistical.  The
oracle runs 16 independent chains (spawned worker processes) and each GPU form
16, all started from the parameter values the synthetic counts were drawn from.
Each side uses its own seed: two forms given the same seed read the same
Philox words in different roles, and their chains would not be independent.
The MCSE of each side is the standard error of its chain means: the slowest
hyperparameters (sigma^2_3, sigma^2_4 at N=16) have integrated autocorrelation
times near 120 iterations, so shorter batches inside one chain would
underestimate it, while each oracle chain spans more than 10 of them.  Every hyperparameter must be within 4 MCSE.
For beta only parameters whose oracle effective sample size is at least 100
are compared (below that the MCSE estimate itself is unreliable); among them at
most 1% may exceed 4 MCSE (chance alone gives about 0.1%), and none of the well
mixed ones (oracle ESS at least 1000) may exceed the t(15) quantile of a
familywise level of 1e-3 (the MCSE of each side comes from 16 chain means).  A systematic error
shows up in the fraction; a lone large z of a slowly mixing, skewed parameter
in short oracle chains does not indicate one."""
import multiprocessing as mp

import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_ORACLE_CHAINS = 16
N_GPU_CHAINS = 16


def _truth_state(d):
    t = d["truth"]
    return {"eps": t["eps"], "beta": t["beta"], "gam": t["gam"], "phi": t["phi"]}


def _dataset(cfg, G):
    """Configuration cfg's inputs with G genes; cfg = ("batch", i): dataset i of
    configuration 3's batch (G is then the dataset's own)."""
    if isinstance(cfg, tuple):
        return synthetic.make_batch(cfg[1] + 1)[cfg[1]]
    return synthetic.make_config(cfg, G=G)


def _oracle_chain(args):
    cfg, G, iters, burnin, seed, chain = args
    import oracle
    d = _dataset(cfg, G)
    ch = oracle.Chain(d["y"], d["X"], d["h"], d["priors"], seed=seed, chain=chain,
                      burnin=burnin, tune_start=burnin // 2).init_default()
    ch.set_state(**_truth_state(d))
    tr = ch.run(iters, thin=1, trace_cap=iters, trace_beta=True)
    ess = np.array([oracle.ess(tr["beta"][:, g, l]) for g in range(tr["beta"].shape[1])
                    for l in range(tr["beta"].shape[2])]).reshape(tr["beta"].shape[1:])
    return tr["phi"], tr["beta"], ess


def _stats(traces):
    """Mean and mean square over chains with the standard errors of the chain means."""
    m1 = np.stack([tr.mean(0) for tr in traces])
    m2 = np.stack([(tr ** 2).mean(0) for tr in traces])
    k = m1.shape[0]
    return {"m1": m1.mean(0), "m1_se": m1.std(0, ddof=1) / np.sqrt(k),
            "m2": m2.mean(0), "m2_se": m2.std(0, ddof=1) / np.sqrt(k)}


@pytest.fixture(scope="module")
def pool():
    ctx = mp.get_context("spawn")
    with ctx.Pool(N_ORACLE_CHAINS) as p:
        yield p


def _compare(a, b, ess, label):
    """z = difference / hypot of the two sides' standard errors of the chain
    means.  With 16 chains per side each standard error has 15 degrees of
    freedom, so z has heavier tails than a normal variate: a gross error of a
    single well-mixed beta_gl is flagged beyond the t(15) quantile of a
    familywise level of 1e-3 over the compared parameters (about 9.5 for 10^4);
    a systematic error shows in the fraction beyond 4 (t(15): 0.1% by chance)."""
    from scipy import stats
    ok, well = ess >= 100, ess >= 1000
    n_well = max(2 * int(well.sum()), 1)
    z_max = float(stats.t.isf(0.5e-3 / n_well, df=N_GPU_CHAINS - 1))
    for m in ("m1", "m2"):
        z = np.abs(a["phi"][m] - b["phi"][m]) / np.hypot(a["phi"][m + "_se"], b["phi"][m + "_se"])
        assert np.all(z < 4.0), (label, "phi", m, z)
        z = np.abs(a["beta"][m] - b["beta"][m]) / np.hypot(a["beta"][m + "_se"],
                                                           b["beta"][m + "_se"])
        worst = np.unravel_index(np.argmax(np.where(ok, z, 0)), z.shape)
        info = (label, "beta", m, "worst (gene, l)", tuple(int(v) for v in worst),
                float(z[worst]), "ess", float(ess[worst]))
        assert np.mean(z[ok] > 4.0) <= 0.01, info + (float(np.mean(z[ok] > 4.0)),)
        assert np.all(z[well] < z_max), info + (z_max,)


_ORACLE_RUNS = {}


def _oracle_runs(pool, cfg, G, orc_iters):
    """Posterior means of the oracle's chains (computed once per configuration)
    and the summed effective sample sizes of the beta_gl.  The oracle's burn-in
    (a third of the run, 800 sweeps) spans more than 7 autocorrelation times of
    the slowest hyperparameter."""
    key = (cfg, G, orc_iters)
    if key not in _ORACLE_RUNS:
        orc_burn = orc_iters // 3
        jobs = [(cfg, G, orc_iters, orc_burn, 101, c) for c in range(N_ORACLE_CHAINS)]
        res = pool.map(_oracle_chain, jobs)
        orc = {"phi": _stats([r[0] for r in res]), "beta": _stats([r[1] for r in res])}
        _ORACLE_RUNS[key] = (orc, sum(r[2] for r in res))
    return _ORACLE_RUNS[key]


@pytest.mark.parametrize("cfg,G,orc_iters,gpu_iters", [(0, 1000, 2400, 12000),
                                                       (1, 1000, 2400, 12000),
                                                       (2, 2000, 2400, 12000)])
def test_long_runs_agree_with_oracle(pool, cfg, G, orc_iters, gpu_iters):
    """FP64 GPU vs oracle, FP32 GPU vs oracle and FP32 GPU vs FP64 GPU.
    Configuration 2 (the precision stress: N = 32, 8 libraries per variety of the
    paper's design) runs here on a subsample of 2000 genes, which the oracle can
    afford; its full shape is compared with the FP64 GPU path in
    test_gpu_precision_stress.py."""
    orc, ess = _oracle_runs(pool, cfg, G, orc_iters)
    assert (ess >= 100).mean() > 0.5
    d = synthetic.make_config(cfg, G=G)
    gpu_burn, thin = gpu_iters // 6, 10
    rows = (gpu_iters - gpu_burn) // thin
    runs = {}
    for precision in (fbs.FBS_F64, fbs.FBS_F32):
        phis, betas = [], []
        for c in range(N_GPU_CHAINS):
            g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=202 + 1000 * precision,
                            chain=c, precision=precision, trace_cap=rows, trace_beta=1)
            g.set_state(it=0, **_truth_state(d))
            g.run(gpu_iters, burnin=gpu_burn, thin=thin)
            g.sync()
            tr = g.trace(beta=True)
            assert tr["phi"].shape[0] == rows
            cnt = g.counters()
            assert cnt["slice_caps"] == 0 and cnt["nonfinite"] == 0
            phis.append(tr["phi"])
            betas.append(tr["beta"])
            g.close()
        runs[precision] = {"phi": _stats(phis), "beta": _stats(betas)}
        _compare(runs[precision], orc, ess, f"cfg {cfg} precision {precision} vs oracle")
    _compare(runs[fbs.FBS_F32], runs[fbs.FBS_F64], ess, f"cfg {cfg} FP32 vs FP64")


def _learned_params(d, seed=77):
    t = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed, precision=fbs.FBS_F32)
    t.set_state(it=0, **_truth_state(d))
    t.proposal_collect(300, burnin=300, thin=2)
    t.proposal_train(epochs=20, batch=2048, lr=2e-3, seed=seed)
    params = t.proposal_params()
    t.close()
    return params


def _learned_chains(d, params, n_iter, burnin, thin, seed, starts=None, min_accept=0.2):
    """16 chains of the FP32 sampler with the learned move (mode 1); each
    calibrates during the first 100 sweeps of its burn-in.  Returns the traces'
    statistics and the chains' final states."""
    rows = (n_iter - burnin) // thin
    phis, betas, ends = [], [], []
    for c in range(N_GPU_CHAINS):
        g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed, chain=c,
                        precision=fbs.FBS_F32, trace_cap=rows, trace_beta=1)
        g.set_state(it=0, **(starts[c] if starts else _truth_state(d)))
        g.proposal_params(set_to=params)
        g.proposal_calibrate(100, burnin=burnin, min_accept=min_accept)
        g.run(n_iter - 100, burnin=burnin, thin=thin)
        g.sync()
        st = g.proposal_stats()
        assert st["mh_genes"] > 0.8 * d["y"].shape[0]
        assert st["accepted"] > 0.3 * st["tried"]
        tr = g.trace(beta=True)
        assert tr["phi"].shape[0] == rows
        cnt = g.counters()
        assert cnt["slice_caps"] == 0 and cnt["nonfinite"] == 0
        phis.append(tr["phi"])
        betas.append(tr["beta"])
        s = g.get_state()
        ends.append({k: s[k] for k in ("eps", "beta", "gam", "phi")})
        g.close()
    return {"phi": _stats(phis), "beta": _stats(betas)}, ends


def test_learned_long_runs_agree_with_oracle(pool):
    """The FP32 sampler with the learned move of the beta_g block against the
    oracle's plain sampler on configuration 0's design (N = 4, L = 2), where the
    plain chains forget their start within the oracle's run.  The network is
    trained once, on draws of one chain started from the generating values; each
    of the 16 chains then calibrates (every gene tries the move for 100 sweeps of
    the burn-in) and runs with its own seed."""
    cfg, G, orc_iters, gpu_iters = 0, 1000, 2400, 12000
    orc, ess = _oracle_runs(pool, cfg, G, orc_iters)
    d = synthetic.make_config(cfg, G=G)
    learned, _ = _learned_chains(d, _learned_params(d), gpu_iters, gpu_iters // 6, 10, 3030)
    _compare(learned, orc, ess, "learned FP32 vs oracle")


def _overdispersed_start(d, rng):
    """A start spread out relative to the posterior (the paper starts its chains
    overdispersed, §5): least-squares beta_g of log(y + 1) - h on X plus N(0, 0.5^2)
    noise, eps = 0, gamma_g = 1, nu uniform on (1, 9), tau, sigma^2_l scaled by
    log-normal factors and theta_l shifted by N(0, 0.5^2)."""
    X, y, h = d["X"], d["y"], d["h"]
    L = X.shape[1]
    b = np.linalg.lstsq(X, (np.log(y + 1.0) - h).T, rcond=None)[0].T
    beta = b + rng.normal(0, 0.5, b.shape)
    theta = beta.mean(0) + rng.normal(0, 0.5, L)
    sig2 = np.clip(beta.var(0), 1e-4, None) * np.exp(rng.normal(0, 0.7, L))
    phi = np.concatenate([[rng.uniform(1, 9), 0.1 * np.exp(rng.normal(0, 1))], theta, sig2])
    return {"eps": np.zeros_like(y, dtype=np.float64), "beta": beta,
            "gam": np.ones(y.shape[0]), "phi": phi}


def _block_reference_chain(args):
    """One chain of the independent reference: the oracle's plain sweep
    (Algorithm 1) followed by an exact Gibbs update of every beta_g given its
    log-rates (oracle.proposal.block_step), all in FP64 on the CPU.  Returns the
    chain's post-burn-in means and mean squares of phi and beta and the beta_gl's
    effective sample sizes."""
    cfg, G, iters, burnin, seed, chain, start = args
    import oracle
    from oracle import proposal as P
    from paper_1606_06659_gb300 import synthetic as syn
    d = syn.make_config(cfg, G=G)
    X = d["X"]
    L = X.shape[1]
    ch = oracle.Chain(d["y"], X, d["h"], d["priors"], seed=seed, chain=chain, burnin=burnin,
                      tune_start=burnin // 2).init_default()
    rng = np.random.default_rng([seed, chain, 1606])
    ch.set_state(**(_truth_state(d) if start == "truth" else _overdispersed_start(d, rng)))
    rows = iters - burnin
    tphi = np.empty((rows, 2 * L + 2))
    tbeta = np.empty((rows, G, L))
    for m in range(1, iters + 1):
        ch.sweep()
        phi = ch.phi.copy()
        eps, beta = P.block_step(ch.eps, ch.beta, ch.gam, phi[2:2 + L], phi[2 + L:], X,
                                 rng.normal(size=(G, L)))
        ch.set_state(eps=eps, beta=beta)
        if m > burnin:
            tphi[m - burnin - 1] = phi
            tbeta[m - burnin - 1] = beta
    ess = np.array([oracle.ess(tbeta[:, g, l]) for g in range(G) for l in range(L)]).reshape(G, L)
    return {"m1_phi": tphi.mean(0), "m2_phi": (tphi ** 2).mean(0),
            "m1_beta": tbeta.mean(0), "m2_beta": (tbeta ** 2).mean(0), "ess": ess, "M": rows}


def _stats_of_chains(res, key):
    m1 = np.stack([r["m1_" + key] for r in res])
    m2 = np.stack([r["m2_" + key] for r in res])
    k = m1.shape[0]
    return {"m1": m1.mean(0), "m1_se": m1.std(0, ddof=1) / np.sqrt(k),
            "m2": m2.mean(0), "m2_se": m2.std(0, ddof=1) / np.sqrt(k)}


@pytest.mark.parametrize("min_accept", [0.01, 0.2])
def test_learned_agrees_with_independent_block_reference(pool, min_accept):
    """The learned form at the paper's design (N = 16, L = 5, 1000 genes) against
    a reference that shares neither its code nor its start.  At this design the
    plain sampler keeps part of its start for tens of thousands of sweeps (the
    beta_gl of genes with large counts move slowly because eps and beta are
    tightly coupled), so it cannot serve as the reference.  The reference adds to
    the oracle's plain sweep an exact Gibbs update of each beta_g given its
    log-rates, the Gaussian conditional that the learned network approximates,
    derived from the model (§4.1) and pinned by its joint density; 16 chains, 8
    from the generating values and 8 from overdispersed starts.  Their
    Gelman-Rubin factors (§3.1) of every hyperparameter must be below 1.01, which
    shows that the reference forgets its start; pooled, they must agree with the
    learned chains within 4 MCSE for every hyperparameter, and for beta as in the
    other posterior tests.  The learned chains calibrate with the benchmark's
    acceptance threshold (0.01, where the move adds to the slice updates) and
    with configuration 4's 0.2."""
    import oracle
    cfg, G = 1, 1000
    ref_iters, ref_burn = 3000, 1000
    if (cfg, G, "block") not in _ORACLE_RUNS:
        jobs = [(cfg, G, ref_iters, ref_burn, 606, c, "truth" if c % 2 == 0 else "overdispersed")
                for c in range(N_ORACLE_CHAINS)]
        _ORACLE_RUNS[(cfg, G, "block")] = pool.map(_block_reference_chain, jobs)
    res = _ORACLE_RUNS[(cfg, G, "block")]
    M = res[0]["M"]
    rhat = oracle.rhat([r["m1_phi"] for r in res], [r["m2_phi"] for r in res], M)
    assert np.all(rhat < 1.01), rhat
    ref = {"phi": _stats_of_chains(res, "phi"), "beta": _stats_of_chains(res, "beta")}
    ess = sum(r["ess"] for r in res)
    d = synthetic.make_config(cfg, G=G)
    if "params" not in _ORACLE_RUNS:
        _ORACLE_RUNS["params"] = _learned_params(d)
    learned, _ = _learned_chains(d, _ORACLE_RUNS["params"], 12000, 2000, 10,
                                 4040 + int(min_accept * 100), min_accept=min_accept)
    _compare(learned, ref, ess, f"learned FP32 (min_accept {min_accept}) vs block reference")


def test_all_slice_long_runs_agree_with_oracle(pool):
    """The all-slice FP64 variant (gamma_g, tau, sigma_l by slice updates) targets
    the same posterior as the exact draws: its GPU chains against the oracle's
    chains of the exact-draw sampler, at configuration 0."""
    cfg, G, orc_iters, gpu_iters = 0, 1000, 2400, 12000
    orc, ess = _oracle_runs(pool, cfg, G, orc_iters)
    d = synthetic.make_config(cfg, G=G)
    gpu_burn, thin = gpu_iters // 6, 10
    rows = (gpu_iters - gpu_burn) // thin
    phis, betas = [], []
    for c in range(N_GPU_CHAINS):
        g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=303, chain=c, all_slice=1,
                        trace_cap=rows, trace_beta=1)
        g.set_state(it=0, **_truth_state(d))
        g.run(gpu_iters, burnin=gpu_burn, thin=thin)
        g.sync()
        tr = g.trace(beta=True)
        cnt = g.counters()
        assert cnt["slice_caps"] == 0 and cnt["nonfinite"] == 0 and cnt["gamma_caps"] == 0
        assert cnt["evals_gam"] > 0 and cnt["evals_hyp"] > 0
        phis.append(tr["phi"])
        betas.append(tr["beta"])
        g.close()
    _compare({"phi": _stats(phis), "beta": _stats(betas)}, orc, ess,
             "cfg 0 all-slice FP64 vs oracle")


def test_batch_datasets_agree_with_oracle(pool):
    """Configuration 3: datasets 33 (N = 8, G = 1791, L = 5, the paper's design
    with two libraries per variety) and 50 (N = 13, G = 1390, L = 2) of the
    64-dataset batch, each as 16 chains with their own seeds inside one batch of
    32 datasets (one set of launches per sweep, FP32), against 16 oracle chains
    per dataset, as in the single-chain posterior tests."""
    picks = (33, 50)
    orc_iters, gpu_iters = 2400, 12000
    gpu_burn, thin = gpu_iters // 6, 10
    rows = (gpu_iters - gpu_burn) // thin
    sets = [synthetic.make_batch(max(picks) + 1)[i] for i in picks]
    batch, seeds, chains = [], [], []
    for k, d in enumerate(sets):
        for c in range(N_GPU_CHAINS):
            batch.append(d)
            seeds.append(909 + k)
            chains.append(c)
    b = fbs.BatchSampler(batch, seeds=seeds, chains=chains, trace_cap=rows, trace_beta=1)
    for j, d in enumerate(batch):
        b.chain(j).set_state(it=0, **_truth_state(d))
    b.run(gpu_iters, burnin=gpu_burn, thin=thin)
    b.sync()
    for k, i in enumerate(picks):
        orc, ess = _oracle_runs(pool, ("batch", i), None, orc_iters)
        phis, betas = [], []
        for c in range(N_GPU_CHAINS):
            v = b.chain(k * N_GPU_CHAINS + c)
            tr = v.trace(beta=True)
            assert tr["phi"].shape[0] == rows
            cnt = v.counters()
            assert cnt["slice_caps"] == 0 and cnt["nonfinite"] == 0
            phis.append(tr["phi"])
            betas.append(tr["beta"])
        _compare({"phi": _stats(phis), "beta": _stats(betas)}, orc, ess,
                 f"batch dataset {i} vs oracle")
    b.close()
