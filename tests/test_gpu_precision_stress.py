"""Configuration 2 at its full shape (N = 32, G = 200000, L = 5): the FP32 form
(FP32 slice log densities, FP64 reductions and hyperparameters,
Kahan-compensated FP32 moments) against the all-FP64 GPU path, which is itself
matched to the oracle step by step at this shape (test_gpu_parity.py).

Sixteen chains of each form start from the same default state and run the
same schedule; their random numbers differ (the two forms read the Philox words
in different roles), so the comparison is statistical.  The standard error of
each form's mean is that of its 16 chain means, which is valid inside the
burn-in transient too, since the chains are independent; the difference over
the hypot of the two standard errors is then t-distributed with about 30
degrees of freedom.  Every hyperparameter must lie within the t(30) quantile of
a familywise level of 1e-3 over the 12 of them (4.5), and for a subsample of
genes at most 2% of the per-gene means of beta, gamma and eps may lie beyond 4
(0.03% by chance).  The test prints the per-quantity error table: the relative
difference of the means and its size in standard errors.  The oracle's
own comparison at this design runs on a 2000-gene subsample in
test_gpu_posterior.py."""
import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CHAINS, ITERS, BURNIN = 16, 600, 200
GENE_STEP = 200   # every 200th gene: 1000 genes of the subsample


def _run(d, precision, seed):
    N, L = d["X"].shape
    G = d["y"].shape[0]
    P = 2 * L + 2
    rows = ITERS - BURNIN
    genes = np.arange(0, G, GENE_STEP)
    out = {"phi": [], "beta": [], "gam": [], "eps": []}
    for c in range(CHAINS):
        g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed, chain=c,
                        precision=precision, trace_cap=rows)
        g.run(ITERS, burnin=BURNIN, thin=1)
        g.sync()
        tr = g.trace()["phi"]
        assert tr.shape == (rows, P)
        out["phi"].append(tr.mean(0))
        m = g.moments()
        assert m["count"] == rows
        out["beta"].append(m["mean_beta"][genes])
        out["gam"].append(m["mean_gam"][genes])
        out["eps"].append(m["mean_eps"][genes])
        cnt = g.counters()
        assert cnt["slice_caps"] == 0 and cnt["nonfinite"] == 0
        g.close()
    return {k: np.array(v) for k, v in out.items()}


def test_precision_stress_fp32_against_fp64_full_shape():
    d = synthetic.make_config(2)
    assert d["y"].shape == (200000, 32)
    f64 = _run(d, fbs.FBS_F64, seed=2201)
    f32 = _run(d, fbs.FBS_F32, seed=2202)
    L = d["X"].shape[1]
    names = ["nu", "tau"] + [f"theta_{l + 1}" for l in range(L)] + \
            [f"sigma2_{l + 1}" for l in range(L)]
    from scipy import stats
    lines = ["quantity      FP64 mean      FP32 mean      rel. diff   |z| (SE of chain means)"]
    z = np.zeros(len(names))
    for k, nm in enumerate(names):
        a, b = f32["phi"][:, k], f64["phi"][:, k]
        z[k] = abs(a.mean() - b.mean()) / np.hypot(a.std(ddof=1), b.std(ddof=1)) * np.sqrt(CHAINS)
        rel = abs(a.mean() - b.mean()) / max(abs(b.mean()), 1e-300)
        lines.append(f"{nm:10s} {b.mean():14.7g} {a.mean():14.7g} {rel:12.2e} {z[k]:8.2f}")
    z_max = float(stats.t.isf(0.5e-3 / len(names), df=2 * (CHAINS - 1)))
    fracs = {}
    for key in ("beta", "gam", "eps"):
        a, b = f32[key], f64[key]
        se = np.hypot(a.std(0, ddof=1), b.std(0, ddof=1)) / np.sqrt(CHAINS)
        zz = np.abs(a.mean(0) - b.mean(0)) / np.maximum(se, 1e-300)
        rel = np.abs(a.mean(0) - b.mean(0)) / np.maximum(np.abs(b.mean(0)), 1e-12)
        fracs[key] = float(np.mean(zz > 4.0))
        lines.append(f"{key} means ({zz.size} values): median rel. diff {np.median(rel):.2e}, "
                     f"beyond 4 SE {100 * fracs[key]:.2f}%")
    print("\nprecision stress, FP32 vs FP64 GPU, N=32 G=200000 L=5, "
          f"{CHAINS} chains x {ITERS - BURNIN} post-burn-in sweeps each\n" + "\n".join(lines))
    assert np.all(z < z_max), (z_max, dict(zip(names, np.round(z, 2))))
    assert all(f <= 0.02 for f in fracs.values()), fracs
