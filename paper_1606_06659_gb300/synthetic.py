"""Seeded synthetic RNA-seq inputs with the shapes of the paper's workloads.

This module generates inputs only: counts, design, offsets, priors, the
parameter values the counts were drawn from, and run lengths.  It holds none
of the sampler's arithmetic, so both the CUDA library and the CPU oracle can be
fed from it without sharing method code.

Generation follows the model of Section 4.1 (Figure 3) forwards:
gamma_g ~ Inverse-Gamma(nu/2, nu tau/2), eps_gn ~ Normal(0, gamma_g),
beta_gl ~ Normal(theta_l, sigma_l^2), y_gn ~ Poisson(exp(h_n + eps_gn + X_n beta_g)),
with h_n ~ Normal(0, 0.1^2).  The Poisson mean is clamped at 2^30 so that counts
fit int32; the number of clamped cells is returned.  The paper's Paschold data
are not available; these draws stand in for them with the same N, G, L, design
and count range.
"""
from __future__ import annotations

import numpy as np

GENERATOR_SEED = 20160621
LAMBDA_CLAMP = float(2 ** 30)


def paper_design(reps: int = 4) -> np.ndarray:
    """The N x 5 model matrix of Section 5: four varieties (B73, Mo17, B73xMo17,
    Mo17xB73) with `reps` libraries each; columns are the parental mean, the two
    hybrid-vs-parent half differences, the hybrid half difference and a +/-1
    flow-cell block split within each variety."""
    base = np.array([[1, 1, -1, 0],
                     [1, -1, 1, 0],
                     [1, 1, 1, 1],
                     [1, 1, 1, -1]], np.float64)
    half = reps // 2
    block = np.array([1.0] * half + [-1.0] * (reps - half))
    left = np.kron(base, np.ones((reps, 1)))
    right = np.kron(np.ones((4, 1)), block.reshape(-1, 1))
    return np.hstack([left, right])


def two_group_design(N: int) -> np.ndarray:
    """Intercept plus a +/-1 treatment split (first half +1, second half -1)."""
    half = N // 2
    return np.stack([np.ones(N), np.array([1.0] * half + [-1.0] * (N - half))], axis=1)


def default_priors(L: int, a=1.0, b=1.0, d=10.0, c=10.0, s=10.0) -> dict:
    return {"a": float(a), "b": float(b), "d": float(d),
            "c": np.full(L, float(c)), "s": np.full(L, float(s))}


def simulate(X, theta, sigma, tau, nu, G, seed, h_sd=0.1, rng=None) -> dict:
    """Draw one dataset from the model with the given parameter values."""
    X = np.asarray(X, np.float64)
    N, L = X.shape
    rng = rng if rng is not None else np.random.default_rng(seed)
    h = rng.normal(0.0, h_sd, size=N)
    # gamma_g ~ IG(nu/2, scale nu*tau/2)  <=>  1/gamma_g ~ Gamma(nu/2, scale 2/(nu*tau))
    gam = 1.0 / rng.gamma(nu / 2.0, 2.0 / (nu * tau), size=G)
    eps = rng.normal(0.0, 1.0, size=(G, N)) * np.sqrt(gam)[:, None]
    beta = rng.normal(np.asarray(theta)[None, :], np.asarray(sigma)[None, :], size=(G, L))
    lam = np.exp(h[None, :] + eps + beta @ X.T)
    clamped = int(np.count_nonzero(~(lam <= LAMBDA_CLAMP)))
    lam = np.minimum(np.nan_to_num(lam, nan=LAMBDA_CLAMP, posinf=LAMBDA_CLAMP), LAMBDA_CLAMP)
    y = rng.poisson(lam).astype(np.int32)
    phi = np.concatenate([[nu, tau], np.asarray(theta, np.float64),
                          np.asarray(sigma, np.float64) ** 2])
    return {"y": y, "X": X, "h": h, "truth": {"eps": eps, "beta": beta, "gam": gam, "phi": phi},
            "clamped": clamped}


CONFIGS = {
    0: dict(name="tiny N=4 G=1000 L=2", N=4, G=1000, L=2, theta=(3.0, 0.0), sigma=(1.5, 0.3),
            tau=0.1, nu=3.0, iters=1000, burnin=500, thin=1),
    1: dict(name="paper-scale N=16 G=40000 L=5", N=16, G=40000, L=5,
            theta=(4.0, 0.0, 0.0, 0.0, 0.0), sigma=(2.0, 0.5, 0.3, 0.2, 0.2), tau=0.1, nu=3.0,
            iters=20000, burnin=10000, thin=10),
    2: dict(name="precision stress N=32 G=200000 L=5", N=32, G=200000, L=5,
            theta=(4.0, 0.0, 0.0, 0.0, 0.0), sigma=(2.0, 0.5, 0.3, 0.2, 0.2), tau=0.1, nu=3.0,
            iters=50000, burnin=25000, thin=10),
}


def make_config(cfg: int, G: int | None = None, seed: int | None = None) -> dict:
    """Inputs for configuration 0, 1 or 2 (optionally with fewer genes)."""
    spec = dict(CONFIGS[cfg])
    if G is not None:
        spec["G"] = int(G)
    N, L = spec["N"], spec["L"]
    if cfg == 0:
        X = two_group_design(N)
    elif cfg == 1:
        X = paper_design(4)
    else:
        X = paper_design(8)
    assert X.shape == (N, L)
    seed = GENERATOR_SEED + cfg if seed is None else seed
    data = simulate(X, spec["theta"], spec["sigma"], spec["tau"], spec["nu"], spec["G"], seed)
    data.update(priors=default_priors(L), spec=spec, seed=seed)
    return data


def make_batch(n_sets: int = 64, seed: int = GENERATOR_SEED + 3, max_G: int = 100000,
               min_G: int = 1000) -> list[dict]:
    """Configuration 3: datasets with N uniform on {4..32}, G log-uniform on
    [min_G, max_G], L in {2, 5}; L = 5 uses the paper's design with N rounded
    down to a multiple of 4 (at least 8)."""
    rng = np.random.default_rng(seed)
    sets = []
    for i in range(n_sets):
        N = int(rng.integers(4, 33))
        G = int(np.exp(rng.uniform(np.log(min_G), np.log(max_G))))
        L = int(rng.choice([2, 5]))
        if L == 5:
            N = max(8, (N // 4) * 4)
            X = paper_design(N // 4)
            theta, sigma = (4.0, 0.0, 0.0, 0.0, 0.0), (2.0, 0.5, 0.3, 0.2, 0.2)
        else:
            X = two_group_design(N)
            theta, sigma = (3.0, 0.0), (1.5, 0.3)
        d = simulate(X, theta, sigma, 0.1, 3.0, G, seed=None, rng=rng)
        d.update(priors=default_priors(X.shape[1]), seed_index=i)
        sets.append(d)
    return sets
