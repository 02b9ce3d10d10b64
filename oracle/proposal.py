"""Plain FP64 numpy oracle of the learned beta_g proposal (test infrastructure only).

The proposal is a multilayer perceptron with two hidden layers and the GELU
activation (tanh form, Hendrycks & Gimpel 2016) mapping per-gene features to a
Gaussian N(mu, C C^T) over the L coefficients beta_g: the first L outputs are
mu, the next L the logs of the diagonal of the lower Cholesky factor C, the
remaining L(L-1)/2 its sub-diagonal entries in row order.  Training minimises
the Gaussian negative log-likelihood
    0.5 ||C^-1 (beta - mu)||^2 + sum_l log C_ll     (+ L/2 log 2 pi),
written here from its definition with explicit backpropagation.

Features of a gene are invariant under the proposal's move, which keeps every
log-rate eta_gn = h_n + eps_gn + X_n beta_g fixed: X^T (eta_g - h) / N (L
values), asinh(X^T y_g) (L), log gamma_g (1), theta (L) and log sigma (L).

The move proposes from the multivariate t distribution with T_DOF degrees of
freedom, centre mu and scale matrix C C^T (the Gaussian's parameters): beta* =
mu + s C xi with xi standard normal and s = sqrt(T_DOF / chi2), chi2 a
chi-square variate with T_DOF degrees of freedom.  Its polynomial tails dominate
the Gaussian tails of the move's target, so the ratio target / proposal is
bounded and the independence sampler is uniformly ergodic (Mengersen & Tweedie
1996), even where the network's scale is too small.
Pinned by scipy's multivariate normal and t densities and by finite differences.

block_conditional / block_step: the exact Gaussian full conditional of beta_g
given its log-rates (the distribution the network learns to approximate) and an
exact Gibbs update from it; the tests use a chain of the oracle's sweeps with
this update added as an independent reference posterior.  Pinned by the joint
density of the model at fixed log-rates (scipy Poisson and Normal terms).
"""
from __future__ import annotations

import numpy as np

SQRT_2_OVER_PI = np.sqrt(2.0 / np.pi)
T_DOF = 8


def n_features(L):
    return 4 * L + 1


def n_outputs(L):
    return L + L * (L + 1) // 2


def features(eps, beta, gam, theta, sigma2, y, X):
    """Feature rows [G][4L+1] from the state (eps [G][N], beta [G][L], gam [G]),
    the hyperparameters and the data."""
    eps, beta, y, X = map(np.asarray, (eps, beta, y, X))
    N = X.shape[0]
    lin = eps + beta @ X.T                       # eta - h
    a = lin @ X / N
    t = np.arcsinh(y.astype(np.float64) @ X)
    G = eps.shape[0]
    return np.hstack([a, t, np.log(np.asarray(gam))[:, None],
                      np.tile(theta, (G, 1)), np.tile(0.5 * np.log(sigma2), (G, 1))])


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(SQRT_2_OVER_PI * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    u = SQRT_2_OVER_PI * (x + 0.044715 * x ** 3)
    t = np.tanh(u)
    du = SQRT_2_OVER_PI * (1.0 + 3 * 0.044715 * x ** 2)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t ** 2) * du


def init_params(n_in, n_out, hidden=64, seed=0):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, np.sqrt(2.0 / n_in), (hidden, n_in)), "b1": np.zeros(hidden),
            "W2": rng.normal(0, np.sqrt(2.0 / hidden), (hidden, hidden)), "b2": np.zeros(hidden),
            "W3": rng.normal(0, 0.1 * np.sqrt(1.0 / hidden), (n_out, hidden)),
            "b3": np.zeros(n_out)}


def forward(p, f):
    z1 = f @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (f, z1, h1, z2, h2)


def unpack(out, L):
    """mu [B][L] and the lower Cholesky factor C [B][L][L] from outputs [B][n_out]."""
    B = out.shape[0]
    mu = out[:, :L]
    C = np.zeros((B, L, L))
    C[:, np.arange(L), np.arange(L)] = np.exp(out[:, L:2 * L])
    k = 2 * L
    for i in range(1, L):
        for j in range(i):
            C[:, i, j] = out[:, k]
            k += 1
    return mu, C


def nll(out, beta, L):
    """Per-row Gaussian negative log-likelihood, without the constant."""
    mu, C = unpack(out, L)
    u = np.linalg.solve(C, (beta - mu)[..., None])[..., 0]
    return 0.5 * np.sum(u * u, axis=1) + np.sum(out[:, L:2 * L], axis=1)


def nll_grad_out(out, beta, L):
    """d(nll)/d(out) per row: with u = C^-1 (beta - mu) and v = C^-T u,
    d/dmu = -v, d/dlogC_ii = 1 - v_i u_i C_ii, d/dC_ij = -v_i u_j (i > j)."""
    mu, C = unpack(out, L)
    u = np.linalg.solve(C, (beta - mu)[..., None])[..., 0]
    v = np.linalg.solve(np.transpose(C, (0, 2, 1)), u[..., None])[..., 0]
    g = np.zeros_like(out)
    g[:, :L] = -v
    g[:, L:2 * L] = 1.0 - v * u * np.exp(out[:, L:2 * L])
    k = 2 * L
    for i in range(1, L):
        for j in range(i):
            g[:, k] = -v[:, i] * u[:, j]
            k += 1
    return g


def loss_and_grads(p, f, beta, L):
    """Mean NLL over the rows and its gradients with respect to every parameter."""
    out, (f, z1, h1, z2, h2) = forward(p, f)
    B = f.shape[0]
    loss = float(np.mean(nll(out, beta, L)))
    go = nll_grad_out(out, beta, L) / B
    g = {"W3": go.T @ h2, "b3": go.sum(0)}
    gh2 = go @ p["W3"]
    gz2 = gh2 * gelu_grad(z2)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(0)
    gh1 = gz2 @ p["W2"]
    gz1 = gh1 * gelu_grad(z1)
    g["W1"] = gz1.T @ f
    g["b1"] = gz1.sum(0)
    return loss, g


def t_log_ratio(out, beta, beta_new, L, dof=T_DOF):
    """log q(beta) - log q(beta_new) for the multivariate t proposal of centre mu
    and scale C C^T (the normalising constants cancel)."""
    mu, C = unpack(out, L)
    u0 = np.linalg.solve(C, (beta - mu)[..., None])[..., 0]
    u1 = np.linalg.solve(C, (beta_new - mu)[..., None])[..., 0]
    a = 0.5 * (dof + L)
    return -a * (np.log1p(np.sum(u0 * u0, 1) / dof) - np.log1p(np.sum(u1 * u1, 1) / dof))


def mh_log_ratio(eps, beta, beta_new, gam, theta, sigma2, X, out):
    """log of the acceptance ratio of the eta-preserving move to beta_new
    (eps_new = eps - X (beta_new - beta)): the Poisson likelihood is unchanged,
    so the ratio holds the Normal(0, gamma) priors of eps, the Normal(theta, sigma^2)
    priors of beta and the t proposal densities q(beta) / q(beta_new)."""
    L = beta.shape[1]
    eps_new = eps - (beta_new - beta) @ X.T
    lp = (-0.5 * np.sum(eps_new ** 2, 1) / gam - 0.5 * np.sum((beta_new - theta) ** 2 / sigma2, 1)
          + 0.5 * np.sum(eps ** 2, 1) / gam + 0.5 * np.sum((beta - theta) ** 2 / sigma2, 1))
    return lp + t_log_ratio(out, beta, beta_new, L)


def mh_move(eps, beta, gam, theta, sigma2, X, out, xi, log_u, chi2):
    """The eta-preserving move of every row from standard normals xi [G][L],
    chi-square variates chi2 [G] (T_DOF degrees of freedom) and log-uniforms
    log_u [G]: beta* = mu + sqrt(T_DOF / chi2) C xi, eps* = eps - X (beta* - beta),
    accepted where log_u < the log ratio of mh_log_ratio.  Returns the new eps,
    beta, the acceptance flags and the log ratios."""
    L = beta.shape[1]
    mu, C = unpack(out, L)
    s = np.sqrt(T_DOF / np.asarray(chi2))
    beta_new = mu + s[:, None] * np.einsum("gij,gj->gi", C, xi)
    la = mh_log_ratio(eps, beta, beta_new, gam, theta, sigma2, X, out)
    acc = log_u < la
    eps_new = np.where(acc[:, None], eps - (beta_new - beta) @ X.T, eps)
    return eps_new, np.where(acc[:, None], beta_new, beta), acc, la


def block_conditional(eps, beta, gam, theta, sigma2, X):
    """The full conditional of beta_g given the log-rates eta_g = h + eps_g + X
    beta_g (and gamma_g, theta, sigma^2), per row: the Poisson likelihood depends
    on (eps_g, beta_g) only through eta_g, so given eta_g the model leaves the
    Normal(0, gamma_g) prior of eps_g = eta_g - h - X beta_g and the
    Normal(theta, sigma^2) prior of beta_g, a Gaussian in beta_g with precision
    X^T X / gamma_g + diag(1 / sigma^2) and mean that precision's inverse times
    X^T (eta_g - h) / gamma_g + theta / sigma^2.  Returns the means [G][L] and
    the covariances [G][L][L]."""
    eps, beta, X = map(np.asarray, (eps, beta, X))
    gam = np.asarray(gam, np.float64)
    lin = eps + beta @ X.T                                 # eta - h
    prec = (X.T @ X)[None] / gam[:, None, None] + np.diag(1.0 / np.asarray(sigma2))[None]
    cov = np.linalg.inv(prec)
    rhs = lin @ X / gam[:, None] + (np.asarray(theta) / np.asarray(sigma2))[None]
    return np.einsum("gij,gj->gi", cov, rhs), cov


def block_step(eps, beta, gam, theta, sigma2, X, z):
    """An exact Gibbs update of every beta_g given its log-rates (Section 4.1's
    model in the coordinates (eta_g, beta_g), whose map from (eps_g, beta_g) has
    unit Jacobian): beta* = mean + chol(cov) z from block_conditional with
    standard normals z [G][L], and eps* = eps - X (beta* - beta), which keeps
    every log-rate.  Returns (eps*, beta*)."""
    mean, cov = block_conditional(eps, beta, gam, theta, sigma2, X)
    beta_new = mean + np.einsum("gij,gj->gi", np.linalg.cholesky(cov), np.asarray(z))
    return np.asarray(eps) - (beta_new - np.asarray(beta)) @ np.asarray(X).T, beta_new
