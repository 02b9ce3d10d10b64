"""Pins for the oracle's three-level model (Section 2.3, Figure 2): K datasets
of the RNA-seq model whose hyperparameters share psi = (b, m_1..m_L) through
tau_k ~ Gamma(a_k, rate b) and theta_kl ~ N(m_l, c_kl^2), with b ~ Gamma(a_b,
rate b_b) and m_l ~ N(0, e_l^2).

Every target is the product of scipy.stats densities of the model's terms,
normalised by quadrature, and the oracle's draws must pass a
Kolmogorov-Smirnov test against it.  A composition test (Geweke) checks that
the psi step and the datasets' tau and theta steps with the top-level priors
fit together into a sampler of the joint distribution."""
import numpy as np
from scipy import stats

import oracle
from tests._quad import GridDist, bracket, ks_pvalue, vectorized
from tests.test_oracle_conditionals import P_MIN, make_chain

K, L = 4, 2
A_K = np.array([2.0, 1.5, 3.0, 2.5])
C_KL = np.array([[1.0, 0.5], [2.0, 0.8], [1.5, 0.6], [0.7, 1.2]])
E = np.array([3.0, 0.4])
A_B, B_B = 2.0, 1.5


def _phi(tau, theta):
    phi = np.zeros((K, 2 * L + 2))
    phi[:, 0] = 3.0
    phi[:, 1] = tau
    phi[:, 2:2 + L] = theta
    phi[:, 2 + L:] = 0.3
    return phi


def _psi_draws(phi, n, seed=5):
    lib = oracle.load()
    import ctypes as C
    pd = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    phi = np.ascontiguousarray(phi)
    a, c, e = (np.ascontiguousarray(v, np.float64) for v in (A_K, C_KL, E))
    psi = np.zeros(1 + L)
    caps = C.c_int64(0)
    out = []
    for it in range(1, n + 1):
        lib.orc_step_psi(K, L, pd(phi), pd(a), pd(c), pd(e), A_B, B_B, seed, it, pd(psi),
                         C.byref(caps))
        out.append(psi.copy())
    assert caps.value == 0
    return np.array(out)


def test_psi_step_matches_posterior():
    tau = np.array([0.8, 1.6, 0.5, 2.2])
    theta = np.array([[1.0, -0.2], [2.5, 0.3], [0.2, 0.1], [1.7, -0.6]])
    draws = _psi_draws(_phi(tau, theta), 5000)

    @vectorized
    def logpost_b(b):
        b = np.asarray(b, float)
        out = stats.gamma.logpdf(b, A_B, scale=1 / B_B)
        for k in range(K):
            out = out + stats.gamma.logpdf(tau[k], A_K[k], scale=1 / np.maximum(b, 1e-300))
        return np.where(b > 0, out, -np.inf)

    lo, hi = bracket(logpost_b, 1.5, 0.05, lo_bound=1e-9)
    assert ks_pvalue(draws[:, 0], GridDist(logpost_b, lo, hi)) > P_MIN
    for l in range(L):
        @vectorized
        def logpost_m(m, l=l):
            m = np.asarray(m, float)
            out = stats.norm.logpdf(m, 0, E[l])
            for k in range(K):
                out = out + stats.norm.logpdf(theta[k, l], m, C_KL[k, l])
            return out

        lo, hi = bracket(logpost_m, theta[:, l].mean(), 0.05)
        assert ks_pvalue(draws[:, 1 + l], GridDist(logpost_m, lo, hi)) > P_MIN


def test_theta_and_tau_steps_use_the_top_level():
    """With psi set, theta_l has the prior N(m_l, c_l^2) and tau the prior
    Gamma(a, rate b)."""
    G = 12
    pri = {"a": 2.0, "b": 3.0, "d": 10.0, "c": np.array([0.5, 2.0]), "s": np.full(2, 10.0)}
    ch = make_chain(G, priors=pri)
    b_top, m_top = 0.7, np.array([2.0, -1.5])
    ch.set_top_level(b_top, m_top)
    rng = np.random.default_rng(1)
    beta = np.stack([rng.normal(1.0, 0.6, G), rng.normal(-0.3, 0.4, G)], 1)
    sig2 = np.array([0.36, 0.16])
    gam = np.array([0.1, 0.3, 0.25, 0.7, 0.05, 0.2, 0.4, 0.15, 0.3, 0.2, 0.6, 0.35])
    nu = 2.5
    th, ta = [], []
    for it in range(1, 4001):
        ch.set_state(beta=beta, gam=gam, phi=[nu, 1.0, 0.0, 0.0, *sig2])
        ch.step_tau(it)
        ch.step_theta(it)
        ta.append(ch.phi[1])
        th.append(ch.phi[2:4].copy())
    th = np.array(th)
    for l in range(2):
        @vectorized
        def logpost(t, l=l):
            t = np.asarray(t, float)
            out = stats.norm.logpdf(t, m_top[l], pri["c"][l])
            for bv in beta[:, l]:
                out = out + stats.norm.logpdf(bv, t, np.sqrt(sig2[l]))
            return out
        lo, hi = bracket(logpost, beta[:, l].mean(), 0.05)
        assert ks_pvalue(th[:, l], GridDist(logpost, lo, hi)) > P_MIN

    @vectorized
    def logpost_tau(t):
        t = np.asarray(t, float)
        out = stats.gamma.logpdf(t, 2.0, scale=1 / b_top)
        for gv in gam:
            out = out + stats.invgamma.logpdf(gv, nu / 2, scale=nu * np.maximum(t, 1e-300) / 2)
        return np.where(t > 0, out, -np.inf)

    lo, hi = bracket(logpost_tau, 0.2, 0.02, lo_bound=1e-9)
    assert ks_pvalue(ta, GridDist(logpost_tau, lo, hi)) > P_MIN


def test_geweke_top_level_composition():
    """Successive-conditional simulation of (psi, tau_k, theta_k) with the other
    parameters of each dataset (gamma, beta, nu, sigma^2) redrawn from the
    model given them: the Gibbs steps (the datasets' tau and theta steps with
    the top-level priors, then psi) must keep the joint prior, so the means of
    psi and of tau_k, theta_kl over the successive draws equal their prior
    means computed by direct forward simulation (|z| < 4.5, batch-mean SE)."""
    rng = np.random.default_rng(11)
    G = 6
    chains = []
    for k in range(K):
        pri = {"a": A_K[k], "b": 1.0, "d": 10.0, "c": C_KL[k], "s": np.full(L, 10.0)}
        chains.append(make_chain(G, priors=pri, seed=20 + k))
    lib = oracle.load()
    import ctypes as C
    pd = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    a, c, e = (np.ascontiguousarray(v, np.float64) for v in (A_K, C_KL, E))
    caps = C.c_int64(0)
    nu, sig2 = 4.0, np.array([0.5, 0.2])

    def forward():
        b = rng.gamma(A_B, 1 / B_B)
        m = rng.normal(0, E)
        tau = rng.gamma(A_K, 1 / b)
        theta = rng.normal(m, C_KL)
        return b, m, tau, theta

    n = 6000
    fw = np.array([np.concatenate([[b], m, tau, theta.ravel()])
                   for b, m, tau, theta in (forward() for _ in range(n))])
    b, m, tau, theta = forward()
    psi = np.concatenate([[b], m])
    sc = []
    for it in range(1, n + 1):
        phi = np.zeros((K, 2 * L + 2))
        for k, ch in enumerate(chains):
            # the rest of dataset k given its tau_k, theta_k
            gam = 1.0 / rng.gamma(nu / 2, 2.0 / (nu * tau[k]), G)
            beta = rng.normal(theta[k], np.sqrt(sig2), (G, L))
            ch.set_top_level(psi[0], psi[1:])
            ch.set_state(gam=gam, beta=beta, phi=[nu, tau[k], *theta[k], *sig2])
            ch.step_tau(it)
            ch.step_theta(it)
            tau[k], theta[k] = ch.phi[1], ch.phi[2:2 + L]
            phi[k] = ch.phi
        lib.orc_step_psi(K, L, pd(np.ascontiguousarray(phi)), pd(a), pd(c), pd(e), A_B, B_B, 77,
                         it, pd(psi), C.byref(caps))
        sc.append(np.concatenate([psi, tau, theta.ravel()]))
    sc = np.array(sc)[500:]
    nb = 50
    bm = sc[: len(sc) // nb * nb].reshape(nb, -1, sc.shape[1]).mean(1)
    se = np.sqrt(bm.var(0, ddof=1) / nb + fw.var(0, ddof=1) / n)
    z = (sc.mean(0) - fw.mean(0)) / se
    assert np.all(np.abs(z) < 4.5), z
