"""The learned proposal of the beta_g block (FP32 handles) against the FP64 oracle
of oracle/proposal.py: the training kernels' loss and gradient, the inference
kernel's outputs, one move of every gene (proposal, acceptance and new state),
and the gain in effective sample size over the plain slice updates.  Long-run
agreement of the learned sampler's posterior with the oracle's is in
test_gpu_posterior.py."""
import numpy as np
import pytest
import oracle
import paper_1606_06659_gb300 as fbs
from oracle import proposal as P
from paper_1606_06659_gb300 import synthetic

pytestmark = pytest.mark.gpu

ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def _flat(p):
    return np.concatenate([np.asarray(p[k], np.float64).ravel() for k in ORDER]).astype(np.float32)


def _unflat(v, F, K, H=64):
    shapes = {"W1": (H, F), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (K, H), "b3": (K,)}
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(v[o:o + n], np.float64).reshape(shapes[k])
        o += n
    assert o == v.size
    return out


def _random_params(L, seed):
    F, K = P.n_features(L), P.n_outputs(L)
    p = P.init_params(F, K, seed=seed)
    rng = np.random.default_rng(seed + 100)
    p["b1"] = rng.normal(0, 0.1, p["b1"].shape)
    p["b2"] = rng.normal(0, 0.1, p["b2"].shape)
    p["W3"] = p["W3"] * 5.0
    p["b3"] = rng.normal(0, 0.2, p["b3"].shape)
    return p


def _truth(d):
    t = d["truth"]
    return {"eps": t["eps"], "beta": t["beta"], "gam": t["gam"], "phi": t["phi"]}


def _oracle_outputs(st, d, params_flat):
    """The oracle's network outputs at a sampler state, with the FP32 parameters
    (inference splits every FP32 operand into two BF16 numbers, which keeps
    about 16 significant bits)."""
    L = d["X"].shape[1]
    P_ = st["phi"]
    theta, sigma2 = P_[2:2 + L], P_[2 + L:2 + 2 * L]
    f = P.features(st["eps"], st["beta"], st["gam"], theta, sigma2, d["y"], d["X"])
    w = _unflat(np.asarray(params_flat, np.float32), P.n_features(L), P.n_outputs(L))
    return P.forward(w, f)[0]


@pytest.mark.parametrize("L,B", [(5, 1000), (2, 37), (8, 300)])
def test_loss_and_gradient_match_oracle(L, B):
    """One forward and backward pass of the training kernels (tensor cores,
    split-BF16 operands, 128 rows per block: a ragged last block in every case)
    against the oracle's explicit backpropagation in FP64; L = 8 is the largest
    shape (33 features with the column of ones in 48, 44 outputs in 48)."""
    F = P.n_features(L)
    p = _random_params(L, seed=L)
    flat = _flat(p)
    assert flat.size == fbs.proposal_param_count(L)
    rng = np.random.default_rng(7)
    feat = rng.normal(0, 1, (B, F)).astype(np.float32)
    beta = rng.normal(0, 0.5, (B, L)).astype(np.float32)
    loss, grad = fbs.proposal_loss_grad(flat, L, feat, beta)
    p32 = _unflat(flat, F, P.n_outputs(L))
    want_loss, want = P.loss_and_grads(p32, feat.astype(np.float64), beta.astype(np.float64), L)
    assert loss == pytest.approx(want_loss, rel=1e-4, abs=1e-4)
    got = _unflat(grad, F, P.n_outputs(L))
    for k in ORDER:
        scale = np.abs(want[k]).max()
        err = np.abs(got[k] - want[k]).max()
        assert err <= 2e-4 * scale + 1e-7, (k, err, scale)


def test_outputs_match_oracle_network():
    """Tensor-core inference kernel (FP32 features, weights and activations as
    BF16 hi/lo pairs, FP32 accumulation in tensor memory) against the oracle's
    features and forward pass in FP64 with the same FP32 parameters, at a state
    the sampler reached: 1000 genes, a ragged last tile of 104 genes."""
    d = synthetic.make_config(1, G=1000)
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=5, precision=fbs.FBS_F32)
    s.set_state(it=0, **_truth(d))
    s.run(20, burnin=20)
    L = d["X"].shape[1]
    flat = _flat(_random_params(L, seed=9))
    s.proposal_params(set_to=flat)
    got = s.proposal_outputs()
    want = _oracle_outputs(s.get_state(), d, flat)
    assert got.shape == want.shape == (1000, P.n_outputs(L))
    assert np.abs(want).max() > 0.5
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-4)
    s.close()


def _design(L, N=16):
    """The paper's N = 16 design for L <= 5; for L > 5 three more columns of
    -1/0/1 entries (a fixed draw of full rank)."""
    base = synthetic.paper_design(4)
    if L <= 5:
        return base[:, :L]
    extra = np.random.default_rng(48).choice([-1.0, 0.0, 1.0], size=(N, 3))
    return np.hstack([base, extra])[:, :L]


@pytest.mark.parametrize("L", [2, 8])
def test_outputs_match_oracle_network_other_widths(L):
    """The inference kernel at the smallest and largest widths (L = 2: 9
    features in 16 columns, 5 outputs in 16; L = 8: 33 in 48, 44 in 48, the
    tensor-memory A operand at its widest) against the oracle's forward pass."""
    X = _design(L)
    assert np.linalg.matrix_rank(X) == L
    theta = [4.0] + [0.0] * (L - 1)
    sigma = [2.0] + [0.3] * (L - 1)
    d = synthetic.simulate(X, theta, sigma, 0.1, 3.0, 1000, seed=900 + L)
    d["priors"] = synthetic.default_priors(L)
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=5, precision=fbs.FBS_F32)
    s.set_state(it=0, **_truth(d))
    s.run(20, burnin=20)
    flat = _flat(_random_params(L, seed=9 + L))
    s.proposal_params(set_to=flat)
    got = s.proposal_outputs()
    want = _oracle_outputs(s.get_state(), d, flat)
    assert got.shape == want.shape == (1000, P.n_outputs(L))
    assert np.abs(want).max() > 0.5
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-4)
    s.close()


def _trained_sampler(d, seed, sweeps=100, epochs=30, **kw):
    s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed, precision=fbs.FBS_F32, **kw)
    s.set_state(it=0, **_truth(d))
    s.proposal_collect(sweeps, burnin=sweeps, thin=1)
    loss = s.proposal_train(epochs=epochs, batch=2048, lr=2e-3, seed=seed)
    assert np.isfinite(loss)
    return s, loss


@pytest.mark.parametrize("kind", [1, 2])
def test_move_matches_oracle_move(kind):
    """One move of every gene: the kernel's t proposal from the network and the
    Philox draws (stream 8, index g: normals from uniforms 0..2L-1, the
    acceptance uniform 2L, the chi-square variate from uniforms 2L+1..2L+4), its
    acceptance decision and the new (eps, beta) against the oracle's move, given
    the same uniforms.  Kind 1 is the network's proposal, kind 2 the
    prior-centred one (centre theta, scale diag(sigma): the oracle's move with
    those as its outputs).  Decisions are compared where the oracle's log ratio
    is clear of the log-uniform by more than the FP32 rounding of its terms."""
    d = synthetic.make_config(1, G=1000)
    s, _ = _trained_sampler(d, seed=21)
    L = d["X"].shape[1]
    G, N = d["y"].shape
    st = s.get_state()
    params = s.proposal_params()
    if kind == 1:
        out = _oracle_outputs(st, d, params)
    else:
        phi = st["phi"]
        out = np.zeros((G, P.n_outputs(L)))
        out[:, :L] = phi[2:2 + L]
        out[:, L:2 * L] = 0.5 * np.log(phi[2 + L:2 + 2 * L])
    it, seed = 4321, 21
    xi = np.empty((G, L))
    log_u = np.empty(G)
    chi2 = np.empty(G)
    for g in range(G):
        u = oracle.uniforms_f32(seed, 0, 8, g, it, 2 * L + 5)
        xi[g] = np.sqrt(-2.0 * np.log(u[0:2 * L:2])) * np.cos(2.0 * np.pi * u[1:2 * L:2])
        log_u[g] = np.log(u[2 * L])
        chi2[g] = -2.0 * np.sum(np.log(u[2 * L + 1:2 * L + 5]))
    phi = st["phi"]
    theta, sigma2 = phi[2:2 + L], phi[2 + L:2 + 2 * L]
    e2, b2, acc, la = P.mh_move(st["eps"], st["beta"], st["gam"], theta, sigma2, d["X"], out,
                                xi, log_u, chi2)
    # magnitude of the terms of the log ratio, for the FP32 rounding margin
    mu, Cc = P.unpack(out, L)
    u_old = np.linalg.solve(Cc, (st["beta"] - mu)[..., None])[..., 0]
    mag = (np.sum(st["eps"] ** 2, 1) / st["gam"] + 0.5 * np.sum(xi ** 2, 1) * P.T_DOF / chi2
           + 0.5 * np.sum(u_old ** 2, 1)
           + np.sum(((b2 - theta) ** 2 + (st["beta"] - theta) ** 2) / sigma2, 1))
    clear = np.abs(la - log_u) > 1e-2 + 1e-4 * mag

    s.proposal_step(it, all_genes=kind)
    got = s.get_state()
    stats = s.proposal_stats()
    assert stats["tried"] == G
    acc_gpu = np.any(got["beta"] != st["beta"], axis=1)
    assert clear.mean() > 0.95
    # the prior-centred proposal suits only genes near their prior: few accept
    assert (0.2 if kind == 1 else 0.002) < acc.mean() < 0.98, acc.mean()
    np.testing.assert_array_equal(acc_gpu[clear], acc[clear])
    assert stats["accepted"] == int(acc_gpu.sum())
    both = clear & acc
    # beta* = mu + C xi carries the rounding of the network's outputs (split-BF16
    # operands keep ~2^-17 of every weight: about 1e-5 of |mu| <= 10) and of the
    # FP32 normals; eps* = eps - X (beta* - beta) inherits beta*'s absolute error.
    np.testing.assert_allclose(got["beta"][both], b2[both], rtol=1e-4, atol=2e-4)
    np.testing.assert_allclose(got["eps"][both], e2[both], rtol=0, atol=5e-4)
    rej = ~acc_gpu
    np.testing.assert_array_equal(got["beta"][rej], st["beta"][rej])
    np.testing.assert_array_equal(got["eps"][rej], st["eps"][rej])
    np.testing.assert_array_equal(got["gam"], st["gam"])
    # every log-rate is kept (up to FP32 rounding of eps)
    X = d["X"]
    np.testing.assert_allclose(got["eps"] + got["beta"] @ X.T, st["eps"] + st["beta"] @ X.T,
                               atol=2e-5)
    s.close()


def test_calibration_selects_genes_and_counts_moves():
    d = synthetic.make_config(1, G=600)
    s, _ = _trained_sampler(d, seed=31, sweeps=60, epochs=60)
    s.proposal_calibrate(40, burnin=200, min_accept=0.2)
    st = s.proposal_stats()
    assert st["tried"] == 0 and st["accepted"] == 0
    assert 0.5 * 600 < st["mh_genes"] <= 600
    assert 0 <= st["prior_genes"] < 0.5 * st["mh_genes"]
    kinds = s.proposal_kinds()
    assert kinds.shape == (600,) and set(np.unique(kinds)) <= {0, 1, 2}
    assert int((kinds > 0).sum()) == st["mh_genes"] and int((kinds == 2).sum()) == st["prior_genes"]
    s.run(30, burnin=200)
    st = s.proposal_stats()
    assert st["tried"] == 30 * st["mh_genes"]
    assert 0.3 * st["tried"] < st["accepted"] < st["tried"]
    s.proposal_mode(0)
    s.run(10, burnin=200)
    assert s.proposal_stats()["tried"] == st["tried"]
    cnt = s.counters()
    assert cnt["nonfinite"] == 0 and cnt["slice_caps"] == 0
    s.close()


def test_fused_network_pass_equals_separate_kernel():
    """The gamma/beta kernel that evaluates the network for its own 128 genes
    (the default) and the separate network kernel followed by the plain
    gamma/beta kernel give bit-identical chains (same tile code, same outputs,
    same moves), through graph segments and direct launches."""
    d = synthetic.make_config(1, G=1000)
    s0, _ = _trained_sampler(d, seed=71, sweeps=40, epochs=20)
    params = s0.proposal_params()
    s0.close()
    runs = []
    for fused in (True, False):
        s = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=72, precision=fbs.FBS_F32,
                        graph_segment=10, trace_cap=5)
        s.set_state(it=0, **_truth(d))
        s.proposal_params(set_to=params)
        s.proposal_fused(fused)
        s.proposal_calibrate(20, burnin=100, min_accept=0.1)
        s.run(25, burnin=100, thin=5)
        s.sync()
        runs.append((s.get_state(), s.proposal_stats(), s.trace()["phi"], s.counters()))
        s.close()
    (sa, pa, ta, ca), (sb, pb, tb, cb) = runs
    for k in ("eps", "beta", "gam", "phi", "w_eps", "w_beta"):
        assert np.array_equal(sa[k], sb[k]), k
    assert pa == pb and np.array_equal(ta, tb) and ca == cb
    assert pa["tried"] > 0 and pa["accepted"] > 0


def _start_after(s):
    st = s.get_state()
    return {k: st[k] for k in ("eps", "beta", "gam", "phi", "w_eps", "waux_eps", "w_beta",
                               "waux_beta", "w_nu", "waux_nu")}


@pytest.mark.parametrize("mode", [1, 2])
def test_learned_move_raises_beta_ess_per_sweep(mode):
    """At the paper's design (N = 16, L = 5, 4000 genes) the learned move must
    raise the effective sample size per sweep of the beta_gl over the plain
    slice updates: by at least 1.5x at the median and 5x at the 5th percentile
    (the plain sampler is slowest for genes with large counts, whose eps and beta
    are strongly coupled).  Mode 1 adds the move to the slice updates, mode 2
    replaces them.  Both chains start from the same state reached after 500
    plain sweeps from the generating values, and are compared over the same
    4000 sweeps (thinned by 10)."""
    d = synthetic.make_config(1, G=4000)
    n, thin = 4000, 10
    kw = {"trace_cap": n // thin, "trace_beta": 1}
    s, _ = _trained_sampler(d, seed=42, sweeps=250, epochs=15)
    s.run(250, burnin=500)
    start = _start_after(s)
    params = s.proposal_params()
    s.close()

    plain = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=41, precision=fbs.FBS_F32, **kw)
    plain.set_state(it=0, **start)
    plain.run(100, burnin=100)
    plain.run(n, burnin=100, thin=thin)
    ess_p = plain.beta_ess()
    plain.close()

    lrn = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=43, precision=fbs.FBS_F32, **kw)
    lrn.set_state(it=0, **start)
    lrn.proposal_params(set_to=params)
    lrn.proposal_calibrate(100, burnin=100, min_accept=0.2)
    lrn.proposal_mode(mode)
    lrn.run(n, burnin=100, thin=thin)
    ess_l = lrn.beta_ess()
    st = lrn.proposal_stats()
    cnt = lrn.counters()
    lrn.close()
    assert cnt["nonfinite"] == 0 and cnt["slice_caps"] == 0
    assert st["mh_genes"] > 0.95 * 4000
    assert st["accepted"] > 0.5 * st["tried"]
    med = np.median(ess_l) / np.median(ess_p)
    p05 = np.percentile(ess_l, 5) / np.percentile(ess_p, 5)
    assert med >= 1.5 and p05 >= 5.0, (med, p05, np.median(ess_l), np.median(ess_p))
