"""GPU parity: the CUDA path against the CPU oracle, element by element, on the
same seeded synthetic inputs.  Sizes span several 128-gene blocks with a
ragged tail; the last tests run the paper-scale workload (N=16, G=40000, L=5)
in the launch configuration the benchmark times."""
import numpy as np
import pytest

import oracle
import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import (ALL_SLICE_KEYS, RTOL, ATOL, STATE_KEYS, assert_state_close, close,
                          make_pair, small_data, sync_gpu_to_oracle)

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------------ RNG and integers
@pytest.mark.parametrize("stream,index0,it,k0", [(1, 0, 1, 0), (5, 123456, 77, 3),
                                                 (3, 0, 2 ** 31 + 5, 250), (7, 4, 9, 256 * 15)])
def test_uniforms_bit_exact(stream, index0, it, k0):
    seed, chain = 0x0123456789ABCDEF, 3
    a = fbs.uniforms(seed, chain, stream, index0, 300, it, k0, 9)
    b = oracle.uniforms(seed, chain, stream, index0, 300, it, k0, 9)
    assert np.array_equal(a, b)


def test_count_sums_bit_exact():
    d = synthetic.make_config(1, G=5000)
    g, o = make_pair(d)
    assert np.array_equal(g.count_sums(), o.count_sums())


# ------------------------------------------------------------------ default start
@pytest.mark.parametrize("cfg", [0, 1])
def test_default_start_matches_oracle(cfg):
    d = small_data(cfg, G=3001)
    g, o = make_pair(d)
    o.init_default()
    gs = g.get_state()
    assert gs["it"] == 0
    assert_state_close(gs, o.get_state(), where="init")


# ------------------------------------------------------------------ lockstep sweeps
COUNTS = ("evals_eps", "evals_beta", "evals_nu", "slice_caps", "gamma_caps", "trunc_caps",
          "evals_gam", "evals_hyp")


def _lockstep(d, n_sweeps, burnin, seed=12345, **opt):
    """Both sides start every sweep from the oracle's state (copied into the GPU),
    run one sweep, and must agree element by element; the evaluation counts,
    being integers, must agree exactly."""
    g, o = make_pair(d, seed=seed, **opt)
    o.init_default()
    o.set_opts(burnin=burnin, tune_start=burnin // 2)
    for it in range(1, n_sweeps + 1):
        sync_gpu_to_oracle(g, o, it - 1)
        c0 = g.counters()
        o0 = o.counters_dict()
        g.run(1, burnin=burnin, thin=1)
        g.sync()
        o.sweep()
        assert_state_close(g.get_state(), o.get_state(), keys=ALL_SLICE_KEYS, where=f"sweep {it}")
        c1, o1 = g.counters(), o.counters_dict()
        for k in COUNTS:
            assert c1[k] - c0[k] == o1[k] - o0[k], (it, k)
    return g, o


@pytest.mark.parametrize("cfg,G", [(0, 1000), (0, 3001), (1, 1537)])
def test_lockstep_sweeps(cfg, G):
    d = small_data(cfg, G=G)
    _lockstep(d, n_sweeps=6, burnin=4)


def test_lockstep_general_design_values():
    """A column with values other than +-1 (and a zero) takes the general class path."""
    rng = np.random.default_rng(3)
    N, G = 6, 700
    X = np.array([[1, 0.5, 1], [1, 2.0, -1], [1, 0.0, 1], [1, 0.5, -1], [1, 2.0, 1], [1, -1.5, -1]])
    d = synthetic.simulate(X, (2.0, 0.3, -0.2), (1.0, 0.3, 0.2), 0.2, 5.0, G, seed=4)
    d["priors"] = synthetic.default_priors(3)
    _lockstep(d, n_sweeps=4, burnin=2)


def test_lockstep_edge_sizes():
    for N, G, L in [(1, 2, 1), (4, 2, 2), (5, 129, 2), (64, 130, 1)]:
        X = synthetic.two_group_design(N) if L == 2 else np.ones((N, 1))
        d = synthetic.simulate(X, (2.0, 0.5)[:L], (1.0, 0.3)[:L], 0.2, 5.0, G, seed=N + G)
        d["priors"] = synthetic.default_priors(L)
        _lockstep(d, n_sweeps=3, burnin=2)


def test_lockstep_zero_and_huge_counts():
    d = small_data(0, G=600)
    d["y"] = d["y"].copy()
    d["y"][:100] = 0
    d["y"][100:130] = 2 ** 30
    _lockstep(d, n_sweeps=3, burnin=0)


# ------------------------------------------------------------------ all-slice variant
@pytest.mark.parametrize("cfg,G", [(0, 1000), (1, 1537)])
def test_all_slice_lockstep_sweeps(cfg, G):
    """gamma_g, tau and sigma_l by slice updates (Section 4.2), through burn-in
    (widths tuned after M_C) and past it."""
    d = small_data(cfg, G=G)
    g, o = _lockstep(d, n_sweeps=8, burnin=4, all_slice=1)
    c = g.counters()
    assert c["evals_gam"] > 0 and c["evals_hyp"] > 0 and c["gamma_caps"] == 0


def test_all_slice_free_running_chain_matches_oracle():
    d = small_data(0, G=2000)
    g, o = make_pair(d, all_slice=1)
    o.init_default()
    burnin = 20
    o.set_opts(burnin=burnin, tune_start=burnin // 2)
    for it in range(1, 41):
        g.run(1, burnin=burnin, thin=1)
        o.sweep()
        assert_state_close(g.get_state(), o.get_state(), keys=ALL_SLICE_KEYS,
                           where=f"iteration {it}")
    gm, om = g.moments(), o.moments_dict()
    for k in ("mean_gam", "msq_gam", "mean_phi", "msq_phi"):
        assert close(gm[k], om[k], 1e-9, 1e-12).all(), k
    gc, oc = g.counters(), o.counters_dict()
    for k in COUNTS:
        assert gc[k] == oc[k], k


def test_all_slice_paper_scale_lockstep_sweep():
    """The paper-scale workload (N=16, G=40000, L=5) in the launch configuration
    the benchmark times, one lockstep sweep during burn-in and one after."""
    d = synthetic.make_config(1)
    _lockstep(d, n_sweeps=2, burnin=1, all_slice=1)


def test_slice_widths_round_trip_and_f32_refuses():
    d = small_data(0, G=300)
    g = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], all_slice=1)
    st = g.get_state()
    assert np.all(st["w_gam"] == 1.0) and np.all(st["w_hyp"] == 1.0)
    assert np.all(st["waux_gam"] == 0.0) and np.all(st["waux_hyp"] == 0.0)
    rng = np.random.default_rng(0)
    want = {"w_gam": rng.uniform(0.1, 2, 300), "waux_gam": rng.uniform(0, 5, 300),
            "w_hyp": rng.uniform(0.1, 2, 3), "waux_hyp": rng.uniform(0, 5, 3)}
    g.set_state(it=7, **want)
    st = g.get_state()
    for k, v in want.items():
        assert np.array_equal(st[k], v), k
    assert st["it"] == 7
    with pytest.raises(ValueError):
        g.set_state(w_hyp=np.ones(5))
    f = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], precision=fbs.FBS_F32)
    assert "w_gam" not in f.get_state()
    with pytest.raises(fbs.FbsError) as e:
        f.set_state(w_gam=np.ones(300))
    assert e.value.code == fbs.FBS_E_ARG


# ------------------------------------------------------------------ free running
def test_free_running_chain_matches_oracle():
    """Both chains run on their own from the same start; compare after every
    iteration until the first slice-branch divergence (none is expected here)."""
    d = small_data(0, G=2000)
    g, o = make_pair(d)
    o.init_default()
    burnin = 20
    o.set_opts(burnin=burnin, tune_start=burnin // 2)
    for it in range(1, 41):
        g.run(1, burnin=burnin, thin=1)
        o.sweep()
        assert_state_close(g.get_state(), o.get_state(), where=f"iteration {it}")
    gm, om = g.moments(), o.moments_dict()
    assert gm["count"] == om["count"] == 20
    for k in ("mean_eps", "msq_eps", "mean_beta", "msq_beta", "mean_gam", "msq_gam", "mean_phi",
              "msq_phi"):
        assert close(gm[k], om[k], 1e-9, 1e-12).all(), k


@pytest.mark.parametrize("all_slice", [0, 1])
def test_graph_segments_equal_direct_launches(all_slice):
    d = small_data(0, G=1500)
    kw = dict(seed=5, all_slice=all_slice)
    a = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], graph_segment=7, **kw)
    b = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], graph_segment=1000, **kw)
    a.run(23, burnin=10, thin=2)   # 3 graph segments + 2 direct sweeps
    b.run(23, burnin=10, thin=2)   # 23 direct sweeps
    sa, sb = a.get_state(), b.get_state()
    for k in ALL_SLICE_KEYS:
        assert np.array_equal(sa[k], sb[k]), k
    assert a.counters() == b.counters()


def test_trace_and_moments_match_oracle():
    d = small_data(0, G=1000)
    g, o = make_pair(d, trace_cap=50, trace_beta=1)
    o.init_default()
    o.set_opts(burnin=10, tune_start=5)
    g.run(30, burnin=10, thin=3)
    tr_o = o.run(30, thin=3, trace_cap=50, trace_beta=True)
    tr_g = g.trace(beta=True)
    assert tr_g["phi"].shape == tr_o["phi"].shape == (6, 6)
    assert close(tr_g["phi"], tr_o["phi"], 1e-9).all()
    assert close(tr_g["beta"], tr_o["beta"], 1e-9).all()
    ess_g = g.beta_ess()
    ess_o = np.array([[oracle.ess(tr_o["beta"][:, gg, l]) for l in range(2)] for gg in range(50)])
    assert close(ess_g[:50], ess_o, 1e-8, 1e-8).all()


def test_resume_equals_one_run():
    d = small_data(0, G=800)
    a = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=9)
    b = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=9)
    a.run(25, burnin=10, thin=1)
    b.run(11, burnin=10, thin=1)
    b.run(14, burnin=10, thin=1)
    sa, sb = a.get_state(), b.get_state()
    for k in STATE_KEYS:
        assert np.array_equal(sa[k], sb[k]), k
    ma, mb = a.moments(), b.moments()
    for k in ma:
        assert np.array_equal(np.asarray(ma[k]), np.asarray(mb[k])), k


# ------------------------------------------------------------------ paper-scale workload
@pytest.mark.slow
def test_paper_scale_lockstep_sweep():
    """N=16, G=40000, L=5 in the benchmark's launch configuration: two lockstep
    sweeps over every gene (the oracle finishes one sweep in about a second)."""
    d = synthetic.make_config(1)
    _lockstep(d, n_sweeps=2, burnin=10)


def test_precision_stress_scale_lockstep_sweep():
    """Configuration 2's shape, N=32 (8 libraries per variety), G=200000, L=5:
    one lockstep sweep over every gene against the oracle (a few seconds)."""
    d = synthetic.make_config(2)
    assert d["y"].shape == (200000, 32)
    _lockstep(d, n_sweeps=1, burnin=10)
