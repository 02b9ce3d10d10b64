"""The C-ABI library loads and exports every entry point include/*.h declares;
argument validation needs no GPU (it fails before any CUDA call)."""
import glob
import os
import re

import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(fbs_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = fbs.load_library()
    names = declared_symbols()
    assert len(names) >= 16
    assert names <= set(fbs.EXPORTED) | names
    for n in sorted(names):
        assert getattr(lib, n) is not None, n
    assert set(fbs.EXPORTED) == names


def test_default_options():
    o = fbs.default_options()
    assert (o.precision, o.w0, o.step_out_max, o.shrink_max, o.moments_eps) == (0, 1.0, 100, 100, 1)
    assert o.all_slice == 0


def _args(**over):
    N, G, L = 4, 10, 2
    a = dict(y=np.ones((G, N), np.int32),
             X=np.stack([np.ones(N), [1.0, 1.0, -1.0, -1.0]], 1), h=np.zeros(N),
             priors={"a": 1.0, "b": 1.0, "d": 10.0, "c": np.full(L, 10.0), "s": np.full(L, 10.0)})
    a.update(over)
    return a


@pytest.mark.parametrize("case", ["N0", "G1", "L9", "singular", "negative_y", "nan_h",
                                  "bad_prior", "too_many_classes", "bad_precision",
                                  "all_slice_f32", "all_slice_2", "persistent_f64",
                                  "persistent_2"])
def test_invalid_arguments_rejected_before_any_cuda_call(case):
    kw = {}
    a = _args()
    if case == "N0":
        a["y"] = np.ones((10, 0), np.int32); a["X"] = np.ones((0, 2)); a["h"] = np.zeros(0)
    elif case == "G1":
        a["y"] = np.ones((1, 4), np.int32)
    elif case == "L9":
        a["X"] = np.ones((4, 9)); a["priors"]["c"] = np.full(9, 1.0); a["priors"]["s"] = np.full(9, 1.0)
    elif case == "singular":
        a["X"] = np.ones((4, 2))
    elif case == "negative_y":
        a["y"] = a["y"].copy(); a["y"][3, 2] = -1
    elif case == "nan_h":
        a["h"] = np.array([0.0, np.nan, 0.0, 0.0])
    elif case == "bad_prior":
        a["priors"]["d"] = 0.0
    elif case == "too_many_classes":
        N = 12
        a["y"] = np.ones((10, N), np.int32)
        a["X"] = np.stack([np.ones(N), np.arange(N, dtype=float) / 7.0], 1)
        a["h"] = np.zeros(N)
    elif case == "bad_precision":
        kw["precision"] = 7
    elif case == "all_slice_f32":
        kw["precision"], kw["all_slice"] = fbs.FBS_F32, 1
    elif case == "all_slice_2":
        kw["all_slice"] = 2
    elif case == "persistent_f64":
        kw["persistent"] = 1
    elif case == "persistent_2":
        kw["precision"], kw["persistent"] = fbs.FBS_F32, 2
    with pytest.raises(fbs.FbsError) as e:
        fbs.Sampler(a["y"], a["X"], a["h"], a["priors"], workspace="library", **kw)
    assert e.value.code == fbs.FBS_E_ARG


def test_workspace_bytes_grows_with_trace():
    base = fbs.workspace_bytes(16, 40000, 5)
    o = fbs.default_options(trace_cap=10, trace_beta=1)
    assert fbs.workspace_bytes(16, 40000, 5, o) >= base + 10 * 40000 * 5 * 8


def test_null_handles_are_refused_without_cuda():
    """Entry points given a NULL handle return FBS_E_ARG before any CUDA call."""
    lib = fbs.load_library()
    checks = [
        lib.fbs_run(None, 1, 0, 1),
        lib.fbs_get_slice_widths(None, None, None, None, None),
        lib.fbs_set_slice_widths(None, None, None, None, None),
        lib.fbs_batch_three_level(None, None, None),
        lib.fbs_batch_top_level(None, None, None, None, None, 0, None, None, None),
        lib.fbs_proposal_fused(None, 1),
        lib.fbs_proposal_wait_limit(None, 0),
        lib.fbs_proposal_mode(None, 1),
        lib.fbs_estimates(None, None),
        lib.fbs_estimates_pooled(0, None, None),
    ]
    assert all(rc == fbs.FBS_E_ARG for rc in checks), checks


def test_bench_ess_matches_oracle_ess():
    """The benchmark's host ESS of the hyperparameter trace is Geyer's initial
    monotone sequence estimator, as the oracle's is (AR(1) series)."""
    import bench
    import oracle
    rng = np.random.default_rng(4)
    x = np.zeros((1500, 3))
    for t in range(1, 1500):
        x[t] = np.array([0.5, 0.9, -0.3]) * x[t - 1] + rng.normal(size=3)
    got = bench.geyer_ess(x)
    want = [oracle.ess(x[:, i]) for i in range(3)]
    np.testing.assert_allclose(got, want, rtol=1e-10)


def test_estimates_argument_checks_without_cuda():
    """fbs_estimates_pooled refuses a bad chain count, a missing output struct,
    NULL handles and a non-positive z before touching the device."""
    import ctypes as C
    lib = fbs.load_library()
    o = fbs.EstimatesOut()
    o.z = 1.96
    hs = (C.c_void_p * 2)(None, None)
    assert lib.fbs_estimates_pooled(2, hs, C.byref(o)) == fbs.FBS_E_ARG
    assert lib.fbs_estimates_pooled(fbs.FBS_MAX_RHAT_CHAINS + 1, hs, C.byref(o)) == fbs.FBS_E_ARG
    o.z = 0.0
    assert lib.fbs_estimates_pooled(1, hs, C.byref(o)) == fbs.FBS_E_ARG
    o.z = float("nan")
    assert lib.fbs_estimates_pooled(1, hs, C.byref(o)) == fbs.FBS_E_ARG
    assert fbs.FBS_E_SLICE_CAP == -4


def test_noalloc_rejects_inconsistent_moment_count_without_cuda():
    """fbs_sweep_noalloc refuses n_mom above the post-burn-in iterations before
    `it` (it - 1 - burnin) before touching the device."""
    from paper_1606_06659_gb300 import synthetic
    dev = dict(y=1, T=1, eps=1, w_eps=1, waux_eps=1, beta=1, w_beta=1, waux_beta=1, gam=1, hyp=1)
    for it, burnin, n_mom in [(3, 1, 2), (2, 5, 1), (1, 0, 1)]:
        with pytest.raises(fbs.FbsError) as e:
            fbs.sweep_noalloc(np.ones((2, 1)), np.zeros(2), synthetic.default_priors(1), seed=1,
                              it=it, burnin=burnin, n_mom=n_mom, G=10, **dev)
        assert e.value.code == fbs.FBS_E_ARG and "n_mom" in str(e.value)
