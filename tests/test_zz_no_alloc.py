"""fbs_sweep_noalloc: one sweep on caller-owned device arrays that allocates
nothing, for callers that cannot call cudaMalloc when they sweep (its scratch
is a fixed static device array inside the library).  Two calls in a row must
give what two fbs_run iterations of a handle give on the same state.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import RTOL, ATOL, close

pytestmark = pytest.mark.gpu


def test_noalloc_sweeps_match_fbs_run():
    import torch
    d = synthetic.make_config(1, G=5000)
    N, L, G = 16, 5, 5000
    seed, burnin = 31, 1
    ref = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed)
    st = ref.get_state()

    # the caller's own device arrays, in the device layout (genes fastest)
    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda()

    T = (d["y"].astype(np.int64) @ d["X"].astype(np.int64)).astype(np.float64)
    arr = {"y": dev(d["y"].astype(np.int32)), "T": dev(T), "eps": dev(st["eps"]),
           "w_eps": dev(st["w_eps"]), "waux_eps": dev(st["waux_eps"]), "beta": dev(st["beta"]),
           "w_beta": dev(st["w_beta"]), "waux_beta": dev(st["waux_beta"]),
           "gam": torch.from_numpy(st["gam"].copy()).cuda(),
           "hyp": torch.from_numpy(np.concatenate([st["phi"], st["w_nu"], st["waux_nu"]])).cuda()}
    mom = {"m_eps": torch.zeros(N, G, dtype=torch.float64, device="cuda"),
           "q_eps": torch.zeros(N, G, dtype=torch.float64, device="cuda"),
           "m_beta": torch.zeros(L, G, dtype=torch.float64, device="cuda"),
           "q_beta": torch.zeros(L, G, dtype=torch.float64, device="cuda"),
           "m_gam": torch.zeros(G, dtype=torch.float64, device="cuda"),
           "q_gam": torch.zeros(G, dtype=torch.float64, device="cuda"),
           "m_phi": torch.zeros(2 * L + 2, dtype=torch.float64, device="cuda"),
           "q_phi": torch.zeros(2 * L + 2, dtype=torch.float64, device="cuda")}
    ptrs = {k: v.data_ptr() for k, v in (arr | mom).items()}
    stream = torch.cuda.current_stream().cuda_stream
    # iteration 1 tunes the widths (it <= burnin); iteration 2 folds the first
    # post-burn-in draw into the moments
    for it in (1, 2):
        fbs.sweep_noalloc(d["X"], d["h"], d["priors"], seed=seed, it=it, burnin=burnin,
                          n_mom=max(0, it - 1 - burnin), stream=stream, G=G, **ptrs)
    torch.cuda.synchronize()

    ref.run(2, burnin=burnin, thin=1)
    got = ref.get_state()
    m = ref.moments()
    hyp = arr["hyp"].cpu().numpy()
    pairs = {
        "eps": (arr["eps"].cpu().numpy().T, got["eps"]),
        "w_eps": (arr["w_eps"].cpu().numpy().T, got["w_eps"]),
        "waux_eps": (arr["waux_eps"].cpu().numpy().T, got["waux_eps"]),
        "beta": (arr["beta"].cpu().numpy().T, got["beta"]),
        "w_beta": (arr["w_beta"].cpu().numpy().T, got["w_beta"]),
        "gam": (arr["gam"].cpu().numpy(), got["gam"]),
        "phi": (hyp[:2 * L + 2], got["phi"]),
        "w_nu": (hyp[2 * L + 2:], np.concatenate([got["w_nu"], got["waux_nu"]])),
        "mean_eps": (mom["m_eps"].cpu().numpy().T, m["mean_eps"]),
        "mean_beta": (mom["m_beta"].cpu().numpy().T, m["mean_beta"]),
        "msq_gam": (mom["q_gam"].cpu().numpy(), m["msq_gam"]),
        "mean_phi": (mom["m_phi"].cpu().numpy(), m["mean_phi"]),
    }
    for k, (a, b) in pairs.items():
        assert close(a, b, RTOL, ATOL).all(), k
    assert m["count"] == 1
    assert not np.array_equal(pairs["eps"][0], st["eps"])  # the sweeps did move the chain


def test_noalloc_rejects_too_many_genes():
    with pytest.raises(fbs.FbsError) as e:
        fbs.sweep_noalloc(np.ones((2, 1)), np.zeros(2), synthetic.default_priors(1), seed=1,
                          it=1, burnin=0, G=fbs.NOALLOC_MAX_GENES + 1, y=1, T=1, eps=1, w_eps=1,
                          waux_eps=1, beta=1, w_beta=1, waux_beta=1, gam=1, hyp=1)
    assert e.value.code == fbs.FBS_E_ARG and "FBS_NOALLOC_MAX_GENES" in str(e.value)
