"""fbs_sweep_noalloc: one sweep on caller-owned device arrays that allocates
nothing, for callers that cannot call cudaMalloc when they sweep (its scratch
is a fixed static device array inside the library).  Calls in a row must give
what fbs_run gives on the same state: every state array, width and tuning sum,
and every running moment, within the FP64 parity tolerance.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic
from tests._pairs import RTOL, ATOL, close

pytestmark = pytest.mark.gpu

N, L = 16, 5


def _arrays(d, st, G, eps_moments=True):
    import torch

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda()

    T = (d["y"].astype(np.int64) @ d["X"].astype(np.int64)).astype(np.float64)
    arr = {"y": dev(d["y"].astype(np.int32)), "T": dev(T), "eps": dev(st["eps"]),
           "w_eps": dev(st["w_eps"]), "waux_eps": dev(st["waux_eps"]), "beta": dev(st["beta"]),
           "w_beta": dev(st["w_beta"]), "waux_beta": dev(st["waux_beta"]),
           "gam": torch.from_numpy(st["gam"].copy()).cuda(),
           "hyp": torch.from_numpy(np.concatenate([st["phi"], st["w_nu"], st["waux_nu"]])).cuda()}
    z = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device="cuda")  # noqa: E731
    mom = {"m_beta": z(L, G), "q_beta": z(L, G), "m_gam": z(G), "q_gam": z(G),
           "m_phi": z(2 * L + 2), "q_phi": z(2 * L + 2)}
    if eps_moments:
        mom.update(m_eps=z(N, G), q_eps=z(N, G))
    status = torch.zeros(1 + fbs.NUM_COUNTERS, dtype=torch.int64, device="cuda")
    return arr, mom, status


def _sweeps(d, G, seed, burnin, n_calls, eps_moments=True, status_every=False):
    import torch
    ref = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=seed,
                      moments_eps=int(eps_moments))
    st = ref.get_state()
    arr, mom, status = _arrays(d, st, G, eps_moments)
    ptrs = {k: v.data_ptr() for k, v in (arr | mom).items()}
    stream = torch.cuda.current_stream().cuda_stream
    statuses = []
    for it in range(1, n_calls + 1):
        fbs.sweep_noalloc(d["X"], d["h"], d["priors"], seed=seed, it=it, burnin=burnin,
                          n_mom=max(0, it - 1 - burnin), stream=stream, G=G,
                          status=status.data_ptr(), **ptrs)
        statuses.append(status.clone())
    torch.cuda.synchronize()
    ref.run(n_calls, burnin=burnin, thin=1)
    return ref, st, arr, mom, [s.cpu().numpy() for s in statuses]


def _compare(ref, arr, mom, eps_moments=True):
    got = ref.get_state()
    m = ref.moments()
    hyp = arr["hyp"].cpu().numpy()
    P = 2 * L + 2
    pairs = {
        "eps": (arr["eps"].cpu().numpy().T, got["eps"]),
        "w_eps": (arr["w_eps"].cpu().numpy().T, got["w_eps"]),
        "waux_eps": (arr["waux_eps"].cpu().numpy().T, got["waux_eps"]),
        "beta": (arr["beta"].cpu().numpy().T, got["beta"]),
        "w_beta": (arr["w_beta"].cpu().numpy().T, got["w_beta"]),
        "waux_beta": (arr["waux_beta"].cpu().numpy().T, got["waux_beta"]),
        "gam": (arr["gam"].cpu().numpy(), got["gam"]),
        "phi": (hyp[:P], got["phi"]),
        "w_nu": (hyp[P:], np.concatenate([got["w_nu"], got["waux_nu"]])),
        "mean_beta": (mom["m_beta"].cpu().numpy().T, m["mean_beta"]),
        "msq_beta": (mom["q_beta"].cpu().numpy().T, m["msq_beta"]),
        "mean_gam": (mom["m_gam"].cpu().numpy(), m["mean_gam"]),
        "msq_gam": (mom["q_gam"].cpu().numpy(), m["msq_gam"]),
        "mean_phi": (mom["m_phi"].cpu().numpy(), m["mean_phi"]),
        "msq_phi": (mom["q_phi"].cpu().numpy(), m["msq_phi"]),
    }
    if eps_moments:
        pairs["mean_eps"] = (mom["m_eps"].cpu().numpy().T, m["mean_eps"])
        pairs["msq_eps"] = (mom["q_eps"].cpu().numpy().T, m["msq_eps"])
    for k, (a, b) in pairs.items():
        assert close(a, b, RTOL, ATOL).all(), k
    return m["count"]


def test_noalloc_sweeps_match_fbs_run():
    """Two calls: iteration 1 tunes the widths (it <= burnin), iteration 2 folds
    the first post-burn-in draw into the moments."""
    G = 5000
    d = synthetic.make_config(1, G=G)
    ref, st, arr, mom, stats = _sweeps(d, G, seed=31, burnin=1, n_calls=2)
    assert _compare(ref, arr, mom) == 1
    assert not np.array_equal(arr["eps"].cpu().numpy().T, st["eps"])  # the chain moved
    for s in stats:  # flags word 0, one sweep each, evaluations counted
        assert s[0] == 0 and s[1 + 7] == 1 and s[1 + 0] > 0 and s[1 + 1] > 0


def test_noalloc_chained_calls_through_burn_in_and_moments():
    """Eight calls with burn-in 4: the widths tune after M_C = 2 sweeps, then the
    moments take four draws (n_mom = 0..3); and the same without eps moments."""
    G = 3001
    d = synthetic.make_config(1, G=G)
    ref, _, arr, mom, stats = _sweeps(d, G, seed=77, burnin=4, n_calls=8)
    assert _compare(ref, arr, mom) == 4
    assert all(s[0] == 0 for s in stats)
    ref2, _, arr2, mom2, _ = _sweeps(d, G, seed=78, burnin=4, n_calls=6, eps_moments=False)
    assert _compare(ref2, arr2, mom2, eps_moments=False) == 2


def test_noalloc_reports_a_nonfinite_start():
    """A NaN in the caller's eps is reported in the status word (bit 0) and
    counted, as fbs_sync reports it for a handle."""
    import torch
    G = 1000
    d = synthetic.make_config(1, G=G)
    ref = fbs.Sampler(d["y"], d["X"], d["h"], d["priors"], seed=5)
    st = ref.get_state()
    st["eps"] = st["eps"].copy()
    st["eps"][7, 3] = np.nan
    arr, mom, status = _arrays(d, st, G)
    ptrs = {k: v.data_ptr() for k, v in (arr | mom).items()}
    fbs.sweep_noalloc(d["X"], d["h"], d["priors"], seed=5, it=1, burnin=0, G=G,
                      stream=torch.cuda.current_stream().cuda_stream, status=status.data_ptr(),
                      **ptrs)
    torch.cuda.synchronize()
    s = status.cpu().numpy()
    assert s[0] & 1 and s[1 + 6] >= 1
    # the next call starts from a cleared scratch: a finite state reports nothing
    st2 = ref.get_state()
    arr2, mom2, status2 = _arrays(d, st2, G)
    ptrs2 = {k: v.data_ptr() for k, v in (arr2 | mom2).items()}
    fbs.sweep_noalloc(d["X"], d["h"], d["priors"], seed=5, it=1, burnin=0, G=G,
                      stream=torch.cuda.current_stream().cuda_stream, status=status2.data_ptr(),
                      **ptrs2)
    torch.cuda.synchronize()
    assert status2.cpu().numpy()[0] == 0
    ref.close()


def test_noalloc_rejects_too_many_genes():
    with pytest.raises(fbs.FbsError) as e:
        fbs.sweep_noalloc(np.ones((2, 1)), np.zeros(2), synthetic.default_priors(1), seed=1,
                          it=1, burnin=0, G=fbs.NOALLOC_MAX_GENES + 1, y=1, T=1, eps=1, w_eps=1,
                          waux_eps=1, beta=1, w_beta=1, waux_beta=1, gam=1, hyp=1)
    assert e.value.code == fbs.FBS_E_ARG and "FBS_NOALLOC_MAX_GENES" in str(e.value)
