"""Helpers that set up the GPU sampler and the CPU oracle on the same seeded
synthetic inputs and compare them element by element."""
import numpy as np

import oracle
import paper_1606_06659_gb300 as fbs
from paper_1606_06659_gb300 import synthetic

# FP64 tolerance: states of both sides agree to 1e-10 relative per step
# (the slice mechanics are bit-identical; only exp/log/lgamma/cos rounding and
# reduction order differ, at the 1e-15 level); the absolute floor covers values
# that are exactly or nearly zero.
RTOL, ATOL = 1e-10, 1e-12
STATE_KEYS = ("eps", "beta", "gam", "phi", "w_eps", "waux_eps", "w_beta", "waux_beta", "w_nu",
              "waux_nu")
# with the widths of gamma_g, tau and sigma_l (FP64 handles; all-slice variant)
ALL_SLICE_KEYS = STATE_KEYS + ("w_gam", "waux_gam", "w_hyp", "waux_hyp")


def make_pair(data, seed=12345, chain=0, **opt):
    g = fbs.Sampler(data["y"], data["X"], data["h"], data["priors"], seed=seed, chain=chain, **opt)
    kw = {}
    for k in ("step_out_max", "shrink_max", "w0", "all_slice"):
        if k in opt:
            kw[k] = opt[k]
    o = oracle.Chain(data["y"], data["X"], data["h"], data["priors"], seed=seed, chain=chain, **kw)
    return g, o


def close(a, b, rtol=RTOL, atol=ATOL):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b) <= rtol * np.maximum(np.abs(a), np.abs(b)) + atol


def assert_state_close(gs, os_, keys=STATE_KEYS, rtol=RTOL, atol=ATOL, where=""):
    for k in keys:
        a, b = np.asarray(gs[k], float), np.asarray(os_[k], float)
        ok = close(a, b, rtol, atol)
        if not ok.all():
            idx = np.argwhere(~ok)[:5]
            raise AssertionError(
                f"{where} {k}: {np.count_nonzero(~ok)} of {ok.size} differ; first at "
                f"{idx.tolist()}: gpu {a[tuple(idx[0])]!r} oracle {b[tuple(idx[0])]!r}")


def sync_gpu_to_oracle(g, o, it):
    st = o.get_state()
    g.set_state(it=it, **st)


def small_data(cfg=0, G=3001, seed=None):
    return synthetic.make_config(cfg, G=G, seed=seed)
