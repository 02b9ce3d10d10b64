"""GB300 Gibbs sampler for the fully Bayesian RNA-seq hierarchical model of
Landau & Niemi, "A fully Bayesian strategy for high-dimensional hierarchical
modeling using massively parallel computing" (arXiv 1606.06659).

This module is a thin ctypes binding of the C ABI in ``include/fbs.h`` (the
library ``_build/libfbs.so``, built by ``paper_1606_06659_gb300.build``).  It
only marshals arguments: every step of a sweep runs in the library's CUDA
kernels.  PyTorch, when given, provides the device workspace (caching
allocator) and the CUDA stream.  There is no CPU fallback: importing fails if
the library has not been built, and creating a sampler fails without a GPU.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfbs.so")

FBS_OK, FBS_E_ARG, FBS_E_CUDA, FBS_E_OOM, FBS_E_SLICE_CAP, FBS_E_NONFINITE = 0, -1, -2, -3, -4, -5
FBS_F64, FBS_F32 = 0, 1
FBS_MAX_CONTRASTS, FBS_MAX_CONTRAST_TERMS = 8, 4
FBS_MAX_RHAT_CHAINS = 64
MAX_N, MAX_L, MAX_CLASSES = 64, 8, 8
COUNTER_NAMES = ("evals_eps", "evals_beta", "evals_nu", "slice_caps", "gamma_caps",
                 "trunc_caps", "nonfinite", "sweeps", "evals_gam", "evals_hyp")
NUM_COUNTERS = len(COUNTER_NAMES)

# symbols declared in include/fbs.h
EXPORTED = ("fbs_default_options", "fbs_workspace_bytes", "fbs_init", "fbs_run", "fbs_sync",
            "fbs_moments", "fbs_get_state", "fbs_set_state", "fbs_trace", "fbs_beta_ess",
            "fbs_count_sums", "fbs_counters", "fbs_profile", "fbs_uniforms", "fbs_free",
            "fbs_last_error_string", "fbs_sweep_noalloc", "fbs_batch_init", "fbs_batch_run",
            "fbs_batch_sync", "fbs_batch_chain", "fbs_batch_set_schedule", "fbs_batch_autotune",
            "fbs_batch_free", "fbs_proposal_param_count", "fbs_proposal_collect",
            "fbs_proposal_train", "fbs_proposal_calibrate", "fbs_proposal_mode",
            "fbs_proposal_params", "fbs_proposal_stats", "fbs_proposal_loss_grad",
            "fbs_proposal_outputs", "fbs_proposal_step", "fbs_set_contrasts",
            "fbs_contrast_probs", "fbs_rhat", "fbs_proposal_kinds", "fbs_get_slice_widths",
            "fbs_set_slice_widths", "fbs_batch_three_level", "fbs_batch_top_level",
            "fbs_proposal_fused", "fbs_estimates", "fbs_estimates_pooled",
            "fbs_proposal_wait_limit", "fbs_measure_peaks")
NOALLOC_MAX_GENES = 2048 * 128


class FbsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fbs error {code}: {msg}")
        self.code = code


class Priors(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("d", C.c_double),
                ("c", C.POINTER(C.c_double)), ("s", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("w0", C.c_double), ("step_out_max", C.c_int),
                ("shrink_max", C.c_int), ("chain", C.c_uint32), ("moments_eps", C.c_int),
                ("trace_cap", C.c_int64), ("trace_beta", C.c_int), ("block", C.c_int),
                ("graph_segment", C.c_int), ("all_slice", C.c_int), ("persistent", C.c_int)]


_PD = C.POINTER(C.c_double)
_PI64 = C.POINTER(C.c_int64)


class TopPrior(C.Structure):
    _fields_ = [("a_b", C.c_double), ("b_b", C.c_double), ("e", _PD), ("seed", C.c_uint64)]
_lib = None


class Dataset(C.Structure):
    """fbs_dataset: one dataset of a batch."""
    _fields_ = [("N", C.c_int), ("G", C.c_int), ("L", C.c_int), ("y", C.POINTER(C.c_int32)),
                ("X", _PD), ("h", _PD), ("priors", Priors), ("seed", C.c_uint64),
                ("chain", C.c_uint32)]


class SweepArgs(C.Structure):
    """fbs_sweep_args: one sweep on caller-owned device arrays (fbs_sweep_noalloc)."""
    _fields_ = [("N", C.c_int), ("G", C.c_int), ("L", C.c_int), ("X", _PD), ("h", _PD),
                ("priors", Priors), ("seed", C.c_uint64), ("chain", C.c_uint32),
                ("step_out_max", C.c_int), ("shrink_max", C.c_int), ("it", C.c_int64),
                ("burnin", C.c_int64), ("n_mom", C.c_int64), ("y", C.c_void_p),
                ("T", C.c_void_p)] + [(n, C.c_void_p) for n in (
                    "eps", "w_eps", "waux_eps", "beta", "w_beta", "waux_beta", "gam", "hyp",
                    "m_eps", "q_eps", "m_beta", "q_beta", "m_gam", "q_gam", "m_phi", "q_phi",
                    "stream", "status")]


class EstimatesOut(C.Structure):
    """fbs_estimates_out: pooled posterior means, sds and intervals (§3.1)."""
    _fields_ = ([("z", C.c_double)] +
                [(f"{q}_{v}", _PD) for v in ("eps", "beta", "gam", "phi")
                 for q in ("mean", "sd", "lo", "hi")] +
                [("trace_phi", _PD), ("trace_rows_max", C.c_int64), ("trace_rows", C.c_int64),
                 ("count", C.c_int64), ("counters", C.c_int64 * 10),
                 ("mh_accepted", C.c_int64), ("mh_tried", C.c_int64)])


def load_library(path: str = LIB_PATH):
    """Load libfbs.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1606_06659_gb300.build`")
    lib = C.CDLL(path)
    vp, i32, i64, u32, u64, d = C.c_void_p, C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    lib.fbs_default_options.argtypes = [C.POINTER(Options)]
    lib.fbs_default_options.restype = None
    lib.fbs_workspace_bytes.argtypes = [i32, i32, i32, C.POINTER(Options), C.POINTER(C.c_size_t)]
    lib.fbs_init.argtypes = [C.POINTER(vp), C.POINTER(C.c_int32), i32, i32, i32, _PD, i32, _PD,
                             C.POINTER(Priors), C.POINTER(Options), u64, vp, C.c_size_t, vp]
    lib.fbs_run.argtypes = [vp, i64, i64, i64]
    lib.fbs_sync.argtypes = [vp]
    lib.fbs_moments.argtypes = [vp] + [_PD] * 8 + [_PI64]
    lib.fbs_get_state.argtypes = [vp] + [_PD] * 10 + [_PI64]
    lib.fbs_set_state.argtypes = [vp] + [_PD] * 10 + [i64]
    lib.fbs_get_slice_widths.argtypes = [vp] + [_PD] * 4
    lib.fbs_set_slice_widths.argtypes = [vp] + [_PD] * 4
    lib.fbs_trace.argtypes = [vp, i64, _PD, _PD, _PI64]
    lib.fbs_beta_ess.argtypes = [vp, _PD]
    lib.fbs_count_sums.argtypes = [vp, _PI64]
    lib.fbs_counters.argtypes = [vp, _PI64]
    lib.fbs_profile.argtypes = [vp, i64, i64, i64, _PD]
    lib.fbs_uniforms.argtypes = [u64, u32, u32, u32, i32, u32, u32, i32, _PD]
    lib.fbs_measure_peaks.argtypes = [_PD]
    lib.fbs_sweep_noalloc.argtypes = [C.POINTER(SweepArgs)]
    lib.fbs_batch_init.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(Dataset), C.POINTER(Options),
                                   vp]
    lib.fbs_batch_run.argtypes = [vp, i64, i64, i64]
    lib.fbs_batch_sync.argtypes = [vp]
    lib.fbs_batch_chain.argtypes = [vp, C.c_int]
    lib.fbs_batch_chain.restype = vp
    lib.fbs_batch_set_schedule.argtypes = [vp, C.c_int, C.c_int]
    lib.fbs_batch_autotune.argtypes = [vp, C.c_int, i64, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_double)]
    lib.fbs_batch_free.argtypes = [vp]
    lib.fbs_batch_three_level.argtypes = [vp, C.POINTER(TopPrior), _PD]
    lib.fbs_batch_top_level.argtypes = [vp, _PD, _PD, _PD, _PI64, i64, _PD, _PI64, _PI64]
    lib.fbs_batch_free.restype = None
    _PF = C.POINTER(C.c_float)
    lib.fbs_proposal_param_count.argtypes = [C.c_int]
    lib.fbs_proposal_collect.argtypes = [vp, i64, i64, i64]
    lib.fbs_proposal_train.argtypes = [vp, C.c_int, C.c_int, C.c_double, u64, _PD]
    lib.fbs_proposal_calibrate.argtypes = [vp, i64, i64, C.c_double]
    lib.fbs_proposal_mode.argtypes = [vp, C.c_int]
    lib.fbs_proposal_fused.argtypes = [vp, C.c_int]
    lib.fbs_proposal_wait_limit.argtypes = [vp, u32]
    lib.fbs_proposal_params.argtypes = [vp, _PF, _PF, C.c_int]
    lib.fbs_proposal_stats.argtypes = [vp, _PI64, _PI64, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.fbs_proposal_loss_grad.argtypes = [_PF, C.c_int, C.c_int, _PF, _PF, _PD, _PF]
    lib.fbs_proposal_outputs.argtypes = [vp, _PF]
    lib.fbs_proposal_step.argtypes = [vp, C.c_int64, C.c_int]
    lib.fbs_set_contrasts.argtypes = [vp, C.c_int, C.POINTER(C.c_int), _PD, _PD]
    lib.fbs_contrast_probs.argtypes = [vp, _PD, _PI64]
    lib.fbs_rhat.argtypes = [C.c_int, C.POINTER(vp), _PD, _PD, _PD, _PD]
    lib.fbs_estimates.argtypes = [vp, C.POINTER(EstimatesOut)]
    lib.fbs_estimates_pooled.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(EstimatesOut)]
    lib.fbs_proposal_kinds.argtypes = [vp, C.POINTER(C.c_uint8)]
    lib.fbs_free.argtypes = [vp]
    lib.fbs_free.restype = None
    lib.fbs_last_error_string.argtypes = []
    lib.fbs_last_error_string.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc):
    if rc != FBS_OK:
        msg = load_library().fbs_last_error_string().decode()
        raise FbsError(rc, msg)


def _pd(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_PD)


def default_options(**kw) -> Options:
    o = Options()
    load_library().fbs_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def workspace_bytes(N, G, L, options: Options | None = None) -> int:
    n = C.c_size_t(0)
    _check(load_library().fbs_workspace_bytes(N, G, L, C.byref(options or default_options()),
                                              C.byref(n)))
    return n.value


def uniforms(seed, chain, stream, index0, n_index, it, k0, n_k) -> np.ndarray:
    """Uniforms generated on the device exactly as the sampler draws them."""
    out = np.empty((n_index, n_k), np.float64)
    _check(load_library().fbs_uniforms(seed, chain, stream, index0, n_index, it, k0, n_k,
                                       _pd(out)))
    return out


PEAK_NAMES = ("ffma", "ex2", "lg2", "imulhi", "dfma")


def measure_peaks() -> dict:
    """Measured throughput of the arithmetic pipes on the current device
    (instructions per second summed over lanes): FP32 FMA, MUFU ex2 and lg2,
    32-bit multiply-high, FP64 FMA (fbs_measure_peaks)."""
    out = np.zeros(len(PEAK_NAMES))
    _check(load_library().fbs_measure_peaks(_pd(out)))
    return dict(zip(PEAK_NAMES, (float(v) for v in out)))


def sweep_noalloc(X, h, priors, *, seed, it, burnin, n_mom=0, chain=0, step_out_max=100,
                  shrink_max=100, stream=None, **dev):
    """One sweep on caller-owned device arrays with no allocation (fbs_sweep_noalloc).

    ``dev`` maps y, T, eps, w_eps, waux_eps, beta, w_beta, waux_beta, gam, hyp, the
    optional moment arrays (m_eps, q_eps, m_beta, q_beta, m_gam, q_gam, m_phi, q_phi)
    and the optional status array (1 + NUM_COUNTERS uint64: flags, counters) to
    device addresses (ints) in the device layout described in include/fbs.h.
    """
    X = np.ascontiguousarray(X, np.float64)
    N, L = X.shape
    h = np.ascontiguousarray(h, np.float64).reshape(N)
    c = np.ascontiguousarray(np.broadcast_to(priors["c"], (L,)), np.float64)
    s = np.ascontiguousarray(np.broadcast_to(priors["s"], (L,)), np.float64)
    a = SweepArgs()
    a.N, a.G, a.L = N, int(dev.pop("G")), L
    a.X, a.h = _pd(X), _pd(h)
    a.priors = Priors(float(priors["a"]), float(priors["b"]), float(priors["d"]), _pd(c), _pd(s))
    a.seed, a.chain = int(seed), int(chain)
    a.step_out_max, a.shrink_max = int(step_out_max), int(shrink_max)
    a.it, a.burnin, a.n_mom = int(it), int(burnin), int(n_mom)
    for name, ptr in dev.items():
        if name not in dict(SweepArgs._fields_):
            raise TypeError(f"unknown device array {name}")
        setattr(a, name, ptr)
    a.stream = stream
    _check(load_library().fbs_sweep_noalloc(C.byref(a)))


def _pf(a):
    if a is None:
        return None
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_float))


def rhat(chains, eps=False):
    """Gelman-Rubin factors (§3.1) from the running moments of several chains of
    the same model: dict of phi [2L+2], beta [G][L], gam [G] (and eps [G][N])."""
    c0 = chains[0]
    out = {"phi": np.empty(c0.P), "beta": np.empty((c0.G, c0.L)), "gam": np.empty(c0.G)}
    if eps:
        out["eps"] = np.empty((c0.G, c0.N))
    hs = (C.c_void_p * len(chains))(*[c.h for c in chains])
    _check(c0.lib.fbs_rhat(len(chains), hs, _pd(out["phi"]), _pd(out["beta"]), _pd(out["gam"]),
                           _pd(out.get("eps"))))
    return out


Z95 = 1.959963984540054


def estimates(chains, z=Z95, eps=False, trace_rows=0):
    """Posterior means, sds (sqrt(msq - mean^2)) and normal-approximation
    intervals mean -/+ z sd (§3.1) from the running moments of one or several
    chains of the same model, pooled over the chains, computed on the device:
    dict of {mean, sd, lo, hi}_{beta [G][L], gam [G], phi [2L+2]} (and eps [G][N]),
    count, counters, mh_accepted, mh_tried and up to trace_rows phi trace rows of
    the first chain."""
    if isinstance(chains, Sampler):
        chains = [chains]
    c0 = chains[0]
    shapes = {"beta": (c0.G, c0.L), "gam": (c0.G,), "phi": (c0.P,), "eps": (c0.G, c0.N)}
    o = EstimatesOut()
    o.z = float(z)
    res = {}
    for v, shp in shapes.items():
        if v == "eps" and not eps:
            continue
        for q in ("mean", "sd", "lo", "hi"):
            a = np.empty(shp)
            res[f"{q}_{v}"] = a
            setattr(o, f"{q}_{v}", _pd(a))
    tr = np.empty((max(int(trace_rows), 0), c0.P))
    if trace_rows:
        o.trace_phi, o.trace_rows_max = _pd(tr), int(trace_rows)
    hs = (C.c_void_p * len(chains))(*[c.h for c in chains])
    _check(c0.lib.fbs_estimates_pooled(len(chains), hs, C.byref(o)))
    res["count"] = o.count
    res["counters"] = dict(zip(COUNTER_NAMES, (int(v) for v in o.counters)))
    res["mh_accepted"], res["mh_tried"] = o.mh_accepted, o.mh_tried
    if trace_rows:
        res["trace_phi"] = tr[:o.trace_rows]
    return res


def proposal_param_count(L):
    return load_library().fbs_proposal_param_count(int(L))


def proposal_loss_grad(params, L, feat, beta):
    """Loss and gradient of the proposal network on a host batch, through the GPU
    training kernels."""
    params = np.ascontiguousarray(params, np.float32)
    feat = np.ascontiguousarray(feat, np.float32)
    beta = np.ascontiguousarray(beta, np.float32)
    grad = np.zeros_like(params)
    loss = C.c_double()
    _check(load_library().fbs_proposal_loss_grad(_pf(params), int(L), feat.shape[0], _pf(feat),
                                                 _pf(beta), C.byref(loss), _pf(grad)))
    return loss.value, grad


class Sampler:
    """One chain of the GPU sampler.

    y: [G][N] int32 counts (or [N][G] with gene_major=False); X: [N][L];
    h: [N]; priors: dict(a, b, d, c[L], s[L]).  ``workspace="torch"`` takes
    the device memory from the PyTorch caching allocator and orders the work on
    torch's current stream; ``workspace="library"`` lets the library allocate.
    """
    n_contrasts = 0


    def __init__(self, y, X, h, priors, seed=1, gene_major=True, workspace="torch",
                 options: Options | None = None, **option_kw):
        self.lib = load_library()
        y = np.ascontiguousarray(y, np.int32)
        if gene_major:
            self.G, self.N = y.shape
        else:
            self.N, self.G = y.shape
        X = np.ascontiguousarray(X, np.float64)
        if X.ndim != 2:
            X = X.reshape(self.N, -1)
        self.L = X.shape[1]
        h = np.ascontiguousarray(h, np.float64).reshape(self.N)
        self.P = 2 * self.L + 2
        c = np.ascontiguousarray(np.broadcast_to(priors["c"], (self.L,)), np.float64)
        s = np.ascontiguousarray(np.broadcast_to(priors["s"], (self.L,)), np.float64)
        pri = Priors(float(priors["a"]), float(priors["b"]), float(priors["d"]), _pd(c), _pd(s))
        self.options = options or default_options()
        for k, v in option_kw.items():
            setattr(self.options, k, v)
        self._ws = None
        ws_ptr, ws_bytes, stream = None, 0, None
        if workspace == "torch":
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device")
            ws_bytes = workspace_bytes(self.N, self.G, self.L, self.options)
            self._ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
            ws_ptr = self._ws.data_ptr()
            stream = torch.cuda.current_stream().cuda_stream
        handle = C.c_void_p()
        _check(self.lib.fbs_init(C.byref(handle), y.ctypes.data_as(C.POINTER(C.c_int32)), self.N,
                                 self.G, 1 if gene_major else 0, _pd(X), self.L, _pd(h),
                                 C.byref(pri), C.byref(self.options), int(seed), ws_ptr, ws_bytes,
                                 stream))
        self.h = handle

    def close(self):
        if getattr(self, "h", None):
            self.lib.fbs_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- running
    def run(self, n_iter, burnin=0, thin=1):
        _check(self.lib.fbs_run(self.h, int(n_iter), int(burnin), int(thin)))

    def sync(self):
        _check(self.lib.fbs_sync(self.h))

    def profile(self, n_iter, burnin=0, thin=1):
        """Mean milliseconds per iteration inside a replayed graph of n_iter sweeps:
        (eps kernel, gamma/beta kernel, hyperparameter kernel, learned-proposal
        network launched alone or 0, the replay's time per iteration)."""
        ms = np.zeros(5)
        _check(self.lib.fbs_profile(self.h, int(n_iter), int(burnin), int(thin), _pd(ms)))
        return tuple(float(v) for v in ms)

    # --------------------------------------------------------------- state
    def get_state(self):
        G, N, L, P = self.G, self.N, self.L, self.P
        out = {"eps": np.empty((G, N)), "beta": np.empty((G, L)), "gam": np.empty(G),
               "phi": np.empty(P), "w_eps": np.empty((G, N)), "waux_eps": np.empty((G, N)),
               "w_beta": np.empty((G, L)), "waux_beta": np.empty((G, L)), "w_nu": np.empty(1),
               "waux_nu": np.empty(1)}
        it = C.c_int64()
        _check(self.lib.fbs_get_state(self.h, *[_pd(out[k]) for k in (
            "eps", "beta", "gam", "phi", "w_eps", "waux_eps", "w_beta", "waux_beta", "w_nu",
            "waux_nu")], C.byref(it)))
        out["it"] = it.value
        if self.options.precision == FBS_F64:
            wid = {"w_gam": np.empty(G), "waux_gam": np.empty(G), "w_hyp": np.empty(L + 1),
                   "waux_hyp": np.empty(L + 1)}
            _check(self.lib.fbs_get_slice_widths(self.h, *[_pd(v) for v in wid.values()]))
            out.update(wid)
        return out

    def phi(self):
        """Current hyperparameters (nu, tau, theta[L], sigma^2[L])."""
        out = np.empty(self.P)
        _check(self.lib.fbs_get_state(self.h, None, None, None, _pd(out), None, None, None, None,
                                      None, None, None))
        return out

    def set_state(self, it=0, **arrays):
        """State arrays by name (as get_state returns them); the gamma, tau and
        sigma widths w_gam, waux_gam [G], w_hyp, waux_hyp [1+L] exist in FP64 only."""
        names = ("eps", "beta", "gam", "phi", "w_eps", "waux_eps", "w_beta", "waux_beta", "w_nu",
                 "waux_nu")
        widths = ("w_gam", "waux_gam", "w_hyp", "waux_hyp")
        unknown = set(arrays) - set(names) - set(widths)
        if unknown:
            raise TypeError(f"unknown state arrays {unknown}")
        conv = {k: np.ascontiguousarray(np.atleast_1d(v), np.float64) for k, v in arrays.items()
                if v is not None}
        for k, n in (("w_gam", self.G), ("waux_gam", self.G), ("w_hyp", self.L + 1),
                     ("waux_hyp", self.L + 1)):
            if k in conv and conv[k].size != n:
                raise ValueError(f"{k} needs {n} values")
        _check(self.lib.fbs_set_state(self.h, *[_pd(conv.get(k)) for k in names], int(it)))
        if any(k in conv for k in widths):
            _check(self.lib.fbs_set_slice_widths(self.h, *[_pd(conv.get(k)) for k in widths]))

    def moments(self):
        G, N, L, P = self.G, self.N, self.L, self.P
        out = {"mean_eps": np.empty((G, N)), "msq_eps": np.empty((G, N)),
               "mean_beta": np.empty((G, L)), "msq_beta": np.empty((G, L)),
               "mean_gam": np.empty(G), "msq_gam": np.empty(G), "mean_phi": np.empty(P),
               "msq_phi": np.empty(P)}
        cnt = C.c_int64()
        _check(self.lib.fbs_moments(self.h, *[_pd(v) for v in out.values()], C.byref(cnt)))
        out["count"] = cnt.value
        return out

    def trace(self, max_rows=None, beta=False):
        cap = int(self.options.trace_cap) if max_rows is None else int(max_rows)
        phi = np.empty((max(cap, 0), self.P))
        bt = np.empty((max(cap, 0), self.G, self.L)) if beta else None
        rows = C.c_int64()
        _check(self.lib.fbs_trace(self.h, cap, _pd(phi), _pd(bt), C.byref(rows)))
        out = {"phi": phi[:rows.value]}
        if beta:
            out["beta"] = bt[:rows.value]
        return out

    def beta_ess(self):
        ess = np.empty((self.G, self.L))
        _check(self.lib.fbs_beta_ess(self.h, _pd(ess)))
        return ess

    def estimates(self, z=Z95, eps=False, trace_rows=0):
        """fbs_estimates of this chain (see the module function estimates)."""
        return estimates([self], z=z, eps=eps, trace_rows=trace_rows)

    def count_sums(self):
        T = np.empty((self.G, self.L), np.int64)
        _check(self.lib.fbs_count_sums(self.h, T.ctypes.data_as(_PI64)))
        return T

    def counters(self):
        c = np.zeros(NUM_COUNTERS, np.int64)
        _check(self.lib.fbs_counters(self.h, c.ctypes.data_as(_PI64)))
        return dict(zip(COUNTER_NAMES, (int(v) for v in c)))

    # --------------------------------------------------------------- learned proposal
    # --------------------------------------------------------------- contrasts
    def set_contrasts(self, props):
        """props: list of propositions, each a list of (v, b) with v of length L:
        the proposition holds when v . beta_g > b for every pair."""
        n = len(props)
        T = FBS_MAX_CONTRAST_TERMS
        terms = np.zeros(max(n, 1), np.int32)
        v = np.zeros((max(n, 1), T, self.L))
        b = np.zeros((max(n, 1), T))
        for q, prop in enumerate(props):
            terms[q] = len(prop)
            if len(prop) > T:
                raise FbsError(FBS_E_ARG, "a proposition has more than FBS_MAX_CONTRAST_TERMS terms")
            for k, (vk, bk) in enumerate(prop):
                v[q, k] = vk
                b[q, k] = bk
        _check(self.lib.fbs_set_contrasts(self.h, n, terms.ctypes.data_as(C.POINTER(C.c_int)),
                                          _pd(v), _pd(b)))
        self.n_contrasts = n

    def contrast_probs(self):
        """[G][n] posterior probabilities and the number of iterations counted."""
        out = np.empty((self.G, self.n_contrasts))
        m = C.c_int64()
        _check(self.lib.fbs_contrast_probs(self.h, _pd(out), C.byref(m)))
        return out, m.value

    def proposal_collect(self, n_sweeps, burnin=0, thin=1):
        _check(self.lib.fbs_proposal_collect(self.h, int(n_sweeps), int(burnin), int(thin)))

    def proposal_train(self, epochs=20, batch=4096, lr=1e-3, seed=1):
        loss = C.c_double()
        _check(self.lib.fbs_proposal_train(self.h, int(epochs), int(batch), float(lr), int(seed),
                                           C.byref(loss)))
        return loss.value

    def proposal_calibrate(self, n_sweeps, burnin=0, min_accept=0.2):
        _check(self.lib.fbs_proposal_calibrate(self.h, int(n_sweeps), int(burnin),
                                               float(min_accept)))

    def proposal_mode(self, mode):
        _check(self.lib.fbs_proposal_mode(self.h, int(mode)))

    def proposal_wait_limit(self, polls):
        """Bound of each tensor-core wait of the network pass (0: give up at once)."""
        _check(self.lib.fbs_proposal_wait_limit(self.h, int(polls)))

    def proposal_fused(self, on):
        _check(self.lib.fbs_proposal_fused(self.h, int(bool(on))))

    def proposal_params(self, set_to=None):
        n = proposal_param_count(self.L)
        out = np.zeros(n, np.float32)
        s = None if set_to is None else np.ascontiguousarray(set_to, np.float32)
        _check(self.lib.fbs_proposal_params(self.h, _pf(out), _pf(s), n))
        return out

    def proposal_outputs(self):
        K = self.L + self.L * (self.L + 1) // 2
        out = np.zeros((self.G, K), np.float32)
        _check(self.lib.fbs_proposal_outputs(self.h, _pf(out)))
        return out

    def proposal_step(self, it, all_genes=1):
        """all_genes: 0 the calibrated per-gene choice, 1 every gene with the
        network's proposal, 2 every gene with the prior-centred one."""
        _check(self.lib.fbs_proposal_step(self.h, int(it), int(all_genes)))

    def proposal_kinds(self):
        """Per gene: 0 slice updates only, 1 the network's proposal, 2 the
        prior-centred one."""
        out = np.zeros(self.G, np.uint8)
        _check(self.lib.fbs_proposal_kinds(self.h, out.ctypes.data_as(C.POINTER(C.c_uint8))))
        return out

    def proposal_stats(self):
        a, t, u, up = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        _check(self.lib.fbs_proposal_stats(self.h, C.byref(a), C.byref(t), C.byref(u),
                                           C.byref(up)))
        return {"accepted": a.value, "tried": t.value, "mh_genes": u.value,
                "prior_genes": up.value}


class ChainView(Sampler):
    """One dataset of a BatchSampler, with the Sampler accessors (state, moments,
    trace, counters).  Running happens through the batch."""

    def __init__(self, lib, handle, N, G, L, options):
        self.lib, self.h = lib, C.c_void_p(handle)
        self.N, self.G, self.L, self.P = N, G, L, 2 * L + 2
        self.options = options
        self._ws = None

    def close(self):
        self.h = None

    def run(self, *a, **k):
        raise FbsError(FBS_E_ARG, "a batch dataset runs with BatchSampler.run")


class BatchSampler:
    """Many datasets (different N, G, L) and chains swept together in the FP32 form.

    datasets: list of dicts with y [G][N], X [N][L], h [N], priors; seeds and
    chains: one per dataset.
    """

    def __init__(self, datasets, seeds=None, chains=None, options: Options | None = None,
                 **option_kw):
        self.lib = load_library()
        C_ = len(datasets)
        seeds = list(seeds) if seeds is not None else [1 + i for i in range(C_)]
        chains = list(chains) if chains is not None else [0] * C_
        self.options = options or default_options(precision=FBS_F32)
        for k, v in option_kw.items():
            setattr(self.options, k, v)
        self._keep = []
        arr = (Dataset * C_)()
        self.shapes = []
        for i, d in enumerate(datasets):
            y = np.ascontiguousarray(d["y"], np.int32)
            G, N = y.shape
            X = np.ascontiguousarray(d["X"], np.float64).reshape(N, -1)
            L = X.shape[1]
            h = np.ascontiguousarray(d["h"], np.float64).reshape(N)
            c = np.ascontiguousarray(np.broadcast_to(d["priors"]["c"], (L,)), np.float64)
            s = np.ascontiguousarray(np.broadcast_to(d["priors"]["s"], (L,)), np.float64)
            self._keep += [y, X, h, c, s]
            pr = d["priors"]
            arr[i] = Dataset(N, G, L, y.ctypes.data_as(C.POINTER(C.c_int32)), _pd(X), _pd(h),
                             Priors(float(pr["a"]), float(pr["b"]), float(pr["d"]), _pd(c),
                                    _pd(s)), int(seeds[i]), int(chains[i]))
            self.shapes.append((N, G, L))
        stream = None
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        handle = C.c_void_p()
        _check(self.lib.fbs_batch_init(C.byref(handle), C_, arr, C.byref(self.options), stream))
        self.b = handle
        self.views = [ChainView(self.lib, self.lib.fbs_batch_chain(self.b, i), *self.shapes[i],
                                self.options) for i in range(C_)]

    def __len__(self):
        return len(self.views)

    def chain(self, c) -> ChainView:
        return self.views[c]

    def run(self, n_iter, burnin=0, thin=1):
        _check(self.lib.fbs_batch_run(self.b, int(n_iter), int(burnin), int(thin)))

    def sync(self):
        _check(self.lib.fbs_batch_sync(self.b))

    def set_schedule(self, eps_block, gb_block):
        _check(self.lib.fbs_batch_set_schedule(self.b, int(eps_block), int(gb_block)))

    def three_level(self, e, a_b, b_b, seed, psi0=None):
        """Make the datasets the groups of the three-level model: their phi_k share
        psi = (b, m_1..m_L) with tau_k ~ Gamma(a_k, rate b), theta_kl ~ N(m_l,
        c_kl^2), b ~ Gamma(a_b, rate b_b), m_l ~ N(0, e_l^2).  e=None switches it off."""
        if e is None:
            _check(self.lib.fbs_batch_three_level(self.b, None, None))
            return
        L = self.shapes[0][2]
        self._top_e = np.ascontiguousarray(np.broadcast_to(e, (L,)), np.float64)
        pri = TopPrior(float(a_b), float(b_b), _pd(self._top_e), int(seed))
        p0 = None if psi0 is None else np.ascontiguousarray(psi0, np.float64).reshape(L + 1)
        _check(self.lib.fbs_batch_three_level(self.b, C.byref(pri), _pd(p0)))

    def top_level(self, max_rows=None):
        """psi = (b, m_1..m_L), its running mean / mean square and count, its
        thinned trace and the count of b draws that ran out of attempts."""
        n = self.shapes[0][2] + 1   # the library refuses a batch that is not three-level
        cap = int(self.options.trace_cap) if max_rows is None else int(max_rows)
        psi, mean, msq = np.empty(n), np.empty(n), np.empty(n)
        tr = np.empty((max(cap, 0), n))
        cnt, rows, caps = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self.lib.fbs_batch_top_level(self.b, _pd(psi), _pd(mean), _pd(msq), C.byref(cnt),
                                            cap, _pd(tr), C.byref(rows), C.byref(caps)))
        return {"psi": psi, "mean": mean, "msq": msq, "count": cnt.value,
                "trace": tr[:rows.value], "gamma_caps": caps.value}

    def autotune(self, sweeps=5, burnin=0):
        e, g, ms = C.c_int(), C.c_int(), C.c_double()
        _check(self.lib.fbs_batch_autotune(self.b, int(sweeps), int(burnin), C.byref(e),
                                           C.byref(g), C.byref(ms)))
        return e.value, g.value, ms.value

    def close(self):
        if getattr(self, "b", None):
            self.lib.fbs_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
