"""Plain FP64 CPU oracle for the Gibbs sweep of Landau & Niemi (arXiv 1606.06659).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package; the GPU library
(``paper_1606_06659_gb300``) never does, and this package never imports it.

The arithmetic lives in ``fbs_oracle.c`` (plain C, no FMA contraction), built
here with gcc into ``oracle/_build/libfbs_oracle.so`` and called through
ctypes.  What each C function follows in the paper is stated beside it there:
Section 4.1 / Figure 3 (model), Algorithm 1 (sweep order), Algorithm 2
(slice sampler and width tuning), Section 3.1 (running moments).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbs_oracle.c")
_HDR = os.path.join(_HERE, "fbs_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfbs_oracle.so")
_lock = threading.Lock()
_lib = None

STREAM_EPS, STREAM_GAMMA, STREAM_NU, STREAM_TAU = 1, 2, 3, 4
STREAM_BETA, STREAM_THETA, STREAM_SIGMA, STREAM_TEST = 5, 6, 7, 200

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]


def build(src: str = _SRC, out: str = _LIB_PATH, defines=()) -> str:
    """Compile the oracle with gcc (plain IEEE double, no contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    newest = max(os.path.getmtime(src), os.path.getmtime(_HDR))
    if os.path.exists(out) and os.path.getmtime(out) >= newest and not defines:
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", *CFLAGS, *[f"-D{d}" for d in defines], "-I", _HERE, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Model(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("G", C.c_int), ("L", C.c_int),
        ("y", C.POINTER(C.c_int32)), ("X", C.POINTER(C.c_double)), ("h", C.POINTER(C.c_double)),
        ("a", C.c_double), ("b", C.c_double), ("d", C.c_double),
        ("c", C.POINTER(C.c_double)), ("s", C.POINTER(C.c_double)),
        ("theta_mean", C.POINTER(C.c_double)),
    ]


_PD = C.POINTER(C.c_double)


STATE_NAMES = ("eps", "beta", "gam", "phi", "w_eps", "waux_eps", "w_beta", "waux_beta", "w_nu",
               "waux_nu", "w_gam", "waux_gam", "w_hyp", "waux_hyp")


class State(C.Structure):
    _fields_ = [(n, _PD) for n in ("eps", "beta", "gam", "phi", "w_eps", "waux_eps",
                                   "w_beta", "waux_beta", "w_nu", "waux_nu", "w_gam",
                                   "waux_gam", "w_hyp", "waux_hyp")]


class Opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("chain", C.c_uint32), ("step_out_max", C.c_int),
                ("shrink_max", C.c_int), ("burnin", C.c_int64), ("tune_start", C.c_int64),
                ("w0", C.c_double), ("all_slice", C.c_int)]


class Moments(C.Structure):
    _fields_ = [(n, _PD) for n in ("mean_eps", "msq_eps", "mean_beta", "msq_beta",
                                   "mean_gam", "msq_gam", "mean_phi", "msq_phi")] + [
        ("count", C.c_int64)]


class Counters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("evals_eps", "evals_beta", "evals_nu", "slice_caps",
                                         "gamma_caps", "trunc_caps", "nonfinite", "evals_gam",
                                         "evals_hyp")]


def _declare(lib):
    u32, u64, i64, d = C.c_uint32, C.c_uint64, C.c_int64, C.c_double
    pM, pS, pO = C.POINTER(Model), C.POINTER(State), C.POINTER(Opts)
    pMo, pCn = C.POINTER(Moments), C.POINTER(Counters)
    lib.orc_philox4x32_10.argtypes = [C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_set_threads.restype = None
    lib.orc_get_threads.argtypes = []
    lib.orc_get_threads.restype = C.c_int
    lib.orc_uniform.argtypes = [u64, u32, u32, u32, u32, u32]
    lib.orc_uniform.restype = d
    lib.orc_normal.argtypes = [u64, u32, u32, u32, u32, u32]
    lib.orc_normal.restype = d
    lib.orc_gamma.argtypes = [d, u64, u32, u32, u32, u32, u32, C.POINTER(i64)]
    lib.orc_gamma.restype = d
    lib.orc_fill_uniforms.argtypes = [u64, u32, u32, u32, C.c_int, u32, u32, C.c_int, _PD]
    lib.orc_fill_gamma.argtypes = [d, u64, u32, u32, u32, C.c_int, u32, _PD]
    lib.orc_fill_normal.argtypes = [u64, u32, u32, u32, C.c_int, u32, _PD]
    for name in ("orc_logf_eps",):
        getattr(lib, name).argtypes = [pM, pS, C.c_int, C.c_int, d]
        getattr(lib, name).restype = d
    lib.orc_logf_beta.argtypes = [pM, pS, C.c_int, C.c_int, d]
    lib.orc_logf_beta.restype = d
    lib.orc_logf_nu.argtypes = [pM, pS, d]
    lib.orc_logf_nu.restype = d
    lib.orc_slice_textbook.argtypes = [C.c_int, d, d, C.c_int, _PD, d, C.c_int, C.c_int, u64,
                                       u32, _PD, C.POINTER(i64)]
    for name in ("orc_step_eps", "orc_step_gamma", "orc_step_nu", "orc_step_tau",
                 "orc_step_beta", "orc_step_theta", "orc_step_sigma"):
        getattr(lib, name).argtypes = [pM, pS, pO, i64, pCn]
    lib.orc_step_beta_l.argtypes = [pM, pS, pO, i64, C.c_int, pCn]
    lib.orc_sweep.argtypes = [pM, pS, pO, i64, pMo, pCn]
    lib.orc_run.argtypes = [pM, pS, pO, i64, i64, i64, pMo, pCn, _PD, _PD, i64]
    lib.orc_run.restype = i64
    lib.orc_init_state.argtypes = [pM, pS, pO]
    lib.orc_init_state.restype = C.c_int
    lib.orc_count_sums.argtypes = [pM, C.POINTER(i64)]
    lib.orc_ess.argtypes = [_PD, i64]
    lib.orc_ess.restype = d
    lib.orc_step_psi.argtypes = [C.c_int, C.c_int, _PD, _PD, _PD, _PD, d, d, u64, i64, _PD,
                                 C.POINTER(i64)]
    return lib


def load(path: str | None = None):
    """Build (if needed) and load the oracle shared library."""
    global _lib
    if path is not None:
        return _declare(C.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _pd(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_PD)


def set_threads(n: int, lib=None) -> int:
    """Host threads (OpenMP) of the oracle's per-gene loops in this process;
    returns the previous number.  The states do not depend on it."""
    lib = lib or load()
    old = lib.orc_get_threads()
    lib.orc_set_threads(int(n))
    return old


# --------------------------------------------------------------------------- RNG helpers
def philox(ctr, key, lib=None):
    lib = lib or load()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniforms(seed, chain, stream, index0, n_index, it, k0, n_k, lib=None):
    lib = lib or load()
    out = np.empty((n_index, n_k), np.float64)
    lib.orc_fill_uniforms(seed, chain, stream, index0, n_index, it, k0, n_k, _pd(out))
    return out


def uniforms_f32(seed, chain, stream, index, it, n_k, lib=None):
    """The FP32 form's uniforms k = 0..n_k-1 of one (stream, index, iteration):
    Philox4x32-10 with key (seed lo, seed hi) and counter (index,
    stream << 24 | k >> 2, it, chain); word k mod 4 of the block, x, maps to
    (floor(x / 2^9) + 1/2) 2^-23, strictly inside (0, 1) and exact in FP32."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    out = np.empty(n_k, np.float64)
    for b in range((n_k + 3) // 4):
        w = philox((index, (stream << 24) | b, it, chain), key, lib)
        for j in range(4):
            if 4 * b + j < n_k:
                out[4 * b + j] = ((w[j] >> 9) + 0.5) * 2.0 ** -23
    return out


def rhat(means, msqs, M):
    """Gelman-Rubin potential scale reduction (§3.1) from C chains' running means
    and mean squares over M draws each (arrays [C][...]): B = M/(C-1) sum_c
    (mean_c - mean)^2, S_c^2 = M/(M-1) (msq_c - mean_c^2), W = mean_c S_c^2,
    Rhat = sqrt(1 + (B/W - 1)/M); NaN where W <= 0."""
    means = np.asarray(means, np.float64)
    msqs = np.asarray(msqs, np.float64)
    C = means.shape[0]
    grand = means.mean(0)
    B = M / (C - 1) * ((means - grand) ** 2).sum(0)
    W = (M / (M - 1) * (msqs - means ** 2)).mean(0)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(W > 0, np.sqrt(1 + (B / W - 1) / M), np.nan)


def contrast_probs(beta_draws, props, dtype=np.float64):
    """Posterior probabilities of contrasts (§3.1): for draws beta [M][G][L] and
    propositions [[(v, b), ...], ...], the fraction of the M draws in which
    v . beta_g > b holds for every pair of the proposition, per gene ([G][n]).
    The dot product is summed over l in order in `dtype`, one rounding per
    operation."""
    beta = np.asarray(beta_draws).astype(dtype)
    M, G, L = beta.shape
    out = np.zeros((G, len(props)))
    for q, prop in enumerate(props):
        ok = np.ones((M, G), bool)
        for v, b in prop:
            s = np.zeros((M, G), dtype)
            for l in range(L):
                s = (s + (dtype(v[l]) * beta[:, :, l]).astype(dtype)).astype(dtype)
            ok &= s > dtype(b)
        out[:, q] = ok.sum(0) / M if M else 0.0
    return out


def gamma_draws(shape, seed, chain, stream, index0, n, it, lib=None):
    lib = lib or load()
    out = np.empty(n, np.float64)
    lib.orc_fill_gamma(float(shape), seed, chain, stream, index0, n, it, _pd(out))
    return out


def normal_draws(seed, chain, stream, index0, n, it, lib=None):
    lib = lib or load()
    out = np.empty(n, np.float64)
    lib.orc_fill_normal(seed, chain, stream, index0, n, it, _pd(out))
    return out


def slice_textbook(kind, p0, p1, x0, w=1.0, K=100, shrink_max=100, seed=1, it=1, lib=None):
    lib = lib or load()
    x0 = np.ascontiguousarray(x0, np.float64)
    out = np.empty_like(x0)
    ev = C.c_int64(0)
    lib.orc_slice_textbook(kind, p0, p1, x0.size, _pd(x0), w, K, shrink_max, seed, it,
                           _pd(out), C.byref(ev))
    return out, ev.value


def ess(x, lib=None):
    lib = lib or load()
    x = np.ascontiguousarray(x, np.float64)
    return lib.orc_ess(_pd(x), x.size)


# --------------------------------------------------------------------------- chain
class Chain:
    """One chain of the sampler on host arrays; every call goes to the C oracle.

    y: int32 [G][N]; X: [N][L]; h: [N]; priors: dict(a, b, d, c[L], s[L]).
    all_slice: slice-sample gamma_g, tau and sigma_l too (their widths are w_gam
    [G] and w_hyp [1+L] = tau, sigma_1..sigma_L).
    """

    def __init__(self, y, X, h, priors, seed=1, chain=0, step_out_max=100, shrink_max=100,
                 burnin=0, tune_start=None, w0=1.0, all_slice=False, lib=None):
        self.lib = lib or load()
        self.y = np.ascontiguousarray(y, np.int32)
        self.G, self.N = self.y.shape
        self.X = np.ascontiguousarray(X, np.float64).reshape(self.N, -1)
        self.L = self.X.shape[1]
        self.h = np.ascontiguousarray(h, np.float64).reshape(self.N)
        L = self.L
        self.c = np.ascontiguousarray(np.broadcast_to(priors["c"], (L,)), np.float64)
        self.s = np.ascontiguousarray(np.broadcast_to(priors["s"], (L,)), np.float64)
        self.theta_mean = None
        self.model = Model(self.N, self.G, L, self.y.ctypes.data_as(C.POINTER(C.c_int32)),
                           _pd(self.X), _pd(self.h), float(priors["a"]), float(priors["b"]),
                           float(priors["d"]), _pd(self.c), _pd(self.s), None)
        G, N = self.G, self.N
        self.eps = np.zeros((G, N))
        self.beta = np.zeros((G, L))
        self.gam = np.ones(G)
        self.phi = np.zeros(2 * L + 2)
        self.w_eps = np.full((G, N), w0)
        self.waux_eps = np.zeros((G, N))
        self.w_beta = np.full((G, L), w0)
        self.waux_beta = np.zeros((G, L))
        self.w_nu = np.full(1, w0)
        self.waux_nu = np.zeros(1)
        self.w_gam = np.full(G, w0)
        self.waux_gam = np.zeros(G)
        self.w_hyp = np.full(1 + L, w0)
        self.waux_hyp = np.zeros(1 + L)
        self.state = State(*[_pd(getattr(self, n)) for n in STATE_NAMES])
        if tune_start is None:
            tune_start = burnin // 2
        self.opts = Opts(seed, chain, step_out_max, shrink_max, burnin, tune_start, w0,
                         int(bool(all_slice)))
        self.mean_eps, self.msq_eps = np.zeros((G, N)), np.zeros((G, N))
        self.mean_beta, self.msq_beta = np.zeros((G, L)), np.zeros((G, L))
        self.mean_gam, self.msq_gam = np.zeros(G), np.zeros(G)
        self.mean_phi, self.msq_phi = np.zeros(2 * L + 2), np.zeros(2 * L + 2)
        self.moments = Moments(*[_pd(getattr(self, n)) for n in (
            "mean_eps", "msq_eps", "mean_beta", "msq_beta", "mean_gam", "msq_gam", "mean_phi",
            "msq_phi")], 0)
        self.counters = Counters()
        self.it = 0

    # state ---------------------------------------------------------------
    def init_default(self):
        rc = self.lib.orc_init_state(C.byref(self.model), C.byref(self.state), C.byref(self.opts))
        if rc != 0:
            raise ValueError("X^T X is singular")
        return self

    def set_state(self, it=None, **arrays):
        unknown = set(arrays) - set(STATE_NAMES)
        if unknown:
            raise TypeError(f"unknown state arrays {unknown}")
        for name, val in arrays.items():
            if val is not None:
                getattr(self, name)[...] = np.asarray(val, np.float64).reshape(
                    getattr(self, name).shape)
        if it is not None:
            self.it = int(it)
        return self

    def get_state(self):
        return {n: getattr(self, n).copy() for n in STATE_NAMES}

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)

    def set_top_level(self, b, theta_mean):
        """Priors that the three-level model's top level sets: tau ~ Gamma(a, rate
        b) and theta_l ~ N(theta_mean_l, c_l^2)."""
        if self.theta_mean is None:
            self.theta_mean = np.zeros(self.L)
            self.model.theta_mean = _pd(self.theta_mean)
        self.theta_mean[...] = np.asarray(theta_mean, np.float64).reshape(self.L)
        self.model.b = float(b)

    # steps -----------------------------------------------------------------
    def _step(self, name, it, *extra):
        getattr(self.lib, name)(C.byref(self.model), C.byref(self.state), C.byref(self.opts),
                                int(it), *extra, C.byref(self.counters))

    def step_eps(self, it): self._step("orc_step_eps", it)
    def step_gamma(self, it): self._step("orc_step_gamma", it)
    def step_nu(self, it): self._step("orc_step_nu", it)
    def step_tau(self, it): self._step("orc_step_tau", it)
    def step_beta(self, it): self._step("orc_step_beta", it)
    def step_beta_l(self, it, l): self._step("orc_step_beta_l", it, int(l))
    def step_theta(self, it): self._step("orc_step_theta", it)
    def step_sigma(self, it): self._step("orc_step_sigma", it)

    def sweep(self):
        self.it += 1
        self.lib.orc_sweep(C.byref(self.model), C.byref(self.state), C.byref(self.opts), self.it,
                           C.byref(self.moments), C.byref(self.counters))

    def run(self, n_iter, thin=1, trace_cap=0, trace_beta=False):
        P = 2 * self.L + 2
        tphi = np.zeros((max(trace_cap, 1), P))
        tbeta = np.zeros((max(trace_cap, 1), self.G, self.L)) if trace_beta else None
        rows = self.lib.orc_run(C.byref(self.model), C.byref(self.state), C.byref(self.opts),
                                self.it, int(n_iter), int(thin), C.byref(self.moments),
                                C.byref(self.counters), _pd(tphi),
                                _pd(tbeta) if tbeta is not None else None, int(trace_cap))
        self.it += int(n_iter)
        out = {"phi": tphi[:rows]}
        if tbeta is not None:
            out["beta"] = tbeta[:rows]
        return out

    # densities / sums -----------------------------------------------------
    def logf_eps(self, g, n, x):
        return self.lib.orc_logf_eps(C.byref(self.model), C.byref(self.state), g, n, x)

    def logf_beta(self, g, l, b):
        return self.lib.orc_logf_beta(C.byref(self.model), C.byref(self.state), g, l, b)

    def logf_nu(self, nu):
        return self.lib.orc_logf_nu(C.byref(self.model), C.byref(self.state), nu)

    def count_sums(self):
        T = np.zeros((self.G, self.L), np.int64)
        self.lib.orc_count_sums(C.byref(self.model), T.ctypes.data_as(C.POINTER(C.c_int64)))
        return T

    def moments_dict(self):
        return {n: getattr(self, n).copy() for n in (
            "mean_eps", "msq_eps", "mean_beta", "msq_beta", "mean_gam", "msq_gam", "mean_phi",
            "msq_phi")} | {"count": self.moments.count}

    def counters_dict(self):
        return {n: getattr(self.counters, n) for n, _ in Counters._fields_}


# --------------------------------------------------------------------------- three levels
class ThreeLevel:
    """The three-level model (Section 2.3) over K datasets of the RNA-seq model:
    dataset k keeps its own phi_k = (nu_k, tau_k, theta_k, sigma^2_k) and the
    phi_k share psi = (b, m_1..m_L) through tau_k ~ Gamma(a_k, rate b) and
    theta_kl ~ N(m_l, c_kl^2), with b ~ Gamma(a_b, rate b_b), m_l ~ N(0, e_l^2).

    One sweep runs Algorithm 1 on every dataset given psi (a Chain each, with its
    own seed and chain number), then draws psi given the phi_k (orc_step_psi).
    datasets: dicts with y, X, h, priors, seed, chain; every X has the same L.
    """

    def __init__(self, datasets, e, a_b, b_b, psi_seed, psi0=None, burnin=0, lib=None):
        self.lib = lib or load()
        self.chains = [Chain(d["y"], d["X"], d["h"], d["priors"], seed=d["seed"],
                             chain=d.get("chain", 0), burnin=burnin, lib=self.lib)
                       for d in datasets]
        Ls = {ch.L for ch in self.chains}
        if len(Ls) != 1:
            raise ValueError("every dataset of a three-level model needs the same L")
        self.K, self.L = len(self.chains), Ls.pop()
        self.e = np.ascontiguousarray(np.broadcast_to(e, (self.L,)), np.float64)
        self.a_b, self.b_b, self.seed = float(a_b), float(b_b), int(psi_seed)
        self.a = np.array([float(d["priors"]["a"]) for d in datasets])
        self.c = np.ascontiguousarray(np.stack([ch.c for ch in self.chains]), np.float64)
        self.psi = (np.asarray(psi0, np.float64).copy() if psi0 is not None
                    else np.array([self.a_b / self.b_b] + [0.0] * self.L))
        self.burnin = int(burnin)
        self.it = 0
        self.gamma_caps = C.c_int64(0)
        for ch in self.chains:
            ch.set_top_level(self.psi[0], self.psi[1:])

    def init_default(self):
        for ch in self.chains:
            ch.init_default()
        return self

    def phis(self):
        return np.stack([ch.phi for ch in self.chains])

    def step_psi(self, it):
        phi = np.ascontiguousarray(self.phis())
        self.lib.orc_step_psi(self.K, self.L, _pd(phi), _pd(self.a), _pd(self.c), _pd(self.e),
                              self.a_b, self.b_b, self.seed, int(it), _pd(self.psi),
                              C.byref(self.gamma_caps))

    def sweep(self):
        self.it += 1
        for ch in self.chains:
            ch.set_top_level(self.psi[0], self.psi[1:])
            ch.sweep()
        self.step_psi(self.it)

    def run(self, n_iter, thin=1):
        """n_iter sweeps; returns the post-burn-in rows of every thin-th
        iteration: psi [rows][1+L] and phi [rows][K][2L+2]."""
        tp, tf = [], []
        for _ in range(int(n_iter)):
            self.sweep()
            if self.it > self.burnin and (self.it - self.burnin) % thin == 0:
                tp.append(self.psi.copy())
                tf.append(self.phis())
        P = 2 * self.L + 2
        return {"psi": np.array(tp).reshape(-1, 1 + self.L),
                "phi": np.array(tf).reshape(-1, self.K, P)}
