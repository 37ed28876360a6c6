"""GB300 GEER engine: epsilon-approximate pairwise effective resistance
(arXiv 2312.06123, Algorithm 3) with hand-written CUDA kernels for sm_103a.

This module is the thin Python binding of the C ABI declared in
``include/geer.h``: it only marshals arguments. Every step of a query runs in
the library ``libgeer.so`` built from ``csrc/``; there is no CPU fallback --
if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np

from ._build import LIB as _LIB_PATH, build as build_library

GER_OK = 0
GER_ERR = {
    -1: "GER_ERR_INVALID", -2: "GER_ERR_NODE_RANGE", -3: "GER_ERR_CSR", -4: "GER_ERR_DISCONNECTED",
    -5: "GER_ERR_BIPARTITE", -6: "GER_ERR_OOM", -7: "GER_ERR_CUDA", -8: "GER_ERR_TIMEOUT",
    -9: "GER_ERR_CAPACITY", -10: "GER_ERR_NO_LAMBDA",
}
GER_FP64, GER_FP32 = 0, 1
GER_SWITCH_RULE, GER_SWITCH_MLP, GER_SWITCH_FIXED = 0, 1, 2
MLP_INPUTS, MLP_HIDDEN, MLP_PARAMS = 6, 64, 4673
LOG_WIDTH = 8
GER_ELL_REFINED, GER_ELL_PENG = 0, 1
GER_ENGINE_SPARSE, GER_ENGINE_DENSE, GER_ENGINE_HYBRID = 0, 1, 2


class GeerError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{GER_ERR.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("tau", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("per_query", ctypes.c_int32), ("switch_policy", ctypes.c_int32),
                ("fixed_ell_b", ctypes.c_int32), ("ell_formula", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("sparse_cap", ctypes.c_int64), ("smm_engine", ctypes.c_int32),
                ("dense_width", ctypes.c_int32), ("dense_switch", ctypes.c_int64), ("dense_budget_mb", ctypes.c_int32),
                ("mlp_at_start", ctypes.c_int32)]


class QueryStats(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int32), ("ell_b", ctypes.c_int32), ("batches", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("eta0", ctypes.c_int64), ("walks", ctypes.c_int64),
                ("walk_steps", ctypes.c_int64), ("r_b", ctypes.c_double), ("r_f", ctypes.c_double),
                ("psi", ctypes.c_double), ("f_last", ctypes.c_double), ("volume", ctypes.c_double),
                ("h", ctypes.c_double), ("checksum", ctypes.c_uint64)]


class MlpTrainOptions(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("dense_width", ctypes.c_int32), ("reserved", ctypes.c_int32), ("dense_switch", ctypes.c_int64),
                ("width_ms", ctypes.c_float * 3), ("switch_ms", ctypes.c_float * 5),
                ("switch_candidates", ctypes.c_int64 * 5), ("tau", ctypes.c_int32),
                ("tau_ms", ctypes.c_float * 8)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


STATS_DTYPE = np.dtype([(n, np.dtype(t._type_)) for n, t in QueryStats._fields_], align=True)
assert STATS_DTYPE.itemsize == ctypes.sizeof(QueryStats)

_lib = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _LIB_PATH


def load_library(build_if_missing: bool = True):
    """Load libgeer.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        build_library()
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH}")
    L = ctypes.CDLL(_LIB_PATH)
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.ger_default_options.argtypes = [ctypes.POINTER(Options)]
    L.ger_default_options.restype = None
    L.ger_load_csr.argtypes = [i64, _P, _P, ctypes.c_int, ctypes.POINTER(_P)]
    L.ger_free.argtypes = [_P]
    L.ger_free.restype = None
    L.ger_graph_size.argtypes = [_P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.ger_spectral_bound.argtypes = [_P, ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(f64)]
    L.ger_set_spectral_bound.argtypes = [_P, f64]
    L.ger_spectral_bound_info.argtypes = [_P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(f64),
                                          ctypes.POINTER(f64)]
    L.ger_query_batch.argtypes = [_P, i64, _P, _P, f64, ctypes.POINTER(Options), _P, _P]
    L.ger_query_batch_eps.argtypes = [_P, i64, _P, _P, _P, ctypes.POINTER(Options), _P, _P]
    L.ger_query_batch_dev.argtypes = [_P, i64, _P, _P, _P, ctypes.POINTER(Options), _P, _P, _P]
    L.ger_query_batch_dev_noalloc.argtypes = [_P, i64, _P, _P, _P, ctypes.POINTER(Options), _P, _P, _P]
    L.ger_last_error.argtypes = []
    L.ger_last_error.restype = ctypes.c_char_p
    L.ger_test_fail_alloc.argtypes = [i64]
    L.ger_test_fail_alloc.restype = ctypes.c_int
    L.ger_launch_count.argtypes = []
    L.ger_launch_count.restype = i64
    L.ger_profile_enable.argtypes = [ctypes.c_int]
    L.ger_profile_enable.restype = ctypes.c_int
    L.ger_profile_read.argtypes = [ctypes.POINTER(KernelProfile), ctypes.c_int]
    L.ger_profile_read.restype = ctypes.c_int
    L.ger_set_switch_mlp.argtypes = [_P, _P, _P]
    L.ger_autotune.argtypes = [_P, i64, _P, _P, _P, ctypes.POINTER(Options), ctypes.POINTER(Tuning)]
    L.ger_smm_trace.argtypes = [_P, i64, _P, _P, _P, ctypes.POINTER(Options), i32, _P, _P]
    L.ger_query_batch_lb.argtypes = [_P, i64, _P, _P, _P, _P, ctypes.POINTER(Options), _P, _P]
    L.ger_mlp_forward.argtypes = [i64, _P, _P, _P]
    L.ger_mlp_gradient.argtypes = [i64, _P, _P, _P, _P, _P]
    L.ger_default_mlp_train_options.argtypes = [ctypes.POINTER(MlpTrainOptions)]
    L.ger_default_mlp_train_options.restype = None
    L.ger_mlp_train.argtypes = [i64, _P, _P, ctypes.POINTER(MlpTrainOptions), _P, _P]
    for name in ("ger_load_csr", "ger_graph_size", "ger_spectral_bound", "ger_set_spectral_bound",
                 "ger_spectral_bound_info",
                 "ger_query_batch", "ger_query_batch_eps", "ger_query_batch_dev",
                 "ger_query_batch_dev_noalloc", "ger_set_switch_mlp", "ger_smm_trace", "ger_mlp_forward",
                 "ger_mlp_gradient", "ger_mlp_train", "ger_autotune", "ger_query_batch_lb"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != GER_OK:
        raise GeerError(rc, load_library(False).ger_last_error().decode(errors="replace"))


def default_options(**kw) -> Options:
    o = Options()
    load_library().ger_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def launch_count() -> int:
    return int(load_library().ger_launch_count())


def test_fail_alloc(countdown: int):
    """Testing hook (ger_test_fail_alloc): make the countdown-th next
    workspace allocation fail; 0 disarms."""
    _check(load_library().ger_test_fail_alloc(int(countdown)))


def profile_enable(on: bool = True):
    """Time every kernel launch with CUDA events on its launch stream."""
    _check(load_library().ger_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{family: (launches, total_ms)} since the last profile_enable(True)."""
    buf = (KernelProfile * 32)()
    k = load_library().ger_profile_read(buf, 32)
    if k < 0:
        _check(k)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(k, 32))}


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _fp16_bits(w) -> np.ndarray:
    """FP16 weights as their IEEE binary16 bit patterns (uint16)."""
    w = np.asarray(w)
    if w.dtype == np.uint16:
        out = np.ascontiguousarray(w)
    else:
        out = np.ascontiguousarray(w, dtype=np.float16).view(np.uint16)
    if out.shape != (MLP_PARAMS,):
        raise ValueError(f"expected {MLP_PARAMS} weights")
    return out


def mlp_forward(x, weights) -> np.ndarray:
    """Network outputs for normalised inputs x[rows][6] (GPU kernel)."""
    x = _arr(x, np.float32).reshape(-1, MLP_INPUTS)
    w = _fp16_bits(weights)
    y = np.zeros(x.shape[0], dtype=np.float32)
    _check(load_library().ger_mlp_forward(x.shape[0], x.ctypes.data_as(_P), w.ctypes.data_as(_P),
                                          y.ctypes.data_as(_P)))
    return y


def mlp_gradient(x, target, weights):
    """(gradient over the MLP_PARAMS parameters, loss) of the mean squared
    error, computed by the GPU backward kernels."""
    x = _arr(x, np.float32).reshape(-1, MLP_INPUTS)
    t = _arr(target, np.float32)
    w = _fp16_bits(weights)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(load_library().ger_mlp_gradient(x.shape[0], x.ctypes.data_as(_P), t.ctypes.data_as(_P),
                                           w.ctypes.data_as(_P), g.ctypes.data_as(_P), ctypes.byref(loss)))
    return g, float(loss.value)


def mlp_train_options(**kw) -> MlpTrainOptions:
    o = MlpTrainOptions()
    load_library().ger_default_mlp_train_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def mlp_train(x, target, weights, options: MlpTrainOptions | None = None):
    """Train on the GPU (Adam, FP16 weights in the passes); returns
    (trained FP16 weights as uint16 bits, per-epoch loss)."""
    x = _arr(x, np.float32).reshape(-1, MLP_INPUTS)
    t = _arr(target, np.float32)
    w = _fp16_bits(weights).copy()
    o = options if options is not None else mlp_train_options()
    loss = np.zeros(max(o.epochs, 1), dtype=np.float32)
    _check(load_library().ger_mlp_train(x.shape[0], x.ctypes.data_as(_P), t.ctypes.data_as(_P), ctypes.byref(o),
                                        w.ctypes.data_as(_P), loss.ctypes.data_as(_P)))
    return w, loss[:o.epochs]


# ---------------------------------------------------------------------------
# spectral-bound sidecar: lambda depends on the graph alone (Section 3.1 computes it
# once per graph), so it is kept in a small JSON file keyed by a hash of the CSR
# ---------------------------------------------------------------------------
LAMBDA_FORMAT = "geer-lambda-2"


def csr_key(row_ptr, col_idx) -> str:
    """Content key of a CSR graph: BLAKE2b-256 over n, nnz and both arrays."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = hashlib.blake2b(digest_size=32)
    h.update(np.array([rp.shape[0] - 1, ci.shape[0]], np.int64).tobytes())
    h.update(memoryview(rp).cast("B"))
    h.update(memoryview(ci).cast("B"))
    return h.hexdigest()


def _lambda_path(cache_dir: str, key: str) -> str:
    return os.path.join(cache_dir, f"lambda-{key}.json")


def read_lambda_sidecar(cache_dir: str, key: str, n: int, nnz: int):
    """(lambda, lambda_2, lambda_n) stored for this graph, or None (absent,
    unreadable, written for another graph, or not marked as a converged
    Lanczos result)."""
    try:
        with open(_lambda_path(cache_dir, key)) as f:
            d = json.load(f)
        if d.get("format") != LAMBDA_FORMAT or d.get("key") != key or d.get("n") != n or d.get("nnz") != nnz:
            return None
        if d.get("converged") is not True:
            return None
        lam, l2, ln = float(d["lambda"]), float(d["lambda_2"]), float(d["lambda_n"])
    except (OSError, ValueError, KeyError, TypeError):
        return None
    if not (0.0 <= lam < 1.0):
        return None
    return lam, l2, ln


def write_lambda_sidecar(cache_dir: str, key: str, n: int, nnz: int, lam: float, l2: float, ln: float,
                         converged: bool = True, steps: int = 0) -> str:
    """Store the graph's spectral bound (written to a temporary file, then
    renamed), with whether its Lanczos run converged; only converged values
    are read back."""
    os.makedirs(cache_dir, exist_ok=True)
    path = _lambda_path(cache_dir, key)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump({"format": LAMBDA_FORMAT, "key": key, "n": int(n), "nnz": int(nnz), "lambda": float(lam),
                   "lambda_2": float(l2), "lambda_n": float(ln), "converged": bool(converged),
                   "steps": int(steps)}, f)
    os.replace(tmp, path)
    return path


class Graph:
    """A graph resident on one GPU (ger_load_csr ... ger_free). With
    keyed=True the CSR's content key is computed at load (a pass over the
    arrays), so that spectral_bound(cache_dir=...) can keep lambda beside it."""

    def __init__(self, row_ptr, col_idx, device: int = 0, keyed: bool = False):
        L = load_library()
        self._rp = _arr(row_ptr, np.int64)
        self._ci = _arr(col_idx, np.int32)
        self.key = csr_key(self._rp, self._ci) if keyed else None
        h = _P()
        n = self._rp.shape[0] - 1
        _check(L.ger_load_csr(n, self._rp.ctypes.data_as(_P), self._ci.ctypes.data_as(_P), int(device),
                              ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.nnz = int(self._rp[-1])
        self._rp = self._ci = None  # the library holds its own copy

    @classmethod
    def from_csr(cls, g, device: int = 0, keyed: bool = False) -> "Graph":
        return cls(g.row_ptr, g.col_idx, device, keyed)

    def close(self):
        if getattr(self, "_h", None):
            load_library().ger_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spectral_bound(self, cache_dir: str | None = None):
        """(lambda, lambda_2, lambda_n) computed on the GPU (Section 3.1). With
        cache_dir (and a keyed graph) a stored value is injected instead
        (ger_set_spectral_bound), and a computed one is stored."""
        use_cache = cache_dir is not None and self.key is not None
        if use_cache:
            hit = read_lambda_sidecar(cache_dir, self.key, self.n, self.nnz)
            if hit is not None:
                self.set_spectral_bound(hit[0])
                return hit
        lam, l2, ln = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load_library().ger_spectral_bound(self._h, ctypes.byref(lam), ctypes.byref(l2), ctypes.byref(ln)))
        if use_cache:
            info = self.spectral_info()
            write_lambda_sidecar(cache_dir, self.key, self.n, self.nnz, lam.value, l2.value, ln.value,
                                 converged=info["converged"], steps=info["steps"])
        return lam.value, l2.value, ln.value

    def spectral_info(self) -> dict:
        """How lambda was obtained (ger_spectral_bound_info): Lanczos steps (0
        when set by the caller), convergence, and the residual bounds of the
        two extreme Ritz pairs (lambda is widened by them when unconverged)."""
        conv, steps = ctypes.c_int32(), ctypes.c_int32()
        rh, rl = ctypes.c_double(), ctypes.c_double()
        _check(load_library().ger_spectral_bound_info(self._h, ctypes.byref(conv), ctypes.byref(steps),
                                                      ctypes.byref(rh), ctypes.byref(rl)))
        return {"converged": bool(conv.value), "steps": int(steps.value), "resid_hi": rh.value,
                "resid_lo": rl.value}

    def set_spectral_bound(self, lam: float):
        _check(load_library().ger_set_spectral_bound(self._h, float(lam)))

    def query(self, s, t, eps, options: Options | None = None, stats: bool = False):
        """r'(s,t) for host arrays s, t (eps scalar or per query). Returns r
        (float64 array) or (r, stats record array)."""
        L = load_library()
        s = _arr(s, np.int32)
        t = _arr(t, np.int32)
        q = s.shape[0]
        if t.shape[0] != q:
            raise ValueError("s and t differ in length")
        r = np.zeros(q, dtype=np.float64)
        st = np.zeros(q, dtype=STATS_DTYPE) if stats else None
        opt = options if options is not None else default_options()
        sp = st.ctypes.data_as(_P) if st is not None else None
        if np.ndim(eps) == 0:
            rc = L.ger_query_batch(self._h, q, s.ctypes.data_as(_P), t.ctypes.data_as(_P), float(eps),
                                   ctypes.byref(opt), r.ctypes.data_as(_P), sp)
        else:
            e = _arr(eps, np.float64)
            if e.shape[0] != q:
                raise ValueError("eps length differs from q")
            rc = L.ger_query_batch_eps(self._h, q, s.ctypes.data_as(_P), t.ctypes.data_as(_P),
                                       e.ctypes.data_as(_P), ctypes.byref(opt), r.ctypes.data_as(_P), sp)
        _check(rc)
        return (r, st) if stats else r

    def set_switch_mlp(self, norm, weights):
        """Install the learned switch: norm = (mean[6], std[6]) of the raw
        inputs, FP16 weights; None removes it."""
        L = load_library()
        if weights is None:
            _check(L.ger_set_switch_mlp(self._h, None, None))
            return
        nv = _arr(norm, np.float32).reshape(2 * MLP_INPUTS)
        w = _fp16_bits(weights)
        _check(L.ger_set_switch_mlp(self._h, nv.ctypes.data_as(_P), w.ctypes.data_as(_P)))

    def autotune(self, s, t, eps, options: Options | None = None) -> dict:
        """Time the dense block widths and the hybrid switch sizes on these
        queries (ger_autotune); the choices stay on the graph."""
        s = _arr(s, np.int32)
        t = _arr(t, np.int32)
        e = _arr(np.broadcast_to(eps, s.shape), np.float64)
        res = Tuning()
        opt = options if options is not None else default_options()
        _check(load_library().ger_autotune(self._h, s.shape[0], s.ctypes.data_as(_P), t.ctypes.data_as(_P),
                                           e.ctypes.data_as(_P), ctypes.byref(opt), ctypes.byref(res)))
        return {"dense_width": res.dense_width, "dense_switch": int(res.dense_switch),
                "width_ms": list(res.width_ms), "switch_ms": list(res.switch_ms),
                "switch_candidates": [int(x) for x in res.switch_candidates], "tau": int(res.tau),
                "tau_ms": list(res.tau_ms)}

    def query_lb(self, s, t, eps, ell_b, options: Options | None = None, stats: bool = False):
        """r'(s,t) with query i running min(ell_b[i], l) SMM iterations in
        place of Eq. (17)'s switch (ger_query_batch_lb; ell_b[i] < 0: the
        options' policy). Returns r or (r, stats)."""
        L = load_library()
        s = _arr(s, np.int32)
        t = _arr(t, np.int32)
        q = s.shape[0]
        e = _arr(np.broadcast_to(eps, (q,)), np.float64)
        lb = _arr(np.broadcast_to(ell_b, (q,)), np.int32)
        r = np.zeros(q, dtype=np.float64)
        st = np.zeros(q, dtype=STATS_DTYPE) if stats else None
        opt = options if options is not None else default_options()
        _check(L.ger_query_batch_lb(self._h, q, s.ctypes.data_as(_P), t.ctypes.data_as(_P), e.ctypes.data_as(_P),
                                    lb.ctypes.data_as(_P), ctypes.byref(opt), r.ctypes.data_as(_P),
                                    st.ctypes.data_as(_P) if st is not None else None))
        return (r, st) if stats else r

    def smm_trace(self, s, t, eps, options: Options | None = None, max_steps: int = 16):
        """Cost log: (log[q][max_steps][LOG_WIDTH], stats) of a batch run
        with min(max_steps, l) SMM iterations; see ger_smm_trace."""
        s = _arr(s, np.int32)
        t = _arr(t, np.int32)
        q = s.shape[0]
        e = _arr(np.broadcast_to(eps, (q,)), np.float64)
        log = np.zeros((q, max_steps, LOG_WIDTH), dtype=np.float32)
        st = np.zeros(q, dtype=STATS_DTYPE)
        opt = options if options is not None else default_options()
        _check(load_library().ger_smm_trace(self._h, q, s.ctypes.data_as(_P), t.ctypes.data_as(_P),
                                            e.ctypes.data_as(_P), ctypes.byref(opt), int(max_steps),
                                            log.ctypes.data_as(_P), st.ctypes.data_as(_P)))
        return log, st

    def query_dev(self, s_dev, t_dev, eps_dev, r_dev, stats_dev=None, options: Options | None = None,
                  stream=None):
        """Device-resident variant: arguments are CUDA tensors (or raw device
        pointers as ints) on this graph's GPU; stats_dev, if given, is a
        uint8 tensor of q * sizeof(ger_query_stats) bytes."""
        def ptr(x):
            if x is None:
                return None
            return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
        q = int(s_dev.shape[0]) if hasattr(s_dev, "shape") else None
        if q is None:
            raise ValueError("s_dev must be a tensor")
        opt = options if options is not None else default_options()
        _check(load_library().ger_query_batch_dev(self._h, q, ptr(s_dev), ptr(t_dev), ptr(eps_dev),
                                                  ctypes.byref(opt), ptr(r_dev), ptr(stats_dev),
                                                  ctypes.c_void_p(stream) if stream else None))

    def query_dev_noalloc(self, s_dev, t_dev, eps_dev, r_dev, stats_dev=None, options: Options | None = None,
                          stream=None):
        """As query_dev, through ger_query_batch_dev_noalloc: for callers
        that cannot allocate device memory. All scratch comes from a static
        32 MiB device array; at most 64 queries per call; the spectral bound
        must already be set or computed. Calls that overlap on the GPU race
        on the shared array."""
        def ptr(x):
            if x is None:
                return None
            return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
        q = int(s_dev.shape[0])
        opt = options if options is not None else default_options()
        _check(load_library().ger_query_batch_dev_noalloc(self._h, q, ptr(s_dev), ptr(t_dev), ptr(eps_dev),
                                                          ctypes.byref(opt), ptr(r_dev), ptr(stats_dev),
                                                          ctypes.c_void_p(stream) if stream else None))
