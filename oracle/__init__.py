"""CPU oracle for the GEER hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path
(``paper_2312_06123_gb300``) and never imports it.

Two layers:
  * ``geer_oracle.c`` (loaded here through ctypes): the algorithm, step by
    step, in plain single-threaded FP64 C -- SMM (Algorithm 2), AMC
    (Algorithm 1), GEER (Algorithm 3), the truncation length (Eq. 6, Eq. 5),
    the spectral bound (Section 3.1) and the walk RNG specification.
  * ``exact.py``: the closed definitions (dense pseudo-inverse, Eq. 1; dense
    matrix powers, Eq. 3/4/11) in numpy, for small graphs.

Every function is pinned by the ``-m "not gpu"`` tests against values the
paper and the mathematics fix (see ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geer_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

i64 = ctypes.c_int64
i32 = ctypes.c_int32
u64 = ctypes.c_uint64
f64 = ctypes.c_double
P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _AmcOut(ctypes.Structure):
    _fields_ = [("psi", f64), ("eta_star", f64), ("eta0", i64), ("batches", i32),
                ("free_batches", i32), ("walks", i64), ("walk_steps", i64), ("r_f", f64),
                ("f_last", f64), ("var_last", f64), ("checksum", u64)]


class _GeerOut(ctypes.Structure):
    _fields_ = [("r", f64), ("r_b", f64), ("r_f", f64), ("ell", i64), ("ell_b", i64),
                ("free_ell_b", i64), ("volume", f64), ("h", f64), ("amc", _AmcOut)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.og_philox4x32_10.argtypes = [P, P, P]
        L.og_walk_hash.argtypes = [i32, i64, ctypes.c_int, ctypes.c_int]
        L.og_walk_hash.restype = u64
        L.og_walk.argtypes = [P, P, i32, ctypes.c_int, u64, i64, ctypes.c_int, ctypes.c_int, i64, P]
        L.og_ell.argtypes = [f64, f64, f64, f64]
        L.og_ell.restype = i64
        L.og_ell_peng.argtypes = [f64, f64]
        L.og_ell_peng.restype = i64
        L.og_eta_star.argtypes = [f64, f64, f64, f64]
        L.og_eta_star.restype = f64
        L.og_bernstein.argtypes = [f64, f64, f64, f64]
        L.og_bernstein.restype = f64
        L.og_apply_P.argtypes = [i64, P, P, P, P]
        L.og_top2.argtypes = [i64, P, P, P]
        L.og_psi.argtypes = [i64, f64, f64, f64, f64, f64, f64]
        L.og_psi.restype = f64
        L.og_smm_terms.argtypes = [i64, P, P, i32, i32, i64, P]
        L.og_smm_terms.restype = ctypes.c_int
        L.og_amc.argtypes = [i64, P, P, i32, i32, P, P, i64, f64, ctypes.c_int, f64, u64, i64,
                             i64, ctypes.c_int, ctypes.POINTER(_AmcOut)]
        L.og_amc.restype = ctypes.c_int
        L.og_geer.argtypes = [i64, P, P, i32, i32, f64, f64, ctypes.c_int, u64, f64, i64, i64,
                              i64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_GeerOut), P]
        L.og_geer.restype = ctypes.c_int
        L.og_spectral_bound.argtypes = [i64, P, P, i64, f64, P, P]
        L.og_spectral_bound.restype = i64
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(P)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    return rp, ci


# ---------------------------------------------------------------------------
# thin wrappers
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().og_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def walk(g, start: int, lf: int, seed: int, q_index: int, b: int, sigma: int, k: int) -> np.ndarray:
    rp, ci = _csr(g)
    out = np.zeros(max(lf, 1), dtype=np.int32)
    lib().og_walk(_ptr(rp), _ptr(ci), int(start), int(lf), int(seed), int(q_index), int(b),
                  int(sigma), int(k), _ptr(out))
    return out[:lf]


def walk_hash(endpoint: int, k: int, sigma: int, b: int) -> int:
    return int(lib().og_walk_hash(int(endpoint), int(k), int(sigma), int(b)))


def ell(ds: float, dt: float, eps: float, lam: float) -> int:
    return int(lib().og_ell(float(ds), float(dt), float(eps), float(lam)))


def ell_peng(eps: float, lam: float) -> int:
    return int(lib().og_ell_peng(float(eps), float(lam)))


def eta_star(psi: float, eps: float, delta: float, tau: float) -> float:
    return float(lib().og_eta_star(psi, eps, delta, tau))


def bernstein(n: float, var: float, psi: float, delta_b: float) -> float:
    return float(lib().og_bernstein(n, var, psi, delta_b))


def apply_P(g, x: np.ndarray) -> np.ndarray:
    rp, ci = _csr(g)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(g.n, dtype=np.float64)
    lib().og_apply_P(g.n, _ptr(rp), _ptr(ci), _ptr(x), _ptr(y))
    return y


def top2(x: np.ndarray) -> tuple[float, float]:
    x = np.ascontiguousarray(x, dtype=np.float64)
    a = np.zeros(1)
    b = np.zeros(1)
    lib().og_top2(x.shape[0], _ptr(x), _ptr(a), _ptr(b))
    return float(a[0]), float(b[0])


def psi(lf, s1, s2, t1, t2, ds, dt) -> float:
    return float(lib().og_psi(int(lf), s1, s2, t1, t2, float(ds), float(dt)))


def smm_terms(g, s: int, t: int, L: int) -> np.ndarray:
    rp, ci = _csr(g)
    out = np.zeros(L + 1)
    rc = lib().og_smm_terms(g.n, _ptr(rp), _ptr(ci), int(s), int(t), int(L), _ptr(out))
    assert rc == 0
    return out


@dataclasses.dataclass
class AmcResult:
    psi: float
    eta_star: float
    eta0: int
    batches: int
    free_batches: int
    walks: int
    walk_steps: int
    r_f: float
    f_last: float
    var_last: float
    checksum: int


def _amc_result(a: _AmcOut) -> AmcResult:
    return AmcResult(a.psi, a.eta_star, a.eta0, a.batches, a.free_batches, a.walks, a.walk_steps,
                     a.r_f, a.f_last, a.var_last, a.checksum)


def amc(g, s, t, xs, xt, lf, eps, tau=5, delta=0.01, seed=3, q_index=0, forced_eta0=0,
        forced_batches=0) -> AmcResult:
    rp, ci = _csr(g)
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    o = _AmcOut()
    rc = lib().og_amc(g.n, _ptr(rp), _ptr(ci), int(s), int(t), _ptr(xs), _ptr(xt), int(lf),
                      float(eps), int(tau), float(delta), int(seed), int(q_index),
                      int(forced_eta0), int(forced_batches), ctypes.byref(o))
    assert rc == 0
    return _amc_result(o)


@dataclasses.dataclass
class GeerResult:
    r: float
    r_b: float
    r_f: float
    ell: int
    ell_b: int
    free_ell_b: int
    volume: float
    h: float
    amc: AmcResult
    trace: np.ndarray | None = None


def geer(g, s, t, eps, lam, delta=0.01, tau=5, seed=3, q_index=0, forced_ell_b=-1,
         forced_eta0=0, forced_batches=0, peng_ell=False, trace=False) -> GeerResult:
    """One GEER query (Algorithm 3). forced_* replay decisions (see the C
    source); q_index is the query's index in its batch (walk RNG key)."""
    rp, ci = _csr(g)
    o = _GeerOut()
    tr = None
    if trace:
        cap = 6 * (max(ell(g.degrees()[s], g.degrees()[t], eps, lam), forced_ell_b, 0) + 2)
        tr = np.zeros(cap)
    rc = lib().og_geer(g.n, _ptr(rp), _ptr(ci), int(s), int(t), float(eps), float(delta),
                       int(tau), int(seed), float(lam), int(q_index), int(forced_ell_b),
                       int(forced_eta0), int(forced_batches), int(bool(peng_ell)),
                       ctypes.byref(o), _ptr(tr) if tr is not None else None)
    if rc != 0:
        raise RuntimeError(f"og_geer failed ({rc})")
    res = GeerResult(o.r, o.r_b, o.r_f, o.ell, o.ell_b, o.free_ell_b, o.volume, o.h,
                     _amc_result(o.amc))
    if tr is not None:
        res.trace = tr[:6 * o.ell_b].reshape(-1, 6)
    return res


def spectral_bound(g, max_steps: int = 300, tol: float = 1e-13) -> tuple[float, float, int]:
    """(lambda_2, lambda_n, lanczos steps) of P = D^-1 A (Section 3.1)."""
    rp, ci = _csr(g)
    a = np.zeros(1)
    b = np.zeros(1)
    k = lib().og_spectral_bound(g.n, _ptr(rp), _ptr(ci), int(max_steps), float(tol), _ptr(a), _ptr(b))
    if k < 0:
        raise RuntimeError(f"og_spectral_bound failed ({k})")
    return float(a[0]), float(b[0]), int(k)


def lam(g, **kw) -> float:
    l2, ln, _ = spectral_bound(g, **kw)
    return max(abs(l2), abs(ln))
