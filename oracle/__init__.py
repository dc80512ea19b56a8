"""ORACLE — test infrastructure only.

Plain FP64 CPU reference of the local diffusion process (LocalGD, Eq. local-gd of
arXiv 2410.21634) for PPR, Katz and the heat kernel, the sequential FIFO push it
is compared with (Algo 1 and the AKatz/AHK updates of Section 2), and dense
closed-form references.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library and
its Python binding never do, and the two share no code.

The C core (``localgd.c``) is compiled with gcc ``-ffp-contract=off`` so each
arithmetic step is one IEEE binary64 operation in the written order.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

from . import dense  # noqa: F401  (re-exported)

PPR, KATZ, HK = 0, 1, 2
KINDS = {"ppr": PPR, "katz": KATZ, "hk": HK}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "localgd.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile localgd.c into _oracle.so.  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Round(ctypes.Structure):
    _fields_ = [("n_active", ctypes.c_int64), ("vol_active", ctypes.c_int64),
                ("rS_l1", ctypes.c_double)]


class _Solve(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("volume", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("resid_l1", ctypes.c_double),
                ("x_l1", ctypes.c_double), ("status", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            I64, D, I = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            rp = ctypes.POINTER(_Round)
            for name in ("oracle_ppr_round", "oracle_katz_round"):
                f = getattr(lib, name)
                f.argtypes = [I64, i64p, i32p, D, D, f64p, f64p, i32p, f64p, rp]
                f.restype = I64
            lib.oracle_hk_round.argtypes = [I64, i64p, i32p, D, I64, I, D, f64p, f64p, f64p,
                                            i32p, f64p, rp]
            lib.oracle_hk_round.restype = I64
            lib.oracle_hk_terms.argtypes = [D, D]
            lib.oracle_hk_terms.restype = I64
            lib.oracle_hk_psi.argtypes = [D, I64, I64]
            lib.oracle_hk_psi.restype = D
            lib.oracle_hk_theta.argtypes = [D, I64, I64, I]
            lib.oracle_hk_theta.restype = D
            lib.oracle_localgd_solve.argtypes = [I64, i64p, i32p, I, D, D, ctypes.c_int32, I, D,
                                                 I64, f64p, ctypes.POINTER(_Solve), ctypes.c_void_p,
                                                 I64]
            lib.oracle_localgd_solve.restype = I
            lib.oracle_localgd_solve_many.argtypes = [I64, i64p, i32p, I, D, D, i32p, I64, I, D,
                                                      I64, f64p, ctypes.c_void_p]
            lib.oracle_localgd_solve_many.restype = I
            lib.oracle_push_fifo.argtypes = [I64, i64p, i32p, I, D, D, ctypes.c_int32, I, D,
                                             f64p, ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_push_fifo.restype = I64
            lib.oracle_gppr_round.argtypes = [I64, i64p, i32p, D, D, D, f64p, f64p, i32p, f64p, rp]
            lib.oracle_gppr_round.restype = I64
            lib.oracle_gppr_solve.argtypes = [I64, i64p, i32p, D, D, D, ctypes.c_int32, I64, f64p, rp,
                                              ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_gppr_solve.restype = I
            lib.oracle_series_round.argtypes = [I64, i64p, i32p, D, I, D, f64p, f64p, f64p, i32p, f64p, rp]
            lib.oracle_series_round.restype = I64
            lib.oracle_series_psi.argtypes = [f64p, I64, I64]
            lib.oracle_series_psi.restype = D
            lib.oracle_series_theta.argtypes = [f64p, I64, I64, I]
            lib.oracle_series_theta.restype = D
            lib.oracle_series_solve.argtypes = [I64, i64p, i32p, f64p, I64, D, ctypes.c_int32, I, I64, f64p,
                                                ctypes.POINTER(_Solve)]
            lib.oracle_series_solve.restype = I
            lib.oracle_localch_solve.argtypes = [I64, i64p, i32p, D, D, ctypes.c_int32, I64, f64p, f64p,
                                                 ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_localch_solve.restype = I64
            lib.oracle_gd_solve.argtypes = [I64, i64p, i32p, I, D, D, ctypes.c_int32, I64, f64p]
            lib.oracle_gd_solve.restype = I64
            _lib = lib
    return _lib


def _kind(kind) -> int:
    return KINDS[kind] if isinstance(kind, str) else int(kind)


# ------------------------------------------------------------- heat kernel ----

HK_TOL = 1e-12


def hk_terms(tau: float, tol: float = HK_TOL) -> int:
    """Smallest N with e^-tau sum_{k>N} tau^k/k! <= tol."""
    return int(_load().oracle_hk_terms(tau, tol))


def hk_psi(tau: float, N: int, k: int) -> float:
    """psi_k(tau) = sum_{j=0}^{N-k} tau^j k!/(k+j)!"""
    return float(_load().oracle_hk_psi(tau, N, k))


def hk_theta(tau: float, N: int, t: int, mode: int = 0) -> float:
    """Threshold scale of layer t: e^tau/((N+1) psi_t) (mode 0) or 1 (mode 1)."""
    return float(_load().oracle_hk_theta(tau, N, t, mode))


# ------------------------------------------------------------------ rounds ----

@dataclass
class RoundResult:
    active: np.ndarray      # S_t, ascending ids
    rho: np.ndarray         # r^(t) on S_t (the pushed snapshot)
    n_active: int
    vol_active: int
    rS_l1: float


def localgd_round(g, kind, param: float, eps: float, x: np.ndarray, r: np.ndarray,
                  t: int = 0, r_next: np.ndarray | None = None, hk_mode: int = 0,
                  hk_tol: float = HK_TOL, eps_theta: float | None = None) -> RoundResult:
    """One synchronous LocalGD round, in place on (x, r[, r_next]) (float64 arrays).

    PPR/Katz: r is the residual.  HK: r is layer t, r_next layer t+1; the layer count
    N and theta_t come from (param=tau, hk_tol, hk_mode) unless eps_theta is given.
    """
    lib = _load()
    k = _kind(kind)
    n = g.n
    active = np.empty(max(n, 1), dtype=np.int32)
    rho = np.empty(max(n, 1), dtype=np.float64)
    st = _Round()
    if k == PPR:
        cnt = lib.oracle_ppr_round(n, g.offsets, g.cols, param, eps, x, r, active, rho, st)
    elif k == KATZ:
        cnt = lib.oracle_katz_round(n, g.offsets, g.cols, param, eps, x, r, active, rho, st)
    else:
        N = hk_terms(param, hk_tol)
        if eps_theta is None:
            eps_theta = hk_theta(param, N, t, hk_mode) * eps
        if r_next is None:
            raise ValueError("heat kernel rounds need r_next")
        cnt = lib.oracle_hk_round(n, g.offsets, g.cols, param, t, int(t < N), eps_theta, x, r,
                                  r_next, active, rho, st)
    return RoundResult(active[:cnt].copy(), rho[:cnt].copy(), st.n_active, st.vol_active,
                       st.rS_l1)


@dataclass
class SolveResult:
    x: np.ndarray
    rounds: int
    volume: int
    pushes: int
    resid_l1: float
    x_l1: float
    status: int
    log: list


def localgd(g, kind, param: float, eps: float, seed: int, hk_mode: int = 0,
            hk_tol: float = HK_TOL, max_rounds: int = 1_000_000, log: bool = False) -> SolveResult:
    """LocalGD from e_seed until the active set is empty.  x is f_PPR, (I-beta A)^-1 e_s
    (Katz) or e^-tau x (HK, so that it approximates the heat-kernel vector)."""
    lib = _load()
    x = np.zeros(g.n, dtype=np.float64)
    res = _Solve()
    cap = min(max_rounds, 1_000_000) if log else 0
    buf = (_Round * cap)() if cap else None
    st = lib.oracle_localgd_solve(g.n, g.offsets, g.cols, _kind(kind), param, eps, int(seed),
                                  hk_mode, hk_tol, max_rounds, x, ctypes.byref(res),
                                  ctypes.cast(buf, ctypes.c_void_p) if buf is not None else None,
                                  cap)
    if st < 0:
        raise MemoryError("oracle_localgd_solve: allocation failed")
    rl = []
    if buf is not None:
        rl = [(buf[i].n_active, buf[i].vol_active, buf[i].rS_l1)
              for i in range(min(res.rounds, cap))]
    return SolveResult(x, res.rounds, res.volume, res.pushes, res.resid_l1, res.x_l1,
                       res.status, rl)


def localgd_many(g, kind, param: float, eps: float, seeds, hk_mode: int = 0,
                 hk_tol: float = HK_TOL, max_rounds: int = 1_000_000):
    """Independent LocalGD solves, one source per OpenMP thread.  Returns (xs [k, n],
    list of per-seed (rounds, volume, pushes, resid_l1, x_l1, status))."""
    lib = _load()
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    k = seeds.shape[0]
    xs = np.zeros((k, g.n), dtype=np.float64)
    res = (_Solve * max(k, 1))()
    st = lib.oracle_localgd_solve_many(g.n, g.offsets, g.cols, _kind(kind), param, eps, seeds, k,
                                       hk_mode, hk_tol, max_rounds, xs.reshape(-1),
                                       ctypes.cast(res, ctypes.c_void_p))
    if st < 0:
        raise MemoryError("oracle_localgd_solve_many: allocation failed")
    info = [(res[i].rounds, res[i].volume, res[i].pushes, res[i].resid_l1, res[i].x_l1,
             res[i].status) for i in range(k)]
    return xs, info


def push_fifo(g, kind, param: float, eps: float, seed: int, hk_mode: int = 0,
              hk_tol: float = HK_TOL):
    """Sequential FIFO push (Algo 1 / AKatz / AHK).  Returns (x, pushes, volume)."""
    lib = _load()
    x = np.zeros(g.n, dtype=np.float64)
    vol = ctypes.c_int64(0)
    p = lib.oracle_push_fifo(g.n, g.offsets, g.cols, _kind(kind), param, eps, int(seed), hk_mode,
                             hk_tol, x, ctypes.byref(vol))
    if p < 0:
        raise MemoryError("oracle_push_fifo: allocation failed")
    return x, int(p), int(vol.value)


def gppr_round(g, alpha: float, beta: float, eps: float, x: np.ndarray, r: np.ndarray) -> RoundResult:
    """One LocalGD round of the generalised propagation M = D^-beta A D^(beta-1), in place."""
    lib = _load()
    n = g.n
    active = np.empty(max(n, 1), dtype=np.int32)
    rho = np.empty(max(n, 1), dtype=np.float64)
    st = _Round()
    cnt = lib.oracle_gppr_round(n, g.offsets, g.cols, alpha, beta, eps, x, r, active, rho, st)
    return RoundResult(active[:cnt].copy(), rho[:cnt].copy(), st.n_active, st.vol_active, st.rS_l1)


def gppr(g, alpha: float, beta: float, eps: float, seed: int, max_rounds: int = 1_000_000):
    """Generalised-propagation LocalGD from e_seed.  Returns (x, rounds, volume, pushes, ||r||_1)."""
    lib = _load()
    x = np.zeros(g.n, dtype=np.float64)
    tot = _Round()
    rounds = ctypes.c_int64()
    st = lib.oracle_gppr_solve(g.n, g.offsets, g.cols, alpha, beta, eps, int(seed), max_rounds, x,
                               ctypes.byref(tot), ctypes.byref(rounds))
    if st < 0:
        raise MemoryError("oracle_gppr_solve: allocation failed")
    return x, int(rounds.value), int(tot.vol_active), int(tot.n_active), float(tot.rS_l1)


def series(g, coef, eps: float, seed: int, mode: int = 0, max_rounds: int = 1_000_000) -> SolveResult:
    """LocalGD on the layered system of f = sum_k coef[k] (A D^-1)^k e_s (coef > 0, N =
    len(coef) - 1); x is returned scaled by coef[0], so that it approximates f."""
    lib = _load()
    c = np.ascontiguousarray(coef, dtype=np.float64)
    x = np.zeros(g.n, dtype=np.float64)
    res = _Solve()
    st = lib.oracle_series_solve(g.n, g.offsets, g.cols, c, c.shape[0] - 1, eps, int(seed), mode,
                                 max_rounds, x, ctypes.byref(res))
    if st < 0:
        raise MemoryError("oracle_series_solve: allocation failed")
    return SolveResult(x, res.rounds, res.volume, res.pushes, res.resid_l1, res.x_l1, res.status, [])


def global_gd(g, kind, param: float, eps: float, seed: int, max_iter: int = 1_000_000):
    """Standard gradient descent (all nodes every iteration) until ||D^-1 r||_inf < eps.
    Returns (x, iterations); its operation count is iterations * nnz."""
    lib = _load()
    x = np.zeros(g.n, dtype=np.float64)
    it = lib.oracle_gd_solve(g.n, g.offsets, g.cols, _kind(kind), param, eps, int(seed), max_iter, x)
    if it < 0:
        raise MemoryError("oracle_gd_solve: allocation failed")
    return x, int(it)


def localch(g, alpha: float, eps: float, seed: int, max_rounds: int = 1_000_000):
    """LocalCH for PPR from e_seed.  Returns (x, r, rounds, volume)."""
    lib = _load()
    x = np.zeros(g.n, dtype=np.float64)
    r = np.zeros(g.n, dtype=np.float64)
    vol = ctypes.c_int64()
    t = lib.oracle_localch_solve(g.n, g.offsets, g.cols, alpha, eps, int(seed), max_rounds, x, r, ctypes.byref(vol))
    if t < 0:
        raise MemoryError("oracle_localch_solve: allocation failed")
    return x, r, int(t), int(vol.value)


def series_round(g, coef, t: int, eps: float, x: np.ndarray, r: np.ndarray, r_next: np.ndarray,
                 mode: int = 0) -> RoundResult:
    """Round t of the series' layered system, in place (r is layer t, r_next layer t+1)."""
    lib = _load()
    c = np.ascontiguousarray(coef, dtype=np.float64)
    N = c.shape[0] - 1
    n = g.n
    active = np.empty(max(n, 1), dtype=np.int32)
    rho = np.empty(max(n, 1), dtype=np.float64)
    st = _Round()
    ratio = c[t + 1] / c[t] if t < N else 0.0
    eps_theta = lib.oracle_series_theta(c, N, t, mode) * eps
    cnt = lib.oracle_series_round(n, g.offsets, g.cols, ratio, int(t < N), eps_theta, x, r, r_next, active, rho, st)
    return RoundResult(active[:cnt].copy(), rho[:cnt].copy(), st.n_active, st.vol_active, st.rS_l1)


def series_theta(coef, t: int, mode: int = 0) -> float:
    c = np.ascontiguousarray(coef, dtype=np.float64)
    return float(_load().oracle_series_theta(c, c.shape[0] - 1, t, mode))


def topk(x: np.ndarray, k: int):
    """The k largest entries of x, value descending, ties by lower id."""
    n = x.shape[0]
    k = min(k, n)
    order = np.lexsort((np.arange(n), -x))[:k]
    return order.astype(np.int32), x[order]


def hk_scale(tau: float) -> float:
    return math.exp(-tau)
