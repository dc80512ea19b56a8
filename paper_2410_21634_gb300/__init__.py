"""Python binding of the GB300 local graph-diffusion library (include/gde.h).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libgde.so`` (built by ``_build.build()``).  The binding refuses to work
when that library is missing — there is no CPU fallback.

Arrays may be numpy arrays (host) or CUDA tensors (device pointers are passed with
``GDE_DEVICE_PTRS``).  PyTorch is only used, when present, to read a tensor's data
pointer and current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

PPR, KATZ, HK, GPPR, SERIES = 0, 1, 2, 3, 4
KINDS = {"ppr": PPR, "katz": KATZ, "hk": HK, "gppr": GPPR, "series": SERIES}
FP64, FP32 = 0, 1
DEVICE_PTRS = 0x1
CHECK_SYMMETRIC = 0x2
OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT = range(6)
SERVE_TRACK = 1
STATUS_NAMES = {0: "GDE_OK", 1: "GDE_EINVAL", 2: "GDE_ENOMEM", 3: "GDE_ECUDA",
                4: "GDE_ENOTCONV", 5: "GDE_ETIMEOUT"}

EXPORTED = ["gde_solve_opts_init", "gde_graph_create", "gde_graph_destroy", "gde_graph_info",
            "gde_solve", "gde_last_error", "gde_session_begin", "gde_session_step",
            "gde_session_read", "gde_session_end", "gde_profile_enable", "gde_profile_read",
            "gde_topk_f32_noalloc", "gde_profile_rounds", "gde_set_tuning", "gde_get_tuning",
            "gde_autotune", "gde_update_edges", "gde_graph_csr", "gde_server_opts_init",
            "gde_server_clock", "gde_server_create", "gde_server_destroy", "gde_server_submit",
            "gde_server_insert_edges", "gde_server_step", "gde_server_poll", "gde_server_info",
            "gde_probe_random_access", "gde_bsession_begin", "gde_bsession_step", "gde_bsession_read",
            "gde_bsession_end", "gde_test_fail_alloc", "gde_test_barrier_fault"]


class GdeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("topk", ctypes.c_int32), ("hk_threshold", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("max_rounds", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_int64),
                ("hk_tol", ctypes.c_double), ("cuda_stream", ctypes.c_void_p), ("prop_beta", ctypes.c_double),
                ("series_coef", ctypes.c_void_p), ("series_terms", ctypes.c_int64),
                ("global_gd", ctypes.c_int32), ("chebyshev", ctypes.c_int32),
                ("katz_minus_source", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("active_volume", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("resid_l1", ctypes.c_double),
                ("mass_l1", ctypes.c_double), ("status", ctypes.c_int32),
                ("fallback", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class StatsList:
    """The per-seed gde_stats of one solve, read from the C array as they are used: item i is a
    dict of seed i's fields (a batch's 1,024 dicts would cost a millisecond to build up front,
    in the time between two solves)."""

    def __init__(self, arr, n: int):
        self._arr = arr
        self._n = n

    def __len__(self):
        return self._n

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[k] for k in range(*i.indices(self._n))]
        i = int(i)
        if i < 0:
            i += self._n
        if not 0 <= i < self._n:
            raise IndexError("seed index out of range")
        return self._arr[i].as_dict()

    def __iter__(self):
        for i in range(self._n):
            yield self._arr[i].as_dict()

    def __repr__(self):
        return repr(list(self))


class Profile(ctypes.Structure):
    _fields_ = [("batch_rounds_ms", ctypes.c_double), ("batch_clear_ms", ctypes.c_double),
                ("batch_topk_ms", ctypes.c_double), ("dense_frontier_ms", ctypes.c_double),
                ("dense_push_ms", ctypes.c_double), ("batch_launches", ctypes.c_int64),
                ("dense_rounds", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("support", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("t1", ctypes.c_int32), ("t2", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("hub_degree", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("rounds_per_step", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("n_eps", ctypes.c_int32), ("eps", ctypes.c_double * 4), ("mem_budget_bytes", ctypes.c_int64),
                ("defer_volume", ctypes.c_int64)]


class ServerResult(ctypes.Structure):
    _fields_ = [("qid", ctypes.c_uint64), ("status", ctypes.c_int32), ("update", ctypes.c_int32),
                ("k", ctypes.c_int32), ("slot", ctypes.c_int32), ("volume", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("ids", ctypes.c_int32 * 64), ("vals", ctypes.c_float * 64)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("running", ctypes.c_int32), ("answered", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("steps", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("edge_batches", ctypes.c_int64), ("cap", ctypes.c_int64), ("volume", ctypes.c_int64),
                ("t_graph", ctypes.c_double), ("t_correct", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_rounds", ctypes.c_double), ("t_results", ctypes.c_double), ("pool_pages", ctypes.c_int64),
                ("pages_used", ctypes.c_int64), ("page_slots", ctypes.c_int64), ("peak_resident", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("readmissions", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("peak_pages", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libgde.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise ImportError(f"CUDA library {p} is missing: run paper_2410_21634_gb300._build.build()")
    lib = ctypes.CDLL(p)
    vp, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.gde_solve_opts_init.argtypes = [ctypes.POINTER(SolveOpts)]
    lib.gde_solve_opts_init.restype = None
    lib.gde_graph_create.argtypes = [I64, vp, vp, ctypes.c_uint32, ctypes.POINTER(vp)]
    lib.gde_graph_destroy.argtypes = [vp]
    lib.gde_graph_info.argtypes = [vp, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32)]
    lib.gde_solve.argtypes = [vp, ctypes.c_int, D, D, vp, I32, ctypes.POINTER(SolveOpts), vp, vp, vp]
    lib.gde_last_error.argtypes = []
    lib.gde_last_error.restype = ctypes.c_char_p
    lib.gde_session_begin.argtypes = [vp, ctypes.c_int, D, D, I32, ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(vp)]
    lib.gde_session_step.argtypes = [vp, ctypes.POINTER(I64)]
    lib.gde_session_read.argtypes = [vp, vp, vp, vp, ctypes.POINTER(I64)]
    lib.gde_session_end.argtypes = [vp]
    lib.gde_bsession_begin.argtypes = [vp, ctypes.c_int, D, D, vp, I32, ctypes.POINTER(SolveOpts),
                                       ctypes.POINTER(vp)]
    lib.gde_bsession_step.argtypes = [vp, ctypes.POINTER(I64)]
    lib.gde_bsession_read.argtypes = [vp, I32, vp, vp, vp, ctypes.POINTER(I64)]
    lib.gde_bsession_end.argtypes = [vp]
    for name in ("gde_bsession_begin", "gde_bsession_step", "gde_bsession_read", "gde_bsession_end"):
        getattr(lib, name).restype = ctypes.c_int
    lib.gde_test_fail_alloc.argtypes = [I64]
    lib.gde_test_fail_alloc.restype = ctypes.c_int
    lib.gde_test_barrier_fault.argtypes = [vp, I64, I32, I32]
    lib.gde_test_barrier_fault.restype = ctypes.c_int
    lib.gde_topk_f32_noalloc.argtypes = [vp, I64, I32, vp, vp, vp]
    lib.gde_topk_f32_noalloc.restype = ctypes.c_int
    lib.gde_profile_rounds.argtypes = [vp, vp, I64, ctypes.POINTER(I64)]
    lib.gde_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.gde_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.gde_autotune.argtypes = [vp, ctypes.c_int, D, D, vp, I32, ctypes.POINTER(SolveOpts),
                                 ctypes.POINTER(Tuning), ctypes.POINTER(D)]
    lib.gde_update_edges.argtypes = [vp, vp, vp, I64, ctypes.c_uint32, ctypes.POINTER(I64)]
    lib.gde_graph_csr.argtypes = [vp, vp, vp, ctypes.c_uint32]
    lib.gde_server_opts_init.argtypes = [ctypes.POINTER(ServerOpts)]
    lib.gde_server_opts_init.restype = None
    lib.gde_server_clock.argtypes = []
    lib.gde_server_clock.restype = D
    lib.gde_server_create.argtypes = [vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.gde_server_destroy.argtypes = [vp]
    lib.gde_server_submit.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, D, I32, I32, ctypes.c_uint32, D]
    lib.gde_server_insert_edges.argtypes = [vp, vp, vp, I64]
    lib.gde_server_step.argtypes = [vp, ctypes.POINTER(I32), ctypes.POINTER(I32)]
    lib.gde_server_poll.argtypes = [vp, ctypes.POINTER(ServerResult), I32, ctypes.POINTER(I32)]
    lib.gde_server_info.argtypes = [vp, ctypes.POINTER(ServerInfo)]
    lib.gde_probe_random_access.argtypes = [vp, ctypes.c_uint64, I64, I32, I32, I32, I32, vp, ctypes.POINTER(D)]
    lib.gde_probe_random_access.restype = ctypes.c_int
    for name in ("gde_server_create", "gde_server_destroy", "gde_server_submit", "gde_server_insert_edges",
                 "gde_server_step", "gde_server_poll", "gde_server_info"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("gde_profile_rounds", "gde_set_tuning", "gde_get_tuning", "gde_autotune",
                 "gde_update_edges", "gde_graph_csr"):
        getattr(lib, name).restype = ctypes.c_int
    lib.gde_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.gde_profile_read.argtypes = [vp, ctypes.POINTER(Profile)]
    for name in ("gde_graph_create", "gde_graph_destroy", "gde_graph_info", "gde_solve",
                 "gde_session_begin", "gde_session_step", "gde_session_read", "gde_session_end",
                 "gde_profile_enable", "gde_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def last_error() -> str:
    return load().gde_last_error().decode()


def _check(st: int):
    if st != OK:
        raise GdeError(st, last_error())


def _kind(kind) -> int:
    return KINDS[kind] if isinstance(kind, str) else int(kind)


def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _ptr(a):
    """(pointer, is_device) of a numpy array or a CUDA tensor (must be contiguous)."""
    if a is None:
        return None, False
    if _is_cuda_tensor(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), True
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous numpy array or a CUDA tensor")
    return a.ctypes.data, False


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def make_opts(precision=FP64, topk=0, hk_threshold=0, batched=0, deterministic=0, flags=0,
              max_rounds=0, mem_budget_bytes=0, hk_tol=0.0, stream=None, prop_beta=0.0,
              series_coef=None, global_gd=0, chebyshev=0, katz_minus_source=0) -> SolveOpts:
    o = SolveOpts()
    load().gde_solve_opts_init(ctypes.byref(o))
    o.precision = FP32 if precision in (FP32, "fp32", "float32") else FP64
    o.topk, o.hk_threshold, o.batched, o.deterministic = topk, hk_threshold, batched, deterministic
    o.flags, o.max_rounds, o.mem_budget_bytes, o.hk_tol = flags, max_rounds, mem_budget_bytes, hk_tol
    o.cuda_stream = stream
    o.prop_beta = float(prop_beta)
    o.global_gd = int(global_gd)
    o.chebyshev = int(chebyshev)
    o.katz_minus_source = int(katz_minus_source)
    if series_coef is not None:
        c = np.ascontiguousarray(series_coef, dtype=np.float64)
        o._series = c  # kept alive with the options
        o.series_coef = c.ctypes.data
        o.series_terms = int(c.shape[0])
    return o


class Graph:
    """A CSR graph resident in HBM (gde_graph_create / gde_graph_destroy)."""

    def __init__(self, n: int, offsets, cols, check_symmetric: bool = False):
        lib = load()
        po, do = _ptr(offsets)
        pc, dc = _ptr(cols)
        if do != dc:
            raise ValueError("offsets and cols must both be host arrays or both CUDA tensors")
        flags = (DEVICE_PTRS if do else 0) | (CHECK_SYMMETRIC if check_symmetric else 0)
        h = ctypes.c_void_p()
        _check(lib.gde_graph_create(int(n), po, pc, flags, ctypes.byref(h)))
        self._h = h
        self.n = int(n)

    @classmethod
    def from_synth(cls, g, **kw):
        return cls(g.n, np.ascontiguousarray(g.offsets, dtype=np.int64),
                   np.ascontiguousarray(g.cols, dtype=np.int32), **kw)

    @property
    def handle(self):
        return self._h

    def info(self):
        n, nnz, md = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(load().gde_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md)))
        return {"n": n.value, "nnz": nnz.value, "max_degree": md.value}

    def update_edges(self, src, dst) -> int:
        """gde_update_edges: insert the undirected edges (src[i], dst[i]); returns the number
        of directed adjacencies added."""
        ps, ds = _ptr(src)
        pd, dd = _ptr(dst)
        if ds != dd or src.shape != dst.shape:
            raise ValueError("src and dst must be alike (both host or both device, same length)")
        added = ctypes.c_int64()
        _check(load().gde_update_edges(self._h, ps, pd, int(src.shape[0]), DEVICE_PTRS if ds else 0,
                                       ctypes.byref(added)))
        return added.value

    def csr(self):
        """gde_graph_csr: (offsets int64 [n+1], cols int32 [nnz]) of the current graph."""
        inf = self.info()
        off = np.zeros(inf["n"] + 1, dtype=np.int64)
        cols = np.zeros(max(inf["nnz"], 1), dtype=np.int32)
        _check(load().gde_graph_csr(self._h, off.ctypes.data, cols.ctypes.data, 0))
        return off, cols[: inf["nnz"]]

    def profile_enable(self, enable: bool = True):
        _check(load().gde_profile_enable(self._h, int(enable)))

    def profile_read(self) -> dict:
        p = Profile()
        _check(load().gde_profile_read(self._h, ctypes.byref(p)))
        return p.as_dict()

    def profile_rounds(self, cap: int = 4096):
        """per-round rows (candidates, volume, ||r_S||_1, ns at round end, ns at frontier end,
        scatter busy ns summed over warps, longest warp ns) of the last batched solve"""
        buf = np.zeros((cap, 7), dtype=np.float64)
        r = ctypes.c_int64()
        _check(load().gde_profile_rounds(self._h, buf.ctypes.data, cap, ctypes.byref(r)))
        return buf[: min(r.value, cap)].copy()

    def set_tuning(self, t1=0, t2=0, chunk=0, blocks_per_sm=0, schedule=0, hub_degree=0):
        t = Tuning(t1, t2, chunk, blocks_per_sm, schedule, hub_degree)
        _check(load().gde_set_tuning(self._h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(load().gde_get_tuning(self._h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def autotune(self, kind, param: float, eps: float, seeds, **opt_kw):
        """gde_autotune on this graph; returns (tuning dict, best ms)."""
        ps, ds = _ptr(seeds)
        flags = opt_kw.pop("flags", 0) | (DEVICE_PTRS if ds else 0)
        if ds and "stream" not in opt_kw:
            opt_kw["stream"] = _current_stream()
        opt_kw.setdefault("topk", 64)
        o = make_opts(flags=flags, precision=FP32, batched=1, **opt_kw)
        t = Tuning()
        ms = ctypes.c_double()
        _check(load().gde_autotune(self._h, _kind(kind), float(param), float(eps), ps, int(seeds.shape[0]),
                                   ctypes.byref(o), ctypes.byref(t), ctypes.byref(ms)))
        return {f: getattr(t, f) for f, _ in t._fields_}, ms.value

    def test_barrier_fault(self, limit_ns: int = 0, block: int = -1, barrier: int = 0):
        """gde_test_barrier_fault: bounded grid-barrier waits of limit_ns and a block that leaves
        at one barrier (tests only; block < 0 turns it off)."""
        _check(load().gde_test_barrier_fault(self._h, int(limit_ns), int(block), int(barrier)))

    def close(self):
        if getattr(self, "_h", None):
            load().gde_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve(graph: Graph, kind, param: float, eps: float, seeds, out_x, out_ids=None,
          stats: bool = True, **opt_kw):
    """gde_solve.  seeds/out_x/out_ids: numpy arrays (host) or CUDA tensors (device).
    Returns (status, per-seed stats: a sequence of dicts, StatsList)."""
    lib = load()
    ps, ds = _ptr(seeds)
    px, dx = _ptr(out_x)
    pi, di = _ptr(out_ids)
    if ds != dx or (out_ids is not None and di != dx):
        raise ValueError("seeds and outputs must all be host arrays or all CUDA tensors")
    nseeds = int(seeds.shape[0])
    flags = opt_kw.pop("flags", 0) | (DEVICE_PTRS if dx else 0)
    if dx and "stream" not in opt_kw:
        opt_kw["stream"] = _current_stream()
    o = make_opts(flags=flags, **opt_kw)
    st_arr = (Stats * max(nseeds, 1))() if stats else None
    st = lib.gde_solve(graph.handle, _kind(kind), float(param), float(eps), ps, nseeds,
                       ctypes.byref(o), px, pi, ctypes.cast(st_arr, ctypes.c_void_p) if stats else None)
    if st not in (OK, ENOTCONV):
        _check(st)
    return st, (StatsList(st_arr, nseeds) if stats else [])


def _check_topk_noalloc_args(x, k, out_ids, out_vals):
    """The checks the C entry point cannot make (it sees only pointers): tensor kinds, dtypes,
    output sizes and one common device.  Raises ValueError."""
    for name, a in (("x", x), ("out_ids", out_ids), ("out_vals", out_vals)):
        if not _is_cuda_tensor(a):
            raise ValueError(f"topk_noalloc: {name} must be a CUDA tensor")
        if not a.is_contiguous():
            raise ValueError(f"topk_noalloc: {name} must be contiguous")
    if str(x.dtype) != "torch.float32" or str(out_vals.dtype) != "torch.float32":
        raise ValueError("topk_noalloc: x and out_vals must be float32")
    if str(out_ids.dtype) != "torch.int32":
        raise ValueError("topk_noalloc: out_ids must be int32")
    k = int(k)
    if out_ids.numel() < k or out_vals.numel() < k:
        raise ValueError(f"topk_noalloc: out_ids and out_vals need at least k = {k} elements")
    if not (x.device == out_ids.device == out_vals.device):
        raise ValueError("topk_noalloc: x, out_ids and out_vals must be on one device")


def topk_noalloc(x, k: int, out_ids, out_vals, stream=None):
    """gde_topk_f32_noalloc: top-k of a dense float CUDA vector without device allocation.
    x (float32), out_ids (int32, >= k elements) and out_vals (float32, >= k elements) must be
    contiguous CUDA tensors on one device; the call runs with that device current and is
    asynchronous on `stream` (default: that device's current torch stream)."""
    _check_topk_noalloc_args(x, k, out_ids, out_vals)
    import torch
    with torch.cuda.device(x.device):
        if stream is None:
            stream = torch.cuda.current_stream(x.device).cuda_stream
        _check(load().gde_topk_f32_noalloc(_ptr(x)[0], int(x.numel()), int(k), _ptr(out_ids)[0],
                                           _ptr(out_vals)[0], stream))


def test_fail_alloc(nth: int):
    """gde_test_fail_alloc: the nth device allocation from now fails with GDE_ENOMEM (0 disarms;
    tests only)."""
    _check(load().gde_test_fail_alloc(int(nth)))


PROBE_MODES = {"load": 0, "load_atomic": 1, "atomic": 2, "red": 3, "atomic64": 4, "red64": 5}


def probe_random_access(buf, nops: int, mode="load_atomic", grid: int = 152 * 8, reps: int = 3,
                        l2_fetch_bytes: int = 0, stream=None) -> float:
    """gde_probe_random_access: mean ms of one launch of `nops` random 32-byte sector accesses
    over the contiguous CUDA tensor `buf` (its contents are overwritten).  mode: "load",
    "load_atomic", "atomic", "red", "atomic64" or "red64" (or 0 .. 5)."""
    if not _is_cuda_tensor(buf):
        raise ValueError("probe_random_access takes a CUDA tensor")
    m = PROBE_MODES.get(mode, mode)
    if stream is None:
        stream = _current_stream()
    ms = ctypes.c_double()
    _check(load().gde_probe_random_access(_ptr(buf)[0], int(buf.numel() * buf.element_size()), int(nops), int(m),
                                          int(grid), int(reps), int(l2_fetch_bytes), stream, ctypes.byref(ms)))
    return ms.value


class Session:
    """Stepping interface: one LocalGD round per step() (gde_session_*)."""

    def __init__(self, graph: Graph, kind, param: float, eps: float, seed: int, **opt_kw):
        lib = load()
        self.graph = graph
        self.precision = FP32 if opt_kw.get("precision", FP64) in (FP32, "fp32") else FP64
        o = make_opts(**opt_kw)
        h = ctypes.c_void_p()
        _check(lib.gde_session_begin(graph.handle, _kind(kind), float(param), float(eps), int(seed),
                                     ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def step(self) -> int:
        k = ctypes.c_int64()
        _check(load().gde_session_step(self._h, ctypes.byref(k)))
        return k.value

    def read(self):
        """(x, r, active S_t of the last step (unordered)) as host numpy arrays."""
        n = self.graph.n
        dt = np.float64 if self.precision == FP64 else np.float32
        x = np.empty(n, dtype=dt)
        r = np.empty(n, dtype=dt)
        act = np.empty(max(n, 1), dtype=np.int32)
        k = ctypes.c_int64()
        _check(load().gde_session_read(self._h, x.ctypes.data, r.ctypes.data, act.ctypes.data,
                                       ctypes.byref(k)))
        return x, r, act[:k.value].copy()

    def close(self):
        if getattr(self, "_h", None):
            load().gde_session_end(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSession:
    """Batched stepping interface (gde_bsession_*): one round of the batched engine per step()
    for every seed of the batch, with each seed's state readable between rounds."""

    def __init__(self, graph: Graph, kind, param: float, eps: float, seeds, **opt_kw):
        lib = load()
        self.graph = graph
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
        if seeds.ndim != 1 or seeds.shape[0] < 1:
            raise ValueError("seeds must be a non-empty 1-d array")
        self.nseeds = int(seeds.shape[0])
        opt_kw.setdefault("precision", FP32)
        o = make_opts(**opt_kw)
        h = ctypes.c_void_p()
        _check(lib.gde_bsession_begin(graph.handle, _kind(kind), float(param), float(eps), seeds.ctypes.data,
                                      self.nseeds, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def step(self) -> int:
        """Runs the next round of every seed; returns the candidates of the round after it."""
        k = ctypes.c_int64()
        _check(load().gde_bsession_step(self._h, ctypes.byref(k)))
        return k.value

    def read(self, j: int):
        """(x float32, r float64, nodes pushed by the last step int32) of seed index j."""
        n = self.graph.n
        x = np.empty(n, dtype=np.float32)
        r = np.empty(n, dtype=np.float64)
        pushed = np.empty(max(n, 1), dtype=np.int32)
        k = ctypes.c_int64()
        _check(load().gde_bsession_read(self._h, int(j), x.ctypes.data, r.ctypes.data, pushed.ctypes.data,
                                        ctypes.byref(k)))
        return x, r, np.sort(pushed[:k.value])

    def close(self):
        if getattr(self, "_h", None):
            load().gde_bsession_end(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_clock() -> float:
    """The steady clock (seconds) that server timestamps use."""
    return float(load().gde_server_clock())


class Server:
    """Continuous-batching server of PPR/Katz queries on a graph with edge insertions
    (gde_server_*).  submit() and insert_edges() queue work; step() runs one device step;
    poll() returns the results emitted so far as dicts."""

    def __init__(self, graph: Graph, slots: int = 256, rounds_per_step: int = 4, topk: int = 64,
                 eps=(1e-6,), mem_budget_bytes: int = 0, defer_volume: int = 0):
        lib = load()
        o = ServerOpts()
        lib.gde_server_opts_init(ctypes.byref(o))
        o.slots, o.rounds_per_step, o.topk = int(slots), int(rounds_per_step), int(topk)
        eps = list(eps)
        if not 1 <= len(eps) <= 4:
            raise ValueError("1 to 4 tolerance classes")
        o.n_eps = len(eps)
        for i, e in enumerate(eps):
            o.eps[i] = float(e)
        o.mem_budget_bytes = int(mem_budget_bytes)
        o.defer_volume = int(defer_volume)
        h = ctypes.c_void_p()
        _check(lib.gde_server_create(graph.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.graph = graph
        self.topk = int(topk)

    def submit(self, qid: int, kind, param: float, eps_class: int, seed: int, track: bool = False,
               t_submit: float = -1.0):
        """Queue a query; track=True keeps it as a standing query (updated after edge batches)."""
        _check(load().gde_server_submit(self._h, int(qid), _kind(kind), float(param), int(eps_class),
                                        int(seed), SERVE_TRACK if track else 0, float(t_submit)))

    def insert_edges(self, src, dst):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if src.shape != dst.shape:
            raise ValueError("src and dst differ in length")
        _check(load().gde_server_insert_edges(self._h, src.ctypes.data, dst.ctypes.data, int(src.shape[0])))

    def step(self):
        """One device step; returns (queries still running, queries still queued)."""
        r, q = ctypes.c_int32(), ctypes.c_int32()
        _check(load().gde_server_step(self._h, ctypes.byref(r), ctypes.byref(q)))
        return r.value, q.value

    def poll(self, cap: int = 4096):
        buf = (ServerResult * cap)()
        n = ctypes.c_int32()
        _check(load().gde_server_poll(self._h, buf, cap, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            k = r.k
            out.append({"qid": r.qid, "status": r.status, "update": bool(r.update), "slot": r.slot,
                        "volume": r.volume, "t_submit": r.t_submit, "t_done": r.t_done,
                        "ids": np.frombuffer(r.ids, dtype=np.int32, count=k).copy(),
                        "vals": np.frombuffer(r.vals, dtype=np.float32, count=k).copy()})
        return out

    def info(self) -> dict:
        i = ServerInfo()
        _check(load().gde_server_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def run_until_idle(self, max_steps: int = 100000):
        """step() until nothing runs or waits; returns the results emitted meanwhile."""
        out = []
        for _ in range(max_steps):
            running, queued = self.step()
            out += self.poll()
            if running == 0 and queued == 0:
                break
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().gde_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
