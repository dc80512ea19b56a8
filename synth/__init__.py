"""Seeded synthetic inputs shared by the oracle's tests and the CUDA path's tests/bench.

The paper evaluates on SNAP/OGB graphs (Section 5, Table 3) that are not available
here.  This module generates undirected, self-loop-free, heavy-tailed graphs of the
sizes the workloads name (Chung-Lu and R-MAT), picks seed nodes, and estimates the
largest adjacency eigenvalue used to set the Katz parameter.  It contains none of the
diffusion method's arithmetic: it only produces CSR arrays and seed lists.

The generator core is C (``gen.c``); this file compiles it on first use with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into _synth.so (gcc, OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            lib.synth_chung_lu_pairs.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_uint64, ctypes.c_int64, i32p, i32p]
            lib.synth_chung_lu_pairs.restype = ctypes.c_int
            lib.synth_rmat_pairs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                             i32p, i32p]
            lib.synth_rmat_pairs.restype = ctypes.c_int
            lib.synth_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, i32p]
            lib.synth_permutation.restype = ctypes.c_int
            lib.synth_relabel.argtypes = [ctypes.c_int64, i32p, i32p, i32p]
            lib.synth_relabel.restype = None
            lib.synth_csr_from_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p,
                                                 i64p, i32p]
            lib.synth_csr_from_pairs.restype = ctypes.c_int64
            lib.synth_lambda_max.argtypes = [ctypes.c_int64, i64p, i32p, ctypes.c_double,
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
            lib.synth_lambda_max.restype = ctypes.c_double
            lib.synth_num_threads.argtypes = []
            lib.synth_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected simple graph in CSR form (int64 row offsets, int32 sorted columns)."""

    n: int
    offsets: np.ndarray
    cols: np.ndarray
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)

    def summary(self) -> dict:
        d = self.degrees()
        return {"name": self.name, "n": int(self.n), "nnz": self.nnz,
                "mean_degree": float(d.mean()) if self.n else 0.0,
                "max_degree": int(d.max()) if self.n else 0,
                "isolated": int((d == 0).sum()), **self.info}


def from_pairs(n: int, src, dst, name: str = "", info: dict | None = None) -> Graph:
    """CSR of the undirected simple graph on n nodes with the given endpoint pairs
    (self-loops dropped, both directions added, duplicates removed, rows sorted)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    if n and m and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("endpoint out of range")
    offsets = np.zeros(n + 1, dtype=np.int64)
    cols = np.empty(max(2 * m, 1), dtype=np.int32)
    nnz = _load().synth_csr_from_pairs(n, m, src, dst, offsets, cols)
    if nnz < 0:
        raise MemoryError("synth_csr_from_pairs: allocation failed")
    return Graph(n, offsets, cols[:nnz].copy(), name, dict(info or {}))


def chung_lu(n: int, mean_deg: float, gamma: float, seed: int, permute: bool = True) -> Graph:
    """Chung-Lu graph: n*mean_deg/2 endpoint pairs drawn with probability proportional
    to w_i = (i+1)^(-1/(gamma-1)), then made simple and undirected, ids permuted."""
    lib = _load()
    m = int(round(n * mean_deg / 2.0))
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if lib.synth_chung_lu_pairs(n, float(mean_deg), float(gamma), seed, m, src, dst) != 0:
        raise MemoryError("synth_chung_lu_pairs: allocation failed")
    if permute:
        perm = np.empty(n, dtype=np.int32)
        lib.synth_permutation(n, seed, perm)
        lib.synth_relabel(m, perm, src, dst)
    return from_pairs(n, src, dst, name=f"chung_lu(n={n},d={mean_deg},gamma={gamma},seed={seed})",
                      info={"generator": "chung_lu", "pairs": m})


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, permute: bool = True) -> Graph:
    """R-MAT graph on 2^scale nodes with edge_factor*2^scale pairs, symmetrised,
    deduplicated, self-loops dropped, ids permuted."""
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.synth_rmat_pairs(scale, a, b, c, seed, m, src, dst)
    if permute:
        perm = np.empty(n, dtype=np.int32)
        lib.synth_permutation(n, seed, perm)
        lib.synth_relabel(m, perm, src, dst)
    return from_pairs(n, src, dst, name=f"rmat(scale={scale},ef={edge_factor},seed={seed})",
                      info={"generator": "rmat", "pairs": m, "abc": (a, b, c)})


def lambda_max(g: Graph, rel_tol: float = 1e-12, max_iter: int = 10000) -> tuple[float, int]:
    """Largest adjacency eigenvalue by power iteration on A + I (FP64).  Returns
    (lambda_max, iterations)."""
    it = ctypes.c_int64(0)
    lam = _load().synth_lambda_max(g.n, g.offsets, g.cols, rel_tol, max_iter, ctypes.byref(it))
    return float(lam), int(it.value)


def num_threads() -> int:
    return int(_load().synth_num_threads())


# ------------------------------------------------------------------ seeds ----

def seeds_by_degree(g: Graph, k: int, seed: int) -> np.ndarray:
    """k source nodes drawn with probability proportional to degree (a uniformly
    random CSR entry's column: the graph is symmetric, so columns appear d_v times)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.integers(0, g.nnz, size=k)
    return g.cols[idx].astype(np.int32)


def seeds_quantile(g: Graph, k: int) -> np.ndarray:
    """k sources spread over the degree distribution: non-isolated nodes sorted by
    (degree, id), the ((i + 1/2) n'/k)-th taken for i < k."""
    d = g.degrees()
    nz = np.nonzero(d > 0)[0]
    order = nz[np.lexsort((nz, d[nz]))]
    npr = order.shape[0]
    pos = ((np.arange(k) + 0.5) * npr / k).astype(np.int64)
    return order[pos].astype(np.int32)


def seeds_mixed(g: Graph, n_uniform: int, n_hub: int, seed: int, hub_frac: float = 0.01) -> np.ndarray:
    """n_uniform sources uniform over non-isolated nodes, then n_hub sources uniform
    over the top hub_frac of nodes by degree (ties by id)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = g.degrees()
    nz = np.nonzero(d > 0)[0]
    uni = rng.choice(nz, size=n_uniform, replace=n_uniform > nz.shape[0])
    ntop = max(1, int(np.ceil(hub_frac * g.n)))
    key = d.astype(np.int64) * (g.n + 1) + (g.n - np.arange(g.n, dtype=np.int64))
    top = np.argpartition(-key, min(ntop, g.n - 1))[:ntop]
    hubs = rng.choice(top, size=n_hub, replace=n_hub > top.shape[0])
    return np.concatenate([uni, hubs]).astype(np.int32)


# ------------------------------------------------------------ tiny graphs ----

def path(n: int) -> Graph:
    e = np.arange(n - 1)
    return from_pairs(n, e, e + 1, name=f"path({n})")


def cycle(n: int) -> Graph:
    e = np.arange(n)
    return from_pairs(n, e, (e + 1) % n, name=f"cycle({n})")


def star(k: int) -> Graph:
    """node 0 joined to leaves 1..k"""
    return from_pairs(k + 1, np.zeros(k, dtype=np.int32), np.arange(1, k + 1), name=f"star({k})")


def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return from_pairs(n, i, j, name=f"complete({n})")


def edge2() -> Graph:
    return from_pairs(2, [0], [1], name="edge2")


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    rng = np.random.Generator(np.random.PCG64(seed))
    i, j = np.triu_indices(n, 1)
    keep = rng.random(i.shape[0]) < p
    return from_pairs(n, i[keep], j[keep], name=f"er(n={n},p={p},seed={seed})")


def with_isolated(g: Graph, extra: int) -> Graph:
    """g plus `extra` isolated nodes appended at the end"""
    off = np.concatenate([g.offsets, np.full(extra, g.offsets[-1], dtype=np.int64)])
    return Graph(g.n + extra, off, g.cols.copy(), g.name + f"+{extra}iso", dict(g.info))


# ----------------------------------------------------- named workloads ----

WORKLOADS = {
    # PPR sanity case: Chung-Lu n=10^4, mean degree 10, exponent 2.5
    "chung_lu_1e4": dict(gen="chung_lu", n=10_000, mean_deg=10.0, gamma=2.5, seed=1),
    # single-seed FP64 form: R-MAT scale 22, edge factor 16
    "rmat22": dict(gen="rmat", scale=22, edge_factor=16, seed=2),
    # precision form: Chung-Lu n=2^24, mean degree 20, exponent 2.1
    "chung_lu_2p24": dict(gen="chung_lu", n=1 << 24, mean_deg=20.0, gamma=2.1, seed=3),
    # batched form: R-MAT scale 24, edge factor 16
    "rmat24": dict(gen="rmat", scale=24, edge_factor=16, seed=4),
    # a smaller graph of the same family (profiling captures, quick checks)
    "rmat20": dict(gen="rmat", scale=20, edge_factor=16, seed=4),
    # serving form: Chung-Lu n=2^23, mean degree 16, exponent 2.3
    "chung_lu_2p23": dict(gen="chung_lu", n=1 << 23, mean_deg=16.0, gamma=2.3, seed=5),
}


def workload_graph(name: str, **override) -> Graph:
    spec = dict(WORKLOADS[name])
    spec.update(override)
    gen = spec.pop("gen")
    if gen == "chung_lu":
        g = chung_lu(spec["n"], spec["mean_deg"], spec["gamma"], spec["seed"])
    else:
        g = rmat(spec["scale"], spec["edge_factor"], seed=spec["seed"])
    g.name = name
    return g


# ------------------------------------------------------------ dynamic graphs ----

def random_edges(n: int, m: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """m endpoint pairs drawn uniformly over the n nodes (an edge-insertion batch of the
    serving workload; self-loops and repeats are left in, the consumer skips them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.integers(0, n, size=m).astype(np.int32), rng.integers(0, n, size=m).astype(np.int32))


def with_edges(g: Graph, src, dst) -> Graph:
    """g plus the undirected edges (src[i], dst[i]) (self-loops and duplicates dropped)."""
    rows = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.offsets))
    return from_pairs(g.n, np.concatenate([rows, np.asarray(src, dtype=np.int32)]),
                      np.concatenate([g.cols, np.asarray(dst, dtype=np.int32)]), name=g.name, info=dict(g.info))


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds, ascending) of a Poisson stream of the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=int(rate_per_s * duration_s * 1.5) + 16)
    t = np.cumsum(gaps)
    return t[t < duration_s]
