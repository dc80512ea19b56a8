"""ORACLE — test infrastructure only.

Dynamic graphs (Section 4, discrete-time snapshots G_0 -> G_1 -> ... with edge-insertion
events, and the Insert procedure of Algorithm 3, LocalGS(Dynamic)): after an edge event the local solver's
state (x, r) is corrected so that the linear-system invariant holds on the new graph, and
LocalGD then continues from the corrected state instead of starting again from e_s.

Unit-mass convention (the rest of the oracle): PPR keeps r = e_s - Q x / alpha with
Q = I - (1 - alpha) A D^-1, Katz keeps r = e_s - (I - beta A) x.

PPR, one new directed adjacency u -> v (column u of A D^-1 gains v; d = the new degree of u):
Algorithm 3's Insert rescales x_u by d / (d - 1), then moves x_u / (alpha d) out of r_u and
(1 - alpha) x_u / (alpha d) into r_v (its p is x / alpha here).  If u had degree 0 its
column was zero (isolated nodes scatter nothing), so x_u stays and r_v gains
(1 - alpha) x_u / alpha.  Katz (derived from its invariant): A gains e_v e_u^T, so r_v
gains beta x_u.  An undirected edge is the two directed adjacencies u -> v, then v -> u.
Residuals may become negative; LocalGD's active test |r_u| >= eps d_u already covers that.

Plain Python loops over the events (batches here are small); every product and quotient is
one binary64 operation in the written order.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from . import KATZ, PPR, _kind, localgd_round


def _csr(n: int, rows: np.ndarray, cols: np.ndarray):
    """CSR with sorted, unique columns per row from directed (row, col) pairs."""
    key = np.unique(rows.astype(np.int64) * n + cols.astype(np.int64))
    r = (key // n).astype(np.int64)
    c = (key % n).astype(np.int32)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, r + 1, 1)
    np.cumsum(off, out=off)
    g = SimpleNamespace(n=n, offsets=off, cols=np.ascontiguousarray(c))
    g.degrees = lambda: np.diff(g.offsets)
    g.nnz = int(off[-1])
    return g


def insert_edges(g, kind, param: float, x: np.ndarray, r: np.ndarray, src, dst):
    """Insert the undirected edges (src[i], dst[i]) in order, correcting (x, r) in place
    after each directed adjacency.  Self-loops and edges already present (in g or earlier in
    the batch) are skipped, so the graph stays simple.  Returns (new graph, number of
    edges inserted)."""
    k = _kind(kind)
    if k not in (PPR, KATZ):
        raise ValueError("edge insertion is defined for PPR and Katz")
    n = g.n
    deg = np.diff(g.offsets).astype(np.int64)
    added = set()

    def present(u, v):
        lo, hi = int(g.offsets[u]), int(g.offsets[u + 1])
        i = lo + int(np.searchsorted(g.cols[lo:hi], v))
        return (i < hi and int(g.cols[i]) == v) or (u, v) in added

    new_rows, new_cols = [], []
    inserted = 0
    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if not (0 <= a < n and 0 <= b < n):
            raise ValueError(f"edge ({a}, {b}) out of range")
        if a == b or present(a, b):
            continue
        for u, v in ((a, b), (b, a)):
            d_old = deg[u]
            d = d_old + 1
            if k == PPR:
                alpha = param
                if d_old == 0:
                    r[v] = r[v] + ((1.0 - alpha) * x[u]) / alpha
                else:
                    x[u] = (x[u] * float(d)) / float(d_old)
                    share = x[u] / (alpha * float(d))
                    r[u] = r[u] - share
                    r[v] = r[v] + (1.0 - alpha) * share
            else:
                r[v] = r[v] + param * x[u]
            deg[u] = d
            added.add((u, v))
            new_rows.append(u)
            new_cols.append(v)
        inserted += 1
    rows = np.concatenate([np.repeat(np.arange(n, dtype=np.int64), np.diff(g.offsets)),
                           np.asarray(new_rows, dtype=np.int64)])
    cols = np.concatenate([g.cols.astype(np.int64), np.asarray(new_cols, dtype=np.int64)])
    return _csr(n, rows, cols), inserted


def localgd_from(g, kind, param: float, eps: float, x: np.ndarray, r: np.ndarray,
                 max_rounds: int = 1_000_000):
    """LocalGD rounds (Eq. local-gd) from the given state until the active set is empty,
    in place.  Returns (rounds, pushed volume)."""
    rounds = vol = 0
    while rounds < max_rounds:
        rr = localgd_round(g, kind, param, eps, x, r)
        if rr.n_active == 0:
            break
        rounds += 1
        vol += rr.vol_active
    return rounds, vol
