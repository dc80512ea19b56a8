"""Synthetic inputs: CSR well-formedness, symmetry, determinism, sizes."""
import numpy as np
import pytest

import synth


def check_simple_undirected(g):
    off, col = g.offsets, g.cols
    assert off[0] == 0 and off[-1] == col.shape[0]
    assert np.all(np.diff(off) >= 0)
    if g.nnz == 0:
        return
    assert col.min() >= 0 and col.max() < g.n
    rows = np.repeat(np.arange(g.n), np.diff(off))
    assert not np.any(rows == col), "self-loop"
    # strictly increasing within each row
    inner = np.diff(col.astype(np.int64))
    same_row = rows[1:] == rows[:-1]
    assert np.all(inner[same_row] > 0), "row not sorted/unique"
    # symmetric: the multiset of (u,v) equals that of (v,u)
    fwd = rows.astype(np.int64) * g.n + col
    bwd = col.astype(np.int64) * g.n + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))


@pytest.mark.parametrize("maker", [
    lambda: synth.chung_lu(3000, 10.0, 2.5, seed=11),
    lambda: synth.rmat(12, 16, seed=5),
    lambda: synth.star(7),
    lambda: synth.path(9),
    lambda: synth.cycle(6),
    lambda: synth.complete(5),
    lambda: synth.erdos_renyi(50, 0.1, 3),
    lambda: synth.with_isolated(synth.cycle(5), 3),
])
def test_csr_simple_undirected(maker):
    check_simple_undirected(maker())


def test_deterministic():
    a = synth.rmat(14, 16, seed=9)
    b = synth.rmat(14, 16, seed=9)
    c = synth.rmat(14, 16, seed=10)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    assert not (a.nnz == c.nnz and np.array_equal(a.cols, c.cols))


def test_chung_lu_sizes_and_tail():
    g = synth.workload_graph("chung_lu_1e4")
    s = g.summary()
    assert s["n"] == 10_000
    # n*d/2 pairs, minus self-loops and duplicates, both directions
    assert 0.9 * 100_000 < s["nnz"] <= 100_000
    d = g.degrees()
    assert d.max() > 20 * np.median(d[d > 0])  # heavy tail


def test_rmat_isolated_and_skew():
    g = synth.rmat(14, 16, seed=2)
    d = g.degrees()
    assert (d == 0).sum() > 0 and d.max() > 50 * d[d > 0].mean() / 10


def test_seed_pickers():
    g = synth.rmat(12, 16, seed=3)
    d = g.degrees()
    q = synth.seeds_quantile(g, 64)
    assert q.shape == (64,) and np.all(d[q] > 0)
    assert np.all(np.diff(d[q]) >= 0)  # ascending degree quantiles
    m = synth.seeds_mixed(g, 16, 16, seed=1)
    thr = np.sort(d)[::-1][int(np.ceil(0.01 * g.n)) - 1]
    assert np.all(d[m[:16]] > 0) and np.all(d[m[16:]] >= thr)
    b = synth.seeds_by_degree(g, 1000, seed=1)
    assert np.all(d[b] > 0) and d[b].mean() > d[d > 0].mean()  # size-biased


def test_lambda_max_matches_eigvalsh():
    g = synth.erdos_renyi(120, 0.08, 4)
    from oracle import dense  # dense adjacency builder only
    lam_ref = np.linalg.eigvalsh(dense.adjacency(g))[-1]
    lam, it = synth.lambda_max(g)
    assert abs(lam - lam_ref) <= 1e-9 * lam_ref and it >= 2
