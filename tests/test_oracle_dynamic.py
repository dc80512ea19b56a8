"""Pins of the dynamic-graph oracle (Section 4; Insert of Algorithm 3 in unit-mass form,
Katz derived from its invariant) against what the linear systems fix:

* after any insertion batch the corrected state satisfies the new graph's invariant
  (PPR: Q' x / alpha + r = e_s with Q' = I - (1-alpha) A' D'^-1; Katz: (I - beta A') x + r
  = e_s), checked with dense matrices built from the new adjacency;
* LocalGD warm-started from the corrected state ends inside the eps bound of the dense
  solution on the new graph (|f' - x| <= eps d' entrywise for PPR, two-sided because
  residuals may be negative);
* a batch's corrections do not depend on the order of its edges (what lets the device
  apply a whole batch at once);
* hand-computed cases: an isolated seed gaining an edge, and self-loops / duplicates skipped.
"""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
from oracle import dynamic
import synth


def state_after_solve(g, kind, param, eps, s):
    x = np.zeros(g.n)
    r = np.zeros(g.n)
    r[s] = 1.0
    dynamic.localgd_from(g, kind, param, eps, x, r)
    return x, r


def invariant_residual(g, kind, param, x, r, s):
    """max |e_s - (system x + r)| on graph g (dense)"""
    e = dense.unit(g.n, s)
    if kind == "ppr":
        lhs = dense.ppr_system(g, param) @ x / param + r
    else:
        lhs = dense.katz_system(g, param) @ x + r
    return float(np.max(np.abs(e - lhs)))


@pytest.fixture(scope="module")
def g0():
    # Erdos-Renyi core plus isolated nodes (so insertions can touch degree-0 nodes)
    return synth.with_isolated(synth.erdos_renyi(120, 0.05, seed=7), 6)


def katz_beta(g):
    return 0.5 / synth.lambda_max(g)[0]


@pytest.mark.parametrize("kind", ["ppr", "katz"])
def test_invariant_holds_after_insertion(g0, kind):
    param = 0.15 if kind == "ppr" else katz_beta(g0)
    s = int(np.argmax(g0.degrees()))
    x, r = state_after_solve(g0, kind, param, 1e-4, s)
    assert invariant_residual(g0, kind, param, x, r, s) < 1e-12
    src, dst = synth.random_edges(g0.n, 40, seed=3)
    src = np.concatenate([src, [s, 121, 122, 5, 7]])   # a seed edge, an isolated pair,
    dst = np.concatenate([dst, [123, 122, 5, 5, 7]])   # a self-loop, a repeat
    g1, m = dynamic.insert_edges(g0, kind, param, x, r, src, dst)
    assert g1.nnz > g0.nnz
    ref = synth.with_edges(g0, src, dst)
    assert np.array_equal(g1.offsets, ref.offsets) and np.array_equal(g1.cols, ref.cols)
    assert m == (ref.nnz - g0.nnz) // 2
    assert invariant_residual(g1, kind, param, x, r, s) < 1e-12
    # and the old graph's invariant is now violated (the correction is not a no-op)
    assert invariant_residual(g0, kind, param, x, r, s) > 1e-6


def test_planted_mistake_breaks_the_invariant(g0):
    """The invariant pin is sensitive: a correction computed with the old degree of u
    (a plausible slip in Insert) leaves a residual error far above rounding."""
    alpha = 0.15
    s = int(np.argmax(g0.degrees()))
    x, r = state_after_solve(g0, "ppr", alpha, 1e-5, s)
    u = s
    v = int(np.nonzero(g0.degrees() == 0)[0][0])
    d = int(g0.degrees()[u])
    x2, r2 = x.copy(), r.copy()
    g1, _ = dynamic.insert_edges(g0, "ppr", alpha, x2, r2, [u], [v])
    assert invariant_residual(g1, "ppr", alpha, x2, r2, s) < 1e-12
    # the slip: share from the old degree d instead of d + 1 on the u -> v direction
    x3, r3 = x2.copy(), r2.copy()
    wrong = x3[u] / (alpha * d) - x3[u] / (alpha * (d + 1))
    r3[u] -= wrong
    r3[v] += (1 - alpha) * wrong
    assert invariant_residual(g1, "ppr", alpha, x3, r3, s) > 1e-6


@pytest.mark.parametrize("kind", ["ppr", "katz"])
def test_warm_start_meets_the_bound(g0, kind):
    param = 0.15 if kind == "ppr" else katz_beta(g0)
    eps = 1e-6
    s = int(synth.seeds_quantile(g0, 8)[6])
    x, r = state_after_solve(g0, kind, param, eps, s)
    src, dst = synth.random_edges(g0.n, 60, seed=11)
    g1, _ = dynamic.insert_edges(g0, kind, param, x, r, src, dst)
    assert (r < 0).any() or kind == "katz"  # PPR corrections create negative residuals
    rounds, vol = dynamic.localgd_from(g1, kind, param, eps, x, r)
    d1 = g1.degrees().astype(float)
    assert np.all(np.abs(r) < eps * d1 + (d1 == 0))  # converged: every |r_u| < eps d_u
    if kind == "ppr":
        f1 = dense.ppr(g1, param, s)
        assert np.all(np.abs(f1 - x) <= eps * d1 + 1e-14)
        # and the result agrees with a fresh solve on the new graph within the same band
        fresh = oracle.localgd(g1, "ppr", param, eps, s).x
        assert np.all(np.abs(fresh - x) <= 2 * eps * d1 + 1e-14)
    else:
        f1 = dense.katz(g1, param, s)
        # Katz: x - f = (I - beta A')^-1 (-r); bounded through the exact inverse
        err = np.linalg.solve(dense.katz_system(g1, param), r)
        assert np.allclose(f1 - x, err, atol=1e-12)
        fresh = oracle.localgd(g1, "katz", param, eps, s).x
        assert np.max(np.abs(fresh - f1)) < 1e-3 and np.max(np.abs(x - f1)) < 1e-3


@pytest.mark.parametrize("kind", ["ppr", "katz"])
def test_batch_corrections_are_order_independent(g0, kind):
    param = 0.15 if kind == "ppr" else katz_beta(g0)
    s = int(np.argmax(g0.degrees()))
    x, r = state_after_solve(g0, kind, param, 1e-5, s)
    src, dst = synth.random_edges(g0.n, 80, seed=5)
    # several edges on the seed and on one node, so degrees change more than once per node
    src = np.concatenate([src, [s, s, s, 121, 121]])
    dst = np.concatenate([dst, [1, 2, 3, 4, 8]])
    xa, ra = x.copy(), r.copy()
    xb, rb = x.copy(), r.copy()
    ga, _ = dynamic.insert_edges(g0, kind, param, xa, ra, src, dst)
    gb, _ = dynamic.insert_edges(g0, kind, param, xb, rb, src[::-1], dst[::-1])
    assert np.array_equal(ga.cols, gb.cols)
    assert np.allclose(xa, xb, rtol=1e-13, atol=1e-16)
    assert np.allclose(ra, rb, rtol=1e-12, atol=1e-16)


def test_isolated_seed_gains_an_edge():
    """An isolated seed s: PPR has x_s = alpha, r = 0.  Inserting (s, v): the first
    adjacency s -> v (old degree 0) leaves x_s and adds (1-alpha) x_s / alpha = 1 - alpha to
    r_v; the second, v -> s, with v of old degree d_v, rescales x_v = 0 (no change)."""
    g = synth.with_isolated(synth.path(4), 2)  # nodes 4, 5 isolated
    alpha = 0.2
    x, r = state_after_solve(g, "ppr", alpha, 1e-3, 4)
    assert x[4] == alpha and not r.any()
    g1, m = dynamic.insert_edges(g, "ppr", alpha, x, r, [4], [1])
    assert m == 1 and x[4] == alpha
    assert r[1] == pytest.approx(1 - alpha, rel=1e-15) and r[4] == 0.0
    assert invariant_residual(g1, "ppr", alpha, x, r, 4) < 1e-12


def test_self_loops_and_duplicates_are_skipped():
    g = synth.path(5)
    x = np.zeros(5)
    r = np.zeros(5)
    r[0] = 1.0
    g1, m = dynamic.insert_edges(g, "ppr", 0.1, x, r, [0, 1, 2, 0, 3], [0, 2, 1, 4, 4])
    assert m == 1  # only (0, 4): (0,0) loop, (1,2) present, (2,1) present, (3,4) present
    assert g1.nnz == g.nnz + 2
