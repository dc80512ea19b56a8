"""Batched FP32 LocalGD for the layered kinds (the heat kernel's Taylor layers and a general
series f = sum_k c_k (A D^-1)^k e_s): every seed of the batch in one persistent launch, layer t
pushed into layer t+1 with the per-layer threshold theta_t eps d_u, x in a per-seed table,
top-k out; against the FP64 oracle through the C ABI.

Both sides satisfy 0 <= f_u - x_u <= eps d_u (the layered bound of Section 3), so a top-k entry
is compared with the oracle's value within eps d_u plus 1e-5 relative (FP32), as for PPR."""
import math

import numpy as np
import pytest

import oracle
import synth
from test_gpu_batched import check_topk, run_batched
from test_gpu_series import ipr_coef

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def c1():
    return synth.workload_graph("chung_lu_1e4")


@pytest.fixture(scope="module")
def rmat16():
    return synth.rmat(16, 16, seed=21)


@pytest.mark.parametrize("hk_mode", [0, 1])
def test_batched_hk(gde, c1, rmat16, hk_mode):
    tau, eps = 5.0, 1e-6
    for g in (c1, rmat16):
        G = gde.Graph.from_synth(g)
        seeds = synth.seeds_mixed(g, 12, 12, seed=5)
        st, stats, ids, vals = run_batched(gde, G, "hk", tau, eps, seeds, hk_threshold=hk_mode)
        assert st == gde.OK and not any(s["fallback"] for s in stats)
        for i in range(0, len(seeds), 3):
            ref = oracle.localgd(g, "hk", tau, eps, int(seeds[i]), hk_mode=hk_mode)
            check_topk(g, ids[i], vals[i], ref.x, eps)
            assert stats[i]["rounds"] <= oracle.hk_terms(tau) + 1
            assert stats[i]["active_volume"] == pytest.approx(ref.volume, rel=0.02, abs=64)
        G.close()


def test_batched_series(gde, rmat16):
    g = rmat16
    c = ipr_coef(1.5)
    eps = 1e-3 * c[0]
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_mixed(g, 8, 8, seed=6)
    st, _, ids, vals = run_batched(gde, G, "series", 0.0, eps, seeds, series_coef=c)
    assert st == gde.OK
    for i in range(0, len(seeds), 3):
        ref = oracle.series(g, c, eps, int(seeds[i]))
        check_topk(g, ids[i], vals[i], ref.x, eps)
    G.close()


def test_hk_equals_its_series(gde, c1):
    """The heat kernel and the series of its Taylor coefficients take the same rounds on
    the batched engine, so their top-k lists agree within FP32 summation order."""
    g = c1
    tau = 5.0
    N = oracle.hk_terms(tau)
    c = [math.exp(-tau)]
    for k in range(N):
        c.append(c[-1] * tau / (k + 1))
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_quantile(g, 6)
    _, _, ids_a, vals_a = run_batched(gde, G, "hk", tau, 1e-6, seeds)
    _, _, ids_b, vals_b = run_batched(gde, G, "series", 0.0, 1e-6, seeds, series_coef=np.array(c))
    assert np.allclose(vals_a, vals_b, rtol=1e-5, atol=0)
    G.close()


def test_alone_equals_in_mix(gde, rmat16):
    g = rmat16
    seeds = synth.seeds_mixed(g, 16, 16, seed=9)
    G = gde.Graph.from_synth(g)
    _, _, ids_b, vals_b = run_batched(gde, G, "hk", 5.0, 1e-6, seeds)
    for i in (0, 7, 20, 31):
        _, _, ids_1, vals_1 = run_batched(gde, G, "hk", 5.0, 1e-6, seeds[i:i + 1])
        # only the order of the seed's float atomics differs: FP32 summation rounding
        assert np.allclose(vals_1[0], vals_b[i], rtol=1e-5, atol=0)
        same = ids_1[0] == ids_b[i]
        assert np.all(same | np.isclose(vals_1[0], vals_b[i], rtol=1e-5, atol=0))
    G.close()


def test_tag_wrap_and_mixed_kinds(gde, rmat16):
    """Every layer takes its own key tag, so a run of layered solves wraps the tag space and
    clears the tables; PPR solves in between share the same workspace.  Every repeat gives
    the first answer again."""
    g = rmat16
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_mixed(g, 8, 8, seed=12)
    _, _, ids0, vals0 = run_batched(gde, G, "hk", 5.0, 1e-6, seeds)
    _, _, pids0, pvals0 = run_batched(gde, G, "ppr", 0.1, 1e-6, seeds)
    for rep in range(14):
        _, _, ids, vals = run_batched(gde, G, "hk", 5.0, 1e-6, seeds)
        assert np.allclose(vals, vals0, rtol=1e-5, atol=0), rep
        if rep % 4 == 3:
            _, _, pids, pvals = run_batched(gde, G, "ppr", 0.1, 1e-6, seeds)
            assert np.allclose(pvals, pvals0, rtol=1e-5, atol=0), rep
    G.close()


def test_overflow_falls_back(gde, rmat16):
    """A budget too small for the touched sets: overflowing seeds are re-solved with dense
    state and the outputs stay correct."""
    g = rmat16
    seeds = synth.seeds_mixed(g, 4, 4, seed=4)
    G = gde.Graph.from_synth(g)
    st, stats, ids, vals = run_batched(gde, G, "hk", 5.0, 1e-6, seeds, mem_budget_bytes=8 * 18 * 4096)
    assert st == gde.OK
    assert any(s["fallback"] for s in stats)
    for i in (0, 5):
        ref = oracle.localgd(g, "hk", 5.0, 1e-6, int(seeds[i]))
        check_topk(g, ids[i], vals[i], ref.x, 1e-6)
    G.close()


def test_isolated_duplicate_and_padding(gde):
    """An isolated seed keeps its unit mass: e^-tau at the seed for the heat kernel and c_0
    for a series, nothing else.  A repeated seed gives the same list twice, and a support
    smaller than k pads with -1."""
    g = synth.with_isolated(synth.star(5), 2)  # nodes 6, 7 isolated
    G = gde.Graph.from_synth(g)
    seeds = np.array([6, 0, 0, 3], dtype=np.int32)
    tau = 2.0
    st, stats, ids, vals = run_batched(gde, G, "hk", tau, 1e-4, seeds, k=8)
    assert st == gde.OK
    assert ids[0, 0] == 6 and vals[0, 0] == pytest.approx(math.exp(-tau), rel=1e-6)
    assert np.all(ids[0, 1:] == -1) and np.all(vals[0, 1:] == 0)
    assert np.array_equal(ids[1], ids[2]) and np.allclose(vals[1], vals[2])
    for i in (1, 3):
        ref = oracle.localgd(g, "hk", tau, 1e-4, int(seeds[i]))
        check_topk(g, ids[i], vals[i], ref.x, 1e-4, k=8)
        assert np.all(ids[i, 6:] == -1)  # the star has 6 nodes
    c = np.array([0.5, 0.25, 0.125, 0.0625])
    st, stats, ids, vals = run_batched(gde, G, "series", 0.0, 1e-4, seeds[:1], k=8, series_coef=c)
    assert st == gde.OK and ids[0, 0] == 6 and vals[0, 0] == pytest.approx(0.5, rel=1e-6)
    G.close()


def test_capped_and_overflowed_solves_leave_a_clean_slab(gde, rmat16):
    """The hub slab is zeroed by the top-k (PPR) or by the layered frontier taking every entry;
    a solve stopped by the round cap, or with an overflowed seed, leaves entries behind and the
    next solve must start from zero counts anyway."""
    g = rmat16
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_mixed(g, 8, 8, seed=17)
    st, stats, ids, vals = run_batched(gde, G, "hk", 5.0, 1e-6, seeds, max_rounds=3)
    assert st == gde.ENOTCONV
    st, stats, ids, vals = run_batched(gde, G, "ppr", 0.1, 1e-6, seeds, max_rounds=2)
    assert st == gde.ENOTCONV
    # a budget so small that some seeds overflow their tables and are re-batched
    run_batched(gde, G, "hk", 5.0, 1e-6, seeds, mem_budget_bytes=16 * 18 * 4096)
    for kind, param in (("hk", 5.0), ("ppr", 0.1), ("hk", 5.0)):
        st, stats, ids, vals = run_batched(gde, G, kind, param, 1e-6, seeds)
        assert st == gde.OK
        for i in (0, 9, 15):
            ref = oracle.localgd(g, kind, param, 1e-6, int(seeds[i]))
            check_topk(g, ids[i], vals[i], ref.x, 1e-6)
    G.close()


def test_slab_capacity_across_kinds_and_batch_sizes(gde, rmat16):
    """The hub slab is reused across solves: two banks for the layered kinds, one for PPR and
    Katz, a seed count that changes from batch to batch.  A layered batch of 4, a PPR batch of
    24, then layered batches of 24 and 4: every batch must start from zero counts and zero x
    wherever it reads, however the one before used the arrays."""
    g = rmat16
    G = gde.Graph.from_synth(g)
    small = synth.seeds_mixed(g, 2, 2, seed=23)
    big = synth.seeds_mixed(g, 12, 12, seed=29)
    for kind, param, seeds in (("hk", 5.0, small), ("ppr", 0.1, big), ("hk", 5.0, big),
                               ("ppr", 0.1, small), ("hk", 5.0, small)):
        st, stats, ids, vals = run_batched(gde, G, kind, param, 1e-6, seeds)
        assert st == gde.OK
        for i in (0, len(seeds) - 1):
            ref = oracle.localgd(g, kind, param, 1e-6, int(seeds[i]))
            check_topk(g, ids[i], vals[i], ref.x, 1e-6)
    G.close()
