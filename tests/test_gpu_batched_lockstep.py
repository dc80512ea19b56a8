"""Round-by-round parity of the batched FP32 engine (the headline path: Eq. local-gd,
Section 3.3, run for every seed of a batch inside one persistent launch, per-seed hash
accumulators) with the FP64 oracle, through the batched stepping interface (gde_bsession_*).

At every round each seed's device state is read back exactly (FP32 table entries widened to
FP64, hub-slab entries as their fixed-point values), the oracle runs that round from it, and
the device's pushed set, x and r must match: S_t identical (up to nodes within one ulp of
their threshold), every entry >= eps d_u within 1e-5 relative, relative L1 within 1e-5.

Every kind is held to the plain 1e-5 bar.  The engine's precision layout is what makes that a
guarantee rather than luck: targets of degree >= 160 accumulate in the exact fixed-point hub
slab, so an FP32 table entry adds at most 159 terms in a round, within 159 * 2^-24 < 1e-5 of
their exact sum.  With the slab turned off (hub_degree = -1) a hub next to a hub seed can add
hundreds of identical float terms (Katz's share beta r_u has no 1/d_u factor; the heat kernel's
first layers push many equal-degree neighbours), and round-to-nearest drifts with their count;
that configuration is stepped for PPR.
"""
import numpy as np
import pytest

import oracle
import synth
from lockstep import run_batched

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def rmat16():
    return synth.rmat(16, 16, seed=21)


@pytest.fixture(scope="module")
def c1():
    return synth.workload_graph("chung_lu_1e4")


def _report(name, rep):
    print(f"\n{name}: {rep}")
    assert rep["rounds"] > 2 and rep["pushes"] > 0 and rep["entries"] > 0


def test_batched_lockstep_ppr_rmat_64_mixed(gde, rmat16):
    """64 seeds (32 uniform, 32 from the top 1% by degree) on R-MAT 16, whose hubs are pushed
    by the merge-path chunks; PPR alpha = 0.1, eps = 1e-6."""
    g = rmat16
    assert g.degrees().max() > 4096
    seeds = synth.seeds_mixed(g, 32, 32, seed=3)
    G = gde.Graph.from_synth(g)
    rep = run_batched(G, g, "ppr", 0.1, 1e-6, seeds)
    _report("ppr rmat16 64 seeds", rep)
    G.close()


def test_batched_lockstep_ppr_c1(gde, c1):
    seeds = synth.seeds_by_degree(c1, 64, seed=5)
    G = gde.Graph.from_synth(c1)
    rep = run_batched(G, c1, "ppr", 0.15, 1e-6, seeds)
    _report("ppr c1 64 seeds", rep)
    G.close()


def test_batched_lockstep_katz(gde, rmat16):
    g = rmat16
    lam, _ = synth.lambda_max(g)
    seeds = synth.seeds_mixed(g, 8, 8, seed=7)
    G = gde.Graph.from_synth(g)
    rep = run_batched(G, g, "katz", 0.5 / lam, 1e-6, seeds)
    _report("katz rmat16", rep)
    G.close()


def test_batched_lockstep_hk_error_bound(gde, rmat16):
    g = rmat16
    seeds = synth.seeds_mixed(g, 8, 8, seed=8)
    G = gde.Graph.from_synth(g)
    rep = run_batched(G, g, "hk", 5.0, 1e-6, seeds, hk_mode=0)
    _report("hk theta rmat16", rep)
    G.close()


def test_batched_lockstep_hk_literal(gde, rmat16):
    """theta_t = 1: most of the graph is active in the middle layers and hubs receive
    thousands of additions in one round, in the exact slab."""
    g = rmat16
    seeds = synth.seeds_mixed(g, 4, 4, seed=9)
    G = gde.Graph.from_synth(g)
    rep = run_batched(G, g, "hk", 5.0, 1e-6, seeds, hk_mode=1)
    _report("hk literal rmat16", rep)
    G.close()


def test_batched_lockstep_ppr_without_slab(gde, rmat16):
    """The hash tables alone (hub_degree = -1): every target in FP32."""
    g = rmat16
    seeds = synth.seeds_mixed(g, 16, 16, seed=3)
    G = gde.Graph.from_synth(g)
    G.set_tuning(hub_degree=-1)
    rep = run_batched(G, g, "ppr", 0.1, 1e-6, seeds)
    _report("ppr rmat16 without slab", rep)
    G.close()


@pytest.mark.parametrize("hub_degree", [2, 64, 1000])
def test_batched_lockstep_other_hub_degrees(gde, rmat16, hub_degree):
    """Other slab thresholds: nearly every node a hub (2), a lower one (64), and one above the
    exact degree codes (1000, rounded up to 1024)."""
    g = rmat16
    seeds = synth.seeds_mixed(g, 8, 8, seed=14)
    G = gde.Graph.from_synth(g)
    G.set_tuning(hub_degree=hub_degree)
    assert G.get_tuning()["hub_degree"] == hub_degree
    rep = run_batched(G, g, "ppr", 0.1, 1e-6, seeds)
    _report(f"ppr rmat16 hub_degree {hub_degree}", rep)
    rep = run_batched(G, g, "hk", 5.0, 1e-6, seeds[::4])
    _report(f"hk rmat16 hub_degree {hub_degree}", rep)
    G.close()


def test_batched_lockstep_series(gde, c1):
    """Table 1's IPR coefficients theta^k/(theta^k + theta^10)^2 on the layered engine."""
    theta = 1.5
    k = np.arange(40, dtype=np.float64)
    coef = theta ** k / (theta ** k + theta ** 10) ** 2
    seeds = synth.seeds_by_degree(c1, 16, seed=6)
    G = gde.Graph.from_synth(c1)
    rep = run_batched(G, c1, "series", 0.0, 1e-7, seeds, coef=coef)
    _report("series c1", rep)
    G.close()


def test_batched_session_rejects_bad_use(gde, c1):
    G = gde.Graph.from_synth(c1)
    with pytest.raises(gde.GdeError) as e:
        gde.BatchSession(G, "ppr", 0.15, 1e-6, np.array([0, c1.n], dtype=np.int32))
    assert e.value.status == gde.EINVAL
    with pytest.raises(gde.GdeError) as e:
        gde.BatchSession(G, "ppr", 0.15, 1e-6, np.array([0], dtype=np.int32), precision="fp64")
    assert e.value.status == gde.EINVAL
    S = gde.BatchSession(G, "ppr", 0.15, 1e-6, np.array([0, 1], dtype=np.int32))
    S.step()
    with pytest.raises(gde.GdeError) as e:
        S.read(2)
    assert e.value.status == gde.EINVAL
    # the graph changes under the session: the next step is refused
    G.update_edges(np.array([0], dtype=np.int32), np.array([c1.n - 1], dtype=np.int32))
    with pytest.raises(gde.GdeError) as e:
        S.step()
    assert e.value.status == gde.EINVAL
    S.close()
    G.close()


def test_batched_session_runs_the_solve(gde, rmat16):
    """Stepping the session to the end gives the same top values as the one-launch solve
    (the same kernel, the same round count) within FP32 atomic-order rounding."""
    g = rmat16
    seeds = synth.seeds_mixed(g, 6, 6, seed=11)
    G = gde.Graph.from_synth(g)
    S = gde.BatchSession(G, "ppr", 0.1, 1e-6, seeds)
    rounds = 0
    while S.step() > 0:
        rounds += 1
    ids = np.zeros((len(seeds), 64), dtype=np.int32)
    vals = np.zeros((len(seeds), 64), dtype=np.float32)
    st, stats = gde.solve(G, "ppr", 0.1, 1e-6, seeds, vals, ids, precision="fp32", topk=64, batched=1)
    assert st == gde.OK
    for j in range(len(seeds)):
        x, _, _ = S.read(j)
        ref_ids, ref_vals = oracle.topk(x.astype(np.float64), 64)
        assert np.allclose(vals[j], ref_vals, rtol=1e-5, atol=0)
    assert max(s["rounds"] for s in stats) == rounds + 1
    S.close()
    G.close()


@pytest.mark.slow
def test_batched_lockstep_full_size_rmat24(gde):
    """Round by round on the benchmark's graph (R-MAT scale 24, hubs of degree up to ~400K)
    with the benchmark's launch shape, PPR alpha=0.1, eps=1e-7: four uniform and four top-1%
    seeds of the benchmark's batch, every entry >= eps d_u within 1e-5 of the FP64 oracle's
    round from the same state, every round of the solve."""
    g = synth.workload_graph("rmat24")
    batch = synth.seeds_mixed(g, 512, 512, seed=4)
    seeds = batch[[0, 1, 2, 3, 512, 513, 514, 515]]
    G = gde.Graph.from_synth(g)
    G.set_tuning(t1=32, t2=128, chunk=512, schedule=4, hub_degree=128)
    rep = run_batched(G, g, "ppr", 0.1, 1e-7, seeds, mem_budget_bytes=512 << 20)
    _report("full size R-MAT 24", rep)
    assert rep["rounds"] >= 8 and rep["entries"] > 10**5
    assert rep["max_rel_r"] <= 1e-5 and rep["max_rel_x"] <= 1e-5
    G.close()


@pytest.mark.slow
@pytest.mark.parametrize("kind,param,eps", [("katz", 0.9, 1e-7), ("hk", 5.0, 1e-6)])
def test_batched_lockstep_full_size_rmat24_katz_hk(gde, kind, param, eps):
    """The benchmark's other kinds on its graph, round by round: Katz (beta = 0.9 / lambda_max,
    the power iteration's estimate) and the heat kernel (tau = 5, error-bound threshold), two
    uniform and two top-1% seeds of the benchmark's batch, at the plain 1e-5 bar."""
    g = synth.workload_graph("rmat24")
    if kind == "katz":
        lam, _ = synth.lambda_max(g, rel_tol=1e-4, max_iter=200)
        param = param / lam
    batch = synth.seeds_mixed(g, 512, 512, seed=4)
    seeds = batch[[0, 1, 512, 513]]
    G = gde.Graph.from_synth(g)
    G.set_tuning(t1=32, t2=128, chunk=512, schedule=4, hub_degree=64)
    rep = run_batched(G, g, kind, param, eps, seeds, mem_budget_bytes=2 << 30)
    _report(f"full size R-MAT 24 {kind}", rep)
    assert rep["max_rel_r"] <= 1e-5 and rep["max_rel_x"] <= 1e-5
    G.close()
