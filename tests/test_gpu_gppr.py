"""Generalised propagation M = D^-b A D^(b-1) (GDE_GPPR: the InstantGNN push of the appendix,
APPNP at b = 1/2) on the device against the FP64 oracle, through the C ABI.

The library runs PPR's round on the scaled residual y = S r (S = max(d, 1)^b); the session
reads r back as y / S, so the round-by-round comparison is in the oracle's variables:
x and r within 1e-12 relative L1 (FP64), S_t identical except nodes whose residual is
within a few ulps of its threshold (the two sides compare y against eps d and r against
eps d^(1-b), which round differently)."""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth
from topk_check import check_bands

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


def rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / den if den > 0 else np.abs(a).sum()


def near_threshold(g, r_before, beta, eps, ids):
    d = g.degrees().astype(np.float64)
    thr = eps * np.power(d[ids], 1.0 - beta)
    return np.abs(np.abs(r_before[ids]) - thr) <= 1e-13 * np.maximum(thr, 1e-300)


def lockstep(gde, g, alpha, beta, eps, seed, precision="fp64"):
    G = gde.Graph.from_synth(g)
    S = gde.Session(G, "gppr", alpha, eps, seed, precision=precision, prop_beta=beta)
    x, r, _ = S.read()
    rounds = 0
    tol = 1e-12 if precision == "fp64" else 1e-5
    try:
        while True:
            xo, ro = x.astype(np.float64), r.astype(np.float64)
            r_before = ro.copy()
            rr = oracle.gppr_round(g, alpha, beta, eps, xo, ro)
            k = S.step()
            x, r, act = S.read()
            dev, ref = set(act.tolist()), set(rr.active.tolist())
            diff = np.array(sorted(dev ^ ref), dtype=np.int64)
            if diff.size:
                assert np.all(near_threshold(g, r_before, beta, eps, diff)), f"round {rounds}: active sets differ"
            if k == 0:
                break
            if diff.size == 0:
                assert rel_l1(x, xo) <= tol and rel_l1(r, ro) <= tol, f"round {rounds}"
            rounds += 1
    finally:
        S.close()
    return rounds


@pytest.fixture(scope="module")
def c1():
    return synth.workload_graph("chung_lu_1e4")


@pytest.fixture(scope="module")
def rmat16():
    return synth.rmat(16, 16, seed=21)


@pytest.mark.parametrize("beta", [0.25, 0.5, 1.0])
def test_lockstep_fp64(gde, c1, rmat16, beta):
    for g in (c1, rmat16):
        d = g.degrees()
        for s in (int(np.argmax(d)), int(synth.seeds_quantile(g, 8)[3])):
            assert lockstep(gde, g, 0.15, beta, 1e-6, s) > 1


def test_lockstep_fp32(gde, c1):
    s = int(synth.seeds_quantile(c1, 8)[6])
    assert lockstep(gde, c1, 0.15, 0.5, 1e-6, s, precision="fp32") > 1


@pytest.mark.parametrize("beta", [0.25, 0.5])
def test_solve_matches_oracle_and_dense_bound(gde, beta):
    g = synth.with_isolated(synth.chung_lu(1500, 8.0, 2.5, seed=5), 2)
    G = gde.Graph.from_synth(g)
    d = g.degrees().astype(np.float64)
    seeds = np.concatenate([synth.seeds_quantile(g, 4), [g.n - 1]]).astype(np.int32)  # an isolated seed too
    out = np.zeros((len(seeds), g.n))
    st, stats = gde.solve(G, "gppr", 0.2, 1e-7, seeds, out, prop_beta=beta)
    assert st == gde.OK
    for i, s in enumerate(seeds):
        ref, rounds, vol, pushes, _ = oracle.gppr(g, 0.2, beta, 1e-7, int(s))
        assert rel_l1(out[i], ref) <= 1e-9
        f = dense.gppr(g, 0.2, beta, int(s))
        err = f - out[i]
        assert err.min() >= -1e-12 and np.all(err < 1e-7 * np.maximum(d, 1.0) ** (1 - beta) + 1e-15)
        assert stats[i]["active_volume"] == pytest.approx(vol, rel=1e-6, abs=16)
    assert out[-1][g.n - 1] == pytest.approx(0.2)  # isolated source: x = alpha e_s


def test_beta_zero_is_ppr_on_the_device(gde, c1):
    G = gde.Graph.from_synth(c1)
    seeds = synth.seeds_quantile(c1, 3)
    a = np.zeros((3, c1.n))
    b = np.zeros((3, c1.n))
    gde.solve(G, "gppr", 0.15, 1e-6, seeds, a, prop_beta=0.0, deterministic=1)
    gde.solve(G, "ppr", 0.15, 1e-6, seeds, b, deterministic=1)
    assert np.array_equal(a, b)


def test_batched_fp32_topk(gde, rmat16):
    g = rmat16
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_mixed(g, 12, 12, seed=6)
    k = 64
    ids = np.zeros((24, k), np.int32)
    vals = np.zeros((24, k), np.float32)
    beta, eps = 0.5, 1e-6
    st, stats = gde.solve(G, "gppr", 0.1, eps, seeds, vals, ids, precision="fp32", topk=k, batched=1,
                          prop_beta=beta)
    assert st == gde.OK
    d = g.degrees().astype(np.float64)
    for i in range(0, 24, 5):
        ref, *_ = oracle.gppr(g, 0.1, beta, eps, int(seeds[i]))
        # the dense bound of this propagation is eps d_u^(1-b) (degree 0 read as 1)
        b = eps * np.maximum(d, 1) ** (1 - beta) + 1e-5 * ref + 1e-12
        check_bands(ids[i], vals[i], ref, b, k)


def test_bad_beta_rejected(gde, c1):
    G = gde.Graph.from_synth(c1)
    out = np.zeros((1, c1.n))
    with pytest.raises(gde.GdeError) as e:
        gde.solve(G, "gppr", 0.15, 1e-6, np.array([1], np.int32), out, prop_beta=1.5)
    assert e.value.status == gde.EINVAL
