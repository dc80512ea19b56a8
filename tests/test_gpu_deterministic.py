"""Deterministic scatter (sort + segmented reduce) of the dense engine.

Each target's contributions are added in ascending source order starting from its
post-frontier residual — the order of the oracle's sequential FP64 round — so in FP64 the
device must reproduce the oracle bit for bit, round by round and for the whole solve, and
repeated runs must be identical in both precisions.
"""
import numpy as np
import pytest

import oracle
import synth

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
    g = synth.rmat(16, 16, seed=21)
    assert g.degrees().max() > 4096
    return g


@pytest.fixture(scope="module")
def c1():
    return synth.workload_graph("chung_lu_1e4")


def lockstep_exact(gde, g, kind, param, eps, seed, hk_mode=0):
    G = gde.Graph.from_synth(g)
    S = gde.Session(G, kind, param, eps, seed, precision="fp64", deterministic=1, hk_threshold=hk_mode)
    x, r, _ = S.read()
    t = 0
    try:
        while True:
            xo, ro = x.copy(), r.copy()
            rn = np.zeros(g.n) if kind == "hk" else None
            rr = oracle.localgd_round(g, kind, param, eps, xo, ro, t=t, r_next=rn, hk_mode=hk_mode)
            k = S.step()
            x, r, act = S.read()
            assert np.array_equal(np.sort(act), rr.active), f"round {t}: active sets differ"
            if k == 0:
                break
            assert np.array_equal(x, xo), f"round {t}: x differs"
            assert np.array_equal(r, rn if kind == "hk" else ro), f"round {t}: r differs"
            t += 1
    finally:
        S.close()
    return t


@pytest.mark.parametrize("kind", ["ppr", "katz", "hk"])
def test_lockstep_bitwise(gde, rmat16, kind):
    param = {"ppr": 0.1, "hk": 5.0}.get(kind)
    if kind == "katz":
        param = 0.5 / synth.lambda_max(rmat16)[0]
    d = rmat16.degrees()
    for s in (int(np.argmax(d)), int(synth.seeds_quantile(rmat16, 8)[5])):
        rounds = lockstep_exact(gde, rmat16, kind, param, 1e-6, s)
        assert rounds > 1


@pytest.mark.parametrize("kind,param", [("ppr", 0.15), ("hk", 5.0)])
def test_solve_bitwise_equals_oracle(gde, c1, kind, param):
    G = gde.Graph.from_synth(c1)
    seeds = synth.seeds_quantile(c1, 4)
    out = np.zeros((4, c1.n))
    st, stats = gde.solve(G, kind, param, 1e-6, seeds, out, deterministic=1)
    assert st == gde.OK
    for i, s in enumerate(seeds):
        ref = oracle.localgd(c1, kind, param, 1e-6, int(s))
        assert np.array_equal(out[i], ref.x)
        assert stats[i]["rounds"] == ref.rounds and stats[i]["active_volume"] == ref.volume


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_runs_are_identical(gde, rmat16, precision):
    G = gde.Graph.from_synth(rmat16)
    seeds = synth.seeds_mixed(rmat16, 3, 3, seed=5)
    dt = np.float64 if precision == "fp64" else np.float32
    outs = []
    for _ in range(3):
        out = np.zeros((6, rmat16.n), dtype=dt)
        gde.solve(G, "ppr", 0.1, 1e-6, seeds, out, precision=precision, deterministic=1)
        outs.append(out)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    # and the FP32 result stays within the FP32 bar of the FP64 oracle
    if precision == "fp32":
        xs, _ = oracle.localgd_many(rmat16, "ppr", 0.1, 1e-6, seeds)
        d = rmat16.degrees().astype(float)
        err = np.abs(outs[0].astype(np.float64) - xs)
        assert np.all(err <= 1e-6 * d[None, :] + 1e-5 * xs + 1e-12)


def test_deterministic_rejects_batched(gde, c1):
    G = gde.Graph.from_synth(c1)
    ids = np.zeros((1, 8), dtype=np.int32)
    vals = np.zeros((1, 8), dtype=np.float32)
    with pytest.raises(gde.GdeError) as e:
        gde.solve(G, "ppr", 0.15, 1e-6, np.array([0], dtype=np.int32), vals, ids, precision="fp32",
                  topk=8, batched=1, deterministic=1)
    assert e.value.status == gde.EINVAL
