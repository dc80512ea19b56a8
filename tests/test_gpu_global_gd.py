"""Standard (global) GD on the device (gde_solve with global_gd = 1: every node every
iteration, a pull SpMV over the whole CSR, until ||D^-1 r||_inf < eps) against the FP64
oracle: the same iteration count and x within 1e-12 relative L1 (the SpMV adds each row in a
different order), on graphs with rows long enough for the block-per-row path; and the
operation ratio of Table 2 (iterations x nnz over LocalGD's sum of vol(S_t))."""
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
    assert g.degrees().max() > 4096  # rows for the block-per-row SpMV
    return g


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("kind", ["ppr", "katz"])
def test_matches_oracle(gde, rmat16, kind):
    for g in (rmat16, synth.workload_graph("chung_lu_1e4")):
        param = 0.1 if kind == "ppr" else 0.5 / synth.lambda_max(g)[0]
        G = gde.Graph.from_synth(g)
        seeds = synth.seeds_quantile(g, 4)[[0, 3]]
        out = np.zeros((2, g.n))
        st, stats = gde.solve(G, kind, param, 1e-6, seeds, out, global_gd=1)
        assert st == gde.OK
        for i, s in enumerate(seeds):
            ref, it = oracle.global_gd(g, kind, param, 1e-6, int(s))
            assert stats[i]["rounds"] == it
            assert stats[i]["active_volume"] == it * g.nnz
            assert rel_l1(out[i], ref) <= 1e-12


def test_fp32(gde, rmat16):
    g = rmat16
    G = gde.Graph.from_synth(g)
    out = np.zeros((1, g.n), np.float32)
    st, stats = gde.solve(G, "ppr", 0.1, 1e-5, synth.seeds_quantile(g, 4)[[1]], out, precision="fp32", global_gd=1)
    ref, it = oracle.global_gd(g, "ppr", 0.1, 1e-5, int(synth.seeds_quantile(g, 4)[1]))
    assert abs(stats[0]["rounds"] - it) <= 1
    assert rel_l1(out[0].astype(np.float64), ref) <= 1e-5


def test_operation_ratio(gde, rmat16):
    """LocalGD touches far fewer edges than GD for a low-degree seed (Table 2's ratio)."""
    g = rmat16
    G = gde.Graph.from_synth(g)
    s = synth.seeds_quantile(g, 8)[[1]]
    out = np.zeros((1, g.n))
    _, gd = gde.solve(G, "ppr", 0.1, 1e-6, s, out, global_gd=1)
    _, lg = gde.solve(G, "ppr", 0.1, 1e-6, s, out)
    assert gd[0]["active_volume"] / lg[0]["active_volume"] > 2.0


def test_rejected_combinations(gde, rmat16):
    G = gde.Graph.from_synth(rmat16)
    ids = np.zeros((1, 8), np.int32)
    vals = np.zeros((1, 8), np.float32)
    with pytest.raises(gde.GdeError):
        gde.solve(G, "ppr", 0.1, 1e-6, np.array([1], np.int32), vals, ids, precision="fp32", topk=8, global_gd=1)
    out = np.zeros((1, rmat16.n))
    with pytest.raises(gde.GdeError):
        gde.solve(G, "hk", 5.0, 1e-6, np.array([1], np.int32), out, global_gd=1)
