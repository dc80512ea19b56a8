"""LocalCH for PPR on the device (gde_solve with chebyshev = 1) against the FP64 oracle of the
same method: the same number of rounds and x within 1e-9 relative L1 (the scatter adds in
another order, and Chebyshev's momentum carries rounding from round to round), inside the
two-sided eps bound of PPR's dense closed form, with fewer pushed edges than LocalGD."""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("eps", [1e-5, 1e-7])
def test_matches_oracle(gde, eps):
    for g in (synth.workload_graph("chung_lu_1e4"), synth.rmat(16, 16, seed=21)):
        G = gde.Graph.from_synth(g)
        seeds = synth.seeds_quantile(g, 4)[[0, 3]]
        out = np.zeros((2, g.n))
        st, stats = gde.solve(G, "ppr", 0.1, eps, seeds, out, chebyshev=1)
        assert st == gde.OK
        for i, s in enumerate(seeds):
            x, r, rounds, vol = oracle.localch(g, 0.1, eps, int(s))
            assert abs(stats[i]["rounds"] - rounds) <= 1
            assert rel_l1(out[i], x) <= 1e-9
            assert stats[i]["active_volume"] == pytest.approx(vol, rel=1e-3)


def test_bound_and_work(gde):
    g = synth.with_isolated(synth.chung_lu(1500, 8.0, 2.5, seed=5), 2)
    G = gde.Graph.from_synth(g)
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    seeds = np.concatenate([synth.seeds_quantile(g, 3), [g.n - 1]]).astype(np.int32)
    out = np.zeros((len(seeds), g.n))
    _, ch = gde.solve(G, "ppr", 0.05, 1e-8, seeds, out, chebyshev=1)
    lg_out = np.zeros_like(out)
    _, lg = gde.solve(G, "ppr", 0.05, 1e-8, seeds, lg_out)
    for i, s in enumerate(seeds):
        f = dense.ppr(g, 0.05, int(s))
        assert np.all(np.abs(f - out[i]) < 1e-8 * d)
        if g.degrees()[s] > 0:
            assert ch[i]["rounds"] < lg[i]["rounds"]
    assert out[-1][g.n - 1] == pytest.approx(0.05)  # isolated source


def test_fp32(gde):
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    out = np.zeros((1, g.n), np.float32)
    s = synth.seeds_quantile(g, 4)[[2]]
    st, stats = gde.solve(G, "ppr", 0.1, 1e-6, s, out, precision="fp32", chebyshev=1)
    assert st == gde.OK
    x, *_ = oracle.localch(g, 0.1, 1e-6, int(s[0]))
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    f = dense.ppr(g, 0.1, int(s[0])) if g.n <= 10000 else x
    assert np.all(np.abs(f - out[0].astype(np.float64)) < 1e-6 * d + 1e-5 * f)


def test_rejects_other_kinds(gde):
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    out = np.zeros((1, g.n))
    with pytest.raises(gde.GdeError):
        gde.solve(G, "katz", 0.001, 1e-6, np.array([1], np.int32), out, chebyshev=1)
