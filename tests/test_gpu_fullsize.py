"""Full-size workloads, sampled seeds against the FP64 oracle (slow: graph generation and
oracle solves on millions of nodes).

* R-MAT scale 22 (4.19M nodes, edge factor 16, symmetrised): plain FP64 local GD, one seed
  per launch, PPR alpha=0.1, Katz beta=0.5/lambda_max, heat kernel tau=5, eps 1e-4..1e-7,
  seeds at degree quantiles.
* Chung-Lu n=2^24, mean degree 20, exponent 2.1: FP32 x/r against FP64 for PPR alpha=0.15
  and the heat kernel tau=10 at eps=1e-7; the error of each result against the FP64
  oracle is checked and reported.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def rmat22():
    return synth.workload_graph("rmat22")


@pytest.fixture(scope="module")
def cl24():
    return synth.workload_graph("chung_lu_2p24")


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("kind", ["ppr", "katz", "hk"])
def test_rmat22_plain_fp64(gde, rmat22, kind):
    g = rmat22
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_quantile(g, 64)[[0, 31, 63]]
    if kind == "ppr":
        param = 0.1
    elif kind == "katz":
        param = 0.5 / synth.lambda_max(g)[0]
    else:
        param = 5.0
    import torch
    out = torch.zeros((1, g.n), dtype=torch.float64, device="cuda")
    for eps in (1e-4, 1e-7):
        for s in seeds:
            st, stats = gde.solve(G, kind, param, eps, torch.tensor([s], dtype=torch.int32, device="cuda"), out)
            assert st == gde.OK
            x = out[0].cpu().numpy()
            ref = oracle.localgd(g, kind, param, eps, int(s))
            assert rel_l1(x, ref.x) <= 1e-9
            assert stats[0]["active_volume"] == pytest.approx(ref.volume, rel=1e-6, abs=64)


@pytest.mark.parametrize("kind,param", [("ppr", 0.15), ("hk", 10.0)])
def test_chung_lu_2p24_fp32_vs_fp64(gde, cl24, kind, param):
    g = cl24
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_quantile(g, 64)[[5, 40, 63]]
    d = g.degrees().astype(np.float64)
    eps = 1e-7
    import torch
    for s in seeds:
        sd = torch.tensor([s], dtype=torch.int32, device="cuda")
        o64 = torch.zeros((1, g.n), dtype=torch.float64, device="cuda")
        o32 = torch.zeros((1, g.n), dtype=torch.float32, device="cuda")
        gde.solve(G, kind, param, eps, sd, o64, precision="fp64")
        gde.solve(G, kind, param, eps, sd, o32, precision="fp32")
        x64 = o64[0].cpu().numpy()
        x32 = o32[0].cpu().numpy().astype(np.float64)
        ref = oracle.localgd(g, kind, param, eps, int(s))
        assert rel_l1(x64, ref.x) <= 1e-9
        # FP32: within the eps error band of the FP64 result (both satisfy the paper's bound)
        err = np.abs(x32 - ref.x)
        band = eps * d + 1e-5 * ref.x + 1e-12
        assert np.all(err <= band), f"max excess {np.max(err - band)}"
        big = (ref.x >= eps * d) & (ref.x > 0)
        rel = err[big] / ref.x[big]
        print(f"{kind} seed {s} (d={int(d[s])}): FP32 vs FP64 oracle rel L1 {rel_l1(x32, ref.x):.2e}, "
              f"max rel on entries >= eps d {rel.max() if big.any() else 0:.2e}")
