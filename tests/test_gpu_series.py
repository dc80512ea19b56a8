"""General power series (GDE_SERIES, f = sum_k c_k (A D^-1)^k e_s on the layered system) on the
device against the FP64 oracle: round by round (x and the current layer within 1e-12
relative L1, identical active sets except at the threshold), whole solves, the dense bound,
and the heat kernel as a special case.  Coefficients: IPR's theta^k/(theta^k+theta^10)^2
(Table 1), truncated where the tail is 1e-12 of the sum."""
import math

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


def ipr_coef(theta):
    k = np.arange(0, 400, dtype=np.float64)
    c = theta ** k / (theta ** k + theta ** 10) ** 2
    tail = np.cumsum(c[::-1])[::-1]
    n = int(np.argmax(tail <= 1e-12 * c.sum()))
    return c[: n + 1]


def rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / den if den > 0 else np.abs(a).sum()


def lockstep(gde, g, coef, eps, seed):
    G = gde.Graph.from_synth(g)
    S = gde.Session(G, "series", 0.0, eps, seed, precision="fp64", series_coef=coef)
    x, r, _ = S.read()
    t = 0
    try:
        while True:
            xo, ro = x.copy(), r.copy()
            rn = np.zeros(g.n)
            rr = oracle.series_round(g, coef, t, eps, xo, ro, rn)
            k = S.step()
            x, r, act = S.read()
            assert np.array_equal(np.sort(act), rr.active), f"round {t}: active sets differ"
            if k == 0:
                break
            assert rel_l1(x, xo) <= 1e-12, f"round {t}: x"
            assert rel_l1(r, rn) <= 1e-12, f"round {t}: next layer"
            t += 1
    finally:
        S.close()
    return t


@pytest.mark.parametrize("theta", [1.3, 2.0])
def test_lockstep_ipr(gde, theta):
    c = ipr_coef(theta)
    for g in (synth.workload_graph("chung_lu_1e4"), synth.rmat(16, 16, seed=21)):
        d = g.degrees()
        eps = 1e-3 * c[0]
        assert lockstep(gde, g, c, eps, int(np.argmax(d))) > 1


def test_solve_matches_oracle_and_dense(gde):
    g = synth.with_isolated(synth.chung_lu(1500, 8.0, 2.5, seed=5), 2)
    G = gde.Graph.from_synth(g)
    c = ipr_coef(1.5)
    eps = 1e-3 * c[0]
    seeds = np.concatenate([synth.seeds_quantile(g, 3), [g.n - 1]]).astype(np.int32)
    out = np.zeros((len(seeds), g.n))
    st, stats = gde.solve(G, "series", 0.0, eps, seeds, out, series_coef=c)
    assert st == gde.OK
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    for i, s in enumerate(seeds):
        ref = oracle.series(g, c, eps, int(s))
        assert rel_l1(out[i], ref.x) <= 1e-9
        assert stats[i]["rounds"] == ref.rounds
        f = dense.series(g, c, int(s))
        assert np.all(f - out[i] >= -1e-15 * c.sum()) and np.all(f - out[i] <= eps * d * (1 + 1e-9))
    assert out[-1][g.n - 1] == pytest.approx(c[0])  # isolated source: c_0 e_s


def test_heat_kernel_as_a_series(gde):
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    tau = 5.0
    N = oracle.hk_terms(tau)
    c = [math.exp(-tau)]
    for k in range(N):
        c.append(c[-1] * tau / (k + 1))
    seeds = synth.seeds_quantile(g, 3)
    a = np.zeros((3, g.n))
    b = np.zeros((3, g.n))
    gde.solve(G, "series", 0.0, 1e-6, seeds, a, series_coef=np.array(c))
    gde.solve(G, "hk", tau, 1e-6, seeds, b)
    for i in range(3):
        assert rel_l1(a[i], b[i]) <= 1e-12


def test_bad_coefficients_rejected(gde):
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    out = np.zeros((1, g.n))
    for c in (np.array([0.5, 0.0, 0.1]), np.array([0.5, -0.1]), np.array([np.nan])):
        with pytest.raises(gde.GdeError) as e:
            gde.solve(G, "series", 0.0, 1e-6, np.array([1], np.int32), out, series_coef=c)
        assert e.value.status == gde.EINVAL
