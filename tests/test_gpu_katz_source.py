"""Katz near its convergence limit, beta = 0.95 / lambda_max and 0.99 / lambda_max, on graphs
where beta d_max > 1 (outside the paper's beta < 1/d_max condition; LocalGD still terminates,
since the Perron-weighted residual falls by (1 - beta lambda) w^T r_S every round).

The Katz vector is f_Katz = x - e_s (Eq. f-katz).  Its source entry is x_s - 1, a small
number recovered from x_s ~ 1: read from an FP32 x_s it would keep only about 6e-8 absolute.
With katz_minus_source = 1 both engines keep x_s - 1 in an FP64 word (starting at -1 and
gaining every residual pushed at s) and return f_Katz; in FP32 mode its source entry must
match the FP64 oracle's to 1e-5 relative, round by round (lock-step) and in the final answer.
"""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth
import lockstep
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
def c1():
    return synth.workload_graph("chung_lu_1e4")


def _beta(g, frac):
    lam, _ = synth.lambda_max(g)
    beta = frac / lam
    assert beta * g.degrees().max() > 1.0
    return beta


@pytest.mark.parametrize("frac", [0.95, 0.99])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_katz_source_entry_lockstep(gde, c1, frac, precision):
    beta = _beta(c1, frac)
    s = int(synth.seeds_quantile(c1, 8)[6])
    G = gde.Graph.from_synth(c1)
    hist, x, _ = lockstep.run(G, c1, "katz", beta, 1e-6, s, precision, katz_minus_source=1)
    assert len(hist) > 20
    G.close()


@pytest.mark.parametrize("frac", [0.95, 0.99])
def test_katz_minus_source_output(gde, c1, frac):
    """f_Katz output against the x output of the same solve: with the deterministic scatter
    both runs do the same arithmetic, so every entry but the source is bitwise equal, and the
    source entry is x_s - 1 (to the FP32 rounding of x_s ~ 1).  (The free-running FP32 and
    FP64 answers of ~1000-round Katz solves may push a near-threshold node in different
    rounds, so their final source entries are compared by the lock-step test instead.)"""
    beta = _beta(c1, frac)
    seeds = synth.seeds_quantile(c1, 4)
    G = gde.Graph.from_synth(c1)
    out_f = np.zeros((len(seeds), c1.n), dtype=np.float32)
    out_x = np.zeros((len(seeds), c1.n), dtype=np.float32)
    st, stats = gde.solve(G, "katz", beta, 1e-7, seeds, out_f, precision="fp32", deterministic=1,
                          katz_minus_source=1)
    assert st == gde.OK
    st, _ = gde.solve(G, "katz", beta, 1e-7, seeds, out_x, precision="fp32", deterministic=1)
    assert st == gde.OK
    for i, s in enumerate(seeds):
        other = np.arange(c1.n) != s
        assert np.array_equal(out_x[i, other], out_f[i, other])
        assert out_f[i, s] > 0
        # the FP32 x_s gains one rounding of up to half an ulp of 1 per push of s; the source
        # word does not, which is what keeps f_s to FP32 relative precision
        assert abs(float(out_x[i, s]) - 1.0 - float(out_f[i, s])) <= (stats[i]["rounds"] + 1) * 2.0 ** -24
    G.close()


def small_graphs():
    return [synth.star(6), synth.erdos_renyi(150, 0.04, 2), synth.chung_lu(400, 6.0, 2.3, seed=4)]


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("frac", [0.95, 0.99])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_katz_minus_source_dense_bound(gde, gi, frac, precision):
    """0 <= f* - f <= eps (I - beta A)^-1 d entrywise (the Katz bound), f = x - e_s, against
    the dense solve (I - beta A)^-1 e_s - e_s; FP32 with 1e-5 relative slack."""
    g = small_graphs()[gi]
    d = g.degrees().astype(float)
    lam = np.linalg.eigvalsh(dense.adjacency(g))[-1]
    beta = frac / lam
    assert beta * d.max() > 1.0
    s = int(np.argmax(d))
    fstar = dense.katz(g, beta, s)
    fstar[s] -= 1.0
    Qinv = np.linalg.inv(dense.katz_system(g, beta))
    G = gde.Graph.from_synth(g)
    eps = 1e-6
    dt = np.float64 if precision == "fp64" else np.float32
    out = np.zeros((1, g.n), dtype=dt)
    st, stats = gde.solve(G, "katz", beta, eps, np.array([s], dtype=np.int32), out, precision=precision,
                          katz_minus_source=1)
    assert st == gde.OK
    err = fstar - out[0].astype(np.float64)
    slack = 1e-12 + (0.0 if precision == "fp64" else 1e-5 * np.abs(fstar))
    assert np.all(err >= -slack)
    assert np.all(err <= eps * (Qinv @ d) + slack)
    G.close()


def katz_bound(g, beta, eps):
    """eps (I - beta A)^-1 d: the Katz error bound of LocalGD (sparse direct solve)"""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.offsets))
    A = sp.csr_matrix((np.ones(g.nnz), (rows, g.cols)), shape=(n, n))
    Q = sp.identity(n, format="csc") - beta * A.tocsc()
    return eps * spl.spsolve(Q, g.degrees().astype(np.float64))


def test_katz_minus_source_batched(gde, c1):
    """The batched engine's f_Katz output: top-k of x - e_s (the source entry from its FP64
    word) against the oracle's, each node within the Katz bound eps ((I - beta A)^-1 d)_u of
    it (both runs satisfy 0 <= f* - f <= that bound); and round by round with the source entry
    at 1e-5."""
    from topk_check import check_bands
    beta = _beta(c1, 0.95)
    seeds = synth.seeds_mixed(c1, 8, 8, seed=31)
    G = gde.Graph.from_synth(c1)
    k = 64
    ids = np.zeros((len(seeds), k), dtype=np.int32)
    vals = np.zeros((len(seeds), k), dtype=np.float32)
    st, stats = gde.solve(G, "katz", beta, 1e-6, seeds, vals, ids, precision="fp32", topk=k, batched=1,
                          katz_minus_source=1)
    assert st == gde.OK
    bound = katz_bound(c1, beta, 1e-6)
    for i in (0, 9, 15):
        ref = oracle.localgd(c1, "katz", beta, 1e-6, int(seeds[i]))
        f = ref.x.copy()
        f[seeds[i]] -= 1.0
        check_bands(ids[i], vals[i], f, bound + 1e-5 * np.abs(f) + 1e-12, k)
    rep = run_batched(G, c1, "katz", beta, 1e-6, seeds[:8], katz_minus_source=1)
    print("\nbatched katz f lock-step:", rep)
    assert rep["max_rel_source"] <= 1e-5
    G.close()


def test_katz_minus_source_rejected_elsewhere(gde, c1):
    G = gde.Graph.from_synth(c1)
    out = np.zeros((1, c1.n))
    for kind, param, kw in (("ppr", 0.15, {}), ("katz", 1e-3, {"global_gd": 1})):
        with pytest.raises(gde.GdeError) as e:
            gde.solve(G, kind, param, 1e-6, np.array([0], dtype=np.int32), out, katz_minus_source=1, **kw)
        assert e.value.status == gde.EINVAL
    G.close()
