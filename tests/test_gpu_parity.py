"""CUDA path against the FP64 oracle (all calls go through the C ABI).

Lock-step per round (tests/lockstep.py), free-running solves against the oracle's
result and against dense closed forms with the eps error bounds, FP32 mode, and
edge cases (isolated and degree-1 seeds, hubs above the merge-path bin threshold,
empty active sets, round caps).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

import lockstep

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
    # hubs well above the warp-bin limit (d > 2048) exercise the merge-path chunks
    g = synth.rmat(16, 16, seed=21)
    assert g.degrees().max() > 4096 * 2
    return g


def c1_seed(g):
    return int(synth.seeds_by_degree(g, 1, seed=1)[0])


# ------------------------------------------------------------- lock-step ----

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lockstep_ppr_c1(gde, c1, precision):
    """Chung-Lu n=10^4, d=10, gamma=2.5, alpha=0.15, eps=1e-6, source drawn by degree."""
    G = gde.Graph.from_synth(c1)
    hist, x, _ = lockstep.run(G, c1, "ppr", 0.15, 1e-6, c1_seed(c1), precision)
    assert len(hist) > 5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed_kind", ["hub", "leaf"])
def test_lockstep_ppr_rmat_hubs(gde, rmat16, precision, seed_kind):
    G = gde.Graph.from_synth(rmat16)
    d = rmat16.degrees()
    s = int(np.argmax(d)) if seed_kind == "hub" else int(np.nonzero(d == 1)[0][0])
    hist, _, _ = lockstep.run(G, rmat16, "ppr", 0.1, 1e-6, s, precision)
    assert sum(h[1] for h in hist) > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lockstep_katz(gde, rmat16, precision):
    lam, _ = synth.lambda_max(rmat16)
    G = gde.Graph.from_synth(rmat16)
    s = int(synth.seeds_quantile(rmat16, 8)[6])
    lockstep.run(G, rmat16, "katz", 0.5 / lam, 1e-6, s, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("hk_mode", [0, 1])
def test_lockstep_hk(gde, rmat16, precision, hk_mode):
    G = gde.Graph.from_synth(rmat16)
    s = int(synth.seeds_quantile(rmat16, 8)[7])
    hist, _, _ = lockstep.run(G, rmat16, "hk", 5.0, 1e-6, s, precision, hk_mode=hk_mode)
    assert len(hist) <= oracle.hk_terms(5.0) + 1


def test_lockstep_hk_c1(gde, c1):
    G = gde.Graph.from_synth(c1)
    lockstep.run(G, c1, "hk", 5.0, 1e-5, c1_seed(c1), "fp64")


# --------------------------------------------------------- free-running ----

def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("kind,param", [("ppr", 0.15), ("katz", None), ("hk", 5.0)])
def test_solve_matches_oracle_c1(gde, c1, kind, param):
    if param is None:
        lam, _ = synth.lambda_max(c1)
        param = 0.5 / lam
    G = gde.Graph.from_synth(c1)
    seeds = synth.seeds_quantile(c1, 4)
    out = np.zeros((4, c1.n))
    st, stats = gde.solve(G, kind, param, 1e-6, seeds, out)
    assert st == gde.OK
    for i, s in enumerate(seeds):
        ref = oracle.localgd(c1, kind, param, 1e-6, int(s))
        assert rel_l1(out[i], ref.x) <= 1e-9
        assert stats[i]["rounds"] == ref.rounds or abs(stats[i]["rounds"] - ref.rounds) <= 1
        assert abs(stats[i]["active_volume"] - ref.volume) <= 1e-6 * ref.volume + 64


def small_graphs():
    return [synth.path(7), synth.cycle(9), synth.star(6), synth.complete(6),
            synth.erdos_renyi(150, 0.04, 2), synth.chung_lu(400, 6.0, 2.3, seed=4)]


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ppr_error_bound_vs_dense(gde, gi, precision):
    """Corollary 3.6: 0 <= f_u - x_u < eps d_u (FP32: up to 1e-5 f_u more)."""
    g = small_graphs()[gi]
    d = g.degrees().astype(float)
    G = gde.Graph.from_synth(g)
    s = np.array([int(np.argmax(d))], dtype=np.int32)
    alpha, eps = 0.15, 1e-5
    f = dense.ppr(g, alpha, int(s[0]))
    out = np.zeros((1, g.n), dtype=np.float64 if precision == "fp64" else np.float32)
    gde.solve(G, "ppr", alpha, eps, s, out, precision=precision)
    err = f - out[0].astype(np.float64)
    slack = 1e-12 if precision == "fp64" else 1e-5 * f + 1e-9
    assert np.all(err >= -slack)
    assert np.all(err < eps * d + slack)


@pytest.mark.parametrize("gi", range(6))
def test_hk_and_katz_vs_dense(gde, gi):
    g = small_graphs()[gi]
    d = g.degrees().astype(float)
    G = gde.Graph.from_synth(g)
    s = np.array([int(np.argmax(d))], dtype=np.int32)
    tau, eps = 3.0, 1e-6
    N = oracle.hk_terms(tau)
    fN = dense.hk_taylor(g, tau, int(s[0]), N)
    out = np.zeros((1, g.n))
    gde.solve(G, "hk", tau, eps, s, out)
    err = fN - out[0]
    assert np.all(err >= -1e-12) and np.all(err <= eps * d + 1e-12)
    lam = np.linalg.eigvalsh(dense.adjacency(g))[-1]
    beta = 0.5 / lam
    xs = dense.katz(g, beta, int(s[0]))
    Qinv = np.linalg.inv(dense.katz_system(g, beta))
    gde.solve(G, "katz", beta, eps, s, out)
    err = xs - out[0]
    assert np.all(err >= -1e-12) and np.all(err <= eps * (Qinv @ d) + 1e-12)


# ---------------------------------------------------------------- edges ----

def test_isolated_seed(gde):
    g = synth.with_isolated(synth.cycle(5), 2)
    G = gde.Graph.from_synth(g)
    out = np.zeros((3, g.n))
    seeds = np.array([5, 6, 0], dtype=np.int32)
    st, stats = gde.solve(G, "ppr", 0.2, 1e-4, seeds, out)
    assert out[0, 5] == 0.2 and out[0].sum() == 0.2 and stats[0]["rounds"] == 1
    assert stats[0]["active_volume"] == 0
    assert out[1, 6] == 0.2
    gde.solve(G, "hk", 2.0, 1e-4, seeds[:1], out[:1])
    assert out[0, 5] == pytest.approx(math.exp(-2.0), rel=1e-15)


def test_seed_not_active(gde):
    """eps so large that even the unit source is below eps d_s: S_0 is empty."""
    g = synth.star(10)
    G = gde.Graph.from_synth(g)
    out = np.ones((1, g.n))
    st, stats = gde.solve(G, "ppr", 0.2, 0.5, np.array([0], dtype=np.int32), out)
    assert st == gde.OK and np.all(out == 0) and stats[0]["rounds"] == 0


def test_round_cap(gde, c1):
    G = gde.Graph.from_synth(c1)
    out = np.zeros((1, c1.n))
    st, stats = gde.solve(G, "ppr", 0.15, 1e-8, np.array([c1_seed(c1)], dtype=np.int32), out,
                          max_rounds=3)
    assert st == gde.ENOTCONV and stats[0]["status"] == gde.ENOTCONV and stats[0]["rounds"] == 3


def test_device_pointers_and_stream(gde, c1):
    import torch
    G = gde.Graph(c1.n, torch.from_numpy(c1.offsets).cuda(), torch.from_numpy(c1.cols).cuda())
    seeds = torch.tensor(synth.seeds_quantile(c1, 3), dtype=torch.int32, device="cuda")
    out = torch.zeros((3, c1.n), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        st, _ = gde.solve(G, "ppr", 0.15, 1e-6, seeds, out)
    s.synchronize()
    host = np.zeros((3, c1.n))
    gde.solve(gde.Graph.from_synth(c1), "ppr", 0.15, 1e-6, seeds.cpu().numpy(), host)
    assert rel_l1(out.cpu().numpy().ravel(), host.ravel()) <= 1e-12


@pytest.mark.parametrize("bad", ["unsorted", "selfloop", "range", "dup", "offsets"])
def test_invalid_csr_rejected(gde, bad):
    off = np.array([0, 2, 4, 6], dtype=np.int64)
    col = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)
    if bad == "unsorted":
        col[0], col[1] = 2, 1
    elif bad == "selfloop":
        col[0] = 0
    elif bad == "range":
        col[5] = 7
    elif bad == "dup":
        col[1] = 1
    else:
        off[1] = 5
    with pytest.raises(gde.GdeError) as e:
        gde.Graph(3, off, col)
    assert e.value.status == gde.EINVAL


def test_asymmetric_rejected_on_request(gde):
    off = np.array([0, 1, 1], dtype=np.int64)
    col = np.array([1], dtype=np.int32)
    gde.Graph(2, off, col)  # accepted without the check
    with pytest.raises(gde.GdeError):
        gde.Graph(2, off, col, check_symmetric=True)


def test_bad_arguments(gde, c1):
    G = gde.Graph.from_synth(c1)
    out = np.zeros((1, c1.n))
    s = np.array([0], dtype=np.int32)
    for kind, param, eps in (("ppr", 1.5, 1e-4), ("ppr", 0.1, 0.0), ("katz", -1.0, 1e-4),
                             ("hk", 0.0, 1e-4)):
        with pytest.raises(gde.GdeError) as e:
            gde.solve(G, kind, param, eps, s, out)
        assert e.value.status == gde.EINVAL
    with pytest.raises(gde.GdeError):
        gde.solve(G, "ppr", 0.1, 1e-4, np.array([c1.n], dtype=np.int32), out)
