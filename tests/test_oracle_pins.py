"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: closed forms on graphs
whose diffusion vectors can be written by hand, dense linear solves and matrix
exponentials (numpy/scipy), exact invariants of LocalGD (Theorem 3.5 and its
proof), the error and work bounds of Corollary 3.6, and library routines
(scipy.stats.poisson for the Taylor truncation).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import dense


def fresh_state(g, seed):
    x = np.zeros(g.n)
    r = np.zeros(g.n)
    r[seed] = 1.0
    return x, r


# ------------------------------------------------------------ closed forms ----

@pytest.mark.parametrize("alpha", [0.15, 0.1, 0.5])
def test_ppr_edge2_rounds(alpha):
    """2-node edge from node 0: round t pushes node t mod 2 with r = (1-alpha)^t
    (Eq. local-gd); x gains alpha (1-alpha)^t there.  f = (1, 1-alpha)/(2-alpha)."""
    g = synth.edge2()
    eps = 1e-9
    x, r = fresh_state(g, 0)
    t, expect_r = 0, 1.0
    while True:
        rr = oracle.localgd_round(g, "ppr", alpha, eps, x, r)
        if rr.n_active == 0:
            break
        assert list(rr.active) == [t % 2]
        assert rr.rho[0] == pytest.approx(expect_r, rel=1e-14)
        assert r[t % 2] == 0.0
        assert r[(t + 1) % 2] == pytest.approx((1 - alpha) * expect_r, rel=1e-14)
        expect_r *= 1 - alpha
        t += 1
    # stops at the first t with (1-alpha)^t < eps * d (d = 1)
    assert (1 - alpha) ** t < eps <= (1 - alpha) ** (t - 1) * (1 + 1e-12)
    f = np.array([1.0, 1.0 - alpha]) / (2.0 - alpha)
    assert np.all(f - x >= -1e-15) and np.all(f - x < eps)


@pytest.mark.parametrize("k", [1, 3, 8])
def test_ppr_star_rounds_from_center(k):
    """Star with k leaves from the centre: even rounds push the centre with
    (1-alpha)^t, odd rounds push every leaf with (1-alpha)^t / k (the share is
    divided by the pushing node's degree, not the receiver's)."""
    g = synth.star(k)
    alpha, eps = 0.2, 1e-7
    x, r = fresh_state(g, 0)
    for t in range(12):
        rr = oracle.localgd_round(g, "ppr", alpha, eps, x, r)
        if t % 2 == 0:
            assert list(rr.active) == [0]
            assert rr.rho[0] == pytest.approx((1 - alpha) ** t, rel=1e-13)
            assert np.allclose(r[1:], (1 - alpha) ** (t + 1) / k, rtol=1e-13)
        else:
            assert list(rr.active) == list(range(1, k + 1))
            assert np.allclose(rr.rho, (1 - alpha) ** t / k, rtol=1e-13)
            assert r[0] == pytest.approx((1 - alpha) ** (t + 1), rel=1e-13)
    # closed form f_c = 1/(2-alpha), f_leaf = (1-alpha)/(k(2-alpha))
    res = oracle.localgd(g, "ppr", alpha, 1e-12, 0)
    f = np.array([1 / (2 - alpha)] + [(1 - alpha) / (k * (2 - alpha))] * k)
    assert np.allclose(res.x, f, rtol=0, atol=1e-11 * k)


@pytest.mark.parametrize("k,beta", [(1, 0.5), (4, 0.3), (9, 0.2)])
def test_katz_star_closed_form(k, beta):
    """(I - beta A) x = e_c on a star: x_c = 1/(1 - k beta^2), x_leaf = beta x_c."""
    g = synth.star(k)
    res = oracle.localgd(g, "katz", beta, 1e-13, 0)
    xc = 1.0 / (1.0 - k * beta * beta)
    f = np.array([xc] + [beta * xc] * k)
    assert np.allclose(res.x, f, rtol=1e-10)
    # Katz pushes the full residual with weight beta (no 1/d_u)
    x, r = fresh_state(g, 0)
    oracle.localgd_round(g, "katz", beta, 1e-9, x, r)
    assert x[0] == 1.0 and np.all(r[1:] == beta) and r[0] == 0.0


@pytest.mark.parametrize("k,tau", [(1, 1.0), (5, 3.0), (4, 5.0)])
def test_hk_star_closed_form(k, tau):
    """Star: M e_c = mean of leaves, M e_leaf = e_c, so
    exp(-tau(I-M)) e_c = e^-tau (cosh(tau) e_c + sinh(tau)/k sum e_leaf)."""
    g = synth.star(k)
    res = oracle.localgd(g, "hk", tau, 1e-14, 0)
    f = math.exp(-tau) * np.array([math.cosh(tau)] + [math.sinh(tau) / k] * k)
    assert np.allclose(res.x, f, rtol=0, atol=2e-12)


def test_hk_edge2_closed_form():
    g = synth.edge2()
    tau = 2.5
    res = oracle.localgd(g, "hk", tau, 1e-15, 0)
    f = np.array([(1 + math.exp(-2 * tau)) / 2, (1 - math.exp(-2 * tau)) / 2])
    assert np.allclose(res.x, f, atol=2e-12)


def test_katz_edge2_closed_form():
    g = synth.edge2()
    beta = 0.7
    res = oracle.localgd(g, "katz", beta, 1e-14, 0)
    assert np.allclose(res.x, np.array([1.0, beta]) / (1 - beta * beta), rtol=1e-12)


# ------------------------------------------------------------- dense solves ----

def graphs_small():
    return [synth.path(7), synth.cycle(9), synth.complete(6), synth.star(5),
            synth.erdos_renyi(60, 0.08, 1), synth.erdos_renyi(150, 0.04, 2),
            synth.with_isolated(synth.erdos_renyi(40, 0.12, 3), 3),
            synth.chung_lu(300, 6.0, 2.5, seed=4)]


@pytest.mark.parametrize("gi", range(8))
@pytest.mark.parametrize("alpha,eps", [(0.15, 1e-4), (0.1, 1e-6), (0.3, 1e-3)])
def test_ppr_error_bound_dense(gi, alpha, eps):
    """Corollary 3.6: 0 <= f_u - x_u < eps d_u for every u, and
    sum_t vol(S_t) <= 1/(alpha eps)."""
    g = graphs_small()[gi]
    d = g.degrees()
    for s in [int(np.argmax(d)), int(np.nonzero(d)[0][0])]:
        f = dense.ppr(g, alpha, s)
        res = oracle.localgd(g, "ppr", alpha, eps, s)
        err = f - res.x
        assert np.all(err >= -1e-13)
        assert np.all(err < eps * d + 1e-13)
        assert res.volume <= 1.0 / (alpha * eps)
        # mass: ||x||_1 + ||r||_1 = 1 (unit source, no isolated node is ever reached)
        assert res.x_l1 + res.resid_l1 == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("gi", range(8))
def test_ppr_converges_to_dense(gi):
    g = graphs_small()[gi]
    s = int(np.argmax(g.degrees()))
    for alpha in (0.15, 0.5):
        f = dense.ppr(g, alpha, s)
        res = oracle.localgd(g, "ppr", alpha, 1e-14, s)
        assert np.allclose(res.x, f, rtol=0, atol=1e-12)


@pytest.mark.parametrize("gi", range(8))
def test_katz_dense(gi):
    """beta = 0.5/lambda_max: LocalGD terminates and 0 <= x* - x <= eps Q^-1 d
    elementwise (x* - x = Q^-1 r with 0 <= r < eps d, Q^-1 >= 0 when beta lambda < 1)."""
    g = graphs_small()[gi]
    A = dense.adjacency(g)
    lam = np.linalg.eigvalsh(A)[-1]
    beta = 0.5 / lam
    d = g.degrees().astype(float)
    s = int(np.argmax(d))
    xs = dense.katz(g, beta, s)
    Qinv = np.linalg.inv(dense.katz_system(g, beta))
    for eps in (1e-3, 1e-6):
        res = oracle.localgd(g, "katz", beta, eps, s)
        assert res.status == 0
        err = xs - res.x
        assert np.all(err >= -1e-12)
        assert np.all(err <= eps * (Qinv @ d) + 1e-12)
    res = oracle.localgd(g, "katz", beta, 1e-15, s)
    assert np.allclose(res.x, xs, atol=1e-12)


@pytest.mark.parametrize("gi", range(8))
@pytest.mark.parametrize("tau", [1.0, 5.0])
def test_hk_dense(gi, tau):
    """HK: Taylor truncation at N (Poisson tail <= 1e-12) against scipy's expm, and
    the layered LocalGD error 0 <= f_N - e^-tau x <= eps d_u (threshold scale
    theta_t = e^tau/((N+1) psi_t))."""
    g = graphs_small()[gi]
    d = g.degrees().astype(float)
    s = int(np.argmax(d))
    N = oracle.hk_terms(tau)
    fN = dense.hk_taylor(g, tau, s, N)
    fe = dense.hk_exact(g, tau, s)
    assert np.abs(fe - fN).sum() <= 1.5e-12
    for eps in (1e-3, 1e-6):
        res = oracle.localgd(g, "hk", tau, eps, s, hk_mode=0)
        err = fN - res.x
        assert np.all(err >= -1e-13)
        assert np.all(err <= eps * d + 1e-13)
    res = oracle.localgd(g, "hk", tau, 1e-15, s)
    assert np.allclose(res.x, fN, atol=1e-12)


# ---------------------------------------------------------------- invariants ----

@pytest.mark.parametrize("gi", [0, 1, 4, 5, 7])
def test_ppr_round_invariants(gi):
    """Every round (Theorem 3.5 and the proof of Corollary 3.6):
    x + alpha Q^-1 r = f with Q = I - (1-alpha) A D^-1;  r >= 0;
    ||r^(t+1)||_1 = ||r^(t)||_1 - alpha ||r_S||_1;  and S_t is exactly
    { u : r_u != 0, r_u >= eps d_u }."""
    g = graphs_small()[gi]
    d = g.degrees()
    alpha, eps = 0.15, 1e-5
    s = int(np.argmax(d))
    f = dense.ppr(g, alpha, s)
    Qinv = np.linalg.inv(dense.ppr_system(g, alpha))
    x, r = fresh_state(g, s)
    gammas = []
    r0 = np.abs(r).sum()
    for t in range(10_000):
        before = r.copy()
        rr = oracle.localgd_round(g, "ppr", alpha, eps, x, r)
        want = np.nonzero((before != 0) & (np.abs(before) >= eps * d))[0]
        assert np.array_equal(rr.active, want)
        if rr.n_active == 0:
            break
        assert np.all(r >= 0)
        assert np.abs(r).sum() == pytest.approx(before.sum() - alpha * rr.rS_l1, abs=1e-14)
        assert np.allclose(x + alpha * Qinv @ r, f, atol=1e-13)
        gammas.append(rr.rS_l1 / before.sum())
    T = len(gammas)
    # Theorem 3.5 with beta P_max = 1 - alpha:  T <= ln(||r0||/||rT||) / (alpha mean gamma)
    assert T <= math.log(r0 / r.sum()) / (alpha * np.mean(gammas)) + 1e-9


def test_jacobi_snapshot_semantics():
    """LocalGD pushes r^(t) on S_t simultaneously (Eq. local-gd): on an edge with
    both ends active, each end receives the other's pre-round residual."""
    g = synth.edge2()
    alpha = 0.25
    x = np.zeros(2)
    r = np.array([1.0, 0.5])
    oracle.localgd_round(g, "ppr", alpha, 0.1, x, r)
    assert np.array_equal(x, alpha * np.array([1.0, 0.5]))
    assert np.array_equal(r, (1 - alpha) * np.array([0.5, 1.0]))


def test_threshold_is_inclusive():
    """An entry exactly at eps d_u is active (|r_u| >= eps d_u, Algo 1's condition)."""
    g = synth.edge2()
    res = oracle.localgd(g, "ppr", 0.5, 0.25, 0, log=True)
    # r: 1, 0.5, 0.25 (== eps d), 0.125 -> three rounds
    assert res.rounds == 3
    assert [e[2] for e in res.log] == [1.0, 0.5, 0.25]


def test_isolated_seed():
    """A degree-0 source moves its mass into x and scatters nothing."""
    g = synth.with_isolated(synth.cycle(4), 2)
    s = 5
    for kind, param, want in (("ppr", 0.15, 0.15), ("katz", 0.3, 1.0),
                              ("hk", 2.0, math.exp(-2.0))):
        res = oracle.localgd(g, kind, param, 1e-6, s)
        assert res.rounds == 1 and res.volume == 0
        e = np.zeros(g.n)
        e[s] = want
        assert np.allclose(res.x, e, rtol=1e-15, atol=0)


def test_katz_perron_weighted_decrease():
    """With A w = lambda w (w > 0): w'r^(t+1) = w'r^(t) - (1 - beta lambda) w'r_S,
    so LocalGD terminates whenever beta lambda < 1 even if beta d_max > 1."""
    g = synth.chung_lu(200, 8.0, 2.2, seed=6)
    A = dense.adjacency(g)
    vals, vecs = np.linalg.eigh(A)
    lam, w = vals[-1], np.abs(vecs[:, -1])
    beta = 0.9 / lam
    assert beta * g.degrees().max() > 1.0  # outside the d_max condition of Corollary 3.4
    s = int(np.argmax(g.degrees()))
    x, r = fresh_state(g, s)
    for t in range(100_000):
        before = w @ r
        rr = oracle.localgd_round(g, "katz", beta, 1e-6, x, r)
        if rr.n_active == 0:
            break
        wS = w[rr.active] @ rr.rho
        assert w @ r == pytest.approx(before - (1 - beta * lam) * wS, rel=1e-9, abs=1e-15)
    else:
        pytest.fail("Katz LocalGD did not terminate")


def test_hk_weighted_mass_and_layer_invariant():
    """Layered system: ||x||_1 + sum_k psi_k ||r_k||_1 = psi_0 every round, and
    x + sum_k P_k r_k = sum_{k<=N} tau^k/k! M^k e_s with P_k = sum_j tau^j k!/(k+j)! M^j."""
    g = synth.erdos_renyi(80, 0.06, 7)
    g = synth.from_pairs(g.n, *np.nonzero(np.triu(dense.adjacency(g) + np.eye(g.n, k=1))))
    tau, eps = 3.0, 1e-5
    N = oracle.hk_terms(tau)
    M = dense.walk_matrix(g)
    psi = [oracle.hk_psi(tau, N, k) for k in range(N + 1)]
    s = 0
    x = np.zeros(g.n)
    layers = [np.zeros(g.n) for _ in range(N + 2)]
    layers[0][s] = 1.0
    target = math.exp(tau) * dense.hk_taylor(g, tau, s, N)
    Pk = []
    for k in range(N + 1):
        P = np.zeros((g.n, g.n))
        Mj = np.eye(g.n)
        c = 1.0
        for j in range(0, N - k + 1):
            if j > 0:
                c *= tau / (k + j)
                Mj = M @ Mj
            P += c * Mj
        Pk.append(P)
    for t in range(N + 1):
        rr = oracle.localgd_round(g, "hk", tau, eps, x, layers[t], t=t, r_next=layers[t + 1])
        mass = x.sum() + sum(psi[k] * layers[k].sum() for k in range(N + 1))
        assert mass == pytest.approx(psi[0], rel=1e-12)
        lhs = x + sum(Pk[k] @ layers[k] for k in range(N + 1))
        assert np.allclose(lhs, target, rtol=1e-12, atol=1e-12)
        if rr.n_active == 0:
            break


def test_hk_terms_against_poisson_tail():
    from scipy.stats import poisson
    for tau, want in ((5.0, 27), (10.0, 39)):
        N = oracle.hk_terms(tau, 1e-12)
        assert N == want
        assert poisson.sf(N, tau) <= 1e-12 < poisson.sf(N - 1, tau)
    for tau in (0.5, 1.0, 2.0, 20.0):
        N = oracle.hk_terms(tau, 1e-12)
        assert poisson.sf(N, tau) <= 1.0000001e-12 and poisson.sf(N - 1, tau) > 0.9999999e-12


def test_hk_psi_definition():
    """psi_N = 1, psi_k = 1 + tau/(k+1) psi_{k+1}, and psi_0 = e^tau P(Poisson(tau) <= N)."""
    from scipy.stats import poisson
    tau = 5.0
    N = oracle.hk_terms(tau)
    psi = [oracle.hk_psi(tau, N, k) for k in range(N + 1)]
    assert psi[N] == 1.0
    for k in range(N):
        assert psi[k] == pytest.approx(1 + tau / (k + 1) * psi[k + 1], rel=1e-14)
    assert psi[0] == pytest.approx(math.exp(tau) * poisson.cdf(N, tau), rel=1e-13)
    th = [oracle.hk_theta(tau, N, k, 0) for k in range(N + 1)]
    assert sum(math.exp(-tau) * psi[k] * th[k] for k in range(N + 1)) == pytest.approx(1.0)
    assert oracle.hk_theta(tau, N, 3, 1) == 1.0


# --------------------------------------------------------------- FIFO push ----

@pytest.mark.parametrize("gi", range(8))
def test_fifo_push_bounds(gi):
    """Algo 1 (APPR, FIFO): ||D^-1 (x - f)||_inf <= eps (Theorem 3.3 with omega = 1),
    and it reaches the same f as LocalGD as eps -> 0."""
    g = graphs_small()[gi]
    d = g.degrees()
    s = int(np.argmax(d))
    alpha = 0.15
    f = dense.ppr(g, alpha, s)
    for eps in (1e-3, 1e-6):
        x, pushes, vol = oracle.push_fifo(g, "ppr", alpha, eps, s)
        err = f - x
        assert np.all(err >= -1e-13) and np.all(err < eps * d + 1e-13)
        assert vol <= 1.0 / (alpha * eps)
    x, _, _ = oracle.push_fifo(g, "ppr", alpha, 1e-14, s)
    assert np.allclose(x, f, atol=1e-12)
    # Katz and HK push variants converge to the same vectors
    lam = np.linalg.eigvalsh(dense.adjacency(g))[-1]
    xk, _, _ = oracle.push_fifo(g, "katz", 0.5 / lam, 1e-15, s)
    assert np.allclose(xk, dense.katz(g, 0.5 / lam, s), atol=1e-11)
    xh, _, _ = oracle.push_fifo(g, "hk", 4.0, 1e-15, s)
    assert np.allclose(xh, dense.hk_taylor(g, 4.0, s, oracle.hk_terms(4.0)), atol=1e-12)


def test_many_matches_single():
    g = synth.chung_lu(2000, 8.0, 2.5, seed=8)
    seeds = synth.seeds_quantile(g, 6)
    xs, info = oracle.localgd_many(g, "ppr", 0.15, 1e-6, seeds)
    for i, s in enumerate(seeds):
        one = oracle.localgd(g, "ppr", 0.15, 1e-6, int(s))
        assert np.array_equal(xs[i], one.x)
        assert info[i][0] == one.rounds and info[i][1] == one.volume


def test_topk_order():
    x = np.array([0.1, 0.5, 0.5, 0.0, 0.3])
    ids, vals = oracle.topk(x, 3)
    assert list(ids) == [1, 2, 4] and list(vals) == [0.5, 0.5, 0.3]
