"""Pins of the generalised-propagation oracle (M = D^-beta A D^(beta-1), the InstantGNN push
of the appendix; beta = 1/2 is APPNP's D^-1/2 A D^-1/2 of Table 1) against what the
mathematics fixes:

* beta = 0 is PPR: the same rounds, bit for bit;
* the dense solution f = alpha (I - (1-alpha) M)^-1 e_s: LocalGD ends with 0 <= f - x and
  (f - x)_u < eps d_u^(1-beta) (the PPR bound carried through the similarity
  M = D^-beta (A D^-1) D^beta, residual y = D^beta r);
* every round keeps the invariant Q x / alpha + r = e_s with Q = I - (1-alpha) M;
* a star, solved by hand, with eps between the two thresholds a wrong exponent would give.
"""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth

GRAPHS = [
    lambda: synth.erdos_renyi(90, 0.07, seed=3),
    lambda: synth.with_isolated(synth.erdos_renyi(60, 0.1, seed=8), 3),
    lambda: synth.star(7),
    lambda: synth.chung_lu(300, 6.0, 2.5, seed=4),
]


def test_beta_zero_is_ppr_bitwise():
    g = synth.chung_lu(2000, 8.0, 2.5, seed=9)
    for s in synth.seeds_quantile(g, 4):
        x, rounds, vol, pushes, _ = oracle.gppr(g, 0.15, 0.0, 1e-6, int(s))
        ref = oracle.localgd(g, "ppr", 0.15, 1e-6, int(s))
        assert np.array_equal(x, ref.x)
        assert rounds == ref.rounds and vol == ref.volume and pushes == ref.pushes


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("beta", [0.25, 0.5, 1.0])
def test_error_bound_against_dense(gi, beta):
    g = GRAPHS[gi]()
    d = g.degrees().astype(np.float64)
    eps = 1e-6
    for s in (int(np.argmax(d)), int(synth.seeds_quantile(g, 4)[1])):
        x, *_ = oracle.gppr(g, 0.15, beta, eps, s)
        f = dense.gppr(g, 0.15, beta, s)
        err = f - x
        assert err.min() >= -1e-15
        bound = eps * np.where(d > 0, d, 1.0) ** (1.0 - beta)
        assert np.all(err < bound)


@pytest.mark.parametrize("beta", [0.25, 0.5])
def test_round_invariant(beta):
    g = synth.erdos_renyi(70, 0.08, seed=12)
    alpha = 0.2
    Q = np.eye(g.n) - (1 - alpha) * dense.gppr_matrix(g, beta)
    s = 3
    x = np.zeros(g.n)
    r = np.zeros(g.n)
    r[s] = 1.0
    for _ in range(200):
        rr = oracle.gppr_round(g, alpha, beta, 1e-7, x, r)
        assert np.max(np.abs(Q @ x / alpha + r - dense.unit(g.n, s))) < 1e-13
        if rr.n_active == 0:
            break
    assert rr.n_active == 0


def test_star_by_hand():
    """Star of 16 leaves, seed at the centre, alpha 0.2, beta 0.25, eps 0.09:
    round 0 pushes the centre (x_c = 0.2; each leaf gets 0.8 / 16^0.75 = 0.1 >= eps);
    round 1 pushes the leaves (x_leaf = 0.02; the centre gets 16 * 0.8 * 0.1 / 16^0.25 =
    0.64); round 2 finds the centre below its threshold 0.09 * 16^0.75 = 0.72 and stops."""
    g = synth.star(16)
    x = np.zeros(g.n)
    r = np.zeros(g.n)
    r[0] = 1.0
    rr = oracle.gppr_round(g, 0.2, 0.25, 0.09, x, r)
    assert list(rr.active) == [0] and x[0] == pytest.approx(0.2, abs=1e-15)
    assert np.allclose(r[1:], 0.1, rtol=1e-14)
    rr = oracle.gppr_round(g, 0.2, 0.25, 0.09, x, r)
    assert list(rr.active) == list(range(1, 17))
    assert np.allclose(x[1:], 0.02, rtol=1e-14) and r[0] == pytest.approx(0.64, rel=1e-14)
    rr = oracle.gppr_round(g, 0.2, 0.25, 0.09, x, r)
    assert rr.n_active == 0
    xs, rounds, *_ = oracle.gppr(g, 0.2, 0.25, 0.09, 0)
    assert rounds == 2 and np.allclose(xs, x, rtol=1e-15)
