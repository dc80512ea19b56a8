"""Pins of the LocalCH oracle (Section 3.3's local Chebyshev method for PPR, with the updates
of the appendix on implementation details) against what the mathematics fixes:

* every update has the form x += xh_S, r -= Q_w xh_S / alpha (Q_w = I - (1-alpha) A D^-1), so
  Q_w x / alpha + r = e_s holds at exit (dense check);
* it stops with every |r_u| < eps d_u, so |f - x| < eps d against PPR's dense closed form
  (two-sided: LocalCH's residuals change sign);
* its first round is LocalGD's first round (x_s = alpha, r = (1-alpha) A D^-1 e_s);
* on these graphs the momentum takes fewer rounds than LocalGD at small eps.
"""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth

GRAPHS = [
    lambda: synth.erdos_renyi(150, 0.05, seed=3),
    lambda: synth.with_isolated(synth.chung_lu(600, 6.0, 2.5, seed=4), 2),
    lambda: synth.cycle(40),
]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("eps", [1e-5, 1e-7])
def test_invariant_and_bound(gi, eps):
    g = GRAPHS[gi]()
    alpha = 0.1
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    Q = np.eye(g.n) - (1 - alpha) * dense.walk_matrix(g)
    for s in (int(np.argmax(g.degrees())), 0):
        x, r, rounds, vol = oracle.localch(g, alpha, eps, s)
        with np.errstate(invalid="ignore", over="ignore"):  # a planted mistake may diverge
            err = np.max(np.abs(Q @ x / alpha + r - dense.unit(g.n, s)))
        assert err < 1e-12
        assert np.all((np.abs(r) < eps * g.degrees()) | (r == 0))
        f = dense.ppr(g, alpha, s)
        assert np.all(np.abs(f - x) < eps * d)


def test_first_round_is_localgd():
    g = synth.erdos_renyi(100, 0.06, seed=9)
    s = int(np.argmax(g.degrees()))
    x, r, rounds, _ = oracle.localch(g, 0.15, 1e-6, s, max_rounds=1)
    x2 = np.zeros(g.n)
    r2 = np.zeros(g.n)
    r2[s] = 1.0
    oracle.localgd_round(g, "ppr", 0.15, 1e-6, x2, r2)
    assert rounds == 1 and np.array_equal(x, x2) and np.allclose(r, r2, rtol=1e-15, atol=0)


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_fewer_rounds_than_localgd(gi):
    g = GRAPHS[gi]()
    s = int(np.argmax(g.degrees()))
    _, _, ch_rounds, _ = oracle.localch(g, 0.05, 1e-8, s)
    gd = oracle.localgd(g, "ppr", 0.05, 1e-8, s)
    assert ch_rounds < gd.rounds
