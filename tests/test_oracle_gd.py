"""Pins of the standard (global) GD oracle, the counterpart LocalGD is compared with in
Section 5 (Table 2's operation ratio, Figure 6's running times):

* it stops with ||D^-1 r||_inf < eps, so PPR's bound 0 <= f - x < eps d holds against the
  dense closed form, and Katz's x stays below (I - beta A)^-1 e_s;
* on a 2-node edge and on a star from its centre the residual alternates between the two
  sides, so the iteration count has a closed form: the first t with (1-alpha)^t / k < eps
  (k = the centre's degree; k = 1 for the edge).
"""
import math

import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth


@pytest.mark.parametrize("g", [synth.erdos_renyi(150, 0.05, seed=2), synth.with_isolated(synth.star(9), 2),
                               synth.chung_lu(400, 6.0, 2.5, seed=7)], ids=["er", "star+iso", "cl"])
def test_ppr_bound(g):
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    for s in (int(np.argmax(g.degrees())), 1):
        x, it = oracle.global_gd(g, "ppr", 0.15, 1e-6, s)
        f = dense.ppr(g, 0.15, s)
        assert it > 0 and (f - x).min() >= -1e-15 and np.all(f - x < 1e-6 * d)


def test_katz_below_the_solution():
    g = synth.erdos_renyi(120, 0.06, seed=4)
    beta = 0.5 / synth.lambda_max(g)[0]
    x, it = oracle.global_gd(g, "katz", beta, 1e-8, 3)
    f = dense.katz(g, beta, 3)
    assert (f - x).min() >= -1e-14 and np.max(f - x) < 1e-5


@pytest.mark.parametrize("k,alpha,eps", [(1, 0.2, 1e-4), (8, 0.2, 3e-5), (20, 0.1, 1e-6)])
def test_iteration_count_closed_form(k, alpha, eps):
    g = synth.edge2() if k == 1 else synth.star(k)
    # the smallest t with (1-alpha)^t / k < eps, away from rounding ties
    t = math.ceil(math.log(eps * k) / math.log(1 - alpha))
    assert abs(math.log(eps * k) / math.log(1 - alpha) - round(math.log(eps * k) / math.log(1 - alpha))) > 1e-6
    x, it = oracle.global_gd(g, "ppr", alpha, eps, 0)
    assert it == t
