"""Pins of the general power-series oracle (f = sum_{k<=N} c_k (A D^-1)^k e_s, the layered
system of Section 2 with layer ratio c_{t+1}/c_t; Table 1's IPR coefficients as the new
case) against what the mathematics fixes:

* with the heat kernel's coefficients c_k = e^-tau tau^k / k! it is the heat-kernel oracle;
* with PPR's c_k = alpha (1-alpha)^k (truncated where the tail is 1e-12) it lands inside the
  eps bound of PPR's dense closed form;
* with IPR's c_k = theta^k / (theta^k + theta^10)^2 it ends inside 0 <= f_N - c_0 x <= eps d_u
  of the dense truncated series (theta_t = 1/((N+1) c_0 psi_t)), and below f_N with the
  literal threshold.
"""
import math

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


def truncate(c, rel=1e-12):
    c = np.asarray(c, dtype=np.float64)
    tail = np.cumsum(c[::-1])[::-1]
    n = int(np.argmax(tail <= rel * c.sum()))
    return c[: max(n, 1) + 1]


def ipr_coef(theta):
    k = np.arange(0, 400, dtype=np.float64)
    return truncate(theta ** k / (theta ** k + theta ** 10) ** 2)


def test_heat_kernel_coefficients_give_the_heat_kernel():
    g = synth.chung_lu(800, 6.0, 2.5, seed=2)
    tau = 5.0
    N = oracle.hk_terms(tau)
    c = [math.exp(-tau)]
    for k in range(N):
        c.append(c[-1] * tau / (k + 1))
    for s in synth.seeds_quantile(g, 3):
        a = oracle.series(g, c, 1e-6, int(s))
        b = oracle.localgd(g, "hk", tau, 1e-6, int(s))
        assert a.rounds == b.rounds
        assert np.abs(a.x - b.x).sum() <= 1e-13 * np.abs(b.x).sum()


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_ppr_coefficients_reach_ppr(gi):
    g = GRAPHS[gi]()
    alpha, eps = 0.2, 1e-6
    c = truncate(alpha * (1 - alpha) ** np.arange(0, 400, dtype=np.float64))
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    s = int(np.argmax(g.degrees()))
    r = oracle.series(g, c, eps, s)
    f = dense.ppr(g, alpha, s)
    assert np.all(f - r.x >= -1e-12) and np.all(f - r.x <= eps * d + 1e-11)


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("theta", [1.3, 2.0])
def test_ipr_bound_against_dense(gi, theta):
    g = GRAPHS[gi]()
    c = ipr_coef(theta)
    d = np.maximum(g.degrees().astype(np.float64), 1.0)
    eps = 1e-3 * c[0]  # tolerance of the size of the series' own scale
    for s in (int(np.argmax(g.degrees())), int(synth.seeds_quantile(g, 4)[1])):
        f = dense.series(g, c, s)
        r = oracle.series(g, c, eps, s)
        err = f - r.x
        assert err.min() >= -1e-15 * c.sum()
        assert np.all(err <= eps * d * (1 + 1e-12))
        lit = oracle.series(g, c, eps, s, mode=1)
        assert (f - lit.x).min() >= -1e-15 * c.sum()


def test_ipr_threshold_scale_is_below_one():
    """theta_t = 1/((N+1) c_0 psi_t) makes the layers' tests stricter than eps d_u where a unit
    of residual still carries much of the series (psi large) and looser at the tail."""
    c = ipr_coef(1.5)
    th = [oracle.series_theta(c, t) for t in range(len(c))]
    assert all(t > 0 for t in th)
    assert oracle.series_theta(c, 0, mode=1) == 1.0
