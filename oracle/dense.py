"""ORACLE — test infrastructure only.  Dense closed-form diffusion vectors for tiny
graphs (n up to a few thousand), from the definitions of Section 2 / Table 1 of
arXiv 2410.21634:

  PPR   f = alpha (I - (1-alpha) A D^-1)^-1 e_s                  (Eq. f-ppr)
  Katz  x = (I - beta A)^-1 e_s,  f_Katz = x - e_s                (Eq. f-katz)
  HK    f = exp(-tau (I - A D^-1)) e_s, and its Taylor truncation
        e^-tau sum_{k<=N} tau^k/k! (A D^-1)^k e_s                (Section 2, heat kernel)

Columns of A D^-1 that belong to degree-0 nodes are zero.
"""
from __future__ import annotations

import math

import numpy as np


def adjacency(g) -> np.ndarray:
    A = np.zeros((g.n, g.n), dtype=np.float64)
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    A[rows, g.cols] = 1.0
    return A


def walk_matrix(g) -> np.ndarray:
    """M = A D^-1 (column u scaled by 1/d_u; zero column when d_u = 0)."""
    A = adjacency(g)
    d = np.diff(g.offsets).astype(np.float64)
    inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    return A * inv[None, :]


def unit(n: int, s: int) -> np.ndarray:
    e = np.zeros(n, dtype=np.float64)
    e[s] = 1.0
    return e


def ppr_system(g, alpha: float) -> np.ndarray:
    """Q = I - (1-alpha) A D^-1"""
    return np.eye(g.n) - (1.0 - alpha) * walk_matrix(g)


def ppr(g, alpha: float, s: int) -> np.ndarray:
    return alpha * np.linalg.solve(ppr_system(g, alpha), unit(g.n, s))


def katz_system(g, beta: float) -> np.ndarray:
    """Q = I - beta A"""
    return np.eye(g.n) - beta * adjacency(g)


def katz(g, beta: float, s: int) -> np.ndarray:
    """x = (I - beta A)^-1 e_s  (the Katz vector is x - e_s)"""
    return np.linalg.solve(katz_system(g, beta), unit(g.n, s))


def hk_taylor(g, tau: float, s: int, N: int) -> np.ndarray:
    """e^-tau sum_{k=0}^{N} tau^k/k! M^k e_s"""
    M = walk_matrix(g)
    v = unit(g.n, s)
    acc = v.copy()
    for k in range(1, N + 1):
        v = (tau / k) * (M @ v)
        acc += v
    return math.exp(-tau) * acc


def hk_exact(g, tau: float, s: int) -> np.ndarray:
    """exp(-tau (I - M)) e_s by scipy's matrix exponential."""
    from scipy.linalg import expm
    M = walk_matrix(g)
    return expm(-tau * (np.eye(g.n) - M)) @ unit(g.n, s)


def gppr_matrix(g, beta: float) -> np.ndarray:
    """M = D^-beta A D^(beta-1) (the generalised propagation of the InstantGNN push; zero
    columns and rows at degree-0 nodes)."""
    A = adjacency(g)
    d = np.diff(g.offsets).astype(np.float64)
    nz = d > 0
    left = np.where(nz, np.power(np.where(nz, d, 1.0), -beta), 0.0)
    right = np.where(nz, np.power(np.where(nz, d, 1.0), beta - 1.0), 0.0)
    return left[:, None] * A * right[None, :]


def gppr(g, alpha: float, beta: float, s: int) -> np.ndarray:
    """f = alpha (I - (1-alpha) M)^-1 e_s = sum_k alpha (1-alpha)^k M^k e_s."""
    M = gppr_matrix(g, beta)
    return alpha * np.linalg.solve(np.eye(g.n) - (1.0 - alpha) * M, unit(g.n, s))


def series(g, coef, s: int) -> np.ndarray:
    """sum_{k<=N} coef[k] (A D^-1)^k e_s"""
    M = walk_matrix(g)
    v = unit(g.n, s)
    f = np.zeros(g.n)
    for c in coef:
        f += c * v
        v = M @ v
    return f
