"""Round-by-round comparison of the CUDA session with the FP64 oracle.

At each round t the device state (x^t, r^t) is read back, the oracle runs one
round of Eq. (local-gd) from exactly that state (FP32 values are widened exactly
to FP64), the device runs its round, and the two results are compared:
  - S_t identical, except nodes whose residual is within 1 ulp of the threshold;
  - FP64: x^(t+1) and r^(t+1) within 1e-12 relative L1 of the oracle's;
  - FP32: per-entry relative error <= 1e-5 on entries >= eps d_u (x and r), widened
    to 2 k_v 2^-24 for entries that receive k_v > ~160 float additions in the round
    (the summation error bound), and relative L1 <= 1e-5 overall.
"""
from __future__ import annotations

import numpy as np

import oracle

FP64_REL_L1 = 1e-12
FP32_REL = 1e-5


def _rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / den if den > 0 else np.abs(a - b).sum()


def contributions(g, active, kind, t, N):
    """number of pushed neighbours of every node in this round (the additions into r_v)"""
    k = np.zeros(g.n, dtype=np.int64)
    if kind == "hk" and t >= N:
        return k
    for u in active:
        k[g.cols[g.offsets[u]:g.offsets[u + 1]]] += 1
    return k


def near_threshold(r, thr):
    """nodes within one ulp of their threshold"""
    return np.abs(r - thr) <= np.spacing(np.maximum(thr, np.finfo(np.float64).tiny))


def run(G, g, kind, param, eps, seed, precision="fp64", hk_mode=0, max_rounds=100000,
        check_every=1):
    import paper_2410_21634_gb300 as gde
    S = gde.Session(G, kind, param, eps, seed, precision=precision, hk_threshold=hk_mode)
    d = g.degrees().astype(np.float64)
    x, r, _ = S.read()
    t = 0
    history = []
    N = oracle.hk_terms(param) if kind == "hk" else None
    try:
        while t < max_rounds:
            xo = x.astype(np.float64)
            ro = r.astype(np.float64)
            rn = np.zeros(g.n) if kind == "hk" else None
            if kind == "hk":
                eps_theta = oracle.hk_theta(param, N, t, hk_mode) * eps
            else:
                eps_theta = eps
            thr = eps_theta * d
            pre_r = ro.copy()
            rr = oracle.localgd_round(g, kind, param, eps, xo, ro, t=t, r_next=rn, hk_mode=hk_mode)
            k = S.step()
            x, r, act = S.read()
            # active sets
            a_dev = np.sort(act)
            if not np.array_equal(a_dev, rr.active):
                diff = np.setxor1d(a_dev, rr.active)
                assert np.all(near_threshold(pre_r[diff], thr[diff])), \
                    f"round {t}: active sets differ at {diff[:10]}"
            assert k == len(act)
            if rr.n_active == 0 or k == 0:
                assert k == 0 or np.all(near_threshold(pre_r[a_dev], thr[a_dev]))
                break
            r_or = rn if kind == "hk" else ro
            xd = x.astype(np.float64)
            rd = r.astype(np.float64)
            if precision == "fp64":
                ex, er = _rel_l1(xd, xo), _rel_l1(rd, r_or)
                assert ex <= FP64_REL_L1, f"round {t}: x rel L1 {ex}"
                assert er <= FP64_REL_L1, f"round {t}: r rel L1 {er}"
            else:
                if kind == "hk":
                    thr_next = oracle.hk_theta(param, N, t + 1, hk_mode) * eps * d if t + 1 <= N else thr
                else:
                    thr_next = thr
                big = (np.abs(r_or) >= thr_next) & (r_or != 0)
                if big.any():
                    # a float sum of k_v positive terms is within (k_v) 2^-24 of the exact sum;
                    # 1e-5 covers up to ~160 contributions, above that the summation bound rules
                    k_v = contributions(g, rr.active, kind, t, N) + 1
                    tol = np.maximum(FP32_REL, 2.0 * k_v * 2.0 ** -24)
                    rel = np.abs(rd - r_or) / np.where(r_or != 0, np.abs(r_or), 1.0)
                    bad = big & (rel > tol)
                    assert not bad.any(), f"round {t}: r per-entry rel {rel[bad].max()} (k_v {k_v[bad].max()})"
                bigx = (np.abs(xo) >= thr) & (xo != 0)
                if bigx.any():
                    relx = np.abs(xd[bigx] - xo[bigx]) / np.abs(xo[bigx])
                    assert relx.max() <= FP32_REL, f"round {t}: x per-entry rel {relx.max()}"
                ex, er = _rel_l1(xd, xo), _rel_l1(rd, r_or)
                assert ex <= FP32_REL and er <= FP32_REL, f"round {t}: rel L1 {ex} {er}"
            history.append((rr.n_active, rr.vol_active, rr.rS_l1))
            t += 1
    finally:
        S.close()
    return history, x, r
