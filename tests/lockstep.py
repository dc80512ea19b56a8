"""Round-by-round comparison of the CUDA session with the FP64 oracle.

At each round t the device state (x^t, r^t) is read back, the oracle runs one
round of Eq. (local-gd) from exactly that state (FP32 values are widened exactly
to FP64), the device runs its round, and the two results are compared:
  - S_t identical, except nodes whose residual is within 1 ulp of the threshold;
  - FP64: x^(t+1) and r^(t+1) within 1e-12 relative L1 of the oracle's;
  - FP32: per-entry relative error <= 1e-5 on entries >= eps d_u (x and r), and
    relative L1 <= 1e-5 overall.  Two cases widen r entries that receive k_v > ~160 float
    additions in the round to 2 k_v 2^-24, the error bound of a float sum of k_v positive
    terms: the heat kernel's literal threshold (theta_t = 1, hk_mode 1), where most of the
    graph is active, and Katz, whose share beta r_u has no 1/d_u factor, so a node next to
    many pushed nodes of equal residual adds hundreds of identical terms and round-to-nearest
    drifts with their count instead of averaging out.  The widened entries are counted and
    printed.
"""
from __future__ import annotations

import numpy as np

import oracle

FP64_REL_L1 = 1e-12
FP32_REL = 1e-5


def _rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / den if den > 0 else np.abs(a - b).sum()


def neighbour_counts(g, active):
    """number of nodes of `active` adjacent to every node (the additions into r_v this round)"""
    active = np.asarray(active, dtype=np.int64)
    beg = g.offsets[active]
    ln = g.offsets[active + 1] - beg
    tot = int(ln.sum())
    if tot == 0:
        return np.zeros(g.n, dtype=np.int64)
    # positions beg[i] .. beg[i] + ln[i] - 1 of every active row, concatenated
    first = np.repeat(beg - np.concatenate(([0], np.cumsum(ln)[:-1])), ln)
    return np.bincount(g.cols[first + np.arange(tot)], minlength=g.n)


def contributions(g, active, kind, t, N):
    """number of pushed neighbours of every node in this round (the additions into r_v)"""
    if kind == "hk" and t >= N:
        return np.zeros(g.n, dtype=np.int64)
    return neighbour_counts(g, active)


def near_threshold(r, thr):
    """nodes within one ulp of their threshold"""
    return np.abs(r - thr) <= np.spacing(np.maximum(thr, np.finfo(np.float64).tiny))


def run(G, g, kind, param, eps, seed, precision="fp64", hk_mode=0, max_rounds=100000,
        check_every=1, katz_minus_source=0):
    """katz_minus_source=1 (Katz): the device reads back f_Katz = x - e_s, its source entry
    from the engine's FP64 source word; the oracle runs on x = f + e_s, and the source entry
    f_s is compared on its own at 1e-5 relative every round (it is small, so the eps d_u mask
    of the other entries would skip it)."""
    import paper_2410_21634_gb300 as gde
    S = gde.Session(G, kind, param, eps, seed, precision=precision, hk_threshold=hk_mode,
                    katz_minus_source=katz_minus_source)
    d = g.degrees().astype(np.float64)
    x, r, _ = S.read()
    t = 0
    history = []
    N = oracle.hk_terms(param) if kind == "hk" else None
    widen = (kind == "hk" and hk_mode == 1) or kind == "katz"
    widened = 0
    try:
        while t < max_rounds:
            xo = x.astype(np.float64)
            if katz_minus_source:
                xo[seed] += 1.0  # the engine's x_s = 1 + f_s
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
            if katz_minus_source:
                xo[seed] -= 1.0  # compare f = x - e_s
                if xo[seed] != 0.0:
                    rel_s = abs(xd[seed] - xo[seed]) / abs(xo[seed])
                    assert rel_s <= FP32_REL, f"round {t}: source entry f_s rel {rel_s:.3g}"
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
                    rel = np.abs(rd - r_or) / np.where(r_or != 0, np.abs(r_or), 1.0)
                    if widen:
                        # a float sum of k_v positive terms is within k_v 2^-24 of the exact
                        # sum; 1e-5 covers up to ~160 contributions, above that the bound rules
                        k_v = contributions(g, rr.active, kind, t, N) + 1
                        tol = np.maximum(FP32_REL, 2.0 * k_v * 2.0 ** -24)
                        widened += int((big & (rel > FP32_REL)).sum())
                    else:
                        k_v = np.zeros(g.n, dtype=np.int64)
                        tol = FP32_REL
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
    if widen:
        print(f"\nlock-step {kind} {precision}: {widened} r entries above 1e-5 within the summation bound")
    return history, x, r


def _oracle_round(g, kind, param, eps, xo, ro, t, hk_mode, coef):
    """one oracle round in place; returns (RoundResult, r_next or None, theta_t eps, theta_t+1 eps)"""
    if kind == "series":
        rn = np.zeros(g.n)
        N = len(coef) - 1
        et = oracle.series_theta(coef, min(t, N), hk_mode) * eps
        en = oracle.series_theta(coef, min(t + 1, N), hk_mode) * eps
        return oracle.series_round(g, coef, t, eps, xo, ro, rn, mode=hk_mode), rn, et, en
    if kind == "hk":
        rn = np.zeros(g.n)
        N = oracle.hk_terms(param)
        et = oracle.hk_theta(param, N, min(t, N), hk_mode) * eps
        en = oracle.hk_theta(param, N, min(t + 1, N), hk_mode) * eps
        return oracle.localgd_round(g, kind, param, eps, xo, ro, t=t, r_next=rn, hk_mode=hk_mode), rn, et, en
    return oracle.localgd_round(g, kind, param, eps, xo, ro, t=t), None, eps, eps


def run_batched(G, g, kind, param, eps, seeds, hk_mode=0, coef=None, widen=False, max_rounds=100000,
                katz_minus_source=0, mem_budget_bytes=0):
    """Lock-step comparison of the batched FP32 engine (every seed of the batch advanced by one
    persistent launch per round) with the FP64 oracle.  At every round t and for every seed j:
    the device state (x^t, r^t) of seed j is widened exactly to FP64, the oracle runs round t
    from it, the device runs round t of all seeds, and
      - the nodes the device pushed equal the oracle's S_t, except nodes within one ulp of
        their threshold (then the round's values are not compared: the two pushed different
        sets);
      - every entry of x^(t+1) and r^(t+1) with |value| >= eps d_u is within 1e-5 relative of
        the oracle's (widen=True: r entries that receive k_v > ~160 float additions get
        2 k_v 2^-24, the summation bound of a float sum);
      - x and r are within 1e-5 relative L1.
    Returns a report: rounds, compared entries, worst relative errors, widened entries and
    rounds skipped for near-threshold differences."""
    import paper_2410_21634_gb300 as gde
    kw = {"hk_threshold": hk_mode, "katz_minus_source": katz_minus_source}
    if mem_budget_bytes:
        kw["mem_budget_bytes"] = int(mem_budget_bytes)
    if coef is not None:
        kw["series_coef"] = np.asarray(coef, dtype=np.float64)
    S = gde.BatchSession(G, kind, param, eps, seeds, **kw)
    d = g.degrees().astype(np.float64)
    ed = eps * d
    ns = len(seeds)
    state = [S.read(j)[:2] for j in range(ns)]
    rep = {"rounds": 0, "entries": 0, "max_rel_r": 0.0, "max_rel_x": 0.0, "widened": 0, "skipped": 0,
           "pushes": 0}
    oracle_kind = "series" if kind == "series" else kind
    layered = kind in ("hk", "series")
    N = (len(coef) - 1) if kind == "series" else (oracle.hk_terms(param) if kind == "hk" else None)
    t = 0
    try:
        while t < max_rounds:
            pre = []
            for j in range(ns):
                x, r = state[j]
                xo = x.astype(np.float64)
                if katz_minus_source:
                    xo[seeds[j]] += 1.0  # the engine's x_s = 1 + f_s
                ro = r.astype(np.float64)
                r0 = ro.copy()
                rr, rn, et, en = _oracle_round(g, oracle_kind, param, eps, xo, ro, t, hk_mode, coef)
                if katz_minus_source:
                    xo[seeds[j]] -= 1.0
                pre.append((xo, rn if layered else ro, rr, r0, et * d))
            ncand = S.step()
            for j in range(ns):
                x, r, pushed = S.read(j)
                state[j] = (x, r)
                xo, r_or, rr, r0, thr = pre[j]
                if not np.array_equal(pushed, rr.active):
                    diff = np.setxor1d(pushed, rr.active)
                    assert np.all(near_threshold(r0[diff], thr[diff])), \
                        f"seed {j} round {t}: pushed sets differ at {diff[:10]}"
                    rep["skipped"] += 1
                    continue
                rep["pushes"] += len(pushed)
                xd = x.astype(np.float64)
                rd = r.astype(np.float64)
                if katz_minus_source and xo[seeds[j]] != 0.0:
                    sj = seeds[j]
                    rel_s = abs(xd[sj] - xo[sj]) / abs(xo[sj])
                    assert rel_s <= FP32_REL, f"seed {j} round {t}: source entry f_s rel {rel_s:.3g}"
                    rep["max_rel_source"] = max(rep.get("max_rel_source", 0.0), rel_s)
                big = (np.abs(r_or) >= ed) & (r_or != 0)
                if big.any():
                    rel = np.abs(rd[big] - r_or[big]) / np.abs(r_or[big])
                    tol = np.full(rel.shape, FP32_REL)
                    if widen:
                        k_v = np.zeros(g.n, dtype=np.int64)
                        if not (layered and t >= N):
                            k_v = neighbour_counts(g, rr.active)
                        tol = np.maximum(tol, 2.0 * (k_v[big] + 1) * 2.0 ** -24)
                        rep["widened"] += int((rel > FP32_REL).sum())
                    bad = rel > tol
                    assert not bad.any(), \
                        f"seed {j} round {t}: r per-entry rel {rel.max():.3g} at node {np.flatnonzero(big)[rel.argmax()]}"
                    rep["max_rel_r"] = max(rep["max_rel_r"], float(rel.max()))
                    rep["entries"] += int(big.sum())
                bigx = (np.abs(xo) >= ed) & (xo != 0)
                if bigx.any():
                    relx = np.abs(xd[bigx] - xo[bigx]) / np.abs(xo[bigx])
                    assert relx.max() <= FP32_REL, f"seed {j} round {t}: x per-entry rel {relx.max():.3g}"
                    rep["max_rel_x"] = max(rep["max_rel_x"], float(relx.max()))
                    rep["entries"] += int(bigx.sum())
                ex, er = _rel_l1(xd, xo), _rel_l1(rd, r_or)
                assert ex <= FP32_REL and er <= FP32_REL, f"seed {j} round {t}: rel L1 {ex:.3g} {er:.3g}"
            t += 1
            rep["rounds"] = t
            if ncand == 0:
                # no candidate left: the oracle finds no active node in any seed's final state
                if not (layered and t > N):
                    for j in range(ns):
                        x, r = state[j]
                        xo, ro = x.astype(np.float64), r.astype(np.float64)
                        if katz_minus_source:
                            xo[seeds[j]] += 1.0
                        r0 = ro.copy()
                        rr, _, et, _ = _oracle_round(g, oracle_kind, param, eps, xo, ro, t, hk_mode, coef)
                        assert rr.n_active == 0 or np.all(near_threshold(r0[rr.active], et * d[rr.active])), \
                            f"seed {j}: the device stopped with active nodes {rr.active[:10]}"
                break
    finally:
        S.close()
    return rep
