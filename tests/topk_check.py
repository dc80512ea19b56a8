"""Checks of a device top-k list against the oracle's x with a band per node.

A free-running FP32 solve and the FP64 oracle both satisfy the method's error bound, but they
may push different near-threshold nodes, so each node u has its own band b_u (for LocalGD
b_u = eps d_u plus FP32 rounding, from 0 <= f_u - x_u < eps d_u, Corollary 3.6).  With every
device value inside its node's band, the i-th largest device value lies between the i-th
largest of x - b and of x + b over all nodes, and a node that fewer than k others can
overtake within their bands is in every valid top-k list.
"""
import numpy as np

import oracle


def check_bands(ids, vals, xref, b, k):
    valid = ids >= 0
    ids_v = ids[valid]
    vals_v = vals[valid].astype(np.float64)
    assert np.all(valid[: len(ids_v)]), "-1 padding before a listed id"
    assert np.all(np.diff(vals_v) <= 0), "values not descending"
    assert len(set(ids_v.tolist())) == len(ids_v), "an id is listed twice"
    assert np.all(np.abs(vals_v - xref[ids_v]) <= b[ids_v]), \
        f"value outside its node's band by {np.max(np.abs(vals_v - xref[ids_v]) - b[ids_v]):.3g}"
    m = len(ids_v)
    if m == 0:
        return
    hi = np.sort(-np.partition(-(xref + b), m - 1)[:m])[::-1]
    lo = np.sort(-np.partition(-(xref - b), m - 1)[:m])[::-1]
    assert np.all(vals_v <= hi) and np.all(vals_v >= lo), "ranking outside the per-node bands"
    if m == k:
        ub = np.sort(xref + b)
        ref_ids, _ = oracle.topk(xref, k)
        listed = set(ids_v.tolist())
        for u in ref_ids.tolist():
            others = ub.size - np.searchsorted(ub, xref[u] - b[u], side="left") - 1
            if others < k:
                assert u in listed, f"node {u} is surely in the top {k} but not listed"
