"""Serving (gde_server_*): continuous batching of PPR and Katz queries with per-query
tolerance classes on a graph that receives edge-insertion batches (Section 4).

* every answer matches the FP64 oracle within the eps band of its class (Corollary 3.6:
  0 <= f - x < eps d for PPR, plus FP32 rounding);
* each query's answer is the same alone and in a mix of queries that arrive while others
  are on the GPU (within FP32 rounding and the eps band);
* after edge insertions, the warm-started updates of resident queries match the oracle's
  solve on the new graph and, on a small graph, the dense solution of the new system;
* queries wait for a slot when all are taken, and every query is answered.
"""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import synth
from topk_check import check_bands

pytestmark = pytest.mark.gpu

EPS = (1e-5, 1e-6)


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def g0():
    return synth.chung_lu(3000, 10.0, 2.5, seed=31)


def beta_of(g):
    return 0.5 / synth.lambda_max(g)[0]


def check_answer(g, res, xref, eps, slack=1.0):
    """top-k of the device against the oracle's x, each node within its own band
    slack eps d_u + 1e-5 |x_u| (the same check as the batched tests, tests/topk_check.py)"""
    d = g.degrees().astype(np.float64)
    check_bands(res["ids"], res["vals"], xref, slack * eps * d + 1e-5 * np.abs(xref) + 1e-12, len(res["ids"]))


def queries(g, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = synth.seeds_by_degree(g, n, seed=seed)
    kinds = rng.integers(0, 2, size=n)
    cls = rng.integers(0, len(EPS), size=n)
    beta = beta_of(g)
    return [(i, "ppr" if kinds[i] == 0 else "katz", 0.15 if kinds[i] == 0 else beta, int(cls[i]), int(seeds[i]))
            for i in range(n)]


def oracle_x(g, q):
    _, kind, param, cls, s = q
    return oracle.localgd(g, kind, param, EPS[cls], s).x


def test_answers_match_the_oracle(gde, g0):
    G = gde.Graph.from_synth(g0)
    S = gde.Server(G, slots=16, rounds_per_step=3, eps=EPS)
    qs = queries(g0, 40, seed=1)
    for q in qs:
        S.submit(*q)
    out = S.run_until_idle()
    first = {r["qid"]: r for r in out if not r["update"]}
    assert sorted(first) == list(range(40))
    for q in qs:
        r = first[q[0]]
        assert r["status"] == gde.OK
        check_answer(g0, r, oracle_x(g0, q), EPS[q[3]])
        assert r["t_done"] >= r["t_submit"]
    inf = S.info()
    # one-shot queries leave their slots at their answers
    assert inf["running"] == 0 and inf["queued"] == 0 and inf["answered"] == 0
    S.close()


def test_same_alone_and_in_the_mix(gde, g0):
    """A query answered alone (one slot, nothing else) and the same query inside a stream of
    others submitted between steps give the same top-k within FP32 rounding."""
    qs = queries(g0, 48, seed=2)
    G = gde.Graph.from_synth(g0)
    alone = {}
    S1 = gde.Server(G, slots=1, rounds_per_step=2, eps=EPS)
    for q in qs[::6]:
        S1.submit(*q)
        alone[q[0]] = [r for r in S1.run_until_idle() if not r["update"]][0]
    S1.close()
    S = gde.Server(G, slots=12, rounds_per_step=2, eps=EPS)
    mixed = {}
    it = iter(qs)
    pending = True
    while pending or S.info()["running"] or S.info()["queued"]:
        for _ in range(5):  # five arrivals between device steps
            q = next(it, None)
            if q is None:
                pending = False
                break
            S.submit(*q)
        S.step()
        for r in S.poll():
            if not r["update"]:
                mixed[r["qid"]] = r
    S.close()
    assert len(mixed) == len(qs)
    for qid, a in alone.items():
        m = mixed[qid]
        # a query's rounds do not depend on the others in the pool; only the order of its
        # float atomics does, so its answer agrees to FP32 summation rounding
        assert np.allclose(a["vals"], m["vals"], rtol=1e-5, atol=0)
        same = a["ids"] == m["ids"]
        assert np.all(same | np.isclose(a["vals"], m["vals"], rtol=1e-5, atol=0))


@pytest.mark.parametrize("kind", ["ppr", "katz"])
def test_warm_start_after_insertions(gde, g0, kind):
    G = gde.Graph.from_synth(g0)
    S = gde.Server(G, slots=8, rounds_per_step=4, eps=EPS)
    param = 0.15 if kind == "ppr" else beta_of(g0)
    seeds = synth.seeds_quantile(g0, 8)
    for i, s in enumerate(seeds):
        S.submit(i, kind, param, 1, int(s), track=True)
    first = [r for r in S.run_until_idle() if not r["update"]]
    assert S.info()["answered"] == 8  # standing queries stay resident
    assert len(first) == 8
    g = g0
    for b in range(2):  # two batches, applied one after the other
        src, dst = synth.random_edges(g0.n, 400, seed=40 + b)
        S.insert_edges(src, dst)
        g = synth.with_edges(g, src, dst)
        upd = {r["qid"]: r for r in S.run_until_idle() if r["update"]}
        assert sorted(upd) == list(range(8))
        inf = S.info()
        assert inf["edge_batches"] == b + 1
    off, cols = G.csr()
    assert np.array_equal(cols, g.cols)
    d = g.degrees().astype(np.float64)
    for i, s in enumerate(seeds):
        r = upd[i]
        assert r["status"] == gde.OK
        fresh = oracle.localgd(g, kind, param, EPS[1], int(s)).x
        # the warm-started answer and a fresh solve both lie within eps d of the new f
        check_answer(g, r, fresh, EPS[1], slack=2.0)
        if kind == "ppr":
            f = dense.ppr(g, param, int(s))
            ids = r["ids"][r["ids"] >= 0]
            assert np.all(np.abs(r["vals"][: len(ids)] - f[ids]) <= EPS[1] * d[ids] + 1e-5 * f[ids] + 1e-12)
    S.close()


def test_queries_wait_for_slots(gde, g0):
    G = gde.Graph.from_synth(g0)
    S = gde.Server(G, slots=3, rounds_per_step=2, eps=EPS)
    qs = queries(g0, 10, seed=5)
    for q in qs:
        S.submit(*q)
    running, queued = S.step()
    assert running + (10 - queued - running) <= 10 and queued >= 7
    out = S.run_until_idle()
    first = {r["qid"]: r for r in out if not r["update"]}
    assert sorted(first) == list(range(10))
    for q in qs[:4]:
        check_answer(g0, first[q[0]], oracle_x(g0, q), EPS[q[3]])
    S.close()


def test_bad_requests_are_rejected(gde, g0):
    G = gde.Graph.from_synth(g0)
    S = gde.Server(G, slots=2, eps=EPS)
    for args in ((0, "ppr", 1.5, 0, 1), (0, "ppr", 0.15, 2, 1), (0, "ppr", 0.15, 0, g0.n), (0, "hk", 5.0, 0, 1)):
        with pytest.raises(gde.GdeError) as e:
            S.submit(*args)
        assert e.value.status == gde.EINVAL
    with pytest.raises(gde.GdeError):
        S.insert_edges(np.array([0], np.int32), np.array([g0.n], np.int32))
    S.close()


def test_queries_in_flight_are_corrected(gde, g0):
    """Edges inserted while queries are mid-solve: their states are corrected (warm start) and
    their first answers match the oracle on the new graph."""
    G = gde.Graph.from_synth(g0)
    S = gde.Server(G, slots=8, rounds_per_step=1, eps=EPS)
    seeds = synth.seeds_quantile(g0, 8)
    for i, s in enumerate(seeds):
        S.submit(i, "ppr", 0.15, 1, int(s))
    S.step()
    S.step()  # two rounds in: every query still running
    assert S.info()["running"] == 8
    src, dst = synth.random_edges(g0.n, 600, seed=77)
    S.insert_edges(src, dst)
    g1 = synth.with_edges(g0, src, dst)
    first = {r["qid"]: r for r in S.run_until_idle() if not r["update"]}
    assert sorted(first) == list(range(8))
    for i, s in enumerate(seeds):
        fresh = oracle.localgd(g1, "ppr", 0.15, EPS[1], int(s)).x
        check_answer(g1, first[i], fresh, EPS[1], slack=2.0)
    S.close()


def test_submit_and_poll_from_another_thread(gde, g0):
    """submit and poll run on a second host thread while the main thread steps (the C calls
    release the interpreter lock, so they really overlap); every query is answered once."""
    import threading
    G = gde.Graph.from_synth(g0)
    S = gde.Server(G, slots=8, rounds_per_step=2, eps=EPS)
    qs = queries(g0, 60, seed=21)
    got = {}
    stop = threading.Event()

    def producer():
        for q in qs:
            S.submit(*q)
        stop.set()

    def consumer():
        while not (stop.is_set() and len(got) == len(qs)):
            for r in S.poll():
                got.setdefault(r["qid"], r)
            if len(got) == len(qs):
                break

    tp = threading.Thread(target=producer)
    tc = threading.Thread(target=consumer)
    tp.start()
    tc.start()
    for _ in range(100000):
        S.step()
        inf = S.info()
        if stop.is_set() and inf["running"] == 0 and inf["queued"] == 0 and len(got) == len(qs):
            break
    tp.join()
    tc.join(timeout=30)
    assert sorted(got) == list(range(len(qs)))
    for q in qs[::7]:
        check_answer(g0, got[q[0]], oracle_x(g0, q), EPS[q[3]])
    S.close()


@pytest.mark.parametrize("defer", [1, 2000])
def test_deferred_heavy_queries(gde, g0, defer):
    """Queries whose last step pushed more than defer_volume edges run one round per step;
    their answers are those of the oracle, and a deferred query needs more steps, never
    different rounds.  defer_volume = 1 defers every query after its first step."""
    G = gde.Graph.from_synth(g0)
    qs = queries(g0, 24, seed=5)
    S = gde.Server(G, slots=8, rounds_per_step=4, eps=EPS, defer_volume=defer)
    for q in qs:
        S.submit(*q)
    out = S.run_until_idle()
    steps_deferred = S.info()["steps"]
    first = {r["qid"]: r for r in out if not r["update"]}
    assert sorted(first) == list(range(24))
    for q in qs:
        check_answer(g0, first[q[0]], oracle_x(g0, q), EPS[q[3]])
    S.close()
    # the same stream without deferral takes no more steps
    S = gde.Server(G, slots=8, rounds_per_step=4, eps=EPS, defer_volume=-1)
    for q in qs:
        S.submit(*q)
    out2 = S.run_until_idle()
    assert S.info()["steps"] <= steps_deferred
    second = {r["qid"]: r for r in out2 if not r["update"]}
    for q in qs:
        a, b = first[q[0]], second[q[0]]
        # deferral spreads a query's rounds over more steps without changing them
        assert np.allclose(a["vals"], b["vals"], rtol=1e-5, atol=0)
    S.close()


def test_admission_by_memory_and_readmission(gde):
    """A pool of eight 64K-slot pages (20 bytes per slot) on Chung-Lu n = 2^17 (tables of 1, 2
    or 4 pages): queries are admitted while their tables fit, so no more than eight run at
    once whatever the slot count; a Katz query from the largest hub touches more nodes than a
    one-page table holds, overflows and is started again with a table four times larger; every
    answer matches the oracle, and the pool is empty at the end."""
    g = synth.chung_lu(1 << 17, 8.0, 2.3, seed=41)
    d = g.degrees()
    G = gde.Graph.from_synth(g)
    pages = 8
    S = gde.Server(G, slots=64, rounds_per_step=2, eps=(1e-5, 1e-7), mem_budget_bytes=pages * (1 << 16) * 20)
    inf = S.info()
    assert inf["pool_pages"] == pages and inf["page_slots"] == 1 << 16 and inf["cap"] == 1 << 18
    beta = beta_of(g)
    hub = int(np.argmax(d))
    qs = [(0, "katz", beta, 1, hub)]
    seeds = synth.seeds_by_degree(g, 23, seed=42)
    for i, s in enumerate(seeds):
        qs.append((i + 1, "ppr", 0.15, 0, int(s)))
    for q in qs:
        S.submit(*q)
    first, peak = {}, 0
    for _ in range(100000):
        running, queued = S.step()
        inf = S.info()
        peak = max(peak, inf["running"])
        assert inf["pages_used"] <= pages
        for r in S.poll():
            if not r["update"]:
                first[r["qid"]] = r
        if running == 0 and queued == 0:
            break
    inf = S.info()
    assert sorted(first) == list(range(len(qs)))
    assert all(r["status"] == gde.OK for r in first.values())
    assert peak <= pages and inf["peak_resident"] <= pages
    assert inf["readmissions"] >= 1 and inf["pages_used"] == 0
    for q in qs[:6]:
        ref = oracle.localgd(g, q[1], q[2], (1e-5, 1e-7)[q[3]], q[4]).x
        check_answer(g, first[q[0]], ref, (1e-5, 1e-7)[q[3]])
    S.close()
    G.close()
