"""Failure detection without a GPU fault.

(a) Grid-barrier timeout: the persistent round kernel's waits are bounded; a test sets a short
limit and lets one block leave at a barrier without arriving (as a block that died would).
The other blocks give up, the solve returns GDE_ETIMEOUT within the limit, writes no output,
and the next solve on the same graph (pool cleared) is correct.

(b) Allocation failure: the host-side injector makes the k-th device allocation fail as an
out-of-memory cudaMalloc would.  Every call that meets it returns GDE_ENOMEM, writes no output
and leaks nothing that breaks later calls; with the injector disarmed the same graph solves
correctly.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from test_gpu_batched import check_topk

pytestmark = pytest.mark.gpu

K = 16


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    yield m
    m.test_fail_alloc(0)


@pytest.fixture(scope="module")
def c1():
    return synth.workload_graph("chung_lu_1e4")


def _batched(gde, G, seeds, kind="ppr", param=0.15, **kw):
    ids = np.full((len(seeds), K), -7, dtype=np.int32)
    vals = np.full((len(seeds), K), -1.0, dtype=np.float32)
    st, stats = gde.solve(G, kind, param, 1e-6, seeds, vals, ids, precision="fp32", topk=K, batched=1, **kw)
    return st, ids, vals


def _check_answers(g, seeds, ids, vals, kind="ppr", param=0.15):
    for i in (0, len(seeds) - 1):
        ref = oracle.localgd(g, kind, param, 1e-6, int(seeds[i]))
        check_topk(g, ids[i], vals[i], ref.x, 1e-6, k=K)


@pytest.mark.parametrize("barrier", [0, 1, 3])
def test_barrier_timeout(gde, c1, barrier):
    seeds = synth.seeds_by_degree(c1, 12, seed=8)
    G = gde.Graph.from_synth(c1)
    st, ids, vals = _batched(gde, G, seeds)  # a good solve first: the pool is in use
    assert st == gde.OK
    G.test_barrier_fault(limit_ns=50_000_000, block=5, barrier=barrier)
    ids = np.full((len(seeds), K), -7, dtype=np.int32)
    vals = np.full((len(seeds), K), -1.0, dtype=np.float32)
    t0 = time.perf_counter()
    with pytest.raises(gde.GdeError) as e:
        gde.solve(G, "ppr", 0.15, 1e-6, seeds, vals, ids, precision="fp32", topk=K, batched=1)
    dt = time.perf_counter() - t0
    assert e.value.status == gde.ETIMEOUT and "timed out" in str(e.value)
    assert dt < 5.0
    assert np.all(ids == -7) and np.all(vals == -1.0), "output written on failure"
    # the same graph, fault off: the next solve clears the pool and is correct
    G.test_barrier_fault(block=-1)
    st, ids, vals = _batched(gde, G, seeds)
    assert st == gde.OK
    _check_answers(c1, seeds, ids, vals)
    G.close()


def test_barrier_timeout_in_a_session_and_a_server(gde, c1):
    G = gde.Graph.from_synth(c1)
    G.test_barrier_fault(limit_ns=50_000_000, block=0, barrier=0)
    S = gde.BatchSession(G, "ppr", 0.15, 1e-6, synth.seeds_by_degree(c1, 4, seed=2))
    with pytest.raises(gde.GdeError) as e:
        S.step()
    assert e.value.status == gde.ETIMEOUT
    S.close()
    srv = gde.Server(G, slots=4, rounds_per_step=2, eps=(1e-6,))
    srv.submit(1, "ppr", 0.15, 0, 7)
    with pytest.raises(gde.GdeError) as e:
        srv.step()
    assert e.value.status == gde.ETIMEOUT
    srv.close()
    G.test_barrier_fault(block=-1)
    seeds = synth.seeds_by_degree(c1, 6, seed=3)
    st, ids, vals = _batched(gde, G, seeds)
    assert st == gde.OK
    _check_answers(c1, seeds, ids, vals)
    G.close()


@pytest.mark.parametrize("nth", [1, 2, 3, 5, 8, 13, 21, 34])
def test_injected_allocation_failure_batched(gde, c1, nth):
    """The first batched solve on a fresh graph allocates its workspace, tables, hub slab and
    staging buffers: the nth of those allocations fails."""
    seeds = synth.seeds_mixed(c1, 4, 4, seed=5)
    G = gde.Graph.from_synth(c1)
    gde.test_fail_alloc(nth)
    ids = np.full((len(seeds), K), -7, dtype=np.int32)
    vals = np.full((len(seeds), K), -1.0, dtype=np.float32)
    try:
        st, _ = gde.solve(G, "ppr", 0.15, 1e-6, seeds, vals, ids, precision="fp32", topk=K, batched=1)
        failed = False
    except gde.GdeError as e:
        failed = True
        assert e.status == gde.ENOMEM and "injected" in str(e)
        assert np.all(ids == -7) and np.all(vals == -1.0), "output written on failure"
    finally:
        gde.test_fail_alloc(0)
    if not failed:
        # fewer than nth allocations: the solve did not meet the failure
        assert st == gde.OK
    st, ids, vals = _batched(gde, G, seeds)
    assert st == gde.OK
    _check_answers(c1, seeds, ids, vals)
    G.close()


@pytest.mark.parametrize("nth", [1, 2, 3, 4])
def test_injected_allocation_failure_graph_plain_and_server(gde, c1, nth):
    # graph creation
    gde.test_fail_alloc(nth)
    try:
        with pytest.raises(gde.GdeError) as e:
            gde.Graph.from_synth(c1)
        assert e.value.status == gde.ENOMEM
    finally:
        gde.test_fail_alloc(0)
    G = gde.Graph.from_synth(c1)
    s = np.array([int(synth.seeds_by_degree(c1, 1, seed=4)[0])], dtype=np.int32)
    # the plain engine's first solve (dense workspace)
    out = np.full((1, c1.n), -1.0)
    gde.test_fail_alloc(nth)
    try:
        with pytest.raises(gde.GdeError) as e:
            gde.solve(G, "ppr", 0.15, 1e-6, s, out)
        assert e.value.status == gde.ENOMEM
        assert np.all(out == -1.0)
    finally:
        gde.test_fail_alloc(0)
    st, _ = gde.solve(G, "ppr", 0.15, 1e-6, s, out)
    assert st == gde.OK
    ref = oracle.localgd(c1, "ppr", 0.15, 1e-6, int(s[0]))
    assert np.abs(out[0] - ref.x).sum() <= 1e-9 * np.abs(ref.x).sum()
    # a server
    gde.test_fail_alloc(nth)
    try:
        with pytest.raises(gde.GdeError) as e:
            gde.Server(G, slots=4, rounds_per_step=2, eps=(1e-6,))
        assert e.value.status == gde.ENOMEM
    finally:
        gde.test_fail_alloc(0)
    srv = gde.Server(G, slots=4, rounds_per_step=2, eps=(1e-6,))
    srv.submit(1, "ppr", 0.15, 0, int(s[0]))
    res = [r for r in srv.run_until_idle() if not r["update"]]
    assert len(res) == 1 and res[0]["status"] == gde.OK
    check_topk(c1, res[0]["ids"][:K], res[0]["vals"][:K], ref.x, 1e-6, k=K)
    srv.close()
    G.close()


def test_injector_arguments(gde):
    with pytest.raises(gde.GdeError) as e:
        gde.test_fail_alloc(-1)
    assert e.value.status == gde.EINVAL
    gde.test_fail_alloc(0)
