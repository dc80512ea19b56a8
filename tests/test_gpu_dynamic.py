"""Edge insertion into the device CSR (gde_update_edges, the dynamic graphs of Section 4):
the rebuilt CSR equals the host-built union of the old graph and the batch (sorted,
deduplicated, self-loops dropped) entry for entry, and solves on the updated graph match the
FP64 oracle on that union."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


def batch_with_edge_cases(g, m, seed):
    src, dst = synth.random_edges(g.n, m, seed)
    # a self-loop, an edge already present, the same new edge twice in both orientations
    u = int(np.argmax(g.degrees()))
    present = int(g.cols[g.offsets[u]])
    extra_s = np.array([5, u, 7, 9], dtype=np.int32)
    extra_d = np.array([5, present, 9, 7], dtype=np.int32)
    return np.concatenate([src, extra_s]), np.concatenate([dst, extra_d])


@pytest.mark.parametrize("name,m", [("chung_lu_1e4", 500), ("rmat16", 20000)])
def test_csr_after_insertions_equals_host_union(gde, name, m):
    g = synth.workload_graph(name) if name != "rmat16" else synth.rmat(16, 16, seed=21)
    G = gde.Graph.from_synth(g)
    ref = g
    for b in range(3):  # three batches in a row
        src, dst = batch_with_edge_cases(ref, m, seed=100 + b)
        added = G.update_edges(src, dst)
        new = synth.with_edges(ref, src, dst)
        assert added == new.nnz - ref.nnz
        off, cols = G.csr()
        assert np.array_equal(off, new.offsets)
        assert np.array_equal(cols, new.cols)
        inf = G.info()
        assert inf["nnz"] == new.nnz and inf["max_degree"] == int(new.degrees().max())
        ref = new


def test_device_pointer_batch_and_empty_batches(gde):
    import torch
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    src, dst = synth.random_edges(g.n, 300, seed=9)
    added = G.update_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    new = synth.with_edges(g, src, dst)
    off, cols = G.csr()
    assert added == new.nnz - g.nnz and np.array_equal(cols, new.cols)
    assert G.update_edges(np.zeros(0, np.int32), np.zeros(0, np.int32)) == 0
    assert G.update_edges(np.array([3], np.int32), np.array([3], np.int32)) == 0  # a self-loop only
    off2, cols2 = G.csr()
    assert np.array_equal(off2, off) and np.array_equal(cols2, cols)


def test_bad_endpoint_leaves_the_graph_unchanged(gde):
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    with pytest.raises(gde.GdeError) as e:
        G.update_edges(np.array([1, 2], np.int32), np.array([4, g.n], np.int32))
    assert e.value.status == gde.EINVAL
    off, cols = G.csr()
    assert np.array_equal(off, g.offsets) and np.array_equal(cols, g.cols)


@pytest.mark.parametrize("kind", ["ppr", "katz", "hk"])
def test_plain_fp64_solve_after_insertions(gde, kind):
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    # solve once first, so cached workspaces exist and must follow the change
    seeds = synth.seeds_quantile(g, 4)
    out = np.zeros((4, g.n))
    gde.solve(G, "ppr", 0.15, 1e-6, seeds, out)
    src, dst = synth.random_edges(g.n, 2000, seed=4)
    G.update_edges(src, dst)
    g1 = synth.with_edges(g, src, dst)
    param = {"ppr": 0.15, "hk": 5.0}.get(kind)
    if kind == "katz":
        param = 0.5 / synth.lambda_max(g1)[0]
    st, stats = gde.solve(G, kind, param, 1e-6, seeds, out)
    assert st == gde.OK
    for i, s in enumerate(seeds):
        ref = oracle.localgd(g1, kind, param, 1e-6, int(s))
        assert np.abs(out[i] - ref.x).sum() <= 1e-9 * np.abs(ref.x).sum()
        assert stats[i]["active_volume"] == pytest.approx(ref.volume, rel=1e-6, abs=64)


def test_batched_solve_after_insertions(gde):
    g = synth.rmat(16, 16, seed=21)
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_mixed(g, 16, 16, seed=3)
    ids = np.zeros((32, 64), np.int32)
    vals = np.zeros((32, 64), np.float32)
    gde.solve(G, "ppr", 0.1, 1e-6, seeds, vals, ids, precision="fp32", topk=64, batched=1)
    src, dst = synth.random_edges(g.n, 30000, seed=8)
    G.update_edges(src, dst)
    g1 = synth.with_edges(g, src, dst)
    st, stats = gde.solve(G, "ppr", 0.1, 1e-6, seeds, vals, ids, precision="fp32", topk=64, batched=1)
    assert st == gde.OK
    xs, info = oracle.localgd_many(g1, "ppr", 0.1, 1e-6, seeds[::5])
    d = g1.degrees().astype(float)
    for n, i in enumerate(range(0, 32, 5)):
        valid = ids[i] >= 0
        band = 1e-6 * d[ids[i][valid]] + 1e-5 * xs[n][ids[i][valid]] + 1e-12
        assert np.all(np.abs(vals[i][valid] - xs[n][ids[i][valid]]) <= band)


def test_packed_columns_carried_through_insertions(gde):
    """On a graph verified symmetric the batched engine's packed columns (node id plus the
    neighbour's degree code) are shifted with the CSR and patched where a degree code changed,
    instead of being rebuilt.  Several batches, one of which pushes the largest hub past the
    next power of two (a change of its logarithmic code), must give the same answers as a
    graph built from scratch on the union, and as the oracle."""
    g = synth.rmat(16, 16, seed=21)
    G = gde.Graph.from_synth(g, check_symmetric=True)
    seeds = synth.seeds_mixed(g, 16, 16, seed=3)
    k = 64
    ids = np.zeros((32, k), np.int32)
    vals = np.zeros((32, k), np.float32)
    gde.solve(G, "ppr", 0.1, 1e-6, seeds, vals, ids, precision="fp32", topk=k, batched=1)  # packs
    d = g.degrees()
    hub = int(np.argmax(d))
    need = (1 << int(np.floor(np.log2(d[hub])) + 1)) - int(d[hub]) + 3
    nbr = set(g.cols[g.offsets[hub]:g.offsets[hub + 1]].tolist()) | {hub}
    fresh = np.array([v for v in range(g.n) if v not in nbr][:need], dtype=np.int32)
    batches = [synth.random_edges(g.n, 5000, seed=40 + b) for b in range(3)]
    batches.insert(1, (np.full(fresh.shape, hub, np.int32), fresh))
    g1 = g
    for src, dst in batches:
        G.update_edges(src, dst)
        g1 = synth.with_edges(g1, src, dst)
        st, _ = gde.solve(G, "ppr", 0.1, 1e-6, seeds, vals, ids, precision="fp32", topk=k, batched=1)
        assert st == gde.OK
    assert g1.degrees()[hub] >= 1 << (int(np.floor(np.log2(d[hub]))) + 1)
    F = gde.Graph.from_synth(g1)
    ids2 = np.zeros_like(ids)
    vals2 = np.zeros_like(vals)
    st, _ = gde.solve(F, "ppr", 0.1, 1e-6, seeds, vals2, ids2, precision="fp32", topk=k, batched=1)
    assert st == gde.OK
    d1 = g1.degrees().astype(float)
    xs, _ = oracle.localgd_many(g1, "ppr", 0.1, 1e-6, seeds)
    for i in range(32):
        for I, V in ((ids[i], vals[i]), (ids2[i], vals2[i])):
            valid = I >= 0
            band = 1e-6 * d1[I[valid]] + 1e-5 * xs[i][I[valid]] + 1e-12
            assert np.all(np.abs(V[valid] - xs[i][I[valid]]) <= band)
        # the two graphs agree on the leaders up to FP32 summation order
        assert np.allclose(vals[i], vals2[i], rtol=1e-4, atol=1e-6 * d1.max())
    F.close()
    G.close()
