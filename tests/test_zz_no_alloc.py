"""gde_topk_f32_noalloc: the top-k entry point that allocates no device memory, for
callers that cannot call cudaMalloc (an application whose device memory is all owned by
its own pool, a serving loop that must not take the allocator's lock or its implicit
synchronisation).  Its output must equal the top-k that gde_solve returns for the same
vector, and the exact ranking (value descending, ties by lower id) computed on the host from
the same vector, on two calls in a row (the scratch array is shared and reused between
calls).

Collected last on purpose (file name), so a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process (the first call on the
device performs the scratch-address set-up).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

K = 64


def _two_calls(gde, x, k):
    import torch
    out = []
    for _ in range(2):
        ids = torch.full((k,), -7, dtype=torch.int32, device=x.device)
        vals = torch.full((k,), -1.0, dtype=torch.float32, device=x.device)
        gde.topk_noalloc(x, k, ids, vals)
        torch.cuda.synchronize()
        out.append((ids.cpu().numpy(), vals.cpu().numpy()))
    return out


def _host_ranking(xs, k):
    """exact top-k of the positive entries on the host: value descending, ties by lower id"""
    ids, vals = oracle.topk(xs.astype(np.float64), k)
    keep = vals > 0
    out_ids = np.full(k, -1, dtype=np.int32)
    out_vals = np.zeros(k, dtype=np.float32)
    out_ids[: keep.sum()] = ids[keep]
    out_vals[: keep.sum()] = xs[ids[keep]]
    return out_ids, out_vals


def test_noalloc_topk_matches_solve_topk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as gde
    g = synth.workload_graph("chung_lu_1e4")
    G = gde.Graph.from_synth(g)
    seed = synth.seeds_by_degree(g, 1, seed=3)
    # the existing entry point: a dense FP32 solve with top-k output
    ids_ref = np.zeros((1, K), dtype=np.int32)
    vals_ref = np.zeros((1, K), dtype=np.float32)
    gde.solve(G, "ppr", 0.15, 1e-6, seed, vals_ref, ids_ref, precision="fp32", topk=K)
    # the same solve with the dense vector as output, ranked by the no-allocation entry point
    x = torch.zeros((1, g.n), dtype=torch.float32, device="cuda")
    gde.solve(G, "ppr", 0.15, 1e-6, torch.from_numpy(seed).cuda(), x, precision="fp32")
    torch.cuda.synchronize()
    xs = x[0].cpu().numpy()
    host_ids, host_vals = _host_ranking(xs, K)
    results = _two_calls(gde, x[0], K)
    for ids, vals in results:
        # the exact host ranking of the same vector: ids and values equal
        assert np.array_equal(ids, host_ids), "ids differ from the host ranking"
        assert np.array_equal(vals, host_vals)
        # the existing entry point, a separate solve: same tolerance as the FP32 parity
        # tests, 1e-5 relative per value (its float atomics may add in another order)
        assert np.allclose(vals, vals_ref[0], rtol=1e-5, atol=0)
    assert np.array_equal(results[0][0], results[1][0]) and np.array_equal(results[0][1], results[1][1])
    G.close()


def test_noalloc_topk_large_vector_with_ties_across_blocks():
    """n = 3e6 takes the 512 partial lists of the scratch (each list ranks 5,860 entries);
    equal values planted on both sides of list boundaries must come out by lower id."""
    import torch
    import paper_2410_21634_gb300 as gde
    n = 3_000_000
    rng = np.random.Generator(np.random.PCG64(23))
    xs = rng.random(n, dtype=np.float32) * 0.5 + 0.25
    xs[rng.random(n) < 0.3] = 0.0          # zeros are never ranked
    per = (n + 511) // 512                 # entries per partial list
    top = np.float32(0.99)
    for b in (1, 7, 100, 511):
        xs[b * per - 3: b * per + 3] = top  # six-way ties straddling a list boundary
    xs[[5, n - 1]] = np.float32(0.995)
    x = torch.from_numpy(xs).cuda()
    host_ids, host_vals = _host_ranking(xs, K)
    assert np.sum(host_vals == top) == 24
    for ids, vals in _two_calls(gde, x, K):
        assert np.array_equal(ids, host_ids)
        assert np.array_equal(vals, host_vals)


def test_noalloc_topk_short_support_and_bad_k():
    import torch
    import paper_2410_21634_gb300 as gde
    small = torch.zeros(100, dtype=torch.float32, device="cuda")
    small[[3, 50, 7]] = torch.tensor([0.5, 0.5, 0.25], device="cuda")
    ids = torch.zeros(8, dtype=torch.int32, device="cuda")
    vals = torch.zeros(8, dtype=torch.float32, device="cuda")
    gde.topk_noalloc(small, 8, ids, vals)
    torch.cuda.synchronize()
    assert ids.cpu().tolist() == [3, 50, 7, -1, -1, -1, -1, -1]
    assert vals.cpu().tolist() == [0.5, 0.5, 0.25, 0.0, 0.0, 0.0, 0.0, 0.0]
    # k beyond the scratch's 64 keys per list: a clear error from the entry point
    big_ids = torch.zeros(65, dtype=torch.int32, device="cuda")
    big_vals = torch.zeros(65, dtype=torch.float32, device="cuda")
    with pytest.raises(gde.GdeError) as e:
        gde.topk_noalloc(small, 65, big_ids, big_vals)
    assert e.value.status == gde.EINVAL and "64" in str(e.value)
