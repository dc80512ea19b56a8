"""gde_topk_f32_noalloc: the top-k entry point that allocates no device memory, for
callers that cannot call cudaMalloc (an application whose device memory is all owned by
its own pool, a serving loop that must not take the allocator's lock or its implicit
synchronisation).  Its output must equal the top-k that gde_solve returns for the same
vector, on two calls in a row (the scratch array is shared and reused between calls).

Collected last on purpose (file name), so a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process (the first call on the
device performs the scratch-address set-up).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

K = 64


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
    results = []
    for _ in range(2):
        ids = torch.full((K,), -7, dtype=torch.int32, device="cuda")
        vals = torch.full((K,), -1.0, dtype=torch.float32, device="cuda")
        gde.topk_noalloc(x[0], K, ids, vals)
        torch.cuda.synchronize()
        results.append((ids.cpu().numpy(), vals.cpu().numpy()))
    for ids, vals in results:
        # same tolerance as the FP32 parity tests: 1e-5 relative per value
        assert np.allclose(vals, vals_ref[0], rtol=1e-5, atol=0)
        same = ids == ids_ref[0]
        assert np.all(same | np.isclose(vals, vals_ref[0], rtol=1e-5)), "ids differ beyond near-ties"
        xs = x[0].cpu().numpy()
        assert np.array_equal(xs[ids], vals)
    assert np.array_equal(results[0][0], results[1][0]) and np.array_equal(results[0][1], results[1][1])
    # a short support pads with -1 / 0, and out-of-range k is rejected with a clear error
    small = torch.zeros(100, dtype=torch.float32, device="cuda")
    small[[3, 50, 7]] = torch.tensor([0.5, 0.5, 0.25], device="cuda")
    ids = torch.zeros(8, dtype=torch.int32, device="cuda")
    vals = torch.zeros(8, dtype=torch.float32, device="cuda")
    gde.topk_noalloc(small, 8, ids, vals)
    torch.cuda.synchronize()
    assert ids.cpu().tolist() == [3, 50, 7, -1, -1, -1, -1, -1]
    assert vals.cpu().tolist()[:3] == [0.5, 0.5, 0.25]
    with pytest.raises(gde.GdeError) as e:
        gde.topk_noalloc(small, 65, ids, vals)
    assert e.value.status == gde.EINVAL and "64" in str(e.value)
