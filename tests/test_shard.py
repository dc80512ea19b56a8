"""Seed sharding over ranks (one process per GPU, graph replicated): block bounds, and the
2-rank path under torch.distributed.run with the gloo backend on CPU, where each rank solves
its block and the top-k lists are gathered on rank 0 in global seed order."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from paper_2410_21634_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("total,world", [(0, 1), (1, 2), (7, 2), (1024, 8), (1023, 8), (5, 8)])
def test_shard_bounds_partition(total, world):
    blocks = [shard.shard_bounds(total, world, r) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == total
    for (a, b), (c, _) in zip(blocks, blocks[1:]):
        assert b == c  # contiguous, no gap or overlap
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_shard_bounds_rejects_bad_requests():
    for args in ((4, 0, 0), (4, 2, 2), (4, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            shard.shard_bounds(*args)


def test_shard_seeds_is_the_block():
    seeds = np.arange(10, dtype=np.int32)
    assert shard.shard_seeds(seeds, 3, 0).tolist() == [0, 1, 2, 3]
    assert shard.shard_seeds(seeds, 3, 2).tolist() == [7, 8, 9]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_gather(tmp_path):
    out = tmp_path / "gather.json"
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}",
           os.path.join(ROOT, "tests", "gloo_shard_worker.py"), str(out)]
    r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(out.read_text())
    assert res["world"] == 2
    assert res["tmax"] == 20.0 and res["tsum"] == 3.0
    g = synth.chung_lu(2000, 8.0, 2.5, seed=11)
    for name, total in (("seven", 7), ("one", 1)):
        block = res[name]
        seeds = synth.seeds_by_degree(g, total, seed=3)
        assert block["seeds"] == seeds.tolist()
        ids = np.array(block["ids"])
        vals = np.array(block["vals"], dtype=np.float32)
        assert ids.shape == (total, 8)
        for i, s in enumerate(seeds):  # row i is seed i's result, whichever rank solved it
            ref = oracle.localgd(g, "ppr", 0.15, 1e-5, int(s))
            ti, tv = oracle.topk(ref.x, 8)
            assert ids[i, : len(ti)].tolist() == list(ti)
            assert np.array_equal(vals[i, : len(tv)], np.asarray(tv, dtype=np.float32))


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
