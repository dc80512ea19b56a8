"""One rank of the seed-sharding check (launched by test_shard.py under torch.distributed.run,
gloo backend, CPU only).  Each rank takes its block of a global seed list, computes the top-k
of its seeds with the FP64 oracle (standing in for the device solve), and the blocks are
gathered on rank 0, which writes them to the JSON file named on the command line."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2410_21634_gb300 import shard  # noqa: E402

K = 8


def block_topk(g, seeds):
    ids = np.full((len(seeds), K), -1, np.int32)
    vals = np.zeros((len(seeds), K), np.float32)
    for i, s in enumerate(seeds):
        ref = oracle.localgd(g, "ppr", 0.15, 1e-5, int(s))
        ti, tv = oracle.topk(ref.x, K)
        ids[i, : len(ti)] = ti
        vals[i, : len(tv)] = tv
    return torch.from_numpy(ids), torch.from_numpy(vals)


def main(out):
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    g = synth.chung_lu(2000, 8.0, 2.5, seed=11)
    result = {"world": world}
    for name, total in (("seven", 7), ("one", 1)):  # ragged blocks; an empty block on rank 1
        seeds = synth.seeds_by_degree(g, total, seed=3)
        mine = shard.shard_seeds(seeds, world, rank)
        ids, vals = block_topk(g, mine)
        got = shard.gather_topk(ids, vals, len(seeds))
        if rank == 0:
            result[name] = {"seeds": seeds.tolist(), "ids": got[0].tolist(), "vals": got[1].tolist()}
    result["tmax"] = shard.max_over_ranks(10.0 * (rank + 1))
    result["tsum"] = shard.sum_over_ranks(float(rank + 1))
    if rank == 0:
        with open(out, "w") as f:
            json.dump(result, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1])
