#!/usr/bin/env python3
"""Benchmark: batched FP32 LocalGD on R-MAT scale 24 (GTEPS and seeds/s at eps=1e-7).

One step = one batched solve of the whole hot path (seed init, every LocalGD round of
every seed in one persistent launch, per-seed top-64) for 1024 PPR sources (512 uniform
+ 512 top-1% hubs), alpha=0.1, eps=1e-7, on the synthetic R-MAT 24 graph (edge factor
16, symmetrised, deduplicated).  Reports seeds/s (value), GTEPS, the plain FP64
one-seed-per-launch path on the same GPU, the roofline of the persistent round kernel,
an end-to-end figure through host buffers, and the FP64 oracle on the host's cores.  Then,
as "serving", it measures the serving workload (Chung-Lu 2^23, PPR/Katz queries arriving
at 2,000/s with eps in {1e-5, 1e-6, 1e-7}, 10,000 random edges inserted every 50 ms):
p50/p99 latency and throughput of the continuous-batching server.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--serve-seconds S]

Under torchrun (N > 1) every rank solves its own 1024 seeds on a replica of the graph
(seed sharding, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GTEPS & seeds/s at eps=1e-7, % HBM peak; batched FP32 vs plain FP64 on same GPU"
ALPHA, EPS, TOPK = 0.1, 1e-7, 64
# algorithmic bytes of the persistent round kernel (FP32 hash accumulators), the method's own
# traffic: sum over rounds of |S_t| B_node + vol(S_t) B_edge + |C_t| B_cand
# per pushed edge: column id 4 + the 8-byte slot word read and its residual written back 4
BYTES_PER_EDGE = 16
# per pushed node: row offsets 16 + frontier record written and read 2 x 12 + x read and
# written 8 + residual zeroed 8 + candidate entry 4 + its append 4
BYTES_PER_PUSH = 64
# per candidate test: its slot word 8 + row offsets 16
BYTES_PER_CAND = 24
# the kernel's own finer model (threshold reads per edge, the degree-bin entries written and
# read by the seed-ordered placement), reported beside it
KERNEL_BYTES_PER_EDGE, KERNEL_BYTES_PER_PUSH = 20, 88


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gde", choices=["gde", "reference"])
    ap.add_argument("--graph", default="rmat24", help="named synthetic workload graph")
    ap.add_argument("--seeds", type=int, default=1024)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default tuning")
    ap.add_argument("--hub-degree", type=int, default=0,
                    help="batched hub-slab degree threshold (0: the library default, -1: no slab)")
    ap.add_argument("--tuning", default="",
                    help='launch shape as JSON, e.g. {"t1": 32, "t2": 128, "chunk": 512, "schedule": 4, '
                         '"hub_degree": 64} (applied before any autotuning)')
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="hash accumulator budget (0: the library default)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="seconds of the serving stream measured after the batched bench (0: skip)")
    ap.add_argument("--no-gd", action="store_true", help="skip the global GD vs LocalGD comparison")
    ap.add_argument("--no-c2", action="store_true",
                    help="skip the plain FP64 sweep on R-MAT 22 (PPR, Katz, heat kernel over eps)")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the FP32-vs-FP64 precision comparison on Chung-Lu 2^24")
    ap.add_argument("--no-kinds", action="store_true", help="skip the batched heat-kernel line")
    ap.add_argument("--no-random-probe", action="store_true",
                    help="skip the random-access calibration of device memory")
    ap.add_argument("--random-probe", action="store_true",
                    help="only run the random-access calibration and print its JSON line")
    ap.add_argument("--serving-only", action="store_true",
                    help="only run the serving workload (--serve-seconds of arrivals) and print its JSON line")
    ap.add_argument("--probe-gb", type=float, default=16.0, help="buffer of the random-access calibration")
    ap.add_argument("--probe-l2-fetch", type=int, default=0,
                    help="L2 fetch-granularity limit during the calibration (0: leave it alone)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_inputs(graph_name, nseeds, rank):
    import synth
    t0 = time.time()
    g = synth.workload_graph(graph_name)
    half = nseeds // 2
    seeds = synth.seeds_mixed(g, nseeds - half, half, seed=4 + 1000 * rank)
    log(f"[bench] graph {g.summary()} generated in {time.time() - t0:.1f}s")
    return g, seeds


def workload_config(g, nseeds, n_gpus):
    return {
        "workload": f"batched PPR top-{TOPK}, R-MAT scale 24 (edge factor 16, a=0.57 b=0.19 c=0.19, "
                    f"symmetrised, deduplicated, int32 CSR), {nseeds} seeds/GPU (half uniform, "
                    f"half top-1% degree), alpha={ALPHA}, eps={EPS}, FP32 hash accumulators"
                    if g.name == "rmat24" else f"batched PPR top-{TOPK} on {g.name}, {nseeds} seeds",
        "graph": g.name, "n": int(g.n), "nnz": int(g.nnz), "max_degree": int(g.degrees().max()),
        "seeds_per_gpu": nseeds, "alpha": ALPHA, "eps": EPS, "topk": TOPK,
        "global_batch": nseeds * n_gpus,
        "parallelism": f"seed-sharded replicas x{n_gpus}",
        "l2": "inputs larger than L2: CSR 2.1 GB read in place, accumulator pool rewritten every step",
    }


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline(g, seeds, budget_s=12.0):
    """The FP64 oracle (as it stands) on a bounded sample of the same seed mix, one seed per
    host thread."""
    import numpy as np

    import oracle
    import synth
    cores = synth.num_threads()
    half = len(seeds) // 2
    # equal numbers of uniform and hub seeds, one round of `cores` seeds first to size the sample
    k = max(2, cores)
    pick = np.concatenate([seeds[: k // 2], seeds[half: half + k - k // 2]])
    t0 = time.time()
    oracle.localgd_many(g, "ppr", ALPHA, EPS, pick)
    dt = time.time() - t0
    reps = max(1, min(8, int(budget_s / max(dt, 1e-3))))
    if reps > 1:
        pick2 = np.concatenate([seeds[: reps * k // 2], seeds[half: half + reps * (k - k // 2)]])
        t0 = time.time()
        oracle.localgd_many(g, "ppr", ALPHA, EPS, pick2)
        dt = time.time() - t0
        pick = pick2
    return {"value": len(pick) / dt, "unit": "seeds/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(pick)} of the {len(seeds)} seeds ({len(pick) // 2} uniform + "
                      f"{len(pick) - len(pick) // 2} hubs), FP64 LocalGD oracle, one seed per thread, "
                      f"{dt:.1f}s wall"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    g, seeds = make_inputs(args.graph, args.seeds, 0)
    import numpy as np

    import oracle
    import synth
    cores = synth.num_threads()
    k = max(2, cores)
    half = len(seeds) // 2
    per_step = np.concatenate([seeds[: k // 2], seeds[half: half + k - k // 2]])
    for _ in range(args.warmup):
        oracle.localgd_many(g, "ppr", ALPHA, EPS, per_step[: max(2, k // 4)])
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        oracle.localgd_many(g, "ppr", ALPHA, EPS, per_step)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = len(per_step) * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "seeds/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(g, args.seeds, args.gpus),
        "cpu_baseline": {"value": value, "unit": "seeds/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step {len(per_step)} of the {len(seeds)} seeds (half uniform, "
                                   f"half hubs), FP64 LocalGD oracle, one seed per host thread"},
        "e2e": {"value": value, "unit": "seeds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


SERVE_SLOTS, SERVE_ROUNDS_PER_STEP = 256, 4
SERVE = {"graph": "chung_lu_2p23", "rate_qps": 2000.0, "batch_edges": 10000, "batch_period_s": 0.05,
         "eps": (1e-5, 1e-6, 1e-7), "alpha": 0.15}


def run_serving(gde, seconds, slots, rounds_per_step, g=None, beta=None, budget_gb=0.0, trace=None,
                defer_volume=0):
    """The serving workload: PPR (alpha 0.15) and Katz (beta = 0.5 / lambda_max) queries
    arriving as a Poisson stream at 2,000/s with eps drawn from {1e-5, 1e-6, 1e-7}, while
    batches of 10,000 uniformly random edges are inserted every 50 ms, on Chung-Lu n=2^23
    (mean degree 16, exponent 2.3).  Latency = answer time - scheduled arrival time, first
    answers only; updates of resident queries after each batch are counted separately."""
    import numpy as np

    import synth
    if g is None:
        g = synth.workload_graph(SERVE["graph"])
    if beta is None:
        beta = 0.5 / synth.lambda_max(g)[0]
    G = gde.Graph.from_synth(g, check_symmetric=True)  # lets insertions keep the packed columns
    # the table pool: 2^31 table slots at 20 bytes (40 GB); queries take power-of-two runs of
    # 64K-slot pages as they are admitted, up to 2n slots each
    budget = int(budget_gb * (1 << 30)) if budget_gb > 0 else (1 << 31) * 20
    S = gde.Server(G, slots=slots, rounds_per_step=rounds_per_step, eps=SERVE["eps"], mem_budget_bytes=budget,
                   defer_volume=defer_volume)
    arrivals = synth.poisson_arrivals(SERVE["rate_qps"], seconds, seed=7)
    nq = len(arrivals)
    rng = np.random.Generator(np.random.PCG64(11))
    kinds = rng.integers(0, 2, size=nq)
    cls = rng.integers(0, len(SERVE["eps"]), size=nq)
    seeds = synth.seeds_by_degree(g, nq, seed=13)
    nb = int(round(seconds / SERVE["batch_period_s"]))
    batches = [synth.random_edges(g.n, SERVE["batch_edges"], seed=1000 + b) for b in range(nb)]

    def params(i):
        return ("ppr", SERVE["alpha"]) if kinds[i] == 0 else ("katz", beta)

    # warm-up outside the timed stream (first launches, thresholds, packed columns), which also
    # leaves `standing` tracked queries resident: they are corrected and re-answered after
    # every edge batch, and their update latency is reported apart from the stream's
    standing = 16
    for i in range(standing):
        k, p = params(i)
        S.submit(10**9 + i, k, p, int(cls[i]), int(seeds[i]), track=True)
    S.run_until_idle()
    clock = gde.server_clock
    t0 = clock()
    qi = bi = steps = failed = 0
    lat, vol, upd_lat = [], 0, []
    while True:
        now = clock() - t0
        while qi < nq and arrivals[qi] <= now:
            k, p = params(qi)
            S.submit(qi, k, p, int(cls[qi]), int(seeds[qi]), t_submit=t0 + float(arrivals[qi]))
            qi += 1
        while bi < nb and (bi + 1) * SERVE["batch_period_s"] <= now:
            S.insert_edges(*batches[bi])
            bi += 1
        ts = clock()
        running, queued = S.step()
        steps += 1
        if trace is not None:
            inf = S.info()
            trace.append((ts - t0, clock() - ts, inf["rounds"], inf["volume"], running, queued, bi))
        for r in S.poll():
            if r["qid"] >= 10**9:
                if r["update"] and r["status"] == gde.OK:
                    upd_lat.append(r["t_done"] - r["t_submit"])
                continue
            if r["status"] != gde.OK:
                failed += 1
            else:
                lat.append(r["t_done"] - r["t_submit"])
                vol += r["volume"]
        if qi == nq and bi == nb and running == 0 and queued == 0:
            break
        if now > 20 * seconds + 30:
            break
    elapsed = clock() - t0
    info = S.info()
    S.close()
    G.close()
    lat = np.sort(np.array(lat)) * 1e3
    return {
        "workload": f"Chung-Lu n=2^23 (mean degree 16, exponent 2.3), Poisson queries at "
                    f"{SERVE['rate_qps']:.0f}/s (PPR alpha={SERVE['alpha']} / Katz beta=0.5/lambda_max, "
                    f"eps in {list(SERVE['eps'])}), {SERVE['batch_edges']} random edges inserted every "
                    f"{SERVE['batch_period_s'] * 1e3:.0f} ms, {seconds:g} s of arrivals",
        "queries": nq, "answered": int(lat.size), "failed": failed,
        "standing_queries": standing, "standing_updates": len(upd_lat),
        "standing_update_p50_ms": float(np.percentile(upd_lat, 50) * 1e3) if upd_lat else None,
        "standing_update_p99_ms": float(np.percentile(upd_lat, 99) * 1e3) if upd_lat else None,
        "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_ms": float(lat.mean()) if lat.size else None,
        "throughput_qps": lat.size / elapsed, "offered_qps": SERVE["rate_qps"],
        "elapsed_s": elapsed, "edge_batches": info["edge_batches"], "steps": steps,
        "rounds": info["rounds"], "slots": slots, "rounds_per_step": rounds_per_step,
        "defer_volume": defer_volume if defer_volume != 0 else 1 << 23,
        "admission": {"budget_gb": round(budget / 2**30, 1), "pool_pages": info["pool_pages"],
                      "page_slots": info["page_slots"], "largest_table_slots": info["cap"],
                      "peak_resident_queries": info["peak_resident"],
                      "peak_gb_in_tables": round(info["peak_pages"] * info["page_slots"] * 20 / 2**30, 2),
                      "readmissions": info["readmissions"],
                      "evictions": info["evictions"], "slots": slots},
        "pushed_edges": info["volume"],
        "step_seconds": {k: round(info[k], 4) for k in ("t_graph", "t_correct", "t_admit", "t_rounds", "t_results")}, "pushed_edges_first_answers": int(vol),
    }


def run_batched_kinds(gde, G, g, seeds_np, dev, sample=32):
    """The batched engine on the other kinds of the paper, on the benchmark's graph and seeds:
    Katz (beta = 0.5 / lambda_max, eps = 1e-7) and the heat kernel (tau = 5, Taylor layers,
    eps = 1e-6), both with 64 GB of tables (a Katz hub seed and the first heat-kernel layers
    touch more nodes than PPR).  Each kind runs on a graph object of its own, autotuned for
    that kind first (the launch shape that suits PPR does not suit the layered heat kernel).
    Each row: batched FP32 seeds/s and GTEPS (CUDA events around 3 solves after one warm-up),
    and the plain FP64 one-seed-per-launch path on `sample` of the seeds (half uniform, half
    hubs)."""
    import numpy as np
    import torch

    import synth
    rows = []
    lam, _ = synth.lambda_max(g, rel_tol=1e-4, max_iter=200)
    nseeds = len(seeds_np)
    seeds = torch.from_numpy(seeds_np).to(dev)
    ids = torch.zeros((nseeds, TOPK), dtype=torch.int32, device=dev)
    vals = torch.zeros((nseeds, TOPK), dtype=torch.float32, device=dev)
    for kind, param, eps, budget_gb in (("katz", 0.5 / lam, 1e-7, 64.0), ("hk", 5.0, 1e-6, 64.0)):
        budget = int(budget_gb * (1 << 30))
        Gk = gde.Graph.from_synth(g)
        tuning, _ = Gk.autotune(kind, param, eps, seeds, topk=TOPK, mem_budget_bytes=budget)

        def solve():
            return gde.solve(Gk, kind, param, eps, seeds, vals, ids, precision="fp32", topk=TOPK, batched=1,
                             mem_budget_bytes=budget)
        solve()
        torch.cuda.synchronize()
        Gk.profile_enable(True)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 3
        for _ in range(reps):
            st, stats = solve()
        e1.record(stream)
        torch.cuda.synchronize()
        prof = Gk.profile_read()
        Gk.profile_enable(False)
        sec = e0.elapsed_time(e1) / 1e3 / reps
        overflow = sum(1 for x in stats if x["fallback"])
        half = nseeds // 2
        smp = np.concatenate([seeds_np[: sample // 2], seeds_np[half: half + sample // 2]])
        out = torch.zeros((1, g.n), dtype=torch.float64, device=dev)
        gde.solve(Gk, kind, param, eps, torch.tensor([int(smp[0])], dtype=torch.int32, device=dev), out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sd in smp:
            gde.solve(Gk, kind, param, eps, torch.tensor([int(sd)], dtype=torch.int32, device=dev), out)
        torch.cuda.synchronize()
        plain = len(smp) / (time.perf_counter() - t0)
        rows.append({"kind": kind, "param": param, "eps": eps, "seeds": nseeds, "budget_gb": budget_gb,
                     "batched_fp32_seeds_per_s": nseeds / sec, "ms_per_solve": sec * 1e3,
                     "gteps": prof["edges"] / reps / sec / 1e9, "fallback_seeds": overflow,
                     "plain_fp64_seeds_per_s": plain, "plain_sample": len(smp),
                     "speedup_vs_plain_fp64": nseeds / sec / plain,
                     "tuning": {k: v for k, v in tuning.items() if k != "blocks_per_sm" or v}})
        Gk.close()
    return {"graph": g.name, "lambda_max": lam, "rows": rows}


def run_gd_compare(gde, g=None):
    """Global GD vs LocalGD (Section 5: Table 2's operation ratio, Figure 6's running time as a
    function of eps), with LocalCH beside them, on R-MAT scale 22, PPR alpha=0.1, plain FP64,
    one seed per solve, 8 seeds at degree quantiles; operation counts are iterations x nnz
    (GD) and sum_t vol(S_t) (LocalGD, LocalCH)."""
    import numpy as np
    import torch

    import synth
    if g is None:
        g = synth.workload_graph("rmat22")
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_quantile(g, 8)
    out = torch.zeros((1, g.n), dtype=torch.float64, device="cuda")
    rows = []
    for eps in (1e-4, 1e-5, 1e-6, 1e-7):
        res = {}
        for name, kw in (("localgd", {}), ("gd", {"global_gd": 1}), ("localch", {"chebyshev": 1})):
            gde.solve(G, "ppr", 0.1, eps, torch.tensor(seeds[:1], dtype=torch.int32, device="cuda"), out, **kw)
            torch.cuda.synchronize()
            ops = 0
            t0 = time.perf_counter()
            for s in seeds:
                _, st = gde.solve(G, "ppr", 0.1, eps, torch.tensor([s], dtype=torch.int32, device="cuda"), out, **kw)
                ops += st[0]["active_volume"]
            torch.cuda.synchronize()
            res[name] = ((time.perf_counter() - t0) / len(seeds), ops / len(seeds))
        rows.append({"eps": eps, "localgd_ms_per_seed": res["localgd"][0] * 1e3, "gd_ms_per_seed": res["gd"][0] * 1e3,
                     "time_ratio_gd_over_localgd": res["gd"][0] / res["localgd"][0],
                     "localgd_ops_per_seed": res["localgd"][1], "gd_ops_per_seed": res["gd"][1],
                     "op_ratio_gd_over_localgd": res["gd"][1] / max(res["localgd"][1], 1),
                     "localch_ms_per_seed": res["localch"][0] * 1e3, "localch_ops_per_seed": res["localch"][1]})
    G.close()
    return {"workload": f"R-MAT scale 22 ({g.n} nodes, {g.nnz} CSR entries), PPR alpha=0.1, plain FP64, "
                        f"8 seeds at degree quantiles, one gde_solve per seed", "rows": rows}


def run_c2(gde, g=None, nseeds=64):
    """Plain FP64 LocalGD, one seed per gde_solve, on R-MAT scale 22 (edge factor 16, int32 CSR):
    PPR alpha=0.1, Katz beta=0.5/lambda_max, heat kernel tau=5 (Taylor layers to 1e-12), at
    eps in {1e-4, 1e-5, 1e-6, 1e-7}, 64 seeds at degree quantiles.  Per row: seeds/s, ms per
    seed and GTEPS (sum_t vol(S_t) over the wall time of the 64 solves, device output)."""
    import torch

    import synth
    if g is None:
        g = synth.workload_graph("rmat22")
    lam, _ = synth.lambda_max(g, rel_tol=1e-9, max_iter=2000)
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_quantile(g, nseeds)
    out = torch.zeros((1, g.n), dtype=torch.float64, device="cuda")
    rows = []
    for kind, param in (("ppr", 0.1), ("katz", 0.5 / lam), ("hk", 5.0)):
        for eps in (1e-4, 1e-5, 1e-6, 1e-7):
            gde.solve(G, kind, param, eps, torch.tensor(seeds[:1], dtype=torch.int32, device="cuda"), out)
            torch.cuda.synchronize()
            vol = rounds = 0
            t0 = time.perf_counter()
            for sd in seeds:
                _, st = gde.solve(G, kind, param, eps, torch.tensor([int(sd)], dtype=torch.int32, device="cuda"), out)
                vol += st[0]["active_volume"]
                rounds += st[0]["rounds"]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            rows.append({"kind": kind, "param": param, "eps": eps, "seeds_per_s": len(seeds) / dt,
                         "ms_per_seed": 1e3 * dt / len(seeds), "gteps": vol / dt / 1e9,
                         "rounds_mean": rounds / len(seeds), "volume_mean": vol / len(seeds)})
    G.close()
    return {"workload": f"R-MAT scale 22 ({g.n} nodes, {g.nnz} CSR entries, edge factor 16, int32 CSR), "
                        f"plain FP64 LocalGD, one gde_solve per seed, {nseeds} seeds at degree quantiles, "
                        f"lambda_max = {lam:.6g}", "rows": rows}


def run_c3(gde, g=None, nseeds=64, sample=8):
    """FP32 vs FP64 on Chung-Lu n=2^24 (mean degree 20, exponent 2.1, int64 offsets / int32
    columns): PPR alpha=0.15 and the heat kernel tau=10 at eps=1e-7, plain engine, 64 seeds at
    degree quantiles.  Per precision: seeds/s and GTEPS over the 64 solves.  Per result on
    `sample` of the seeds, the FP32 answer against the FP64 answer of the same seed (the FP64
    engine equals the FP64 oracle to 1e-9 relative L1 on this graph: tests/test_gpu_fullsize.py):
    relative L1 error, the largest absolute error, the largest relative error over entries
    >= eps d_u, and whether every entry lies inside the method's error band (both answers
    satisfy 0 <= f - x < eps d_u for the exact f, so they differ by less than eps d_u)."""
    import numpy as np
    import torch

    import synth
    if g is None:
        g = synth.workload_graph("chung_lu_2p24")
    G = gde.Graph.from_synth(g)
    seeds = synth.seeds_quantile(g, nseeds)
    pick = seeds[np.linspace(0, nseeds - 1, sample).round().astype(int)]
    d = g.degrees().astype(np.float64)
    band = 1e-7 * np.maximum(d, 1.0)
    rows = []
    eps = 1e-7
    for kind, param in (("ppr", 0.15), ("hk", 10.0)):
        times = {}
        for precision, dt_t in (("fp64", torch.float64), ("fp32", torch.float32)):
            out = torch.zeros((1, g.n), dtype=dt_t, device="cuda")
            gde.solve(G, kind, param, eps, torch.tensor(seeds[:1], dtype=torch.int32, device="cuda"), out,
                      precision=precision)
            torch.cuda.synchronize()
            vol = 0
            t0 = time.perf_counter()
            for sd in seeds:
                _, st = gde.solve(G, kind, param, eps, torch.tensor([int(sd)], dtype=torch.int32, device="cuda"),
                                  out, precision=precision)
                vol += st[0]["active_volume"]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            times[precision] = {"seeds_per_s": len(seeds) / dt, "gteps": vol / dt / 1e9}
        errs = []
        o64 = torch.zeros((1, g.n), dtype=torch.float64, device="cuda")
        o32 = torch.zeros((1, g.n), dtype=torch.float32, device="cuda")
        for sd in pick:
            sdt = torch.tensor([int(sd)], dtype=torch.int32, device="cuda")
            gde.solve(G, kind, param, eps, sdt, o64, precision="fp64")
            gde.solve(G, kind, param, eps, sdt, o32, precision="fp32")
            ref = o64[0].cpu().numpy()
            x = o32[0].double().cpu().numpy()
            diff = np.abs(x - ref)
            big = (np.abs(ref) >= eps * d) & (ref != 0)
            errs.append({"seed": int(sd), "degree": int(d[sd]),
                         "rel_l1": float(diff.sum() / np.abs(ref).sum()),
                         "max_abs": float(diff.max()),
                         "max_rel_entries_ge_eps_d": float((diff[big] / np.abs(ref[big])).max()) if big.any() else 0.0,
                         "within_eps_band": bool(np.all(diff < band + 1e-12))})
        rows.append({"kind": kind, "param": param, "eps": eps,
                     "fp64": times["fp64"], "fp32": times["fp32"],
                     "fp32_speedup": times["fp32"]["seeds_per_s"] / times["fp64"]["seeds_per_s"],
                     "fp32_vs_fp64_max_rel_l1": max(e["rel_l1"] for e in errs),
                     "fp32_vs_fp64_max_rel_entries_ge_eps_d": max(e["max_rel_entries_ge_eps_d"] for e in errs),
                     "fp32_all_within_eps_band": all(e["within_eps_band"] for e in errs),
                     "per_result": errs})
    G.close()
    return {"workload": f"Chung-Lu n=2^24 ({g.n} nodes, {g.nnz} CSR entries, mean degree 20, exponent 2.1, "
                        f"int64 offsets, int32 columns), plain engine, {nseeds} seeds at degree quantiles; "
                        f"errors of the FP32 answers on {sample} of them against the FP64 answers",
            "rows": rows}


PROBE_GRID = 152 * 8
PROBE_ACCESSES = 1 << 30


def traffic_from_capture(traffic_json, kernel_source, tuning, edges_per_launch):
    """DRAM bytes of one round-kernel launch, from the ncu capture of the same kernel source and
    launch shape on a small case of the workload (bytes per pushed edge) times this launch's
    pushed edges.  (None, None) when the file is missing, the source changed since the capture,
    or no capture has this tuning (blocks_per_sm aside: the grid follows the occupancy)."""
    import hashlib
    if not os.path.exists(traffic_json):
        return None, None
    tj = json.load(open(traffic_json))
    src = open(kernel_source, "rb").read()
    if tj.get("kernel") != "k_batch_rounds" or tj.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None, None
    tuned = {k: v for k, v in tuning.items() if k != "blocks_per_sm"}
    for c in tj.get("captures", []):
        if c.get("tuning") == tuned:
            note = (f"{c['bytes_per_edge']:.2f} B per pushed edge from one ncu capture on {tj['graph']} with "
                    f"{tj['seeds']} seeds and this launch's tuning (profiles/traffic.json), times this "
                    f"launch's pushed edges")
            return c["bytes_per_edge"] * edges_per_launch, note
    return None, None


def random_access_ceiling(gde, dev, gb=16.0, l2_fetch=0):
    """Random 32-byte sector rates of device memory (gde_probe_random_access) over a buffer far
    above the L2 size: reads, read + FP32 atomic add (the scatter's insert-or-add), and atomics
    alone, in G accesses/s."""
    import torch
    buf = torch.empty(int(gb * (1 << 30)), dtype=torch.uint8, device=dev)
    out = {"buffer_gb": gb, "accesses_per_launch": PROBE_ACCESSES, "grid": PROBE_GRID,
           "l2_fetch_bytes": l2_fetch or "default"}
    for name in ("load", "load_atomic", "atomic"):
        ms = gde.probe_random_access(buf, PROBE_ACCESSES, name, grid=PROBE_GRID, reps=3, l2_fetch_bytes=l2_fetch)
        out[f"{name}_gaccess_per_s"] = PROBE_ACCESSES / (ms / 1e3) / 1e9
    # the same accesses over the first 32 MB only (L2-resident): the rate of the hits
    l2buf = buf[: 32 << 20]
    out["l2_resident_mb"] = 32
    for name in ("load", "load_atomic", "atomic"):
        ms = gde.probe_random_access(l2buf, PROBE_ACCESSES, name, grid=PROBE_GRID, reps=3)
        out[f"l2_resident_{name}_gaccess_per_s"] = PROBE_ACCESSES / (ms / 1e3) / 1e9
    del buf, l2buf
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving_only:
        import torch
        import paper_2410_21634_gb300 as gde
        torch.cuda.set_device(0)
        gde.load()
        serving = run_serving(gde, args.serve_seconds, SERVE_SLOTS, SERVE_ROUNDS_PER_STEP)
        print(json.dumps({"serving": serving}), flush=True)
        return 0
    if args.random_probe:
        import torch
        import paper_2410_21634_gb300 as gde
        gde.load()
        ra = random_access_ceiling(gde, torch.device("cuda", 0), args.probe_gb, args.probe_l2_fetch)
        print(json.dumps({"random_access": ra}), flush=True)
        return 0
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws != args.gpus:
        log(f"[bench] warning: --gpus {args.gpus} but WORLD_SIZE {ws}")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    import paper_2410_21634_gb300 as gde
    gde.load()
    g, seeds_np = make_inputs(args.graph, args.seeds, rank)
    G = gde.Graph.from_synth(g)
    nseeds = len(seeds_np)
    dev = torch.device("cuda", local)
    seeds = torch.from_numpy(seeds_np).to(dev)
    ids = torch.zeros((nseeds, TOPK), dtype=torch.int32, device=dev)
    vals = torch.zeros((nseeds, TOPK), dtype=torch.float32, device=dev)

    budget = int(args.budget_gb * (1 << 30))
    if args.tuning:
        G.set_tuning(**json.loads(args.tuning))
    if args.hub_degree:
        G.set_tuning(hub_degree=args.hub_degree)

    def step():
        return gde.solve(G, "ppr", ALPHA, EPS, seeds, vals, ids, precision="fp32", topk=TOPK, batched=1,
                         mem_budget_bytes=budget)

    # the project's autotuner picks the push's bin thresholds, hub chunk, order and grid on
    # this batch before anything is timed
    tuning, tune_ms = None, None
    if not args.no_autotune:
        t0 = time.time()
        tuning, tune_ms = G.autotune("ppr", ALPHA, EPS, seeds, topk=TOPK, mem_budget_bytes=budget)
        log(f"[bench] autotune: {tuning} ({tune_ms:.1f} ms) in {time.time() - t0:.1f}s")
    for _ in range(max(args.warmup, 3)):
        st, stats = step()
    overflow = sum(1 for s in stats if s["fallback"])
    torch.cuda.synchronize()
    G.profile_enable(True)
    stream = torch.cuda.current_stream()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        # an NVTX range marks the timed steps, so a profiler can be limited to them
        torch.cuda.nvtx.range_push("bench_timed")
        start.record(stream)
        for _ in range(args.steps):
            st, stats = step()
        stop.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = start.elapsed_time(stop)
    prof = G.profile_read()
    G.profile_enable(False)
    t_max = ms
    edges_step = prof["edges"] / args.steps
    if pg:
        from paper_2410_21634_gb300 import shard
        t_max = shard.max_over_ranks(ms, device=dev)
        edges_total = shard.sum_over_ranks(prof["edges"], device=dev)
    else:
        edges_total = float(prof["edges"])
    sec = t_max / 1e3
    value = nseeds * ws * args.steps / sec
    gteps = edges_total / sec / 1e9
    clk = clocks.summary()

    # roofline of the persistent round kernel (its own CUDA events, on the launching stream)
    peak, peak_kind = measured_peaks()
    launches = max(prof["batch_launches"], 1)
    k_ms = prof["batch_rounds_ms"] / launches
    # candidates tested per launch: the kernel's round log of the last solve (all steps are the
    # same solve)
    rlog = G.profile_rounds()
    cands = float(rlog[:, 0].sum())
    # device time of the last solve's rounds: frontier phase (S_t, pushes placed) vs scatter
    t_end, t_a = rlog[:, 3], rlog[:, 4]
    t_prev = np.concatenate(([0.0], t_end[:-1]))
    phases = {"frontier_ms": float((t_a - t_prev).sum() / 1e6), "scatter_ms": float((t_end - t_a).sum() / 1e6),
              "rounds": int(rlog.shape[0]),
              "heavy_rounds_ms": [round(float(x) / 1e6, 3) for x in (t_end - t_prev)[:4]]}
    alg_bytes = (BYTES_PER_EDGE * prof["edges"] + BYTES_PER_PUSH * prof["pushes"]) / launches \
        + BYTES_PER_CAND * cands
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    kernel_bytes = (KERNEL_BYTES_PER_EDGE * prof["edges"] + KERNEL_BYTES_PER_PUSH * prof["pushes"]) / launches
    traffic, traffic_note = None, None
    if g.name == "rmat24" and nseeds == 1024:
        traffic, traffic_note = traffic_from_capture(
            os.path.join(ROOT, "profiles", "traffic.json"),
            os.path.join(ROOT, "paper_2410_21634_gb300", "csrc", "batched.cu"),
            G.get_tuning(), prof["edges"] / launches)
    roofline = {"bound": "hbm", "kernel": "k_batch_rounds", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "kernel_ms": k_ms, "alg_bytes_per_launch": alg_bytes,
                "bytes_model": f"{BYTES_PER_EDGE} B per pushed edge, {BYTES_PER_PUSH} B per pushed node, "
                               f"{BYTES_PER_CAND} B per candidate",
                "edges_per_launch": prof["edges"] / launches, "pushes_per_launch": prof["pushes"] / launches,
                "candidates_per_launch": cands,
                "phases_last_launch": phases,
                "frac_kernel_model": kernel_bytes / (k_ms / 1e3) / 1e9 / peak,
                "traffic_over_alg": traffic / alg_bytes if traffic else None,
                "traffic_note": traffic_note,
                "share_of_step": prof["batch_rounds_ms"] / ms if ms > 0 else None}

    # end to end through the public API with host buffers (seeds in, top-k out)
    seeds_host = torch.from_numpy(seeds_np).pin_memory()
    ids_h = torch.zeros((nseeds, TOPK), dtype=torch.int32).pin_memory()
    vals_h = torch.zeros((nseeds, TOPK), dtype=torch.float32).pin_memory()
    ids_hn, vals_hn, seeds_hn = ids_h.numpy(), vals_h.numpy(), seeds_host.numpy()
    e2e_steps = max(3, min(args.steps, 20))
    gde.solve(G, "ppr", ALPHA, EPS, seeds_hn, vals_hn, ids_hn, precision="fp32", topk=TOPK, batched=1,
              mem_budget_bytes=budget)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        gde.solve(G, "ppr", ALPHA, EPS, seeds_hn, vals_hn, ids_hn, precision="fp32", topk=TOPK, batched=1,
                  mem_budget_bytes=budget)
    e2e_sec = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": nseeds * ws / e2e_sec, "unit": "seeds/s", "h2d_bytes_per_step": 4 * nseeds,
           "d2h_bytes_per_step": 8 * nseeds * TOPK,
           "note": "host seed ids in, host top-k ids+values out, through gde_solve with host pointers"}

    # the random-access ceiling of this GPU's memory, beside the round kernel's insert rate
    random_access = None
    if not args.no_random_probe and rank == 0:
        random_access = random_access_ceiling(gde, dev, args.probe_gb, args.probe_l2_fetch)
        random_access["round_kernel_inserts_gaccess_per_s"] = prof["edges"] / launches / (k_ms / 1e3) / 1e9

    # the plain FP64 local GD, one seed per launch, on the same GPU and seed mix
    plain = None
    if not args.no_plain and rank == 0:
        out = torch.zeros((1, g.n), dtype=torch.float64, device=dev)
        half = nseeds // 2
        sample = np.concatenate([seeds_np[:128], seeds_np[half:half + 128]])
        for s in sample[:4]:
            gde.solve(G, "ppr", ALPHA, EPS, torch.tensor([s], dtype=torch.int32, device=dev), out)
        torch.cuda.synchronize()
        vol = 0
        t0 = time.perf_counter()
        for s in sample:
            _, st1 = gde.solve(G, "ppr", ALPHA, EPS, torch.tensor([s], dtype=torch.int32, device=dev), out)
            vol += st1[0]["active_volume"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        # a second pass with the library's events around the frontier and push kernels: the
        # share of the wall time the GPU spends in them (the rest is the per-round host sync,
        # the round-info read and the launch gaps that the batched engine amortises)
        G.profile_enable(True)
        t1 = time.perf_counter()
        for s in sample:
            gde.solve(G, "ppr", ALPHA, EPS, torch.tensor([s], dtype=torch.int32, device=dev), out)
        torch.cuda.synchronize()
        dt1 = time.perf_counter() - t1
        pp = G.profile_read()
        G.profile_enable(False)
        busy_ms = pp["dense_frontier_ms"] + pp["dense_push_ms"]
        plain = {"value": len(sample) / dt, "unit": "seeds/s", "gteps": vol / dt / 1e9,
                 "sample": f"{len(sample)} of the {nseeds} seeds (128 uniform + 128 hubs), one gde_solve "
                           f"per seed, dense FP64 x and r, output x written per seed",
                 "dtype": "f64",
                 "rounds_per_seed": pp["dense_rounds"] / len(sample),
                 "kernel_ms_per_seed": busy_ms / len(sample),
                 "wall_ms_per_seed": dt1 * 1e3 / len(sample),
                 "gpu_busy_share": busy_ms / (dt1 * 1e3),
                 "busy_note": "frontier + push kernel time (CUDA events) over wall time, second pass "
                              "with the events on; the rest is per-round host sync and launch gaps"}

    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        cpu = cpu_baseline(g, seeds_np)

    gpu_launches = prof["launches"]  # counted by the library for the timed steps
    tuning_used = G.get_tuning()

    kinds = None
    if not args.no_kinds and rank == 0:
        kinds = run_batched_kinds(gde, G, g, seeds_np, dev)

    # the serving workload (continuous batching with edge insertions), on its own graph
    serving = None
    if args.serve_seconds > 0 and rank == 0 and ws == 1:
        G.close()  # release the batched pool first
        serving = run_serving(gde, args.serve_seconds, SERVE_SLOTS, SERVE_ROUNDS_PER_STEP)
    gd_compare = None
    g22 = None
    if (not args.no_gd or not args.no_c2) and rank == 0 and ws == 1:
        import synth
        g22 = synth.workload_graph("rmat22")
    if not args.no_gd and rank == 0 and ws == 1:
        G.close()
        gd_compare = run_gd_compare(gde, g22)
    c2 = None
    if not args.no_c2 and rank == 0 and ws == 1:
        G.close()
        c2 = run_c2(gde, g22)
    c3 = None
    if not args.no_c3 and rank == 0 and ws == 1:
        G.close()
        c3 = run_c3(gde)
    line = {
        "metric": METRIC, "value": value, "unit": "seeds/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(g, nseeds, ws),
        "gteps": gteps,
        "plain_fp64_one_seed_per_launch": plain,
        "speedup_vs_plain_fp64": (value / ws) / plain["value"] if plain else None,
        "roofline": roofline,
        "random_access": random_access,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "hash_overflow_seeds": overflow,
        "edges_per_step": edges_step,
        "rounds_per_step": prof["rounds"] / launches,
        "tuning": tuning_used,
        "autotuned": tuning is not None,
        "batched_kinds": kinds,
        "serving": serving,
        "global_gd_vs_localgd": gd_compare,
        "c2_plain_fp64_rmat22": c2,
        "c3_fp32_vs_fp64_chung_lu_2p24": c3,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    G.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
