#!/usr/bin/env python3
"""Benchmark of the GB300 Block-Parallel IDA* solver.

Metric: 15-puzzle node expansions/s (and instances/s), batched vs plain,
with every integer result equal to the CPU oracle's.

Workload (default, the headline line): ``mixed15_4096``, 4096 seeded
15-puzzle boards of mixed difficulty (every 20th a uniformly random solvable
permutation, the rest random walks of 20-90 moves), Manhattan heuristic,
all-optimal-solutions mode (the final iteration is searched to completion,
so node counts are order-free). One step solves all 4096 boards:

* batched (headline ``value``): all boards in one solve call (persistent
  search warps shared by every board, per-board limits, the threshold loop
  as one CUDA graph);
* plain (``plain``): one solve call per board, as in the paper's
  one-instance-per-run experiments, timed over fewer steps.

Expansions are the nodes expanded over all iterations of all instances.
Inputs are resident in HBM when a timed step starts; L2 is flushed (a
256 MiB write) between steps. ``e2e`` repeats the batched step from pinned
host boards, copying the boards in and every result back inside the timed
region. Sub-keys measure the other workloads: ``perms15_100`` (100 random
permutations, plain and batched), ``walks24_1024`` (24-puzzle walks with a
node budget), ``serving`` (the continuous-batching service under Poisson
arrivals) and ``first_solution`` (first-solution mode against the oracle's
first-solution mode on one host core, the paper's headline comparison).

Multi-GPU: instances are independent, so each rank solves a contiguous range
of the boards with no collective on the data path, and the result rows are
gathered after the timed steps (strong scaling: the job is the workload);
``--replicas`` has every rank solve the whole workload instead (weak scaling).

``--impl reference`` times the CPU oracle (plain sequential IDA*, one thread
per instance, all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1705_02843_gb300 import inputs as I  # noqa: E402

METRIC = "15-puzzle node expansions/s & instances/s, batched vs plain, oracle-exact"
UNIT = "expansions/s"
WORKLOAD_DESC = {
    "mixed15_4096": "mixed15_4096: 4096 seeded 15-puzzle boards (seeds 100000-104095; every 20th a random "
                    "solvable permutation, 205 in all; the rest random walks of 20-90 moves), Manhattan "
                    "distance, all-optimal-solutions mode",
    "perms15_100": "perms15_100: 100 seeded uniformly random solvable 15-puzzle boards (seeds 1001-1100), "
                   "Manhattan distance, all-optimal-solutions mode",
}

# Instructions per expansion of the search kernel (warp instructions issued
# per node expanded: ncu smsp__inst_executed.sum of one launch over the nodes
# that launch popped, which the host-driven loop logs per launch), its share
# on the integer ALU pipe (16 lanes per scheduler: one warp instruction every
# 2 cycles, so above one half the ALU pipe, not issue, bounds the kernel at
# issue peak / (2 x share)), and DRAM bytes (read + write) of the captured
# launch, for the kernel each form runs.
#   batched: k_search<4,384,0>, a steady-state launch (the first pass of a
#   step, hand-back on) of a batched solve of the 4096-board mix: 331.2 M
#   warp instructions over 77.2 M nodes; ALU share (issue 84.0 %, ALU pipe
#   64.9 % busy) and DRAM bytes from one full capture of such a launch
#   (profiles/k_search_15puzzle_mixed15_4096_batched.txt). Hand-back passes
#   with few nodes issue more per node (4.4-5.4), so issue utilisation
#   computed with this figure is a lower bound;
#   plain: the fused-iteration variant k_search<4,384,1>, the final iteration
#   of board 0 of the mix as one pass
#   (profiles/k_search_15puzzle_plain_fused_final_iteration.txt); its ALU
#   share is the batched kernel's (the same step; a single-board launch's
#   pipe fractions are skewed by its tail).
KERNEL_COUNTERS = {
    "batched": {"kernel": "k_search<4,384,0>", "instr_per_expansion": 4.29, "alu_pipe_share": 0.386,
                "traffic_per_launch": 10233088},
    "plain": {"kernel": "k_search<4,384,1>", "instr_per_expansion": 4.66, "alu_pipe_share": 0.386,
              "traffic_per_launch": None},
}


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name + ".json")


def load_golden(name):
    p = golden_path(name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return {r["index"]: r for r in json.load(f)["instances"]}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, pg=None, device=None):
    """Largest value over the ranks of the process group (the job's time is
    its slowest rank's); the identity without a process group."""
    if pg is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def shard_range(n, world, rank):
    """The instance range [lo, hi) of one rank: n instances cut into world
    contiguous ranges whose sizes differ by at most one."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_rows(rows, pg=None, device=None):
    """The final gather: every rank's result rows (its instance range, in
    order) concatenated in rank order on every rank; the identity without a
    process group."""
    if pg is None:
        return list(rows)
    parts = [None] * pg.get_world_size()
    pg.all_gather_object(parts, list(rows))
    return [r for part in parts for r in part]


def sum_over_ranks(value, pg=None, device=None):
    """Sum of an integer over the ranks (the identity without a process group)."""
    if pg is None:
        return int(value)
    import torch

    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return int(t.item())


def replica_throughput(units_per_rank, seconds_per_rank, world, pg=None, device=None):
    """Whole-job throughput of N independent replicas: every rank processes
    the same amount of work; the job takes as long as the slowest rank."""
    t = max_over_ranks(seconds_per_rank, pg, device)
    return world * units_per_rank / t


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """CPU oracle arm: rank 0 only; other ranks exit without work."""
    if rank != 0:
        return
    import oracle

    insts = I.WORKLOADS[args.workload]()
    gold = load_golden(args.workload)
    sample, cores = pick_cpu_sample(insts, gold, args.cpu_sample_nodes, args.cpu_sample_board_cap)
    tiles = I.tiles_array([insts[i] for i in sample])
    times, nodes_tot = [], 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = oracle.solve_batch(4, tiles, count_all=True, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            nodes_tot = sum(r.total_nodes for r in res)
    t = statistics.mean(times)
    value = nodes_tot / t
    desc = cpu_sample_desc(insts, sample, nodes_tot, args.cpu_sample_board_cap)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "mode": "CPU oracle, one thread per board"},
        "instances_per_s": len(sample) / t,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Continuous batching under Poisson arrivals (98% walks of 30-90 moves,
    2% random permutations): completed requests/s and p50/p99 latency from
    submit to pollable result, per arrival rate; every result checked against
    the same boards solved in one batched call."""
    import torch

    from paper_1705_02843_gb300 import bpida

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rates = [float(r) for r in args.serving_rates.split(",")]
    out = []
    for rate in rates:
        n_req = int(min(args.serving_max_requests, rate * args.serving_seconds))
        summary, results, insts = serve(bpida, rate, n_req, args.serving_slice_us)
        summary["parity"], summary["batched_capacity"] = check_served(bpida, torch, dev, results, insts)
        out.append(summary)
        print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    best = max(out, key=lambda r: r["completed_per_s"])
    print(json.dumps({"metric": "15-puzzle serving: completed requests/s and p50/p99 latency (submit to result)",
                      "unit": "requests/s", "data": "synthetic",
                      "config": {"workload": "Poisson arrivals; 98% walks of 30-90 moves, 2% random permutations",
                                 "slots": 8192, "mode": "continuous batching",
                                 "time_slice_us": args.serving_slice_us if args.serving_slice_us is not None
                                 else "library default (2000)"},
                      "saturation": {"completed_per_s": best["completed_per_s"], "at_rate_per_s": best["rate_per_s"]},
                      "rates": out}), flush=True)


def run_ablation(args):
    """The paper's BPIDA* against this design, on the same workloads, every
    result checked equal: the paper's kernel (block = warp, 8 nodes x 4
    actions per pop, static root shares, no dynamic load balancing) on this
    design's per-iteration root sets (variant 1, also with 16x wider root
    sets), and with the paper's own static load balancing (variant 5: a
    persistent root set split and reassigned after every iteration by the
    repetitions each root took; one board per run, as in the paper). The
    4096-board mix is measured on its first --ablation-mix-boards boards."""
    import torch

    from paper_1705_02843_gb300 import bpida

    torch.cuda.set_device(0)
    out = {}
    for wl in ("perms15_100", "mixed15_4096"):
        insts = I.WORKLOADS[wl]()
        if wl == "mixed15_4096":
            insts = insts[:args.ablation_mix_boards]
        b = torch.from_numpy(I.packed_array(insts).view(np.int64)).cuda()
        res = {}
        wide = 65536 if wl == "perms15_100" else 512
        runs = [("this_design", 0, 0, ("batched", "plain")), ("paper_kernel", 1, 0, ("batched", "plain")),
                ("paper_kernel_wide_roots", 1, wide, ("batched",)),
                ("paper_bpida_static_lb", bpida.BPSTATIC, 0, ("plain",))]
        for name, variant, split, forms in runs:
            cfg = bpida.make_config(4, variant=variant, split_target=split)
            for form in forms:
                for rep in range(2 if variant == 0 else 1):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    if form == "batched" or variant >= bpida.PSIMPLE:
                        # variants 2-5 solve the boards of a call one at a time
                        sols = [bpida.solve(b, 4, cfg)]
                    else:
                        sols = [bpida.solve(b[i:i + 1], 4, cfg) for i in range(len(insts))]
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                hosts = [h for s in sols for h in s.to_host()]
                nodes = sum(sum(h["nodes"]) for h in hosts)
                st = bpida.last_stats()
                res[(name, form)] = (dt, nodes, [(h["length"], h["nodes"], h["moves"]) for h in hosts], st)
        ref = res[("this_design", "batched")][2]
        row = {"boards": len(insts)}
        for (name, form), (dt, nodes, rows, st) in res.items():
            if rows != ref:
                raise RuntimeError("%s (%s) disagrees with this design on %s" % (name, form, wl))
            row["%s_%s" % (name, form)] = {"seconds": dt, "expansions_per_s": nodes / dt,
                                            "instances_per_s": len(insts) / dt}
            if name == "paper_bpida_static_lb":
                row["%s_%s" % (name, form)].update({"search_warps": st["tp_threads"], "final_roots": st["tp_roots"],
                                                    "lb_ratio_last_board": st["lb_ratio"]})
        row["wide_roots_per_instance_cap"] = wide
        out[wl] = row
        print(json.dumps({wl: row}), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "ablation: this design vs the paper's BPIDA* (same drivers, exact results)",
                      "results": out}), flush=True)


def run_thread_parallel(args):
    """The paper's thread-parallel configurations (PSimple, PStaticLB,
    PFullLB: one sequential depth-first search per thread) against this
    design, one board per solve call on the 100-permutation workload, every
    result checked against the stored oracle results. Load balance is the
    paper's maxload / averageload of each board's next-to-last iteration,
    summarised over the boards whose next-to-last iteration expanded at least
    10 nodes per search thread."""
    import torch

    from paper_1705_02843_gb300 import bpida

    torch.cuda.set_device(0)
    insts = I.perms15_100()
    gold = load_golden("perms15_100")
    b = torch.from_numpy(I.packed_array(insts).view(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    names = {bpida.BLOCK_PARALLEL: "this_design", bpida.PSIMPLE: "PSimple", bpida.PSTATICLB: "PStaticLB",
             bpida.PFULLLB: "PFullLB"}
    out = {}
    for v in (bpida.BLOCK_PARALLEL, bpida.PSIMPLE, bpida.PSTATICLB, bpida.PFULLLB):
        cfg = bpida.make_config(4, variant=v)
        bpida.solve(b[:1], 4, cfg)  # warm-up (workspace, graphs)
        torch.cuda.synchronize()
        ms, ratios, nodes, threads = 0.0, [], 0, 0
        for i in range(len(insts)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s = bpida.solve(b[i:i + 1], 4, cfg)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            h = s.to_host()[0]
            if s.status != bpida.OK or (gold and (h["length"] != gold[i]["length"] or h["nodes"] != gold[i]["nodes"])):
                raise RuntimeError("%s: board %d differs from the oracle" % (names[v], i))
            nodes += sum(h["nodes"])
            st = bpida.last_stats()
            if v != bpida.BLOCK_PARALLEL:
                threads = st["tp_threads"]
                if len(h["nodes"]) >= 2 and h["nodes"][-2] >= 10 * threads:
                    ratios.append(st["lb_ratio"])
        row = {"seconds": ms / 1e3, "expansions_per_s": nodes / (ms / 1e3), "instances_per_s": len(insts) / (ms / 1e3)}
        if v != bpida.BLOCK_PARALLEL:
            row.update({"threads": threads, "lb_boards": len(ratios),
                        "lb_mean": statistics.mean(ratios) if ratios else None,
                        "lb_min": min(ratios) if ratios else None, "lb_max": max(ratios) if ratios else None,
                        "lb_sd": statistics.pstdev(ratios) if ratios else None})
        out[names[v]] = row
        print(json.dumps({names[v]: row}), file=sys.stderr, flush=True)
    for k in ("PStaticLB", "PFullLB", "this_design"):
        out[k]["speedup_vs_PSimple"] = out["PSimple"]["seconds"] / out[k]["seconds"]
    out["this_design"]["speedup_vs_PFullLB"] = out["PFullLB"]["seconds"] / out["this_design"]["seconds"]
    print(json.dumps({"metric": "ablation: thread-parallel IDA* (PSimple, PStaticLB, PFullLB) vs this design, "
                                "one board per call, exact results",
                      "config": {"workload": WORKLOAD_DESC["perms15_100"]}, "unit": "seconds for all boards", "results": out}),
          flush=True)


def run_workloads(args):
    """The other workloads: the 4096-board mix (95% random walks of 20-90
    moves, 5% random permutations) solved in one batched call and one board
    per call, and the 1024 24-puzzle walks (40-100 moves) batched with the
    oracle's node budget of 5e7 nodes per board. Every result is checked
    against the stored oracle results. Expansions count the nodes of the
    iterations each board completed."""
    import torch

    from paper_1705_02843_gb300 import bpida

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    def check(name, gold, hosts, idx):
        # a board stopped by the node budget reports its completed
        # iterations; the stored oracle row also holds the partial last one
        for i, h in zip(idx, hosts):
            g = gold[i]
            want = g["nodes"] if g["status"] == 0 else g["nodes"][:-1]
            if h["status"] != g["status"] or h["nodes"] != want or (
                    g["status"] == 0 and (h["length"] != g["length"] or "".join(map(str, h["moves"])) != g["moves"])):
                raise RuntimeError("%s: board %d differs from the oracle" % (name, i))
        return sum(sum(h["nodes"]) for h in hosts)

    out = {}
    # 15-puzzle mix: batched and plain
    insts = I.mixed15_4096()
    gold = load_golden("mixed15_4096")
    n = len(insts)
    b = torch.from_numpy(I.packed_array(insts).view(np.int64)).cuda()
    cfg = bpida.make_config(4)
    bpida.solve(b, 4, cfg)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(1, args.steps)):
        sol, t = timed(lambda: bpida.solve(b, 4, cfg))
        ts.append(t)
    nodes = check("mixed15_4096 batched", gold, sol.to_host(), range(n))
    t_b = statistics.median(ts)
    sols, t_p = timed(lambda: [bpida.solve(b[i:i + 1], 4, cfg) for i in range(n)])
    check("mixed15_4096 plain", gold, [s.to_host()[0] for s in sols], range(n))
    out["mixed15_4096"] = {"boards": n, "expansions": nodes,
                           "batched": {"seconds": t_b, "expansions_per_s": nodes / t_b, "instances_per_s": n / t_b},
                           "plain": {"seconds": t_p, "expansions_per_s": nodes / t_p, "instances_per_s": n / t_p},
                           "batched_over_plain_instances_per_s": t_p / t_b}
    print(json.dumps({"mixed15_4096": out["mixed15_4096"]}), file=sys.stderr, flush=True)
    # 24-puzzle walks with the oracle's node budget
    insts = I.walks24_1024()
    gold = load_golden("walks24_1024")
    n = len(insts)
    b = torch.from_numpy(I.packed_array(insts).view(np.int64).reshape(n, 2)).cuda()
    cfg = bpida.make_config(5, node_budget=50_000_000)
    bpida.solve(b, 5, cfg)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(1, args.steps)):
        sol, t = timed(lambda: bpida.solve(b, 5, cfg))
        ts.append(t)
    hosts = sol.to_host()
    nodes = check("walks24_1024", gold, hosts, range(n))
    t_b = statistics.median(ts)
    solved = sum(1 for h in hosts if h["status"] == 0)
    out["walks24_1024"] = {"boards": n, "solved_within_budget": solved, "node_budget": 50_000_000,
                           "expansions": nodes, "seconds": t_b, "expansions_per_s": nodes / t_b,
                           "instances_per_s": n / t_b}
    print(json.dumps({"walks24_1024": out["walks24_1024"]}), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "15-puzzle mix and 24-puzzle walks: expansions/s and instances/s, oracle-exact",
                      "data": "synthetic", "results": out}), flush=True)


# k_search<4,384,0,1> (the pattern-database search kernel of batched calls):
# warp instructions issued per node expanded, from ncu on the largest launch
# of a batched solve of the 100 boards with hand-back off, over the nodes the
# launch log records for it (profiles/k_search_pdb555_perms15_100_batched.txt).
# DRAM bytes and the ALU share of those launches are not those of the bench's
# launches (hand-back on; a single launch's pipe fractions are skewed by its
# tail), so none here.
INSTR_PER_EXPANSION_PDB = {"555": 13.0, "663": 13.18}
TRAFFIC_PER_LAUNCH_PDB = {}
ALU_PIPE_SHARE_PDB = {}


def run_pdb(args):
    """The pattern-database heuristic (the memory-intensive heuristic the
    paper's Section 7 names as future work) on the 100-permutation workload:
    the tables are built on the device, then the plain step (one call per
    board) and the batched step (one call) are timed as in the default leg
    (L2 flushed between steps, so every step starts with the tables out of
    L2), every result checked against the stored oracle results under the
    same heuristic. The oracle, with tables it builds itself, is timed on the
    host cores over all 100 boards."""
    import torch

    from paper_1705_02843_gb300 import bpida

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    part = args.pdb
    groups = I.PDB_PARTITIONS[part]
    insts = I.perms15_100()
    n = len(insts)
    gold = load_golden("perms15_100_pdb" + part)
    if gold is None:
        raise RuntimeError("no stored oracle results for partition %s: run "
                           "python tests/golden/make_golden.py perms15_100 --pdb %s" % (part, part))
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pdb = bpida.PatternDb(4, groups)
    build_s = time.perf_counter() - t0
    table_bytes = sum(pdb.table_bytes(g) for g in range(len(groups)))

    if args.profile_pdb is not None:
        # host-driven loop (ncu cannot see kernels inside graphs with
        # conditional nodes); -1: the batched call
        # (with --profile-default as in the bench, else hand-back off); the
        # first solve's search launches are printed with their node counts
        b = boards if args.profile_pdb < 0 else boards[args.profile_pdb:args.profile_pdb + 1]
        cfg = bpida.make_config(4, driver=1, exit_fraction_pct=0 if args.profile_default else 100)
        log = None
        for rep in range(2):
            bpida.set_timing(rep == 0)
            s = bpida.solve(b, 4, cfg, pdb=pdb)
            torch.cuda.synchronize(dev)
            if rep == 0:
                log = bpida.launch_log()
        bpida.set_timing(False)
        print(json.dumps({"profile_pdb": args.profile_pdb, "partition": part, "status": s.status,
                          "nodes": int(s.nodes.cpu().numpy().view(np.uint64).sum()),
                          "stats": bpida.last_stats(),
                          "launches": [{"i": i, "ms": ms, "nodes": nd} for i, (ms, nd) in enumerate(log)],
                          "largest_launch": max(range(len(log)), key=lambda i: log[i][1]) if log else None}),
              flush=True)
        return

    cfg = bpida.make_config(4)

    def check(sols):
        tot = 0
        for i, h in enumerate(sols):
            g = gold[i]
            if h["status"] != 0 or h["length"] != g["length"] or h["nodes"] != g["nodes"] or \
                    h["solutions"] != g["solutions"] or "".join(map(str, h["moves"])) != g["moves"]:
                raise RuntimeError("pattern databases %s: board %d differs from the oracle" % (part, i))
            tot += sum(h["nodes"])
        return tot

    def plain_step():
        return [bpida.solve(boards[i:i + 1], 4, cfg, pdb=pdb) for i in range(n)]

    def batched_step():
        return [bpida.solve(boards, 4, cfg, pdb=pdb)]

    def hosts(sols):
        return [h for s in sols for h in s.to_host()]

    def timed(step, k, warm):
        for _ in range(warm):
            step()
        torch.cuda.synchronize(dev)
        ms, sols = [], None
        for _ in range(k):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sols = step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return ms, sols

    with ClockSampler(0) as clk:
        ms_plain, psols = timed(plain_step, args.steps, args.warmup)
        ms_batch, bsols = timed(batched_step, args.steps, args.warmup)
    clocks = clk.summary()
    exp = check(hosts(psols))
    if check(hosts(bsols)) != exp:
        raise RuntimeError("batched and plain expansions differ")
    t_plain = sum(ms_plain) / 1e3 / len(ms_plain)
    t_batch = sum(ms_batch) / 1e3 / len(ms_batch)

    # end to end through host buffers: pinned boards copied to the device and
    # every result copied back inside the timed region (plain step)
    packed = I.packed_array(insts)
    host_boards = torch.from_numpy(packed.view(np.int64)).pin_memory()
    ml, mi = bpida.max_len(4), bpida.max_iters(4)
    host_out = {k: torch.empty(sz, dtype=dt).pin_memory() for k, sz, dt in (
        ("len", n, torch.int32), ("moves", n * ml, torch.uint8), ("nodes", n * mi, torch.int64),
        ("iters", n, torch.int32), ("status", n, torch.int32), ("solutions", n, torch.int64))}

    def e2e_step():
        dboards = host_boards.to(dev, non_blocking=True)
        sols = [bpida.solve(dboards[i:i + 1], 4, cfg, pdb=pdb) for i in range(n)]
        host_out["len"].copy_(torch.cat([x.length for x in sols]), non_blocking=True)
        host_out["moves"].copy_(torch.cat([x.moves.reshape(-1) for x in sols]), non_blocking=True)
        host_out["nodes"].copy_(torch.cat([x.nodes.reshape(-1) for x in sols]), non_blocking=True)
        host_out["iters"].copy_(torch.cat([x.iters for x in sols]), non_blocking=True)
        host_out["status"].copy_(torch.cat([x.inst_status for x in sols]), non_blocking=True)
        host_out["solutions"].copy_(torch.cat([x.solutions for x in sols]), non_blocking=True)
        return sols

    ms_e2e, _ = timed(e2e_step, args.steps, 1)
    if int(host_out["nodes"].numpy().view(np.uint64).sum()) != exp:
        raise RuntimeError("end-to-end expansions differ")
    t_e2e = sum(ms_e2e) / 1e3 / len(ms_e2e)
    e2e = {"value": exp / t_e2e, "unit": UNIT, "instances_per_s": n / t_e2e,
           "h2d_bytes_per_step": host_boards.numel() * 8,
           "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in host_out.values())}

    # the search kernel alone: the batched call through the host-driven
    # loop, every k_search launch bracketed by CUDA events on its stream
    bpida.set_timing(True)
    flush.fill_(1)
    torch.cuda.synchronize(dev)
    s = bpida.solve(boards, 4, bpida.make_config(4, driver=1), pdb=pdb)
    torch.cuda.synchronize(dev)
    st = bpida.last_stats()
    bpida.set_timing(False)
    check(s.to_host())
    kern_rate = st["search_nodes"] / (st["search_ms"] / 1e3)
    roof = None
    I_pdb = INSTR_PER_EXPANSION_PDB.get(part)
    if I_pdb:
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        peak = 152 * 4 * sm_mhz * 1e6
        roof = {"kernel": "k_search<4,384,0,1>", "bound": "alu", "achieved": kern_rate * I_pdb, "peak": peak,
                "unit": "warp-instructions/s", "frac": kern_rate * I_pdb / peak,
                "traffic": TRAFFIC_PER_LAUNCH_PDB.get(part), "instr_per_expansion": I_pdb,
                "alu_pipe": {"share": ALU_PIPE_SHARE_PDB[part], "peak": peak / (2 * ALU_PIPE_SHARE_PDB[part]),
                             "frac": kern_rate * I_pdb / (peak / (2 * ALU_PIPE_SHARE_PDB[part]))}
                if ALU_PIPE_SHARE_PDB.get(part) else None}

    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        t0 = time.perf_counter()
        opdb = oracle.PatternDb(4, groups)
        ob = time.perf_counter() - t0
        t0 = time.perf_counter()
        res = oracle.solve_batch(4, I.tiles_array(insts), pdb=opdb)
        ot = time.perf_counter() - t0
        onodes = sum(r.total_nodes for r in res)
        cpu = {"value": onodes / ot, "unit": "expansions/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "all %d boards, %d expansions, %.1f s (tables built in %.1f s, not included)" % (
                   n, onodes, ot, ob),
               "instances_per_s": n / ot}
    line = {
        "metric": METRIC + " (pattern-database heuristic)",
        "value": exp / t_plain, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_plain * 1e3, "higher_is_better": True, "dtype": "int64", "data": "synthetic",
        "instances_per_s": n / t_plain,
        "batched": {"value": exp / t_batch, "instances_per_s": n / t_batch, "ms_per_step": t_batch * 1e3},
        "expansions_per_step": exp,
        "search_kernel": {"expansions_per_s": kern_rate, "launches": st["passes"], "search_ms": st["search_ms"]},
        "config": {"workload": "perms15_100 (100 seeded random solvable 15-puzzle boards), all-optimal-solutions "
                               "mode, additive pattern databases, groups " + json.dumps(groups),
                   "table_bytes": table_bytes, "device_build_s": build_s, "l2": "flushed between steps"},
        "parity": {"checked": n, "mismatched": 0, "against": "tests/golden/perms15_100_pdb%s.json" % part},
        "e2e": e2e, "roofline": roof, "clocks": clocks, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    pdb.close()


def pick_cpu_sample(insts, gold, budget_nodes, board_cap=None):
    """A bounded sample of a workload for the CPU oracle: the boards in
    workload order whose stored oracle node count is at most ``board_cap``
    (None: any), until ``budget_nodes`` expansions; without stored results,
    the first 8 boards."""
    cores = os.cpu_count() or 1
    if not gold:
        return list(range(min(8, len(insts)))), cores
    sample, acc = [], 0
    for i in range(len(insts)):
        c = sum(gold[i]["nodes"])
        if board_cap and c > board_cap:
            continue
        if acc + c > budget_nodes:
            if sample:
                break
            continue
        sample.append(i)
        acc += c
    return sample, cores


def pick_cheapest(gold, budget_nodes):
    """The cheapest boards by stored oracle node count, up to budget_nodes."""
    order = sorted(gold, key=lambda i: sum(gold[i]["nodes"]))
    sample, acc = [], 0
    for i in order:
        c = sum(gold[i]["nodes"])
        if acc + c > budget_nodes and sample:
            break
        sample.append(i)
        acc += c
    return sorted(sample)


def cpu_sample_desc(insts, sample, nodes, board_cap):
    kinds = {}
    for i in sample:
        kinds[insts[i].kind] = kinds.get(insts[i].kind, 0) + 1
    what = ", ".join("%d %ss" % (v, k) for k, v in sorted(kinds.items()))
    cap = (" among those of at most %.0e stored oracle nodes" % board_cap) if board_cap else ""
    return "%d of %d boards (%s), taken in workload order%s; %d expansions" % (
        len(sample), len(insts), what, cap, nodes)


def replay(W, tiles, moves):
    """The board after applying blank moves (0 up, 1 left, 2 right, 3 down)."""
    b = list(tiles)
    p = b.index(0)
    for m in moves:
        q = p + (-W, -1, 1, W)[m]
        if not 0 <= q < W * W or (m in (1, 2) and q // W != p // W):
            return None
        b[p], b[q] = b[q], b[p]
        p = q
    return b


def same_as_golden(h, g, first_only=False):
    """Per-board parity with the stored oracle result (all-solutions mode:
    length, nodes per iteration, first solution, solution count;
    first-solution mode: length and every iteration but the last)."""
    if h["status"] != g["status"]:
        return False
    if g["status"] != 0:
        return True
    if first_only:
        return h["length"] == g["length"] and h["nodes"][:-1] == g["nodes"][:-1] and \
            h["nodes"][-1] <= g["nodes"][-1] and len(h["nodes"]) == len(g["nodes"])
    return h["length"] == g["length"] and h["nodes"] == g["nodes"] and \
        "".join(map(str, h["moves"])) == g["moves"] and h["solutions"] == g["solutions"]


class Timer:
    """Steps timed with CUDA events on the launching stream, L2 flushed
    before each, barrier + synchronize around the timed region."""

    def __init__(self, torch, dev, stream, pg):
        self.torch, self.dev, self.stream, self.pg = torch, dev, stream, pg
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def run(self, step_fn, k, warm):
        torch = self.torch
        for _ in range(warm):
            step_fn()
        torch.cuda.synchronize(self.dev)
        if self.pg:
            self.pg.barrier()
        ms, aggs, out = [], [], None
        for _ in range(k):
            self.flush.fill_(1)
            torch.cuda.synchronize(self.dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            out, agg = step_fn()
            e1.record(self.stream)
            torch.cuda.synchronize(self.dev)
            ms.append(e0.elapsed_time(e1))
            # solve calls are asynchronous: their statistics are read once
            # the stream is idle
            aggs.append(agg() if callable(agg) else agg)
        torch.cuda.synchronize(self.dev)
        if self.pg:
            self.pg.barrier()
        return ms, aggs, out


AGG_KEYS = ("search_ms", "search_ms_device", "search_nodes", "passes", "launches", "records", "handed_back")


def make_steps(bpida, boards, n, cfg):
    """(batched step, plain step): all boards in one call / one call per board."""

    def stats():
        st = bpida.last_stats()
        return {k: st[k] for k in AGG_KEYS}

    def batched():
        s = bpida.solve(boards, 4, cfg)
        if s.status != bpida.OK:
            raise RuntimeError("solve failed: " + bpida.status_str(s.status))
        return [s], stats

    def plain():
        sols, agg = [], dict.fromkeys(AGG_KEYS, 0)
        for i in range(n):
            s = bpida.solve(boards[i:i + 1], 4, cfg)
            if s.status != bpida.OK:
                raise RuntimeError("solve failed: " + bpida.status_str(s.status))
            sols.append(s)
        # the calls are asynchronous and statistics are those of the last
        # call once the stream is idle: the plain step's are not collected
        return sols, agg

    return batched, plain


def hosts_of(sols):
    return [h for s in sols for h in s.to_host()]


def parity(hosts, gold, first_only=False):
    bad = [i for i, h in enumerate(hosts) if not same_as_golden(h, gold[i], first_only)]
    return {"checked": len(hosts), "mismatched": len(bad), "first_mismatch": bad[0] if bad else None}


def kernel_roofline(bpida, torch, dev, boards, form, clocks, width=4, node_budget=0, counters=None):
    """Roofline of the search kernel of one form: the solve once more through
    the host-driven loop, which brackets every search launch with CUDA events
    on the launching stream; warp instructions per expansion from ncu."""
    counters = counters or KERNEL_COUNTERS[form]
    n = boards.shape[0]
    bpida.set_timing(True)
    torch.cuda.synchronize(dev)
    cfg = bpida.make_config(width, driver=1, node_budget=node_budget)
    ms = nodes = launches = 0
    if form == "batched":
        bpida.solve(boards, width, cfg)
        torch.cuda.synchronize(dev)
        st = bpida.last_stats()
        ms, nodes, launches = st["search_ms"], st["search_nodes"], st["passes"]
    else:
        for i in range(n):
            bpida.solve(boards[i:i + 1], width, cfg)
            torch.cuda.synchronize(dev)
            st = bpida.last_stats()
            ms += st["search_ms"]
            nodes += st["search_nodes"]
            launches += st["passes"]
    bpida.set_timing(False)
    sms = st["sm_count"]
    f_mhz = clocks.get("sm_mhz") or 2070.0
    peak = sms * 4 * f_mhz * 1e6 / 1e9  # G warp-instructions issued per second
    rate = nodes / (ms / 1e3)
    I_exp = counters["instr_per_expansion"]
    achieved = rate * I_exp / 1e9
    share = counters["alu_pipe_share"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s", "frac": achieved / peak,
            "traffic": counters.get("traffic_per_launch"), "kernel": counters["kernel"],
            "instr_per_expansion": I_exp, "expansions_per_s_in_kernel": rate,
            "launch_ms_mean": ms / max(launches, 1), "launches_timed": launches, "nodes_timed": nodes,
            "peak_basis": "%d SMs x 4 schedulers x %.0f MHz median SM clock sampled during the run" % (sms, f_mhz),
            "alu_pipe": {"share": share, "peak": peak / (2 * share), "frac": achieved / (peak / (2 * share)),
                         "basis": "the integer ALU pipe takes a warp instruction every 2 cycles per scheduler; "
                                  "with this share of ALU instructions it caps issue at 1 / (2 x share) per cycle"}}
    if counters.get("instr_per_expansion_all_launches"):
        roof["issue_utilization_all_launches"] = rate * counters["instr_per_expansion_all_launches"] / 1e9 / peak
    return roof


def serve(bpida, rate, n_req, slice_us=None, seed=None):
    """Drives the continuous-batching service with a Poisson stream; returns
    (summary, results by request id, boards)."""
    stream = I.serving_stream(rate, n_req, seed=300000 + int(rate) if seed is None else seed)
    words = [int(w) for w in I.packed_array([x for _, x in stream])]
    lat, results = [], {}
    with bpida.Server(frontier_bytes=2 << 30, max_slots=8192, time_slice_us=slice_us) as sv:
        t0 = bpida.Server.clock()
        i = got = 0
        while got < n_req:
            now = bpida.Server.clock() - t0
            while i < n_req and stream[i][0] <= now:
                sv.submit(words[i], i)
                i += 1
            for r in sv.poll():
                if r["status"] != 0:
                    raise RuntimeError("request %d failed: %s" % (r["req_id"], bpida.status_str(r["status"])))
                lat.append(r["latency_s"])
                results[r["req_id"]] = r
                got += 1
            if i < n_req:
                wait = stream[i][0] - (bpida.Server.clock() - t0)
                if wait > 0.0005:
                    time.sleep(min(wait, 0.002))
            else:
                time.sleep(0.0005)
        t_end = bpida.Server.clock() - t0
        st = sv.stats()
    lat.sort()
    summary = {"rate_per_s": rate, "requests": n_req, "completed_per_s": n_req / t_end,
               "p50_ms": 1e3 * lat[len(lat) // 2], "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
               "device_steps": st["steps"], "sliced_steps": st["sliced_steps"], "max_active": st["max_active"],
               "wall_s": t_end, "arrivals_s": stream[-1][0]}
    return summary, results, [x for _, x in stream]


def check_served(bpida, torch, dev, results, insts):
    """Every served result equals the same board's result from one batched
    solve call (which the parity tests check against the oracle) and replays
    to the goal."""
    b = torch.from_numpy(I.packed_array(insts).view(np.int64)).to(dev)
    bpida.solve(b, 4).synchronize()  # warm-up (the call's graph)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sol = bpida.solve(b, 4)
    e1.record()
    ref = sol.to_host()
    batched_s = e0.elapsed_time(e1) / 1e3
    bad = 0
    for i, x in enumerate(insts):
        r, h = results[i], ref[i]
        if (r["length"], r["nodes"], r["moves"], r["solutions"]) != (h["length"], h["nodes"], h["moves"],
                                                                       h["solutions"]) or \
                replay(4, x.tiles, r["moves"]) != list(range(16)):
            bad += 1
    return {"checked": len(insts), "mismatched": bad,
            "against": "the same boards solved in one batched call, and a replay of every solution"}, \
        {"instances_per_s": len(insts) / batched_s, "ms": batched_s * 1e3,
         "what": "the same requests' boards solved in one batched call (CUDA events): the GPU's throughput "
                 "on this request mix, which bounds the service's completed requests/s"}


def leg_perms(bpida, torch, dev, timer, steps, clocks_hint):
    """perms15_100 (the paper-shaped workload): plain and batched, parity
    against the stored oracle results, and the plain form's search-kernel
    roofline."""
    insts = I.perms15_100()
    gold = load_golden("perms15_100")
    n = len(insts)
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64)).to(dev)
    batched, plain = make_steps(bpida, boards, n, bpida.make_config(4))
    ms_p, _, psols = timer.run(plain, steps, 1)
    ms_b, _, bsols = timer.run(batched, steps, 1)
    hp, hb = hosts_of(psols), hosts_of(bsols)
    exp = sum(sum(h["nodes"]) for h in hp)
    t_p, t_b = sum(ms_p) / 1e3 / steps, sum(ms_b) / 1e3 / steps
    par = parity(hp, gold)
    pb = parity(hb, gold)
    par["mismatched"] += pb["mismatched"]
    par["checked"] += pb["checked"]
    return {"workload": WORKLOAD_DESC["perms15_100"], "expansions_per_step": exp, "steps": steps,
            "plain": {"expansions_per_s": exp / t_p, "instances_per_s": n / t_p, "ms_per_step": t_p * 1e3},
            "batched": {"expansions_per_s": exp / t_b, "instances_per_s": n / t_b, "ms_per_step": t_b * 1e3},
            "batched_over_plain_instances_per_s": t_p / t_b,
            "parity": par,
            "roofline_plain": kernel_roofline(bpida, torch, dev, boards, "plain", clocks_hint)}


# 24-puzzle search kernel k_search<5,384,0>: warp instructions per expansion
# and ALU share of the largest launch (7.25 G nodes, one pass per step) of a
# batched solve of walks24_1024 with the 5e7 node budget
# (profiles/k_search_24puzzle_walks24_1024_batched.txt); DRAM bytes are those
# of that launch, not of the bench's launches (hand-back on), so none here.
KERNEL_COUNTERS_W5 = {"kernel": "k_search<5,384,0>", "instr_per_expansion": 5.91, "alu_pipe_share": 0.42,
                      "traffic_per_launch": None}


def leg_walks24(bpida, torch, dev, timer, steps, clocks_hint):
    """walks24_1024: 1024 24-puzzle walks of 40-100 moves, batched, with the
    oracle's node budget of 5e7 nodes per board; parity against the stored
    oracle results (a board stopped by the budget reports its completed
    iterations)."""
    insts = I.walks24_1024()
    gold = load_golden("walks24_1024")
    n = len(insts)
    budget = 50_000_000
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64).reshape(n, 2)).to(dev)
    cfg = bpida.make_config(5, node_budget=budget)

    def step():
        s = bpida.solve(boards, 5, cfg)
        if s.status != bpida.OK:
            raise RuntimeError("solve failed: " + bpida.status_str(s.status))
        return [s], lambda: {"search_nodes": bpida.last_stats()["search_nodes"]}

    ms, aggs, sols = timer.run(step, steps, 1)
    hosts = hosts_of(sols)
    bad = 0
    for i, h in enumerate(hosts):
        g = gold[i]
        want = g["nodes"] if g["status"] == 0 else g["nodes"][:-1]
        if h["status"] != g["status"] or h["nodes"] != want or (
                g["status"] == 0 and (h["length"] != g["length"] or "".join(map(str, h["moves"])) != g["moves"])):
            bad += 1
    t = sum(ms) / 1e3 / steps
    reported = sum(sum(h["nodes"]) for h in hosts)
    searched = aggs[-1]["search_nodes"]
    roof = kernel_roofline(bpida, torch, dev, boards, "batched", clocks_hint, width=5, node_budget=budget,
                           counters=KERNEL_COUNTERS_W5)
    return {"workload": "walks24_1024: 1024 seeded 24-puzzle random walks of 40-100 moves (seeds 200000-201023), "
                        "node budget 5e7 per board (as the oracle's)",
            "solved_within_budget": sum(1 for h in hosts if h["status"] == 0), "boards": n,
            "ms_per_step": t * 1e3, "instances_per_s": n / t,
            "reported_expansions_per_s": reported / t,
            "searched_expansions_per_s": searched / t,
            "note": "reported = the nodes of the iterations each board completed (what the oracle reports); "
                    "searched = every node the search kernel popped, the iterations the budget cut short included",
            "parity": {"checked": n, "mismatched": bad, "against": "tests/golden/walks24_1024.json"},
            "roofline": roof}


def leg_serving(bpida, torch, dev, rates, n_req):
    out = []
    for rate in rates:
        summary, results, insts = serve(bpida, rate, n_req)
        summary["parity"], summary["batched_capacity"] = check_served(bpida, torch, dev, results, insts)
        out.append(summary)
    return {"workload": "Poisson arrivals; 98% walks of 30-90 moves, 2% random permutations; "
                        "latency from submit to pollable result", "mode": "continuous batching, 2 ms time slices",
            "rates": out}


def leg_first_solution(bpida, torch, dev, budget_nodes):
    """First-solution mode (count_all = 0, Section 6's main timing
    experiment) against the oracle's first-solution mode on one host core
    (the paper's sequential-solver setting), and the same for all-solutions
    mode (its count-all experiment), on the cheapest boards of perms15_100;
    one board per solve call on the GPU, as in the paper."""
    import oracle

    insts = I.perms15_100()
    gold = load_golden("perms15_100")
    idx = pick_cheapest(gold, budget_nodes)
    sub = [insts[i] for i in idx]
    boards = torch.from_numpy(I.packed_array(sub).view(np.int64)).to(dev)
    tiles = I.tiles_array(sub)
    out = {"boards": len(idx), "sample": "the %d cheapest boards of perms15_100 (stored all-solutions node count, "
                                         "%d nodes in all)" % (len(idx), sum(sum(gold[i]["nodes"]) for i in idx))}
    stream = torch.cuda.current_stream(dev)
    for mode, count_all in (("first_solution", False), ("all_solutions", True)):
        cfg = bpida.make_config(4, count_all=count_all)
        for i in range(len(idx)):  # warm-up (graphs, workspace)
            bpida.solve(boards[i:i + 1], 4, cfg)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sols = [bpida.solve(boards[i:i + 1], 4, cfg) for i in range(len(idx))]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_gpu = e0.elapsed_time(e1) / 1e3
        t0 = time.perf_counter()
        ref = oracle.solve_batch(4, tiles, count_all=count_all, nthreads=1)
        t_cpu = time.perf_counter() - t0
        hosts = hosts_of(sols)
        bad = 0
        for x, h, r in zip(sub, hosts, ref):
            ok = h["status"] == 0 and h["length"] == r.length and h["nodes"][:-1] == r.nodes[:-1] and \
                len(h["nodes"]) == len(r.nodes) and replay(4, x.tiles, h["moves"]) == list(range(16))
            if count_all:
                ok = ok and h["nodes"] == r.nodes and h["moves"] == r.moves
            bad += 0 if ok else 1
        out[mode] = {"gpu_s": t_gpu, "cpu_one_core_s": t_cpu, "speedup": t_cpu / t_gpu,
                     "gpu_instances_per_s": len(idx) / t_gpu, "cpu_instances_per_s": len(idx) / t_cpu,
                     "gpu_expansions": sum(sum(h["nodes"]) for h in hosts),
                     "cpu_expansions": sum(r.total_nodes for r in ref),
                     "parity": {"checked": len(idx), "mismatched": bad,
                                "against": "the oracle's %s mode on the same boards (length, %s, replay)" % (
                                    "first-solution" if not count_all else "all-solutions",
                                    "every iteration but the last" if not count_all
                                    else "every iteration, first solution")}}
    out["paper"] = "Section 6: 4.98x (first solution) and 6.78x (all solutions) over one Xeon E5-2670 core, on a " \
                   "GRID K520, Korf's 100 boards (context only)"
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="mixed15_4096", choices=["mixed15_4096", "perms15_100"])
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs: every GPU solves the whole workload (weak scaling) instead of its "
                         "instance range")
    ap.add_argument("--plain-steps", type=int, default=3,
                    help="timed steps of the plain form (one call per board; slower, so fewer)")
    ap.add_argument("--sub-steps", type=int, default=3, help="timed steps of each sub-workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the sub-workload legs")
    ap.add_argument("--cpu-sample-nodes", type=float, default=8e8)
    ap.add_argument("--cpu-sample-board-cap", type=float, default=5e7)
    ap.add_argument("--first-solution-nodes", type=float, default=3e8,
                    help="all-solutions node count of the boards the first-solution leg runs on one core")
    ap.add_argument("--ablation", action="store_true",
                    help="compare against the paper's BPIDA* kernel instead")
    ap.add_argument("--ablation-mix-boards", type=int, default=512,
                    help="with --ablation: boards of the 4096-board mix to run (its first ones)")
    ap.add_argument("--workloads", action="store_true",
                    help="measure the 4096-board mix (batched and plain) and the 24-puzzle walks instead")
    ap.add_argument("--thread-parallel", action="store_true",
                    help="compare the paper's thread-parallel configurations with this design instead")
    ap.add_argument("--serving", action="store_true",
                    help="run the continuous-batching service under Poisson arrivals instead")
    ap.add_argument("--serving-rates", default="1000,2000,5000,10000,20000,50000")
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--serving-max-requests", type=int, default=20000)
    ap.add_argument("--serving-slice-us", type=int, default=None,
                    help="time slice of a device step in microseconds (0 = none; default: the library's)")
    ap.add_argument("--sub-serving-rates", default="2000,10000,50000",
                    help="arrival rates of the default line's serving leg")
    ap.add_argument("--sub-serving-requests", type=int, default=4000)
    ap.add_argument("--pdb", default=None, choices=sorted(I.PDB_PARTITIONS),
                    help="time the pattern-database heuristic with this tile partition")
    ap.add_argument("--profile-pdb", type=int, default=None, metavar="IDX",
                    help="with --pdb: solve board IDX (-1: all, one call) twice through the host-driven loop")
    ap.add_argument("--driver", default="graph", choices=["graph", "host"],
                    help="graph: each solve call is one CUDA graph launch (default); host: the "
                         "host launches every kernel (same kernels; ncu can list them)")
    ap.add_argument("--profile-case", type=int, default=None, metavar="IDX",
                    help="solve board IDX alone, twice, through the host-driven loop with one "
                         "search pass per step, print the first solve's search launches (duration, "
                         "nodes) and statistics and exit (for ncu captures)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="solve all boards of the workload in one call, twice, through the host-driven loop "
                         "with one search pass per step, print the first solve's search launches and exit "
                         "(for ncu captures of the search kernel at full occupancy)")
    ap.add_argument("--profile-default", action="store_true",
                    help="with --profile-case or --profile-batched: keep the default hand-back (as in the bench)")
    ap.add_argument("--profile-width", type=int, default=4, choices=[4, 5],
                    help="with --profile-case or --profile-batched: 5 = the 24-puzzle walk workload")
    ap.add_argument("--profile-variant", type=int, default=0, metavar="V",
                    help="with --profile-case: solve with bpida_config.variant V (2-4: the thread-parallel "
                         "configurations; the final iteration's k_search_tp launch is number iters-1)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()

    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.serving:
        run_serving(args)
        return
    if args.ablation:
        run_ablation(args)
        return
    if args.thread_parallel:
        run_thread_parallel(args)
        return
    if args.pdb:
        run_pdb(args)
        return
    if args.workloads:
        run_workloads(args)
        return

    import torch

    from paper_1705_02843_gb300 import bpida

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    insts = I.WORKLOADS[args.workload]()
    if args.profile_batched or args.profile_case is not None:
        # for ncu: two solves through the host-driven loop (ncu cannot see
        # kernels inside graphs that hold conditional nodes), by default with
        # hand-back off (one search pass per step, plus passes for stack
        # overflows); the first solve's search launches are printed with
        # their durations and node counts, so that a profiler's instruction
        # count of launch i (ncu -k regex:k_search -s i -c 1) over the nodes
        # that the same run prints for launch i gives instructions per
        # expansion (the launch sequence can differ between runs where
        # passes end by timing, so take both from one run).
        #   --profile-batched: all boards of the workload in one call (width
        #   5: the 24-puzzle walks with the oracle's node budget);
        #   --profile-case IDX: board IDX alone.
        W = args.profile_width
        pool = I.walks24_1024() if W == 5 else insts
        x = pool if args.profile_batched else [pool[args.profile_case]]
        b = torch.from_numpy(I.packed_array(x).view(np.int64)).to(dev)
        budget = 50_000_000 if W == 5 else 0
        if args.profile_variant >= 2:
            cfg = bpida.make_config(W, variant=args.profile_variant)
        else:
            cfg = bpida.make_config(W, exit_fraction_pct=0 if args.profile_default else 100, driver=1,
                                    variant=args.profile_variant, node_budget=budget)
        log = None
        for rep in range(2):
            bpida.set_timing(rep == 0)
            s = bpida.solve(b, W, cfg)
            torch.cuda.synchronize(dev)
            if rep == 0:
                log = bpida.launch_log()
        bpida.set_timing(False)
        st = bpida.last_stats()
        out = {"profile": "batched" if args.profile_batched else "case %d" % args.profile_case, "width": W,
               "boards": len(x), "status": s.status, "stats": st,
               "launches": [{"i": i, "ms": ms, "nodes": nd} for i, (ms, nd) in enumerate(log)]}
        if args.profile_case is not None:
            h = s.to_host()[0]
            out.update(length=h["length"], iters=h["iters"], nodes=h["nodes"])
        else:
            out["nodes"] = int(s.nodes.cpu().numpy().view(np.uint64).sum())
        if log:
            out["largest_launch"] = max(range(len(log)), key=lambda i: log[i][1])
        print(json.dumps(out), flush=True)
        return

    gold = load_golden(args.workload)
    # Multi-GPU: the instances are independent, so each rank solves its own
    # instance range with no collective on the data path; the results are
    # gathered at the end (strong scaling: the whole job is the workload).
    # --replicas: every rank solves the whole workload (weak scaling).
    n_all = len(insts)
    copies = world if (world > 1 and args.replicas) else 1
    lo, hi = (0, n_all) if copies > 1 else shard_range(n_all, world, rank)
    insts = insts[lo:hi]
    n = len(insts)
    packed = I.packed_array(insts)
    boards = torch.from_numpy(packed.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)
    timer = Timer(torch, dev, stream, pg)
    base_cfg = bpida.make_config(4, driver=1 if args.driver == "host" else 0)
    batched_step, plain_step = make_steps(bpida, boards, n, base_cfg)
    k = args.steps

    def mx(v):
        return max_over_ranks(v, pg, dev)

    def job_rows(hosts):
        # the final gather (outside the timed region): every board of the job, in order
        return hosts if copies > 1 else gather_rows(hosts, pg, dev)

    # headline: the batched form, K timed steps
    with ClockSampler(local) as clk:
        ms_b, agg_b, bsols = timer.run(batched_step, k, args.warmup)
    clocks = clk.summary()
    hb = hosts_of(bsols)
    exp_rank = sum(sum(h["nodes"]) for h in hb)
    exp_per_step = copies * sum_over_ranks(exp_rank, pg if copies == 1 else None, dev)
    rows_b = job_rows(hb)
    par_b = parity(rows_b, gold) if gold else None
    t_batch = mx(sum(ms_b)) / 1e3
    n_job = copies * n_all
    value = exp_per_step * k / t_batch
    inst_s = n_job * k / t_batch

    # the plain form: one call per board, fewer timed steps
    kp = max(1, min(args.plain_steps, k))
    ms_p, _, psols = timer.run(plain_step, kp, 1)
    hp = hosts_of(psols)
    if sum(sum(h["nodes"]) for h in hp) != exp_rank:
        raise RuntimeError("batched and plain expansions differ")
    rows_p = job_rows(hp)
    par_p = parity(rows_p, gold) if gold else None
    t_plain = mx(sum(ms_p)) / 1e3
    plain_inst_s = n_job * kp / t_plain

    # end to end through the host-buffer path: pinned boards copied in and
    # every result copied back inside the timed region (batched form)
    host_boards = torch.from_numpy(packed.view(np.int64)).pin_memory()
    ml, mi = bpida.max_len(4), bpida.max_iters(4)
    host_out = {key: torch.empty(sz, dtype=dt).pin_memory() for key, sz, dt in (
        ("len", n, torch.int32), ("moves", n * ml, torch.uint8), ("nodes", n * mi, torch.int64),
        ("iters", n, torch.int32), ("status", n, torch.int32), ("solutions", n, torch.int64))}
    h2d = host_boards.numel() * 8
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())

    def e2e_step():
        dboards = host_boards.to(dev, non_blocking=True)
        s = bpida.solve(dboards, 4, base_cfg)
        if s.status != bpida.OK:
            raise RuntimeError(bpida.status_str(s.status))
        host_out["len"].copy_(s.length, non_blocking=True)
        host_out["moves"].copy_(s.moves.reshape(-1), non_blocking=True)
        host_out["nodes"].copy_(s.nodes.reshape(-1), non_blocking=True)
        host_out["iters"].copy_(s.iters, non_blocking=True)
        host_out["status"].copy_(s.inst_status, non_blocking=True)
        host_out["solutions"].copy_(s.solutions, non_blocking=True)
        return [s], {}

    ms_e2e, _, _ = timer.run(e2e_step, k, 1)
    if int(host_out["nodes"].numpy().view(np.uint64).sum()) != exp_rank:
        raise RuntimeError("end-to-end expansions differ")
    t_e2e = mx(sum(ms_e2e)) / 1e3
    e2e_value = exp_per_step * k / t_e2e

    launches_job = sum_over_ranks(sum(a["launches"] for a in agg_b), pg, dev)

    # roofline of the dominant kernel (the batched form's k_search)
    roof = kernel_roofline(bpida, torch, dev, boards, "batched", clocks)
    dev_ms = sum(a["search_ms_device"] for a in agg_b)
    dev_nodes = sum(a["search_nodes"] for a in agg_b)
    roof["expansions_per_s_in_kernel_timed_steps"] = dev_nodes / (dev_ms / 1e3) if dev_ms else None
    roof["search_share_of_step"] = dev_ms / sum(ms_b) if dev_ms else None

    # HBM traffic of the frontiers and the hand-back queue (the only DRAM
    # traffic of the method: a subtree's search stays in shared memory): each
    # 24-byte record is written once and read once
    fq_bytes = 2 * 24 * sum(a["records"] + a["handed_back"] for a in agg_b) / k
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    fq_gbs = fq_bytes / (t_batch / k) / 1e9
    hbm = {"bytes_per_step": fq_bytes, "gbs": fq_gbs, "peak_gbs": hbm_peak,
           "frac": fq_gbs / hbm_peak if hbm_peak else None,
           "what": "frontier records (splitter writes, first pass reads) and hand-back queue records, "
                   "24 B each, written once and read once, batched form"}

    sub = {}
    if rank == 0 and not args.no_sub:
        ks = max(1, args.sub_steps)
        if args.workload != "perms15_100":
            sub["perms15_100"] = leg_perms(bpida, torch, dev, timer, ks, clocks)
        sub["walks24_1024"] = leg_walks24(bpida, torch, dev, timer, ks, clocks)
        sub["serving"] = leg_serving(bpida, torch, dev, [float(r) for r in args.sub_serving_rates.split(",")],
                                     args.sub_serving_requests)
        if world == 1:
            sub["first_solution"] = leg_first_solution(bpida, torch, dev, args.first_solution_nodes)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        sample, cores = pick_cpu_sample(insts, gold, args.cpu_sample_nodes, args.cpu_sample_board_cap)
        t0 = time.perf_counter()
        res = oracle.solve_batch(4, I.tiles_array([insts[i] for i in sample]), count_all=True, nthreads=cores)
        dt = time.perf_counter() - t0
        cn = sum(r.total_nodes for r in res)
        cpu = {"value": cn / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": cpu_sample_desc(insts, sample, cn, args.cpu_sample_board_cap) + ", %.1f s" % dt,
               "instances_per_s": len(sample) / dt,
               "note": "instances/s of the sample only: its boards are cheaper than the workload's average, so "
                       "this is not comparable with the GPU's instances/s over the whole workload"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": k,
            "warmup": args.warmup, "ms_per_step": t_batch * 1e3 / k, "higher_is_better": True,
            "scaling": "weak" if (world == 1 or copies > 1) else "strong",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload],
                       "mode": "batched: each GPU's boards in one solve call",
                       "driver": args.driver,
                       "parallelism": ("replicas: every GPU solves all %d boards" % n_all) if copies > 1 else
                                      ("instance ranges: %d GPUs, %d-%d boards each, results gathered" % (
                                          world, n_all // world, -(-n_all // world)) if world > 1 else "single GPU"),
                       "l2": "flushed between steps (256 MiB write)"},
            "instances_per_s": inst_s,
            "expansions_per_step": exp_per_step,
            "plain": {"value": exp_per_step * kp / t_plain, "unit": UNIT, "instances_per_s": plain_inst_s,
                      "ms_per_step": t_plain * 1e3 / kp, "steps": kp, "mode": "one solve call per board"},
            "batched_over_plain_instances_per_s": inst_s / plain_inst_s,
            "parity": {"batched": par_b, "plain": par_p,
                       "against": "tests/golden/%s.json: stored oracle results (length, nodes per iteration, "
                                  "first solution, solution count) of every board" % args.workload},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": t_e2e * 1e3 / k, "instances_per_s": n_job * k / t_e2e},
            "roofline": roof,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                       "reasons": clocks["reasons"]},
            "gpu_launches": launches_job,
            "hbm_frontier_queue": hbm,
            "cpu_baseline": cpu,
        }
        line.update(sub)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
