"""Write the oracle's results for a named seeded workload to JSON.

Calls only ``oracle`` (plain sequential IDA*, count-all mode) and the seeded
input generators, never the CUDA path. Instances are solved one per worker
thread (the C call releases the GIL) and the file is rewritten as results
arrive, so an interrupted run keeps what it finished; a rerun skips the
instances already present.

usage: python tests/golden/make_golden.py WORKLOAD [--threads N]
       [--budget NODES] [--only-kind walk|perm] [--pdb PARTITION]

With --pdb the heuristic is the oracle's pattern databases for that tile
partition (inputs.PDB_PARTITIONS) and the file is WORKLOAD_pdbPARTITION.json.
"""
import argparse
import json
import os
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1705_02843_gb300 import inputs as I  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(I.WORKLOADS))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--budget", type=int, default=0, help="per-instance node budget (0 = none)")
    ap.add_argument("--only-kind", default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--pdb", default=None, choices=sorted(I.PDB_PARTITIONS))
    args = ap.parse_args()

    insts = I.WORKLOADS[args.workload]()
    name = args.workload + ("_pdb" + args.pdb if args.pdb else "")
    pdb = oracle.PatternDb(insts[0].W, I.PDB_PARTITIONS[args.pdb]) if args.pdb else None
    path = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json")
    done = {}
    if os.path.exists(path):
        with open(path) as f:
            for rec in json.load(f)["instances"]:
                done[rec["index"]] = rec
    todo = [i for i, x in enumerate(insts)
            if i not in done and (args.only_kind is None or x.kind == args.only_kind)]
    lock = threading.Lock()

    def save():
        doc = {
            "workload": args.workload,
            "generator": "paper_1705_02843_gb300.inputs." + I.WORKLOADS[args.workload].__name__,
            "oracle": "oracle/ida_oracle.c (count-all mode)",
            "heuristic": ("pattern databases, groups %s" % I.PDB_PARTITIONS[args.pdb]) if args.pdb
                         else "Manhattan distance",
            "node_budget": args.budget,
            "instances": [done[k] for k in sorted(done)],
        }
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(doc, f, separators=(",", ":"))
        os.replace(tmp, path)

    def work(i):
        x = insts[i]
        t0 = time.time()
        r = oracle.solve(x.W, x.tiles, count_all=True, node_budget=args.budget, pdb=pdb)
        rec = {
            "index": i, "seed": x.seed, "kind": x.kind, "walk_len": x.walk_len,
            "status": r.status, "length": r.length, "h0": r.h0, "iters": r.iters,
            "nodes": r.nodes, "limits": r.limits, "solutions": r.solutions,
            "moves": "".join(str(m) for m in r.moves), "oracle_s": round(time.time() - t0, 3),
        }
        with lock:
            done[i] = rec
            save()
        print("%5d %-4s len=%3d nodes=%14d %.1fs" % (i, x.kind, r.length, r.total_nodes, time.time() - t0),
              flush=True)

    with ThreadPoolExecutor(max_workers=args.threads) as ex:
        list(ex.map(work, todo))
    with lock:
        save()


if __name__ == "__main__":
    main()
