"""Autotuner for the solver's launch knobs.

Tunes the frontier cap (root-split size), warps per block, per-warp stack
size, hand-back threshold and minimum rounds before hand-back by coordinate
descent on measured throughput (instances/s) of a sample workload, in either
form: "plain" (one solve call per board) or "batched" (one call for all).
A candidate is accepted only if every result (length, nodes per iteration,
first solution, status) equals the expected results given by the caller
(normally the stored oracle results of the sample), so tuning can never
trade exactness for speed. The best configuration is cached per (GPU name,
SM count, width, form) in a JSON file.

    python -m paper_1705_02843_gb300.autotune --workload perms15_100 --form plain
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import bpida
from . import inputs as I

KNOBS = {
    "split_target": [1024, 2048, 4096, 8192],
    "warps_per_block": [2, 4, 8],
    "stack_entries": [384, 512, 768],
    "exit_fraction_pct": [5, 10, 25],
    "min_rounds": [32, 64, 128],
}
DEFAULT = {"split_target": 4096, "warps_per_block": 4, "stack_entries": 512,
           "exit_fraction_pct": 10, "min_rounds": 64}


def cache_path() -> str:
    return os.environ.get("BPIDA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bpida", "tune.json"))


def device_key(width: int, form: str) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|%d|w%d|%s" % (p.name, p.multi_processor_count, width, form)


def _config(width: int, knobs: Dict[str, int]) -> bpida.Config:
    return bpida.make_config(width, **knobs)


def _run(boards: torch.Tensor, width: int, form: str, knobs: Dict[str, int]):
    cfg = _config(width, knobs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if form == "batched":
        sols = [bpida.solve(boards, width, cfg)]
    else:
        sols = [bpida.solve(boards[i:i + 1], width, cfg) for i in range(boards.shape[0])]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if any(s.status != bpida.OK for s in sols):
        return None, dt
    res = []
    for s in sols:
        res.extend(s.to_host())
    return res, dt


def _same(res: Sequence[dict], expected: Sequence[dict]) -> bool:
    keys = ("status", "length", "nodes", "moves")
    return len(res) == len(expected) and all(all(r[k] == e[k] for k in keys) for r, e in zip(res, expected))


def tune(boards: torch.Tensor, width: int, form: str, expected: Sequence[dict],
         repeats: int = 2, rounds: int = 2, log=print) -> Dict[str, int]:
    """Coordinate descent from DEFAULT; returns the best knob setting whose
    results equal `expected` (per-board dicts with status/length/nodes/moves)."""
    n = boards.shape[0]

    def score(knobs):
        best = None
        for _ in range(repeats):
            res, dt = _run(boards, width, form, knobs)
            if res is None or not _same(res, expected):
                return None
            best = dt if best is None else min(best, dt)
        return n / best

    _run(boards, width, form, DEFAULT)  # warm-up (graphs, workspace)
    cur = dict(DEFAULT)
    cur_s = score(cur)
    if cur_s is None:
        raise RuntimeError("the default configuration does not reproduce the expected results")
    log("default %s: %.1f inst/s" % (cur, cur_s))
    for _ in range(rounds):
        improved = False
        for knob, values in KNOBS.items():
            for v in values:
                if v == cur[knob]:
                    continue
                cand = dict(cur, **{knob: v})
                s = score(cand)
                log("  %s=%s: %s" % (knob, v, "rejected" if s is None else "%.1f inst/s" % s))
                if s is not None and s > cur_s * 1.01:
                    cur, cur_s, improved = cand, s, True
        if not improved:
            break
    log("best %s: %.1f inst/s" % (cur, cur_s))
    return cur


def save(width: int, form: str, knobs: Dict[str, int], path: Optional[str] = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    doc = {}
    if os.path.exists(path):
        with open(path) as f:
            doc = json.load(f)
    doc[device_key(width, form)] = knobs
    with open(path, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)


def load_config(width: int, form: str, path: Optional[str] = None) -> Optional[bpida.Config]:
    """The cached configuration for this GPU, width and form, or None."""
    path = path or cache_path()
    if not os.path.exists(path):
        return None
    with open(path) as f:
        doc = json.load(f)
    knobs = doc.get(device_key(width, form))
    return _config(width, knobs) if knobs else None


def _golden_expected(workload: str, indices: List[int]) -> Optional[List[dict]]:
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = os.path.join(here, "tests", "golden", workload + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        by_index = {r["index"]: r for r in json.load(f)["instances"]}
    out = []
    for i in indices:
        r = by_index[i]
        out.append({"status": r["status"], "length": r["length"], "nodes": r["nodes"],
                    "moves": [int(c) for c in r["moves"]]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="perms15_100", choices=sorted(I.WORKLOADS))
    ap.add_argument("--form", default="plain", choices=["plain", "batched"])
    ap.add_argument("--sample", type=int, default=40, help="boards of the workload to tune on")
    ap.add_argument("--no-save", action="store_true")
    args = ap.parse_args()
    insts = I.WORKLOADS[args.workload]()
    W = insts[0].W
    idx = list(range(min(args.sample, len(insts))))
    sample = [insts[i] for i in idx]
    arr = I.packed_array(sample)
    boards = torch.from_numpy(arr.view(np.int64)).cuda()
    expected = _golden_expected(args.workload, idx)
    if expected is None:
        # no stored oracle results: the default configuration's results,
        # which the parity tests check against the oracle, are the reference
        res, _ = _run(boards, W, args.form, DEFAULT)
        expected = res
    best = tune(boards, W, args.form, expected)
    if not args.no_save:
        save(W, args.form, best)
        print("saved to", cache_path())


if __name__ == "__main__":
    main()
