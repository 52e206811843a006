"""Autotuner for the solver's launch knobs.

Tunes the search mode (a warp or a block per subtree group: bpida_config
variant 0 or 6), the frontier cap (root-split size), warps per block,
per-warp stack size, hand-back threshold and minimum rounds before
hand-back by coordinate descent on measured throughput (instances/s) of a
sample workload, in either form: "plain" (one solve call per board) or
"batched" (one call for all). A candidate is accepted only if every result
(length, nodes per iteration, first solution, status) equals the expected
results given by the caller (normally the stored oracle results of the
sample), so tuning can never trade exactness for speed. The best
configuration is cached per (GPU name, SM count, width, form) in a JSON file
(BPIDA_TUNE_CACHE, else ~/.cache/bpida/tune.json), which bpida.solve reads
to fill the configuration fields a caller leaves at 0.

    python -m paper_1705_02843_gb300.autotune --workload perms15_100 --form plain
    python -m paper_1705_02843_gb300.autotune --workload walks24_1024 --form batched --budget 50000000
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
    "variant": [0, 6],
    "split_target": [1024, 2048, 4096, 8192],
    "warps_per_block": [2, 4, 8],
    "stack_entries": [384, 480, 512, 768],
    "exit_fraction_pct": [5, 10, 25],
    "min_rounds": [32, 64, 128],
}
# The library's defaults (bpida.cu) for each width.
DEFAULT = {"variant": 0, "split_target": 4096, "warps_per_block": 4, "stack_entries": 384,
           "exit_fraction_pct": 10, "min_rounds": 64}


def defaults(width: int) -> Dict[str, int]:
    d = dict(DEFAULT)
    if width == 3:
        d["stack_entries"] = 512
    return d


def knob_values(width: int) -> Dict[str, List[int]]:
    """The values tried for each knob (block mode is for widths 3 and 4)."""
    k = {name: list(v) for name, v in KNOBS.items()}
    if width == 5:
        k["variant"] = [0]
        k["stack_entries"] = [256, 384, 512, 768, 1024]
    return k


def cache_path() -> str:
    return bpida.tune_cache_path()


def device_key(width: int, form: str) -> str:
    return bpida.tune_key(width, form)


def _config(width: int, knobs: Dict[str, int], node_budget: int = 0) -> bpida.Config:
    return bpida.make_config(width, node_budget=node_budget, **knobs)


def _run(boards: torch.Tensor, width: int, form: str, knobs: Dict[str, int], node_budget: int = 0):
    cfg = _config(width, knobs, node_budget)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if form == "batched":
        sols = [bpida.solve(boards, width, cfg, tuned=False)]
    else:
        sols = [bpida.solve(boards[i:i + 1], width, cfg, tuned=False) for i in range(boards.shape[0])]
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
         repeats: int = 2, rounds: int = 2, log=print, node_budget: int = 0) -> Dict[str, int]:
    """Coordinate descent from the library's defaults; returns the best knob
    setting whose results equal `expected` (per-board dicts with
    status/length/nodes/moves)."""
    n = boards.shape[0]
    start = defaults(width)
    values = knob_values(width)

    def score(knobs):
        best = None
        for _ in range(repeats):
            res, dt = _run(boards, width, form, knobs, node_budget)
            if res is None or not _same(res, expected):
                return None
            best = dt if best is None else min(best, dt)
        return n / best

    _run(boards, width, form, start, node_budget)  # warm-up (graphs, workspace)
    cur = dict(start)
    cur_s = score(cur)
    if cur_s is None:
        raise RuntimeError("the default configuration does not reproduce the expected results")
    log("default %s: %.1f inst/s" % (cur, cur_s))
    for _ in range(rounds):
        improved = False
        for knob, vals in values.items():
            for v in vals:
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
    knobs = bpida.tuned_knobs(width, form, path)
    return _config(width, knobs) if knobs else None


def _golden_expected(workload: str, indices: List[int]) -> Optional[List[dict]]:
    """Stored oracle results; a board the oracle stopped at its node budget
    reports only its completed iterations."""
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = os.path.join(here, "tests", "golden", workload + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        by_index = {r["index"]: r for r in json.load(f)["instances"]}
    out = []
    for i in indices:
        r = by_index[i]
        ok = r["status"] == 0
        out.append({"status": r["status"], "length": r["length"] if ok else -1,
                    "nodes": r["nodes"] if ok else r["nodes"][:-1],
                    "moves": [int(c) for c in r["moves"]] if ok else []})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="perms15_100", choices=sorted(I.WORKLOADS))
    ap.add_argument("--form", default="plain", choices=["plain", "batched"])
    ap.add_argument("--sample", type=int, default=40, help="boards of the workload to tune on")
    ap.add_argument("--budget", type=int, default=0, help="node budget per board (as the stored results' oracle)")
    ap.add_argument("--rounds", type=int, default=2)
    ap.add_argument("--no-save", action="store_true")
    args = ap.parse_args()
    insts = I.WORKLOADS[args.workload]()
    W = insts[0].W
    idx = list(range(min(args.sample, len(insts))))
    sample = [insts[i] for i in idx]
    arr = I.packed_array(sample)
    boards = torch.from_numpy(arr.view(np.int64)).cuda()
    if W == 5:
        boards = boards.reshape(-1, 2)
    expected = _golden_expected(args.workload, idx)
    if expected is None:
        # no stored oracle results: the default configuration's results,
        # which the parity tests check against the oracle, are the reference
        res, _ = _run(boards, W, args.form, defaults(W), args.budget)
        expected = res
    best = tune(boards, W, args.form, expected, rounds=args.rounds, node_budget=args.budget)
    if not args.no_save:
        save(W, args.form, best)
        print("saved to", cache_path())


if __name__ == "__main__":
    main()
