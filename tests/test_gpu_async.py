"""The solve calls are stream-ordered and asynchronous.

A graph-driven call enqueues its work on the caller's stream and returns
without waiting; calls on different streams take different workspaces and
may overlap on the device. Every result is checked against the oracle or
its stored results once the streams are synchronised.
"""
import json
import os
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1705_02843_gb300 import bpida
from paper_1705_02843_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _mix_golden():
    with open(os.path.join(GOLDEN, "mixed15_4096.json")) as f:
        return {r["index"]: r for r in json.load(f)["instances"]}


def _boards(insts):
    return torch.from_numpy(I.packed_array(insts).view(np.int64)).to("cuda:0")


def _check(sol, want):
    got = sol.to_host()
    assert len(got) == len(want)
    for g, (length, nodes, moves) in zip(got, want):
        assert g["status"] == bpida.OK
        assert (g["length"], g["nodes"], "".join(map(str, g["moves"]))) == (length, nodes, moves)


def _golden_want(gold, idx):
    return [(gold[i]["length"], gold[i]["nodes"], gold[i]["moves"]) for i in idx]


def test_two_streams_overlap_and_match_the_oracle():
    """Two batches enqueued on two streams before either is synchronised."""
    gold = _mix_golden()
    mix = I.mixed15_4096()
    idx_a = list(range(0, 1024))
    idx_b = list(range(1024, 2048))
    a, b = _boards([mix[i] for i in idx_a]), _boards([mix[i] for i in idx_b])
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(sa):
        ra = bpida.solve(a, 4, stream=sa)
    with torch.cuda.stream(sb):
        rb = bpida.solve(b, 4, stream=sb)
    assert ra.status == bpida.OK and rb.status == bpida.OK
    torch.cuda.synchronize()
    _check(ra, _golden_want(gold, idx_a))
    _check(rb, _golden_want(gold, idx_b))


def test_a_call_returns_before_its_work_finishes():
    """The host gets control back long before the device finishes (after a
    first call has built the graph and sized the workspace)."""
    gold = _mix_golden()
    mix = I.mixed15_4096()
    idx = [i for i in range(4096) if mix[i].kind == "perm"][:64]
    b = _boards([mix[i] for i in idx])
    bpida.solve(b, 4).synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol = bpida.solve(b, 4)
    t_enqueue = time.perf_counter() - t0
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    assert sol.status == bpida.OK
    assert t_enqueue < 0.25 * t_all, (t_enqueue, t_all)
    _check(sol, _golden_want(gold, idx))


def test_back_to_back_calls_on_one_stream_without_synchronising():
    """Many calls on one stream reuse one workspace in stream order; nothing
    is synchronised until the end."""
    insts = I.walks15_16x40()
    ref = oracle.solve_batch(4, I.tiles_array(insts), count_all=True)
    b = _boards(insts)
    sols = [bpida.solve(b[i:i + 1], 4) for i in range(len(insts))]
    sols.append(bpida.solve(b, 4))
    torch.cuda.synchronize()
    want = [(r.length, r.nodes, "".join(map(str, r.moves))) for r in ref]
    for i, s in enumerate(sols[:-1]):
        _check(s, want[i:i + 1])
    _check(sols[-1], want)


def test_more_streams_than_pooled_workspaces():
    """Six streams share a pool of four workspaces: the calls that find every
    workspace busy wait on the device for one, and every result stays exact.
    The configuration also differs between streams (different graphs)."""
    gold = _mix_golden()
    mix = I.mixed15_4096()
    streams = [torch.cuda.Stream() for _ in range(6)]
    batches = [list(range(300 * k, 300 * k + 300)) for k in range(6)]
    boards = [_boards([mix[i] for i in idx]) for idx in batches]
    torch.cuda.synchronize()
    sols = []
    for k, (st, b) in enumerate(zip(streams, boards)):
        with torch.cuda.stream(st):
            cfg = bpida.make_config(4, split_target=1024 if k % 2 else 0)
            sols.append(bpida.solve(b, 4, cfg, stream=st))
    torch.cuda.synchronize()
    for s, idx in zip(sols, batches):
        assert s.status == bpida.OK
        _check(s, _golden_want(gold, idx))


def test_statistics_are_read_after_synchronising():
    """bpida_get_stats gives the last call's loop counts once its stream is
    idle (graph driver: copied back at the end of the call)."""
    insts = I.walks15_16x40()
    b = _boards(insts)
    sol = bpida.solve(b, 4)
    sol.synchronize()
    st = bpida.last_stats()
    assert st["steps"] > 0 and st["passes"] >= st["steps"]
    assert st["launches"] == 3 + 2 * st["steps"] + st["passes"]
    # the search kernel's pops: the counted iterations' (less the
    # splitter's) and the path-recovery steps'
    assert st["search_nodes"] > 0 and st["records"] > 0
