"""bpida_solve_noalloc: the solve for callers that cannot allocate device
memory (a device whose memory a framework's pool allocator already holds,
loops that cannot take cudaMalloc's device synchronisation). Its workspace
is a fixed __device__ array inside the library, so the library allocates
nothing during the call.

Checked through the C ABI against bpida_solve_ex on two calls in a row, with
different batch sizes so that state left in the shared array by the first
call cannot leak into the second. Results must be identical (integers:
bit-exact), and both must equal the CPU oracle or its stored results. Also:
the largest batch it takes (BPIDA_NOALLOC_MAX_BOARDS, with random
permutations), null optional outputs, and device memory unchanged by a call.
This file is named to run after every other test file.
"""
import ctypes
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1705_02843_gb300 import bpida
from paper_1705_02843_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _boards(insts):
    return torch.from_numpy(I.packed_array(insts).view(np.int64)).to("cuda:0")


def _strip(rows):
    for x in rows:
        x.pop("solutions")  # only bpida_solve_ex reports solution counts
    return rows


def test_noalloc_matches_solve_on_two_calls_in_a_row():
    batches = [
        I.walks15_16x40() + [I.make_walk(4, 9100 + i, 20 + i) for i in range(24)],
        [I.make_walk(4, 9300 + i, 30 + (i % 9)) for i in range(7)],
    ]
    for insts in batches:
        b = _boards(insts)
        ref = bpida.solve(b, 4)
        got = bpida.solve_noalloc(b)
        torch.cuda.synchronize()
        assert ref.status == bpida.OK
        assert got.status == bpida.OK, bpida.status_str(got.status)
        r, g = _strip(ref.to_host()), _strip(got.to_host())
        assert g == r
        orc = oracle.solve_batch(4, I.tiles_array(insts), count_all=True)
        for gi, oi in zip(g, orc):
            assert gi["length"] == oi.length and gi["nodes"] == oi.nodes and gi["moves"] == oi.moves


def test_noalloc_largest_batch_with_random_permutations():
    """BPIDA_NOALLOC_MAX_BOARDS boards: the 30 cheapest random permutations of
    the 100-board workload (stored oracle results) and walks of 20-60 moves
    (oracle), in one call, then again; both calls equal bpida_solve_ex."""
    with open(os.path.join(GOLDEN, "perms15_100.json")) as f:
        gold = {r["index"]: r for r in json.load(f)["instances"]}
    perms = I.perms15_100()
    cheap = sorted(gold, key=lambda i: sum(gold[i]["nodes"]))[:30]
    n = bpida.NOALLOC_MAX_BOARDS
    walks = [I.make_walk(4, 9500 + i, 20 + (i % 41)) for i in range(n - len(cheap))]
    insts = [perms[i] for i in cheap] + walks
    b = _boards(insts)
    ref = _strip(bpida.solve(b, 4).to_host())
    orc = oracle.solve_batch(4, I.tiles_array(walks), count_all=True)
    for _ in range(2):
        got = bpida.solve_noalloc(b)
        torch.cuda.synchronize()
        assert got.status == bpida.OK, bpida.status_str(got.status)
        g = _strip(got.to_host())
        assert g == ref
        for i, gi in zip(cheap, g):
            assert gi["length"] == gold[i]["length"] and gi["nodes"] == gold[i]["nodes"]
            assert "".join(map(str, gi["moves"])) == gold[i]["moves"]
        for gi, oi in zip(g[len(cheap):], orc):
            assert gi["length"] == oi.length and gi["nodes"] == oi.nodes and gi["moves"] == oi.moves


def test_noalloc_null_optional_outputs_and_no_device_memory_change():
    """out_num_iters and out_status may be NULL; a call (after a first one on
    this device) leaves the device's free memory unchanged."""
    lib = bpida.load()
    insts = I.walks15_16x40()
    n = len(insts)
    b = _boards(insts)
    full = bpida.solve_noalloc(b)  # first call on the device: address look-up
    torch.cuda.synchronize()
    assert full.status == bpida.OK
    ml, mi = bpida.max_len(4), bpida.max_iters(4)
    out_len = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    out_moves = torch.full((n, ml), 9, dtype=torch.uint8, device="cuda:0")
    out_nodes = torch.full((n, mi), -1, dtype=torch.int64, device="cuda:0")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stream = torch.cuda.current_stream()
    rc = lib.bpida_solve_noalloc(b.data_ptr(), n, out_len.data_ptr(), out_moves.data_ptr(), out_nodes.data_ptr(),
                                 None, None, ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == bpida.OK
    assert free1 == free0
    assert torch.equal(out_len, full.length)
    assert torch.equal(out_moves, full.moves)
    assert torch.equal(out_nodes, full.nodes)


def test_noalloc_rejects_too_many_boards():
    n = bpida.NOALLOC_MAX_BOARDS + 1
    b = torch.zeros(n, dtype=torch.int64, device="cuda:0")
    got = bpida.solve_noalloc(b)
    assert got.status == bpida.EINVAL
