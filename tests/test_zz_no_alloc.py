"""bpida_solve_noalloc: the solve for callers that cannot allocate device
memory (work issued during another component's graph capture, devices whose
memory a framework pool already holds, loops that cannot take cudaMalloc's
device synchronisation). Its workspace is a fixed __device__ array inside the
library, so the library allocates nothing during the call.

Checked through the C ABI against bpida_solve_ex on two calls in a row, with
different batch sizes so that state left in the shared array by the first
call cannot leak into the second. Results must be identical (integers:
bit-exact), and both must equal the CPU oracle. This file is named to run
after every other test file.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1705_02843_gb300 import bpida
from paper_1705_02843_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _boards(insts):
    return torch.from_numpy(I.packed_array(insts).view(np.int64)).to("cuda:0")


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
        r, g = ref.to_host(), got.to_host()
        for x in r + g:
            x.pop("solutions")  # only bpida_solve_ex reports solution counts
        assert g == r
        orc = oracle.solve_batch(4, I.tiles_array(insts), count_all=True)
        for gi, oi in zip(g, orc):
            assert gi["length"] == oi.length and gi["nodes"] == oi.nodes and gi["moves"] == oi.moves


def test_noalloc_rejects_too_many_boards():
    n = bpida.NOALLOC_MAX_BOARDS + 1
    b = torch.zeros(n, dtype=torch.int64, device="cuda:0")
    got = bpida.solve_noalloc(b)
    assert got.status == bpida.EINVAL
