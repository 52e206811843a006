"""Continuous-batching service (bpida_server_*): requests submitted in waves
while earlier ones are still on the GPU must come back with exactly the
results the same boards get when solved alone (and the oracle's), and the
service must actually overlap them (several instances searched in one
step, fewer device steps than the requests need one by one)."""
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


def _alone(inst):
    t = torch.from_numpy(I.packed_array([inst]).view(np.int64)).to("cuda:0")
    sol = bpida.solve(t, 4)
    torch.cuda.synchronize()
    r = sol.to_host()[0]
    st = bpida.last_stats()
    return r, st["steps"]


def _drain(sv, want, deadline_s=180.0):
    got = {}
    t_end = time.time() + deadline_s
    while len(got) < want:
        for r in sv.poll():
            got[r["req_id"]] = r
        if time.time() > t_end:
            raise AssertionError("service did not finish in time: %d of %d" % (len(got), want))
        time.sleep(0.001)
    return got


def test_serving_matches_solo_results_in_the_mix():
    rng = I.Xoshiro256ss(4242)
    insts = [I.make_walk(4, 60000 + i, rng.uniform_int(20, 56)) for i in range(96)]
    with open(os.path.join(GOLDEN, "perms15_100.json")) as f:
        doc = json.load(f)
    cheap = sorted(doc["instances"], key=lambda r: sum(r["nodes"]))[:4]
    perms = I.perms15_100()
    insts += [perms[r["index"]] for r in cheap]
    solo = [_alone(x) for x in insts]
    packed = [int(w) for w in I.packed_array(insts)]
    with bpida.Server(frontier_bytes=256 << 20, max_slots=64) as sv:
        waves = [range(0, 30), range(30, 60), range(60, 100)]
        for w in waves:
            for i in w:
                sv.submit(packed[i], i)
            time.sleep(0.02)
        got = _drain(sv, len(insts))
        stats = sv.stats()
    for i, (r, _) in enumerate(solo):
        g = got[i]
        assert g["status"] == r["status"] == 0
        assert g["length"] == r["length"]
        assert g["nodes"] == r["nodes"]
        assert g["moves"] == r["moves"]
        assert g["solutions"] == r["solutions"]
    ref = oracle.solve_batch(4, I.tiles_array(insts))
    for i, o in enumerate(ref):
        assert got[i]["length"] == o.length and got[i]["nodes"] == o.nodes and got[i]["moves"] == o.moves
    # the requests overlapped on the device
    assert stats["completed"] == len(insts)
    assert stats["max_active"] > 1
    assert stats["steps"] < sum(steps for _, steps in solo)
    assert stats["slots"] == 64  # more requests than slots: admission waited for free slots


def test_serving_rejects_bad_boards_and_keeps_going():
    good = I.make_walk(4, 77, 30)
    bad = list(good.tiles)
    a, b = [p for p in range(16) if bad[p]][:2]
    bad[a], bad[b] = bad[b], bad[a]
    with bpida.Server(frontier_bytes=64 << 20, max_slots=8) as sv:
        sv.submit(I.pack(4, bad)[0], 1)
        sv.submit(I.pack(4, good.tiles)[0], 2)
        got = _drain(sv, 2)
    assert got[1]["status"] == bpida.EINVAL and got[1]["length"] == -1
    ref = oracle.solve(4, good.tiles)
    assert got[2]["status"] == 0 and got[2]["nodes"] == ref.nodes and got[2]["moves"] == ref.moves


def _mix_with_perms(n_walks, perm_ranks):
    rng = I.Xoshiro256ss(777)
    insts = [I.make_walk(4, 61000 + i, rng.uniform_int(20, 56)) for i in range(n_walks)]
    with open(os.path.join(GOLDEN, "perms15_100.json")) as f:
        doc = json.load(f)
    order = sorted(doc["instances"], key=lambda r: sum(r["nodes"]))
    perms = I.perms15_100()
    return insts + [perms[order[k]["index"]] for k in perm_ranks]


def test_time_sliced_steps_give_the_same_results():
    """With a 50-microsecond time slice the permutations' iterations run over
    many steps, their open nodes carried from step to step, while the walks
    advance and finish: every result equals the board's solo result and the
    oracle's."""
    insts = _mix_with_perms(60, [0, 1, 2, 3, 40, 60])
    solo = [_alone(x)[0] for x in insts]
    packed = [int(w) for w in I.packed_array(insts)]
    with bpida.Server(frontier_bytes=256 << 20, max_slots=48, time_slice_us=50) as sv:
        for i, w in enumerate(packed):
            sv.submit(w, i)
            if i % 20 == 19:
                time.sleep(0.005)
        got = _drain(sv, len(insts))
        stats = sv.stats()
    for i, r in enumerate(solo):
        g = got[i]
        assert g["status"] == r["status"] == 0
        assert (g["length"], g["nodes"], g["moves"], g["solutions"]) == (r["length"], r["nodes"], r["moves"],
                                                                          r["solutions"]), i
    ref = oracle.solve_batch(4, I.tiles_array(insts))
    for i, o in enumerate(ref):
        assert got[i]["nodes"] == o.nodes and got[i]["moves"] == o.moves
    assert stats["sliced_steps"] > 0


def _easy_latencies(slice_us):
    insts = _mix_with_perms(40, [99])
    packed = [int(w) for w in I.packed_array(insts)]
    with bpida.Server(frontier_bytes=256 << 20, max_slots=64, time_slice_us=slice_us) as sv:
        sv.submit(packed[-1], len(insts) - 1)  # the hardest board first (~1e10 nodes)
        time.sleep(0.02)                      # it is into its long iterations by now
        for i in range(len(insts) - 1):
            sv.submit(packed[i], i)
        got = _drain(sv, len(insts))
    lat = sorted(got[i]["latency_s"] for i in range(len(insts) - 1))
    return lat[len(lat) // 2], got


def test_time_slices_let_short_requests_pass_a_long_one():
    """Forty easy walks submitted while the hardest permutation is in its long
    iterations: with a 500-microsecond slice they are admitted and finish
    while the permutation still searches; without slices every step waits
    for the permutation's iteration."""
    sliced, got_s = _easy_latencies(500)
    whole, got_w = _easy_latencies(0)
    for i in got_s:
        assert got_s[i]["nodes"] == got_w[i]["nodes"] and got_s[i]["moves"] == got_w[i]["moves"]
    assert sliced < 0.5 * whole, (sliced, whole)
