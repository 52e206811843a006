"""CUDA path vs the CPU oracle, bit-exact on every integer result.

Every test calls the C ABI (libbpida.so) through the Python binding on
seeded synthetic boards and compares, per instance: status, optimal length,
nodes expanded in every iteration (all-solutions mode, so the final
iteration's count is order-free) and the first solution, which must be the
oracle's (the lexicographically first optimal move sequence in U<L<R<D
order) and must replay to the goal.
"""
import json
import os
import random

import numpy as np
import pytest
import torch

import oracle
from paper_1705_02843_gb300 import bpida
from paper_1705_02843_gb300 import inputs as I
from tests import puzzle_ref as P

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gpu_solve(W, boards_tiles, **cfg):
    packed = [I.pack(W, t) for t in boards_tiles]
    arr = np.array(packed, dtype=np.uint64).reshape(-1) if W <= 4 else np.array(packed, dtype=np.uint64).reshape(-1, 2)
    t = torch.from_numpy(arr.view(np.int64)).to("cuda:0")
    sol = bpida.solve(t, W, bpida.make_config(W, **cfg))
    torch.cuda.synchronize()
    return sol.status, sol.to_host()


def check_against(W, tiles, got, ref):
    assert len(got) == len(ref)
    for i, (g, r) in enumerate(zip(got, ref)):
        assert g["status"] == r.status, (i, g["status"], r.status)
        if r.status != oracle.OK:
            continue
        assert g["length"] == r.length, (i, g["length"], r.length)
        assert g["nodes"] == r.nodes, (i, g["nodes"], r.nodes)
        assert g["iters"] == r.iters
        assert g["moves"] == r.moves, (i, g["moves"], r.moves)
        assert g["solutions"] == r.solutions, (i, g["solutions"], r.solutions)
        assert P.replay(W, tiles[i], g["moves"]) == list(range(W * W))


def test_walks15_16x40():
    insts = I.walks15_16x40()
    tiles = [x.tiles for x in insts]
    rc, got = gpu_solve(4, tiles)
    assert rc == bpida.OK
    check_against(4, tiles, got, oracle.solve_batch(4, np.array(tiles, dtype=np.uint8)))


def test_edge_cases_15():
    goal = list(range(16))
    one = [1, 0] + list(range(2, 16))
    two = [1, 2, 0] + list(range(3, 16))
    walk = I.walks15_16x40()[3].tiles
    unsolvable = list(walk)
    a, b = [p for p in range(16) if unsolvable[p]][:2]
    unsolvable[a], unsolvable[b] = unsolvable[b], unsolvable[a]
    notperm = [1] * 16
    tiles = [goal, one, unsolvable, two, notperm, walk]
    rc, got = gpu_solve(4, tiles)
    assert rc == bpida.OK
    assert got[0]["length"] == 0 and got[0]["nodes"] == [1] and got[0]["moves"] == []
    assert got[1]["length"] == 1 and got[1]["nodes"] == [2] and got[1]["moves"] == [1]
    assert got[3]["length"] == 2 and got[3]["nodes"] == [3] and got[3]["moves"] == [1, 1]
    for i in (2, 4):
        assert got[i]["status"] == bpida.EINVAL and got[i]["length"] == -1
    ref = oracle.solve_batch(4, np.array([t if i not in (4,) else goal for i, t in enumerate(tiles)], dtype=np.uint8))
    for i in (0, 1, 3, 5):
        assert got[i]["nodes"] == ref[i].nodes and got[i]["moves"] == ref[i].moves


def test_empty_batch():
    t = torch.zeros(0, dtype=torch.int64, device="cuda:0")
    sol = bpida.solve(t, 4)
    assert sol.status == bpida.OK and sol.length.numel() == 0


@pytest.mark.parametrize("n", [1, 33, 257])
def test_ragged_batches(n):
    rng = random.Random(n)
    insts = [I.make_walk(4, 7000 + i, rng.randint(0, 36)) for i in range(n)]
    tiles = [x.tiles for x in insts]
    rc, got = gpu_solve(4, tiles)
    assert rc == bpida.OK
    check_against(4, tiles, got, oracle.solve_batch(4, np.array(tiles, dtype=np.uint8)))


def test_all_8puzzle_states():
    dist, count, order = P.bfs8()
    tiles = [list(s) for s in order]
    rc, got = gpu_solve(3, tiles)
    assert rc == bpida.OK
    ref = oracle.solve_batch(3, np.array(tiles, dtype=np.uint8))
    for i, (s, g, r) in enumerate(zip(order, got, ref)):
        assert g["length"] == dist[s]
        assert g["nodes"] == r.nodes, (i, g["nodes"], r.nodes)
        assert g["moves"] == r.moves
        # all-solutions mode counts every shortest path (BFS path counting)
        assert g["solutions"] == count[s], (i, g["solutions"], count[s])
    rs = random.Random(1)
    for i in rs.sample(range(len(order)), 2000):
        assert P.replay(3, tiles[i], got[i]["moves"]) == list(range(9))


@pytest.mark.parametrize("cfg", [
    dict(stack_entries=256), dict(stack_entries=1024), dict(warps_per_block=8),
    dict(split_target=1), dict(split_target=2, min_rounds=32, exit_fraction_pct=1),
    dict(split_target=64, exit_fraction_pct=90),
    dict(driver=1), dict(driver=1, split_target=1, stack_entries=1024),
    dict(min_pass_us=-1, exit_fraction_pct=1, min_rounds=32), dict(min_pass_us=1000),
    dict(variant=1), dict(variant=1, driver=1), dict(variant=1, split_target=1),
    dict(variant=6), dict(variant=6, warps_per_block=8), dict(variant=6, warps_per_block=1, stack_entries=256),
    dict(variant=6, driver=1, split_target=1), dict(variant=6, min_pass_us=-1, exit_fraction_pct=1, min_rounds=32),
])
def test_tuning_knobs_do_not_change_results(cfg):
    insts = I.walks15_16x40()[:8]
    tiles = [x.tiles for x in insts]
    rc, got = gpu_solve(4, tiles, **cfg)
    assert rc == bpida.OK
    check_against(4, tiles, got, oracle.solve_batch(4, np.array(tiles, dtype=np.uint8)))


def test_block_size_changes_between_calls():
    """The search kernel is shared by every block size: a call with small
    blocks must not leave its shared-memory limit too low for the next call
    with larger ones."""
    insts = I.walks15_16x40()[:4]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    for wpb in (4, 1, 4, 8, 2, 8):
        rc, got = gpu_solve(4, tiles, warps_per_block=wpb)
        assert rc == bpida.OK, wpb
        check_against(4, tiles, got, ref)


def test_many_configurations_cycle_through_the_graph_cache():
    """More distinct launch configurations than cached graphs: evicted
    graphs are rebuilt on reuse and every call stays exact."""
    insts = I.walks15_16x40()[:3]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    targets = [16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768]
    for st in targets + targets[:3]:
        rc, got = gpu_solve(4, tiles, split_target=st)
        assert rc == bpida.OK, st
        check_against(4, tiles, got, ref)


def test_node_budget():
    insts = I.walks15_16x40()[:2]
    tiles = [x.tiles for x in insts]
    rc, got = gpu_solve(4, tiles, node_budget=50)
    assert all(g["status"] == bpida.EBUDGET and g["length"] == -1 for g in got)
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    for g, r in zip(got, ref):
        # completed iterations before the budget ran out are exact
        assert g["nodes"] == r.nodes[:len(g["nodes"])]


@pytest.mark.parametrize("which", [0, 6, 14])
def test_node_budget_boundary_matches_oracle(which):
    """A budget equal to the oracle's total solves the board; one node less
    must stop it, on the GPU as in the oracle, including when the budget runs
    out in the middle of a large iteration."""
    x = I.walks15_16x40()[which]
    r = oracle.solve(4, x.tiles)
    total = r.total_nodes
    assert oracle.solve(4, x.tiles, node_budget=total).status == oracle.OK
    assert oracle.solve(4, x.tiles, node_budget=total - 1).status == oracle.BUDGET
    rc, got = gpu_solve(4, [x.tiles], node_budget=total)
    assert got[0]["status"] == bpida.OK and got[0]["nodes"] == r.nodes
    rc, got = gpu_solve(4, [x.tiles], node_budget=total - 1)
    assert got[0]["status"] == bpida.EBUDGET and got[0]["nodes"] == r.nodes[:-1]
    mid = sum(r.nodes[:-1]) + r.nodes[-1] // 3
    rc, got = gpu_solve(4, [x.tiles], node_budget=mid)
    assert got[0]["status"] == bpida.EBUDGET and got[0]["nodes"] == r.nodes[:-1]


def test_budget_drops_only_the_instance_over_budget():
    insts = I.walks15_16x40()[:6]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    budget = sorted(r.total_nodes for r in ref)[3]
    rc, got = gpu_solve(4, tiles, node_budget=budget)
    for g, r in zip(got, ref):
        if r.total_nodes <= budget:
            assert g["status"] == bpida.OK and g["nodes"] == r.nodes and g["moves"] == r.moves
        else:
            assert g["status"] == bpida.EBUDGET and g["nodes"] == r.nodes[:len(g["nodes"])]


def test_24puzzle_walks():
    insts = [I.make_walk(5, 900 + s, 30 + 2 * s) for s in range(12)]
    tiles = [x.tiles for x in insts]
    rc, got = gpu_solve(5, tiles)
    assert rc == bpida.OK
    check_against(5, tiles, got, oracle.solve_batch(5, np.array(tiles, dtype=np.uint8)))


@pytest.mark.parametrize("cfg", [
    dict(exit_fraction_pct=1, min_rounds=1),
    dict(exit_fraction_pct=1, min_rounds=1, split_target=8, warps_per_block=4),
    dict(exit_fraction_pct=5, min_rounds=16, split_target=64, stack_entries=512),
])
def test_24puzzle_hand_backs(cfg):
    """24-puzzle batches with busy warps handing their stacks back early
    and often (many passes per step): open nodes leave the search stacks as
    records and come back, so the stack's board form is converted both ways
    many times. Results against the oracle; the host driver reports the
    passes."""
    insts = [I.make_walk(5, 930 + s, 36 + 2 * s) for s in range(10)]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(5, np.array(tiles, dtype=np.uint8))
    rc, got = gpu_solve(5, tiles, driver=1, **cfg)
    assert rc == bpida.OK
    st = bpida.last_stats()
    assert st["passes"] > st["steps"]
    check_against(5, tiles, got, ref)


def _golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle results for " + name)
    with open(path) as f:
        return json.load(f)


def _check_golden(W, insts, got, recs):
    """Compare with stored oracle results; boards the oracle stopped at its
    node budget must stop on the GPU too, with the completed iterations
    equal."""
    checked = 0
    for r in recs:
        g = got[r["index"]]
        assert g["status"] == r["status"], (r["index"], g["status"], r["status"])
        if r["status"] == oracle.OK:
            assert g["length"] == r["length"], r["index"]
            assert g["nodes"] == r["nodes"], r["index"]
            assert "".join(map(str, g["moves"])) == r["moves"], r["index"]
            assert g["solutions"] == r["solutions"], r["index"]
            assert P.replay(W, insts[r["index"]].tiles, g["moves"]) == list(range(W * W))
        else:
            assert g["nodes"] == r["nodes"][:-1], r["index"]
        checked += 1
    return checked


def test_perms15_100_full_plain_and_batched():
    """All 100 random permutations, one solve call per board (the benchmark's
    launch form) and all in one call."""
    doc = _golden("perms15_100")
    insts = I.perms15_100()
    rc, batched = gpu_solve(4, [x.tiles for x in insts])
    assert rc == bpida.OK
    assert _check_golden(4, insts, batched, doc["instances"]) == 100
    plain = []
    for x in insts:
        rc, g = gpu_solve(4, [x.tiles])
        assert rc == bpida.OK
        plain.extend(g)
    assert plain == batched


def test_mixed15_4096_full():
    doc = _golden("mixed15_4096")
    insts = I.mixed15_4096()
    rc, got = gpu_solve(4, [x.tiles for x in insts])
    assert rc == bpida.OK
    assert _check_golden(4, insts, got, doc["instances"]) >= 4095
    for i, (x, g) in enumerate(zip(insts, got)):
        # properties that hold for every board, stored result or not
        assert g["status"] == 0
        assert P.replay(4, x.tiles, g["moves"]) == list(range(16))
        if x.kind == "walk":
            assert g["length"] <= x.walk_len and (x.walk_len - g["length"]) % 2 == 0


def test_walks24_1024_with_node_budget():
    doc = _golden("walks24_1024")
    budget = doc["node_budget"]
    insts = I.walks24_1024()
    rc, got = gpu_solve(5, [x.tiles for x in insts], node_budget=budget)
    assert rc == bpida.OK
    assert _check_golden(5, insts, got, doc["instances"]) == 1024
    assert sum(g["status"] == 0 for g in got) > 500


def test_graph_and_host_drivers_agree_on_batch():
    insts = I.walks15_16x40() + [I.make_walk(4, 8800 + i, 30 + i) for i in range(20)]
    tiles = [x.tiles for x in insts]
    rc0, a = gpu_solve(4, tiles, driver=0)
    rc1, b = gpu_solve(4, tiles, driver=1)
    assert rc0 == rc1 == bpida.OK
    assert a == b


def test_launch_log_of_a_host_driven_call():
    """With timing on, a host-driven call logs every search launch: one entry
    per pass, and the nodes of the entries add up to the nodes the search
    kernel popped; a graph-driven call logs nothing."""
    insts = I.walks15_16x40()
    tiles = [x.tiles for x in insts]
    bpida.set_timing(True)
    try:
        rc, got = gpu_solve(4, tiles, driver=1)
        st = bpida.last_stats()
        log = bpida.launch_log()
        assert rc == bpida.OK
        assert len(log) == st["passes"] > 0
        assert sum(nd for _, nd in log) == st["search_nodes"]
        assert all(ms > 0 for ms, _ in log)
        rc, _ = gpu_solve(4, tiles, driver=0)
        assert rc == bpida.OK and bpida.launch_log() == []
    finally:
        bpida.set_timing(False)


def test_small_stacks_report_queue_overflow_not_wrong_results():
    """A 256-entry stack spills so often on the 100 random permutations in
    one batched call that the hand-back queue overflows: the instances it
    hits end with BPIDA_ENOMEM, and every instance that ends with BPIDA_OK
    has the oracle's exact results."""
    doc = _golden("perms15_100")
    gold = {r["index"]: r for r in doc["instances"]}
    tiles = [x.tiles for x in I.perms15_100()]
    rc, got = gpu_solve(4, tiles, stack_entries=256)
    assert rc == bpida.OK
    statuses = {g["status"] for g in got}
    assert statuses <= {bpida.OK, bpida.ENOMEM}
    for i, g in enumerate(got):
        if g["status"] == bpida.OK:
            r = gold[i]
            assert g["length"] == r["length"] and g["nodes"] == r["nodes"], i
            assert "".join(map(str, g["moves"])) == r["moves"], i


def test_repeated_plain_calls_reuse_the_graph():
    insts = I.walks15_16x40()[:6]
    ref = oracle.solve_batch(4, np.array([x.tiles for x in insts], dtype=np.uint8))
    for x, r in zip(insts, ref):
        rc, got = gpu_solve(4, [x.tiles])
        assert rc == bpida.OK
        assert got[0]["nodes"] == r.nodes and got[0]["moves"] == r.moves


def test_first_solution_mode():
    """Stop at the first goal (Section 6's first-solution timing): optimal
    length and every non-final iteration exact, the final iteration no larger
    than in all-solutions mode, and the returned moves an optimal solution."""
    doc = _golden("perms15_100")
    cheap = sorted(doc["instances"], key=lambda r: sum(r["nodes"]))[:30]
    perms = I.perms15_100()
    insts = I.walks15_16x40() + [perms[r["index"]] for r in cheap]
    tiles = [x.tiles for x in insts]
    rc, got = gpu_solve(4, tiles, count_all=False)
    assert rc == bpida.OK
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), count_all=True)
    first = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), count_all=False)
    for t, g, r, f in zip(tiles, got, ref, first):
        assert g["status"] == 0 and g["length"] == r.length == f.length
        assert g["nodes"][:-1] == r.nodes[:-1] == f.nodes[:-1]
        assert 1 <= g["nodes"][-1] <= r.nodes[-1]
        assert len(g["moves"]) == g["length"]
        assert P.replay(4, t, g["moves"]) == list(range(16))


def test_block_mode_on_permutations_budgets_and_first_solutions():
    """Block per subtree group (variant 6): the 40 cheapest random
    permutations against the stored oracle results, a node budget that stops
    one board in the middle of an iteration, and first-solution mode."""
    doc = _golden("perms15_100")
    cheap = sorted(doc["instances"], key=lambda r: sum(r["nodes"]))[:40]
    perms = I.perms15_100()
    insts = [perms[r["index"]] for r in cheap]
    rc, got = gpu_solve(4, [x.tiles for x in insts], variant=6)
    assert rc == bpida.OK
    for r, g in zip(cheap, got):
        assert g["length"] == r["length"] and g["nodes"] == r["nodes"] and g["solutions"] == r["solutions"]
        assert "".join(map(str, g["moves"])) == r["moves"]
    x = I.walks15_16x40()[6]
    ref = oracle.solve(4, x.tiles)
    mid = sum(ref.nodes[:-1]) + ref.nodes[-1] // 3
    rc, got = gpu_solve(4, [x.tiles], variant=6, node_budget=mid)
    assert got[0]["status"] == bpida.EBUDGET and got[0]["nodes"] == ref.nodes[:-1]
    rc, got = gpu_solve(4, [x.tiles], variant=6, node_budget=ref.total_nodes)
    assert got[0]["status"] == bpida.OK and got[0]["nodes"] == ref.nodes
    tiles = [x.tiles for x in insts[:12]]
    rc, got = gpu_solve(4, tiles, variant=6, count_all=False)
    full = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    for t, g, r in zip(tiles, got, full):
        assert g["status"] == 0 and g["length"] == r.length and g["nodes"][:-1] == r.nodes[:-1]
        assert 1 <= g["nodes"][-1] <= r.nodes[-1]
        assert P.replay(4, t, g["moves"]) == list(range(16))


def test_paper_kernel_matches_on_permutations():
    """The paper's BPIDA* kernel (ablation) gives the same exact results."""
    doc = _golden("perms15_100")
    cheap = sorted(doc["instances"], key=lambda r: sum(r["nodes"]))[:40]
    perms = I.perms15_100()
    insts = [perms[r["index"]] for r in cheap]
    rc, got = gpu_solve(4, [x.tiles for x in insts], variant=1)
    assert rc == bpida.OK
    for r, g in zip(cheap, got):
        assert g["length"] == r["length"] and g["nodes"] == r["nodes"]
        assert "".join(map(str, g["moves"])) == r["moves"]


def test_fused_iterations_match_one_iteration_per_step():
    """Calls of at most 8 boards fuse their small early iterations into one
    step (one search at the highest limit, node counts split by slack); a
    16-board call runs one iteration per step. Every result must be the same
    and the oracle's, and the fused calls must take fewer steps than
    iterations."""
    insts = I.walks15_16x40()
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    rc, whole = gpu_solve(4, tiles)
    assert rc == bpida.OK
    check_against(4, tiles, whole, ref)
    steps_fused, iters = 0, 0
    for i in range(16):
        rc, one = gpu_solve(4, [tiles[i]])
        assert rc == bpida.OK
        steps_fused += bpida.last_stats()["steps"]
        iters += one[0]["iters"]
        check_against(4, [tiles[i]], one, [ref[i]])
    assert steps_fused < iters
    for lo in (0, 8):
        rc, eight = gpu_solve(4, tiles[lo:lo + 8])
        assert rc == bpida.OK
        check_against(4, tiles[lo:lo + 8], eight, ref[lo:lo + 8])
    # 8-puzzle states up to the diameter, one per call
    dist, count, order = P.bfs8()
    for s in [order[-1], order[-2], order[1000], order[50000]]:
        rc, one = gpu_solve(3, [list(s)])
        r = oracle.solve(3, list(s))
        assert one[0]["length"] == dist[s] and one[0]["nodes"] == r.nodes and one[0]["solutions"] == count[s]
        assert one[0]["moves"] == r.moves


def test_fused_iterations_24puzzle():
    """The 24-puzzle's fused-iteration kernel (calls of at most 8 boards):
    one board per call and four per call, against the oracle."""
    insts = [I.make_walk(5, 900 + s, 30 + 2 * s) for s in range(12)]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(5, np.array(tiles, dtype=np.uint8))
    steps, iters = 0, 0
    for i in range(12):
        rc, one = gpu_solve(5, [tiles[i]])
        assert rc == bpida.OK
        steps += bpida.last_stats()["steps"]
        iters += one[0]["iters"]
        check_against(5, [tiles[i]], one, [ref[i]])
    assert steps < iters
    for lo in (0, 4, 8):
        rc, four = gpu_solve(5, tiles[lo:lo + 4])
        assert rc == bpida.OK
        check_against(5, tiles[lo:lo + 4], four, ref[lo:lo + 4])


def test_first_solution_mode_one_board_per_call():
    """First-solution mode, one board per call (the plain form): the length and
    every non-final iteration exact, the final one at most the all-solutions
    count, the moves an optimal solution."""
    doc = _golden("perms15_100")
    cheap = sorted(doc["instances"], key=lambda r: sum(r["nodes"]))[:12]
    perms = I.perms15_100()
    insts = I.walks15_16x40() + [perms[r["index"]] for r in cheap]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), count_all=True)
    for t, r in zip(tiles, ref):
        rc, got = gpu_solve(4, [t], count_all=False)
        g = got[0]
        assert rc == bpida.OK and g["status"] == 0 and g["length"] == r.length
        assert g["nodes"][:-1] == r.nodes[:-1]
        assert 1 <= g["nodes"][-1] <= r.nodes[-1]
        assert P.replay(4, t, g["moves"]) == list(range(16))


def test_first_solution_mode_with_fused_steps():
    """One-board calls in first-solution mode fuse small thresholds into one
    step, and a fused step runs to completion: lengths and non-final counts
    are the oracle's, the final count is at most the all-solutions count and
    equals it when the final iteration was fused (small walks: here most of
    them); every path replays."""
    insts = I.walks15_16x40()
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), count_all=True)
    equal = 0
    for t, r in zip(tiles, ref):
        rc, got = gpu_solve(4, [t], count_all=False)
        g = got[0]
        assert rc == bpida.OK and g["status"] == 0 and g["length"] == r.length
        assert g["nodes"][:-1] == r.nodes[:-1]
        assert 1 <= g["nodes"][-1] <= r.nodes[-1]
        assert P.replay(4, t, g["moves"]) == list(range(16))
        equal += g["nodes"][-1] == r.nodes[-1]
    assert equal >= len(tiles) // 2


@pytest.mark.parametrize("cap", [30000, 32000000])
def test_fused_step_cap_does_not_change_results(cap):
    """bpida_set_fuse_nodes only moves thresholds between steps: one-board
    calls (fused) give the oracle's results at a small and a large cap."""
    insts = I.walks15_16x40()[:6] + I.perms15_100()[:2]
    tiles = [x.tiles for x in insts]
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8))
    bpida.set_fuse_nodes(cap)
    try:
        for t, r in zip(tiles, ref):
            rc, got = gpu_solve(4, [t])
            assert rc == bpida.OK
            check_against(4, [t], got, [r])
    finally:
        bpida.set_fuse_nodes(0)


def test_bpida_solve_default_entry_point():
    """bpida_solve, the call of the problem statement with the default
    configuration, called directly through the C ABI (no configuration
    struct, no per-instance status): 16 walks and two random permutations
    of the 4096-board mix against the oracle and the stored oracle results."""
    import ctypes

    lib = bpida.load()
    doc = {r["index"]: r for r in _golden("mixed15_4096")["instances"]}
    mix = I.mixed15_4096()
    insts = I.walks15_16x40() + [mix[20], mix[40]]
    n = len(insts)
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64)).to("cuda:0")
    ml, mi = bpida.max_len(4), bpida.max_iters(4)
    out_len = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    out_moves = torch.full((n, ml), 9, dtype=torch.uint8, device="cuda:0")
    out_nodes = torch.full((n, mi), -1, dtype=torch.int64, device="cuda:0")
    stream = torch.cuda.current_stream()
    rc = lib.bpida_solve(ctypes.c_void_p(boards.data_ptr()), n, ctypes.c_void_p(out_len.data_ptr()),
                         ctypes.c_void_p(out_moves.data_ptr()), ctypes.c_void_p(out_nodes.data_ptr()),
                         ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    assert rc == bpida.OK
    L = out_len.cpu().tolist()
    mv = out_moves.cpu().numpy()
    nd = out_nodes.cpu().numpy().view(np.uint64)
    ref = oracle.solve_batch(4, I.tiles_array(insts[:16]), count_all=True)
    want = [(r.length, r.nodes, "".join(map(str, r.moves))) for r in ref] + \
        [(doc[i]["length"], doc[i]["nodes"], doc[i]["moves"]) for i in (20, 40)]
    for i, (length, nodes, moves) in enumerate(want):
        assert L[i] == length
        assert [int(x) for x in nd[i, :len(nodes)]] == nodes and not nd[i, len(nodes):].any()
        assert "".join(str(int(x)) for x in mv[i, :length]) == moves and not mv[i, length:].any()
