"""Pattern-database heuristic on the GPU vs the CPU oracle, bit-exact.

The tables built by bpida_pdb_create must equal the oracle's byte for byte
(including the 255 entries that are no abstract state), and every solve
through bpida_solve_pdb must return the oracle's status, length, nodes per
iteration, solution count and first solution under the same heuristic.
"""
import random

import numpy as np
import pytest
import torch

import oracle
from paper_1705_02843_gb300 import bpida
from paper_1705_02843_gb300 import inputs as I
from tests import puzzle_ref as P

pytestmark = pytest.mark.gpu

G8 = [[1, 2, 3, 4], [5, 6, 7, 8]]
G8B = [[1, 5], [2, 3, 6], [4, 7, 8]]
G555 = [[1, 2, 3, 4, 5], [6, 7, 8, 9, 10], [11, 12, 13, 14, 15]]
G663 = [[1, 2, 3, 4, 5, 6], [7, 8, 9, 10, 11, 12], [13, 14, 15]]


@pytest.fixture(scope="module")
def pdb8():
    return oracle.PatternDb(3, G8), bpida.PatternDb(3, G8)


@pytest.fixture(scope="module")
def pdb555():
    return oracle.PatternDb(4, G555), bpida.PatternDb(4, G555)


def gpu_solve(W, tiles, pdb, **cfg):
    packed = np.array([I.pack(W, t) for t in tiles], dtype=np.uint64).reshape(-1)
    t = torch.from_numpy(packed.view(np.int64)).to("cuda:0")
    sol = bpida.solve(t, W, bpida.make_config(W, **cfg), pdb=pdb)
    torch.cuda.synchronize()
    return sol.status, sol.to_host()


def check(W, tiles, got, ref, final_counts=True):
    assert len(got) == len(ref)
    for i, (g, r) in enumerate(zip(got, ref)):
        assert g["status"] == r.status, (i, g["status"], r.status)
        if r.status != oracle.OK:
            continue
        assert g["length"] == r.length, (i, g["length"], r.length)
        assert g["iters"] == r.iters, (i, g["iters"], r.iters)
        if final_counts:
            assert g["nodes"] == r.nodes, (i, g["nodes"], r.nodes)
            assert g["moves"] == r.moves, (i, g["moves"], r.moves)
            assert g["solutions"] == r.solutions
        else:
            assert g["nodes"][:-1] == r.nodes[:-1]
        assert P.replay(W, tiles[i], g["moves"]) == list(range(W * W))


G6 = [[1], [2], [3], [4, 5, 6], [7, 8, 9, 10, 11], [12, 13, 14, 15]]  # the largest number of groups


@pytest.mark.parametrize("W,groups", [(3, G8), (3, G8B), (4, G555), (4, G6)])
def test_tables_equal_oracle_and_walks(W, groups):
    ref = oracle.PatternDb(W, groups)
    with bpida.PatternDb(W, groups) as pdb:
        for g in range(len(groups)):
            tab = pdb.table(g).numpy()
            assert tab.size == ref.tables[g].size
            assert np.array_equal(tab, ref.tables[g]), g
            assert pdb.max_value(g) == ref.max_values[g]
        rng = random.Random(W * 10 + len(groups))
        tiles = [I.make_walk(W, 500 + i, rng.randint(0, 40)).tiles for i in range(40)]
        rc, got = gpu_solve(W, tiles, pdb)
        assert rc == bpida.OK
        check(W, tiles, got, oracle.solve_batch(W, np.array(tiles, dtype=np.uint8), pdb=ref))


def test_six_tile_tables_equal_oracle():
    """6-6-3: two 256 MB tables, larger than L2."""
    ref = oracle.PatternDb(4, G663)
    with bpida.PatternDb(4, G663) as pdb:
        for g in range(3):
            assert pdb.table_bytes(g) == ref.tables[g].size
            assert np.array_equal(pdb.table(g).numpy(), ref.tables[g]), g
        w = I.walks15_16x40()
        tiles = [x.tiles for x in w]
        rc, got = gpu_solve(4, tiles, pdb)
        assert rc == bpida.OK
        check(4, tiles, got, oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), pdb=ref))


def test_all_8puzzle_states(pdb8):
    ref_pdb, pdb = pdb8
    dist, count, order = P.bfs8()
    tiles = [list(s) for s in order]
    rc, got = gpu_solve(3, tiles, pdb)
    assert rc == bpida.OK
    ref = oracle.solve_batch(3, np.array(tiles, dtype=np.uint8), pdb=ref_pdb)
    for i, (s, g, r) in enumerate(zip(order, got, ref)):
        assert g["length"] == dist[s]
        assert g["nodes"] == r.nodes, (i, g["nodes"], r.nodes)
        assert g["moves"] == r.moves
        assert g["solutions"] == count[s]


@pytest.fixture(scope="module")
def perms_cheap(pdb555):
    """The 24 cheapest of the 100 random permutations under the 5-5-5
    heuristic, with the oracle's results."""
    ref_pdb, _ = pdb555
    w = I.perms15_100()
    res = oracle.solve_batch(4, I.tiles_array(w), pdb=ref_pdb)
    order = sorted(range(len(w)), key=lambda i: res[i].total_nodes)[:24]
    return [w[i].tiles for i in order], [res[i] for i in order]


@pytest.mark.parametrize("cfg", [dict(), dict(driver=1), dict(stack_entries=256), dict(stack_entries=512),
                                 dict(split_target=1, min_pass_us=-1, exit_fraction_pct=1, min_rounds=32),
                                 dict(warps_per_block=8)])
def test_perms_batched(pdb555, perms_cheap, cfg):
    _, pdb = pdb555
    tiles, ref = perms_cheap
    rc, got = gpu_solve(4, tiles, pdb, **cfg)
    assert rc == bpida.OK
    check(4, tiles, got, ref)


def test_perms_one_board_per_call(pdb555, perms_cheap):
    """Calls of at most 8 boards fuse the small iterations of a step."""
    _, pdb = pdb555
    tiles, ref = perms_cheap
    for i in range(0, 12):
        rc, got = gpu_solve(4, [tiles[i]], pdb)
        assert rc == bpida.OK
        check(4, [tiles[i]], got, [ref[i]])
    rc, got = gpu_solve(4, tiles[:8], pdb)
    assert rc == bpida.OK
    check(4, tiles[:8], got, ref[:8])


def test_walks_and_edge_cases(pdb555):
    ref_pdb, pdb = pdb555
    goal = list(range(16))
    one = [1, 0] + list(range(2, 16))
    walk = I.walks15_16x40()[3].tiles
    unsolvable = list(walk)
    a, b = [p for p in range(16) if unsolvable[p]][:2]
    unsolvable[a], unsolvable[b] = unsolvable[b], unsolvable[a]
    tiles = [goal, one, unsolvable] + [x.tiles for x in I.walks15_16x40()]
    rc, got = gpu_solve(4, tiles, pdb)
    assert rc == bpida.OK
    assert got[0]["length"] == 0 and got[0]["nodes"] == [1]
    assert got[1]["length"] == 1 and got[1]["nodes"] == [2] and got[1]["moves"] == [1]
    assert got[2]["status"] == bpida.EINVAL and got[2]["length"] == -1
    ref = oracle.solve_batch(4, np.array([goal, one, goal] + tiles[3:], dtype=np.uint8), pdb=ref_pdb)
    check(4, tiles[3:], got[3:], ref[3:])


@pytest.mark.parametrize("n", [1, 33, 257])
def test_ragged_batches(pdb555, n):
    ref_pdb, pdb = pdb555
    rng = random.Random(100 + n)
    tiles = [I.make_walk(4, 9000 + i, rng.randint(0, 50)).tiles for i in range(n)]
    rc, got = gpu_solve(4, tiles, pdb)
    assert rc == bpida.OK
    check(4, tiles, got, oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), pdb=ref_pdb))


def test_first_solution_mode(pdb555, perms_cheap):
    _, pdb = pdb555
    tiles, ref = perms_cheap
    rc, got = gpu_solve(4, tiles, pdb, count_all=False)
    assert rc == bpida.OK
    check(4, tiles, got, ref, final_counts=False)


def test_node_budget(pdb555, perms_cheap):
    ref_pdb, pdb = pdb555
    tiles, _ = perms_cheap
    budget = 40000
    rc, got = gpu_solve(4, tiles, pdb, node_budget=budget)
    assert rc == bpida.OK
    ref = oracle.solve_batch(4, np.array(tiles, dtype=np.uint8), node_budget=budget, pdb=ref_pdb)
    assert {r.status for r in ref} == {oracle.OK, oracle.BUDGET}
    for i, (g, r) in enumerate(zip(got, ref)):
        assert g["status"] == r.status, i
        if r.status == oracle.OK:
            assert g["nodes"] == r.nodes and g["moves"] == r.moves
        else:
            # the completed iterations are reported
            assert g["nodes"] == r.nodes[:-1], i


def test_empty_call_and_bad_arguments(pdb555, pdb8):
    _, pdb = pdb555
    t = torch.zeros(0, dtype=torch.int64, device="cuda:0")
    assert bpida.solve(t, 4, pdb=pdb).status == bpida.OK
    one = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    assert bpida.solve(one, 3, bpida.make_config(3), pdb=pdb).status == bpida.EINVAL   # width mismatch
    assert bpida.solve(one, 4, bpida.make_config(4, variant=1), pdb=pdb).status == bpida.EINVAL
    assert bpida.solve(one, 4, bpida.make_config(4, stack_entries=768), pdb=pdb).status == bpida.EINVAL
    assert bpida.solve(one, 4, bpida.make_config(4), pdb=pdb8[1]).status == bpida.EINVAL
