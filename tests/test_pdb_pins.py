"""Pins of the oracle's pattern-database heuristic (the memory-intensive
heuristic named as future work in the paper's conclusion, Section 7)
against facts fixed independently of it.

* the tables equal an independent 0-1 breadth-first search of each abstract
  space (``tests/puzzle_ref.py``), entry by entry, and hold exactly the
  16!/(16-k-1)! (or 9!/(9-k-1)!) abstract states of a k-tile group;
* special case: singleton groups give the Manhattan distance;
* the heuristic is 0 at the goal, never above the true distance, never below
  the Manhattan distance, has its parity, and changes by exactly 1 along
  every 8-puzzle edge (so limits rise by exactly 2, as with the Manhattan
  distance);
* IDA* with it returns every 8-puzzle state's BFS distance, its number of
  shortest paths and its lexicographically smallest shortest path; the first
  limit is h(start) and every later one the smallest pruned f;
* the nodes popped per iteration equal an independent memoised tree-size
  recurrence with the same heuristic;
* on 15-puzzle walks with the 5-5-5 partition: any admissible heuristic
  gives the same optimal length, the same number of optimal solutions and
  the same first solution as the Manhattan distance, which is pinned on its
  own.
"""
import math
import random

import numpy as np
import pytest

import oracle
from paper_1705_02843_gb300 import inputs as I
from tests import puzzle_ref as P

G8 = [[1, 2, 3, 4], [5, 6, 7, 8]]
G8B = [[1, 5], [2, 3, 6], [4, 7, 8]]
G15_3 = [[1, 2, 3], [4, 8, 12], [5, 6, 7], [9, 10, 11], [13, 14, 15]]
G15_555 = [[1, 2, 3, 4, 5], [6, 7, 8, 9, 10], [11, 12, 13, 14, 15]]


def _index(pos, blank):
    idx = 0
    for j, p in enumerate(pos):
        idx |= p << (4 * j)
    return idx | (blank << (4 * len(pos)))


@pytest.fixture(scope="module")
def bfs():
    return P.bfs8()


@pytest.fixture(scope="module")
def pdb8():
    return oracle.PatternDb(3, G8)


@pytest.fixture(scope="module")
def h8(bfs, pdb8):
    dist, count, order = bfs
    h = pdb8.h_batch(np.array(order, dtype=np.uint8))
    return {s: int(v) for s, v in zip(order, h)}


@pytest.mark.parametrize("W,groups", [(3, G8), (3, G8B), (4, G15_3),
                                      # 5- and 6-tile groups: the 24- and 28-bit indices of the
                                      # 15-puzzle partitions used by the benchmarks
                                      (3, [[1, 2, 3, 4, 5], [6, 7, 8]]), (3, [[2, 3, 5, 6, 7, 8], [1, 4]])])
def test_tables_equal_independent_01bfs(W, groups):
    pdb = oracle.PatternDb(W, groups)
    N = W * W
    for g, tab in zip(groups, pdb.tables):
        ref = P.pattern_distances(W, g)
        k = len(g)
        assert len(ref) == math.perm(N, k + 1)
        assert tab.size == 16 ** (k + 1)
        assert int((tab != 255).sum()) == len(ref)
        idx = np.array([_index(pos, b) for pos, b in ref], dtype=np.int64)
        want = np.array(list(ref.values()), dtype=np.uint8)
        assert np.array_equal(tab[idx], want)
    assert pdb.max_values == [max(P.pattern_distances(W, g).values()) for g in groups]


@pytest.mark.parametrize("seed", range(6))
def test_random_8puzzle_partitions_equal_independent_01bfs(seed):
    """Seeded random partitions of the 8 tiles into groups of 1 to 4 tiles."""
    rng = random.Random(seed)
    tiles = list(range(1, 9))
    rng.shuffle(tiles)
    groups = []
    while tiles:
        k = rng.randint(1, min(4, len(tiles)))
        groups.append(sorted(tiles[:k]))
        tiles = tiles[k:]
    pdb = oracle.PatternDb(3, groups)
    for g, tab in zip(groups, pdb.tables):
        ref = P.pattern_distances(3, g)
        assert int((tab != 255).sum()) == len(ref) == math.perm(9, len(g) + 1)
        idx = np.array([_index(pos, b) for pos, b in ref], dtype=np.int64)
        assert np.array_equal(tab[idx], np.array(list(ref.values()), dtype=np.uint8)), groups


def test_singleton_groups_reduce_to_manhattan(bfs):
    dist, count, order = bfs
    pdb = oracle.PatternDb(3, [[t] for t in range(1, 9)])
    h = pdb.h_batch(np.array(order, dtype=np.uint8))
    assert all(int(v) == P.manhattan_py(3, s) for s, v in zip(order, h))
    pdb = oracle.PatternDb(4, [[t] for t in range(1, 16)])
    rng = random.Random(5)
    boards = []
    for _ in range(200):
        t = list(range(16))
        rng.shuffle(t)
        boards.append(t)
    h = pdb.h_batch(np.array(boards, dtype=np.uint8))
    assert [int(v) for v in h] == [P.manhattan_py(4, s) for s in boards]


def test_admissible_consistent_dominates_manhattan_8puzzle(bfs, h8):
    dist, count, order = bfs
    assert h8[tuple(range(9))] == 0
    steps = set()
    for s in order:
        hs = h8[s]
        assert P.manhattan_py(3, s) <= hs <= dist[s]
        for _, n in P.neighbours(3, s):
            steps.add(h8[n] - hs)
    # a cost-1 abstract move shifts one of the group's tiles by one cell and
    # a cost-0 move none, so d_G has the parity of the group's Manhattan
    # distance and every real move changes h by exactly 1
    assert steps == {-1, 1}
    assert all((hs - P.manhattan_py(3, s)) % 2 == 0 for s, hs in h8.items())


@pytest.fixture(scope="module")
def all8_pdb(bfs, pdb8):
    dist, count, order = bfs
    return oracle.solve_batch(3, np.array(order, dtype=np.uint8), count_all=True, pdb=pdb8)


def test_ida_pdb_all_8puzzle(bfs, h8, all8_pdb):
    dist, count, order = bfs
    rises = set()
    for s, r in zip(order, all8_pdb):
        assert r.status == oracle.OK
        assert r.length == dist[s]
        assert r.solutions == count[s]
        assert r.h0 == h8[s]
        assert r.limits[0] == r.h0 and r.limits[-1] == r.length
        rises |= {b - a for a, b in zip(r.limits, r.limits[1:])}
    assert rises == {2}
    rng = random.Random(11)
    for i in rng.sample(range(len(order)), 300):
        assert all8_pdb[i].moves == P.lexmin_shortest_path(order[i], dist)


def test_tree_size_recurrence_pdb_8puzzle(bfs, pdb8, all8_pdb):
    dist, count, order = bfs
    tabs = [P.pattern_distances(3, g) for g in G8]
    h = lambda s: P.pattern_h(3, G8, tabs, s)
    rng = random.Random(4)
    for i in rng.sample(range(len(order)), 40):
        s, r = order[i], all8_pdb[i]
        for it, (L, n) in enumerate(zip(r.limits, r.nodes)):
            nodes, goals, fmin = P.tree_size_h(3, s, L, h)
            assert nodes == n
            if it + 1 < r.iters:
                assert goals == 0 and fmin == r.limits[it + 1]
            else:
                assert goals == r.solutions


@pytest.fixture(scope="module")
def walks16():
    w = I.walks15_16x40()
    return w, oracle.solve_batch(4, I.tiles_array(w), count_all=True)


def test_tree_size_recurrence_pdb_15puzzle(walks16):
    w, md = walks16
    pdb = oracle.PatternDb(4, G15_3)
    tabs = [P.pattern_distances(4, g) for g in G15_3]
    h = lambda s: P.pattern_h(4, G15_3, tabs, s)
    res = oracle.solve_batch(4, I.tiles_array(w), count_all=True, pdb=pdb)
    checked = 0
    for x, r, m in zip(w, res, md):
        assert (r.length, r.solutions, r.moves) == (m.length, m.solutions, m.moves)
        assert r.h0 == h(tuple(x.tiles))
        for it, (L, n) in enumerate(zip(r.limits, r.nodes)):
            if n > 60000:
                continue
            nodes, goals, fmin = P.tree_size_h(4, x.tiles, L, h)
            assert nodes == n
            if it + 1 < r.iters:
                assert fmin == r.limits[it + 1]
            else:
                assert goals == r.solutions
            checked += 1
    assert checked >= 40


@pytest.fixture(scope="module")
def pdb555():
    return oracle.PatternDb(4, G15_555)


def test_555_partition_properties(pdb555, walks16):
    w, md = walks16
    assert pdb555.max_values == [25, 21, 25]  # values fit the 6-bit fields of the search kernel
    rng = random.Random(9)
    boards, nexts = [], []
    for x in w:
        s = tuple(x.tiles)
        for _ in range(20):
            ns = P.neighbours(4, s)
            n = ns[rng.randrange(len(ns))][1]
            boards.append(s)
            nexts.append(n)
            s = n
    hb = pdb555.h_batch(np.array(boards, dtype=np.uint8))
    hn = pdb555.h_batch(np.array(nexts, dtype=np.uint8))
    assert set((hn - hb).tolist()) == {-1, 1}
    mh = np.array([P.manhattan_py(4, s) for s in boards])
    assert (hb >= mh).all() and ((hb - mh) % 2 == 0).all()
    # random permutations of the goal's parity class as well as walks
    perms = [x.tiles for x in I.perms15_100()[:50]]
    hp = pdb555.h_batch(np.array(perms, dtype=np.uint8))
    mp = np.array([P.manhattan_py(4, s) for s in perms])
    assert (hp >= mp).all() and ((hp - mp) % 2 == 0).all()
    res = oracle.solve_batch(4, I.tiles_array(w), count_all=True, pdb=pdb555)
    for x, r, m in zip(w, res, md):
        assert r.status == oracle.OK
        assert (r.length, r.solutions, r.moves) == (m.length, m.solutions, m.moves)
        assert m.h0 <= r.h0 <= r.length
        assert r.total_nodes <= m.total_nodes
        assert P.replay(4, x.tiles, r.moves) == list(range(16))


def test_bad_groups_are_rejected():
    with pytest.raises(ValueError):
        oracle.PatternDb(3, [[1, 2, 3, 4], [5, 6, 7]])  # tile 8 in no group
    with pytest.raises(ValueError):
        oracle.PatternDb(3, [[1, 2, 3, 4], [4, 5, 6, 7, 8]])  # tile 4 twice
    with pytest.raises(ValueError):
        oracle.PatternDb(3, [[1, 2, 3, 4, 5, 6, 7], [8]])  # more than 6 tiles


def test_blank_free_tables_would_be_inconsistent(bfs):
    """Why the blank's cell is part of every abstract state: tables that keep
    only the minimum over blank cells are still admissible but change h by up
    to 7 along an 8-puzzle edge (G's tiles can wall the blank in), so the
    search's slack arithmetic (s or s - 2) would not hold."""
    import collections

    dist, count, order = bfs
    tabs = []
    for g in G8:
        m = collections.defaultdict(lambda: 1 << 30)
        for (pos, b), v in P.pattern_distances(3, g).items():
            m[pos] = min(m[pos], v)
        tabs.append(m)

    def h(s):
        where = {v: p for p, v in enumerate(s)}
        return sum(t[tuple(where[x] for x in sorted(g))] for g, t in zip(G8, tabs))

    H = {s: h(s) for s in order}
    steps = {H[n] - H[s] for s in order for _, n in P.neighbours(3, s)}
    assert all(H[s] <= dist[s] for s in order)
    assert max(steps) == 7 and min(steps) == -7
