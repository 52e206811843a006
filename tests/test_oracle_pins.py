"""Pins of the CPU oracle against facts fixed independently of it.

* closed forms: 9!/2 = 181,440 reachable 8-puzzle states; the 8-puzzle with
  the blank in a corner has diameter 31 with exactly two states at distance
  31 (Reinefeld 1993);
* brute force: breadth-first search of the whole 8-puzzle graph gives every
  state's optimal length, its number of shortest paths (= the number of
  optimal solutions the all-solutions mode of Section 6 must count) and its
  lexicographically smallest shortest path (= the first solution a
  depth-first search in U, L, R, D order must return);
* heuristic: Manhattan distance is 0 at the goal, never exceeds the true
  distance and changes by exactly 1 along every edge;
* hand-worked node counts for the first limits of tiny instances;
* an independent memoised tree-size recurrence for the nodes popped per
  iteration (root and goals counted, parent pruning, push iff f <= limit);
* thresholds rise by exactly 2 (every move changes g by 1 and h by 1);
* replay of every returned move sequence; A* optimal lengths; the walk
  bounds opt <= walk length and opt = walk length (mod 2).
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from paper_1705_02843_gb300 import inputs as I
from tests import puzzle_ref as P


@pytest.fixture(scope="module")
def bfs():
    return P.bfs8()


@pytest.fixture(scope="module")
def all8(bfs):
    dist, count, order = bfs
    states = order
    res = oracle.solve_batch(3, np.array(states, dtype=np.uint8), count_all=True)
    return states, res


def test_bfs_closed_forms(bfs):
    dist, count, order = bfs
    assert len(dist) == 181440 == 362880 // 2
    assert max(dist.values()) == 31
    assert sum(1 for d in dist.values() if d == 31) == 2


def test_solvability_rule_equals_reachability_w3(bfs):
    dist, _, _ = bfs
    perms = list(itertools.permutations(range(9)))
    ok = oracle.is_solvable_batch(3, np.array(perms, dtype=np.uint8))
    reach = np.array([p in dist for p in perms])
    assert ok.sum() == 181440
    assert np.array_equal(ok, reach)


def test_solvability_rejects(bfs):
    base = I.walks15_16x40()[0].tiles
    # swap two non-blank tiles: leaves the goal's parity class
    t = list(base)
    i, j = [p for p in range(16) if t[p] != 0][:2]
    t[i], t[j] = t[j], t[i]
    assert oracle.is_solvable(4, base)
    assert not oracle.is_solvable(4, t)
    assert oracle.solve(4, t).status == oracle.INVALID
    assert oracle.solve(4, [1] * 16).status == oracle.INVALID
    assert oracle.solve(4, list(range(15)) + [16]).status == oracle.INVALID


def test_optimal_lengths_all_8puzzle(bfs, all8):
    dist, _, _ = bfs
    states, res = all8
    assert all(r.status == oracle.OK for r in res)
    assert all(r.length == dist[s] for s, r in zip(states, res))


def test_solution_counts_all_8puzzle(bfs, all8):
    _, count, _ = bfs
    states, res = all8
    assert all(r.solutions == count[s] for s, r in zip(states, res))


def test_first_solution_is_lexmin_shortest_path(bfs, all8):
    dist, _, _ = bfs
    states, res = all8
    rng = random.Random(7)
    idx = [i for i, s in enumerate(states) if dist[s] >= 27] + rng.sample(range(len(states)), 3000)
    for i in idx:
        s, r = states[i], res[i]
        assert r.moves == P.lexmin_shortest_path(s, dist)
        assert P.replay(3, s, r.moves) == list(range(9))


def test_thresholds_rise_by_two_all_8puzzle(all8):
    states, res = all8
    for s, r in zip(states, res):
        assert r.h0 == P.manhattan_py(3, s)
        assert r.limits == [r.h0 + 2 * i for i in range(r.iters)]
        assert r.iters == (r.length - r.h0) // 2 + 1
        assert all(a <= b for a, b in zip(r.nodes, r.nodes[1:]))


def test_manhattan_admissible_and_consistent_w3(bfs):
    dist, _, order = bfs
    states = np.array(order, dtype=np.uint8)
    h = oracle.manhattan_batch(3, states)
    assert h[0] == 0 and tuple(order[0]) == tuple(range(9))
    d = np.array([dist[s] for s in order])
    assert np.all(h <= d)
    index = {s: i for i, s in enumerate(order)}
    a, b = [], []
    for i, s in enumerate(order):
        for _, n in P.neighbours(3, s):
            a.append(i)
            b.append(index[n])
    assert np.all(np.abs(h[np.array(a)] - h[np.array(b)]) == 1)


@pytest.mark.parametrize("W", [4, 5])
def test_manhattan_matches_python_and_unit_steps(W):
    rng = I.Xoshiro256ss(99 + W)
    boards = [I.random_permutation(W, rng) for _ in range(300)]
    h = oracle.manhattan_batch(W, np.array(boards, dtype=np.uint8))
    assert [int(x) for x in h] == [P.manhattan_py(W, b) for b in boards]
    for b in boards[:100]:
        hb = P.manhattan_py(W, b)
        for _, n in P.neighbours(W, tuple(b)):
            assert abs(int(oracle.manhattan(W, list(n))) - hb) == 1
    assert oracle.manhattan(W, list(range(W * W))) == 0


def test_hand_worked_counts():
    # start = goal: one node popped, and it is the goal
    r = oracle.solve(4, list(range(16)))
    assert (r.length, r.nodes, r.solutions, r.limits) == (0, [1], 1, [0])
    # blank at position 1 (tile 1 at 0): h0 = 1; root popped, L reaches the
    # goal (f = 1); R and D move tiles 2 and 5 away (f = 3 > 1, pruned);
    # the goal is popped: 2 nodes.
    t = [1, 0] + list(range(2, 16))
    r = oracle.solve(4, t)
    assert (r.length, r.nodes, r.solutions, r.moves) == (1, [2], 1, [1])
    # blank moved R, R from the goal: [1, 2, 0, 3, ...], h0 = 2. Root: L
    # gives h = 1, f = 2 (pushed); R (tile 3) and D (tile 6) give f = 4.
    # That child: L reaches the goal (f = 2), D moves tile 5 up (f = 4), R is
    # the inverse move. Then the goal: 3 nodes, one solution.
    t = [1, 2, 0] + list(range(3, 16))
    r = oracle.solve(4, t)
    assert (r.length, r.nodes, r.solutions, r.moves) == (2, [3], 1, [1, 1])


def test_tree_size_recurrence_8puzzle(bfs, all8):
    dist, _, _ = bfs
    states, res = all8
    rng = random.Random(3)
    picks = rng.sample(range(len(states)), 60)
    for i in picks:
        s, r = states[i], res[i]
        for L, n in zip(r.limits, r.nodes):
            nodes, goals = P.tree_size(3, s, L)
            assert nodes == n
        assert goals == r.solutions


@pytest.fixture(scope="module")
def walks16():
    w = I.walks15_16x40()
    return w, oracle.solve_batch(4, I.tiles_array(w), count_all=True)


def test_walk_bounds_replay_and_astar(walks16):
    w, res = walks16
    for x, r in zip(w, res):
        assert r.status == oracle.OK
        assert r.length <= x.walk_len and (x.walk_len - r.length) % 2 == 0
        assert P.replay(4, x.tiles, r.moves) == list(range(16))
        assert len(r.moves) == r.length
        assert r.limits == [r.h0 + 2 * i for i in range(r.iters)]
        assert all(a <= b for a, b in zip(r.nodes, r.nodes[1:]))
    for x, r in list(zip(w, res))[:8]:
        assert P.astar_length(4, x.tiles) == r.length


def test_tree_size_recurrence_15puzzle(walks16):
    w, res = walks16
    checked = 0
    for x, r in zip(w, res):
        for it, (L, n) in enumerate(zip(r.limits, r.nodes)):
            if n > 60000:
                continue
            nodes, goals = P.tree_size(4, x.tiles, L)
            assert nodes == n
            if it == r.iters - 1:
                assert goals == r.solutions
            checked += 1
    assert checked >= 50


def test_first_solution_mode(walks16):
    w, res = walks16
    first = oracle.solve_batch(4, I.tiles_array(w), count_all=False)
    for a, b in zip(res, first):
        assert b.length == a.length and b.moves == a.moves
        assert b.nodes[:-1] == a.nodes[:-1]
        assert b.nodes[-1] <= a.nodes[-1]
        assert b.solutions == 1


def test_budget_and_limits():
    x = I.walks15_16x40()[0]
    r = oracle.solve(4, x.tiles, node_budget=100)
    assert r.status == oracle.BUDGET


def test_24puzzle_small_walks():
    insts = [I.make_walk(5, 500 + s, 24) for s in range(6)]
    res = oracle.solve_batch(5, I.tiles_array(insts))
    for x, r in zip(insts, res):
        assert r.status == oracle.OK
        assert r.length <= 24 and r.length % 2 == 0
        assert P.replay(5, x.tiles, r.moves) == list(range(25))
        assert r.limits == [r.h0 + 2 * i for i in range(r.iters)]
    x, r = insts[0], res[0]
    for L, n in zip(r.limits, r.nodes):
        if n <= 50000:
            assert P.tree_size(5, x.tiles, L)[0] == n
