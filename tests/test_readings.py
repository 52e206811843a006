"""CPU pins of two readings the CUDA path builds on, checked with code that
shares nothing with it (plain Python enumeration) against the oracle.

1. Fused iterations: because the Manhattan distance is consistent, f never
   decreases along a path, so one depth-first search at limit L + 2J counted
   by f gives the node count of every iteration L' <= L + 2J: the nodes with
   f <= L'.
2. The thread-parallel configurations' root sets (smallest f expanded first,
   nodes replaced in place by their children, goals never expanded): the
   expanded nodes counted at every limit they fit plus the roots' subtrees
   give sequential IDA*'s node counts at every limit.
"""
from collections import Counter

import numpy as np
import pytest

import oracle
from paper_1705_02843_gb300 import inputs as I
from tests import puzzle_ref as P


def _f_histogram(W, tiles, limit):
    """f of every node an f-limited depth-first search pops (goals popped but
    not expanded, the inverse of the last move never applied)."""
    goal = tuple(range(W * W))
    hist = Counter()
    stack = [(tuple(tiles), 0, -1)]
    while stack:
        s, g, last = stack.pop()
        f = g + P.manhattan_py(W, s)
        hist[f] += 1
        if s == goal:
            continue
        for m, c in P.neighbours(W, s):
            if last >= 0 and m == 3 - last:
                continue
            if g + 1 + P.manhattan_py(W, c) <= limit:
                stack.append((c, g + 1, m))
    return hist


@pytest.mark.parametrize("W,which", [(4, 2), (4, 3), (4, 5), (4, 12), (3, None)])
def test_one_search_at_the_top_limit_gives_every_lower_count(W, which):
    if W == 4:
        tiles = I.walks15_16x40()[which].tiles
    else:
        tiles = I.make_walk(3, 31, 24).tiles
    r = oracle.solve(W, tiles)
    h0 = P.manhattan_py(W, tiles)
    top = h0 + 2 * (r.iters - 1)
    hist = _f_histogram(W, tiles, top)
    for it in range(r.iters):
        L = h0 + 2 * it
        assert sum(c for f, c in hist.items() if f <= L) == r.nodes[it], (it, L)


def test_f_never_decreases_along_a_move():
    """The property behind reading 1, on random 15- and 24-puzzle boards:
    every move changes h by exactly 1, so f = g + h changes by 0 or 2."""
    rng = np.random.default_rng(3)
    for W in (4, 5):
        for k in range(40):
            tiles = I.make_walk(W, 500 + k, int(rng.integers(10, 60))).tiles
            s = tuple(tiles)
            h = P.manhattan_py(W, s)
            for _, c in P.neighbours(W, s):
                assert abs(P.manhattan_py(W, c) - h) == 1


@pytest.mark.parametrize("which,T", [(11, 64), (15, 128), (3, 256)])
def test_smallest_f_first_root_sets_are_count_exact(which, T):
    from tests.test_thread_parallel import model

    tiles = I.walks15_16x40()[which].tiles
    r = oracle.solve(4, tiles)
    for variant in (2, 3):  # PSimple, PStaticLB
        per_it, _ = model(4, tiles, variant, T, r.iters)
        assert [n for n, _ in per_it] == r.nodes
