"""Independent checkers used to pin the oracle (test-only helpers).

Nothing here is shared with the oracle or with the CUDA path: breadth-first
search of the 8-puzzle state graph, a Python Manhattan distance, replay of
move sequences, A* search and a memoised tree-size recurrence.
"""
from __future__ import annotations

import heapq
import sys
from collections import deque
from functools import lru_cache
from typing import Dict, List, Sequence, Tuple

DELTA_ROWCOL = {0: (-1, 0), 1: (0, -1), 2: (0, 1), 3: (1, 0)}  # U L R D (blank)


def neighbours(W: int, s: Tuple[int, ...]):
    """(move, next state) pairs for every legal blank move, in U L R D order."""
    b = s.index(0)
    r, c = divmod(b, W)
    out = []
    for m in range(4):
        dr, dc = DELTA_ROWCOL[m]
        rr, cc = r + dr, c + dc
        if 0 <= rr < W and 0 <= cc < W:
            q = rr * W + cc
            n = list(s)
            n[b], n[q] = n[q], 0
            out.append((m, tuple(n)))
    return out


def manhattan_py(W: int, s: Sequence[int]) -> int:
    h = 0
    for p, v in enumerate(s):
        if v:
            pr, pc = divmod(p, W)
            gr, gc = divmod(v, W)
            h += abs(pr - gr) + abs(pc - gc)
    return h


_BFS8 = None


def bfs8():
    """Distances and shortest-path counts to the goal for every reachable
    8-puzzle state (the graph is undirected, so BFS from the goal)."""
    global _BFS8
    if _BFS8 is None:
        goal = tuple(range(9))
        dist: Dict[tuple, int] = {goal: 0}
        order = [goal]
        q = deque([goal])
        while q:
            s = q.popleft()
            for _, n in neighbours(3, s):
                if n not in dist:
                    dist[n] = dist[s] + 1
                    order.append(n)
                    q.append(n)
        count = {goal: 1}
        for s in order[1:]:
            d = dist[s]
            count[s] = sum(count[n] for _, n in neighbours(3, s) if dist[n] == d - 1)
        _BFS8 = (dist, count, order)
    return _BFS8


def lexmin_shortest_path(s, dist) -> List[int]:
    """Lexicographically smallest (U<L<R<D) shortest move sequence to the goal."""
    path = []
    while dist[s] > 0:
        for m, n in neighbours(3, s):
            if dist[n] == dist[s] - 1:
                path.append(m)
                s = n
                break
    return path


def replay(W: int, tiles: Sequence[int], moves: Sequence[int]):
    """Apply blank moves; returns the final board or None if a move is illegal."""
    s = list(tiles)
    b = s.index(0)
    for m in moves:
        if m not in DELTA_ROWCOL:
            return None
        r, c = divmod(b, W)
        dr, dc = DELTA_ROWCOL[m]
        rr, cc = r + dr, c + dc
        if not (0 <= rr < W and 0 <= cc < W):
            return None
        q = rr * W + cc
        s[b], s[q] = s[q], 0
        b = q
    return s


def astar_length(W: int, tiles: Sequence[int]) -> int:
    """Optimal solution length by A* with the Manhattan heuristic and a
    closed set (the heuristic is consistent, so closed nodes are final)."""
    start = tuple(tiles)
    goal = tuple(range(W * W))
    g = {start: 0}
    heap = [(manhattan_py(W, start), 0, start)]
    closed = set()
    while heap:
        f, gs, s = heapq.heappop(heap)
        if s in closed:
            continue
        if s == goal:
            return gs
        closed.add(s)
        for _, n in neighbours(W, s):
            ng = gs + 1
            if n not in closed and ng < g.get(n, 1 << 30):
                g[n] = ng
                heapq.heappush(heap, (ng + manhattan_py(W, n), ng, n))
    return -1


def tree_size(W: int, tiles: Sequence[int], limit: int) -> Tuple[int, int]:
    """(nodes, goals) of the f-limited tree, by the recurrence
    T(s, g, last) = (1, 1) at a goal, else 1 + sum of T over children c
    (moves other than the inverse of ``last``) with g + 1 + h(c) <= limit;
    memoised on (state, g, last)."""
    goal = tuple(range(W * W))
    sys.setrecursionlimit(max(10000, sys.getrecursionlimit()))

    @lru_cache(maxsize=None)
    def T(s, g, last):
        if s == goal:
            return 1, 1
        nodes, goals = 1, 0
        for m, c in neighbours(W, s):
            if last >= 0 and m == 3 - last:
                continue
            if g + 1 + manhattan_py(W, c) <= limit:
                a, b = T(c, g + 1, m)
                nodes += a
                goals += b
        return nodes, goals

    res = T(tuple(tiles), 0, -1)
    T.cache_clear()
    return res


def pattern_distances(W: int, group: Sequence[int]) -> Dict[Tuple[Tuple[int, ...], int], int]:
    """Abstract distances of one pattern group, by a 0-1 breadth-first search
    (deque: cost-0 successors go to the front, cost-1 ones to the back).

    An abstract state is (positions of the group's tiles in increasing tile
    order, blank position); the blank swaps with an adjacent cell, which
    costs 1 if the cell holds one of the group's tiles and 0 otherwise. The
    search starts at the abstract goal (tile t at cell t, blank at 0)."""
    tiles = sorted(group)
    start = (tuple(tiles), 0)
    dist = {start: 0}
    dq = deque([start])
    done = set()
    while dq:
        s = dq.popleft()
        if s in done:
            continue
        done.add(s)
        pos, b = s
        r, c = divmod(b, W)
        for m in range(4):
            dr, dc = DELTA_ROWCOL[m]
            rr, cc = r + dr, c + dc
            if not (0 <= rr < W and 0 <= cc < W):
                continue
            q = rr * W + cc
            if q in pos:
                j = pos.index(q)
                n = (pos[:j] + (b,) + pos[j + 1:], q)
                w = 1
            else:
                n = (pos, q)
                w = 0
            nd = dist[s] + w
            if nd < dist.get(n, 1 << 30):
                dist[n] = nd
                if w == 0:
                    dq.appendleft(n)
                else:
                    dq.append(n)
    return dist


def pattern_h(W: int, groups: Sequence[Sequence[int]], tables: Sequence[dict], s: Sequence[int]) -> int:
    """Sum over groups of the abstract distance of the board's abstraction."""
    where = {v: p for p, v in enumerate(s)}
    h = 0
    for g, tab in zip(groups, tables):
        h += tab[(tuple(where[t] for t in sorted(g)), where[0])]
    return h


def tree_size_h(W: int, tiles: Sequence[int], limit: int, h) -> Tuple[int, int, int]:
    """tree_size with heuristic h(state); also returns the smallest f of a
    pruned child (the next limit of IDA*), or None if nothing was pruned."""
    goal = tuple(range(W * W))
    sys.setrecursionlimit(max(10000, sys.getrecursionlimit()))
    hc = {}

    def H(s):
        v = hc.get(s)
        if v is None:
            v = hc[s] = h(s)
        return v

    @lru_cache(maxsize=None)
    def T(s, g, last):
        if s == goal:
            return 1, 1, None
        nodes, goals, fmin = 1, 0, None
        for m, c in neighbours(W, s):
            if last >= 0 and m == 3 - last:
                continue
            f = g + 1 + H(c)
            if f <= limit:
                a, b, fm = T(c, g + 1, m)
                nodes += a
                goals += b
            else:
                fm = f
            if fm is not None and (fmin is None or fm < fmin):
                fmin = fm
        return nodes, goals, fmin

    res = T(tuple(tiles), 0, -1)
    T.cache_clear()
    return res
