"""Seeded synthetic sliding-tile instances.

This module is the only code shared by the CPU oracle tests and the CUDA
path. It draws random numbers and builds boards; it holds none of the
search's arithmetic (no heuristic, no threshold logic, no node counting).

Board convention (used by every module of this project):

* positions are numbered row-major ``0 .. W*W-1``;
* ``tiles[p]`` is the tile at position ``p``; tile ``0`` is the blank;
* the goal has tile ``t`` at position ``t`` (blank at position 0);
* the blank moves U=0, L=1, R=2, D=3 (position -W, -1, +1, +W); the
  inverse of move ``m`` is ``3 - m``.

Packed form handed to the C ABI: for W <= 4 one ``uint64`` per board with
``tiles[p]`` in bits ``[4p, 4p+4)``; for W == 5 two ``uint64`` words
(low word first) of the 128-bit integer with ``tiles[p]`` in bits
``[5p, 5p+5)``.

The random number generators are SplitMix64 (Steele, Lea & Flood 2014) for
seeding and xoshiro256** (Blackman & Vigna 2018), written here from their
published definitions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence

MASK64 = (1 << 64) - 1

# Blank displacement per move for a width-W board: U, L, R, D.
MOVE_NAMES = "ULRD"


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


def splitmix64(state: int):
    """One SplitMix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Xoshiro256ss:
    """xoshiro256** seeded by four SplitMix64 outputs of ``seed``."""

    def __init__(self, seed: int):
        st = seed & MASK64
        s = []
        for _ in range(4):
            st, out = splitmix64(st)
            s.append(out)
        self.s = s

    def next_u64(self) -> int:
        s0, s1, s2, s3 = self.s
        result = (_rotl((s1 * 5) & MASK64, 7) * 9) & MASK64
        t = (s1 << 17) & MASK64
        s2 ^= s0
        s3 ^= s1
        s1 ^= s2
        s0 ^= s3
        s2 ^= t
        s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return result

    def below(self, n: int) -> int:
        """Unbiased integer in [0, n) by rejection of the top partial block."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = ((1 << 64) // n) * n
        while True:
            x = self.next_u64()
            if x < limit:
                return x % n

    def uniform_int(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def uniform01(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def goal_tiles(W: int) -> List[int]:
    return list(range(W * W))


def _blank_targets(W: int, p: int):
    """Legal (move, new blank position) pairs for a blank at ``p``."""
    r, c = divmod(p, W)
    out = []
    if r > 0:
        out.append((0, p - W))
    if c > 0:
        out.append((1, p - 1))
    if c < W - 1:
        out.append((2, p + 1))
    if r < W - 1:
        out.append((3, p + W))
    return out


def random_walk(W: int, length: int, rng: Xoshiro256ss) -> List[int]:
    """Board reached from the goal by ``length`` uniformly chosen blank moves,
    never undoing the previous move."""
    tiles = goal_tiles(W)
    blank = 0
    last = -1
    for _ in range(length):
        opts = [(m, q) for (m, q) in _blank_targets(W, blank) if last < 0 or m != 3 - last]
        m, q = opts[rng.below(len(opts))]
        tiles[blank], tiles[q] = tiles[q], 0
        blank = q
        last = m
    return tiles


def _reachable_parity_ok(W: int, tiles: Sequence[int]) -> bool:
    """Input filter: keeps permutations in the goal's parity class
    (inversions among non-blank tiles, plus the blank's row when W is even)."""
    seq = [t for t in tiles if t != 0]
    inv = 0
    for i in range(len(seq)):
        for j in range(i + 1, len(seq)):
            if seq[i] > seq[j]:
                inv += 1
    if W % 2 == 1:
        return inv % 2 == 0
    blank_row = tiles.index(0) // W
    return (inv + blank_row) % 2 == 0


def random_permutation(W: int, rng: Xoshiro256ss) -> List[int]:
    """Uniform random board from the goal's parity class (Fisher-Yates,
    redrawn until it passes the parity filter)."""
    n = W * W
    while True:
        tiles = list(range(n))
        for i in range(n - 1, 0, -1):
            j = rng.below(i + 1)
            tiles[i], tiles[j] = tiles[j], tiles[i]
        if _reachable_parity_ok(W, tiles):
            return tiles


def pack(W: int, tiles: Sequence[int]) -> List[int]:
    """Packed words of one board (see module docstring)."""
    if W <= 4:
        v = 0
        for p, t in enumerate(tiles):
            v |= (t & 0xF) << (4 * p)
        return [v]
    if W == 5:
        v = 0
        for p, t in enumerate(tiles):
            v |= (t & 0x1F) << (5 * p)
        return [v & MASK64, v >> 64]
    raise ValueError("unsupported width")


def unpack(W: int, words: Sequence[int]) -> List[int]:
    if W <= 4:
        v = int(words[0])
        return [(v >> (4 * p)) & 0xF for p in range(W * W)]
    if W == 5:
        v = int(words[0]) | (int(words[1]) << 64)
        return [(v >> (5 * p)) & 0x1F for p in range(W * W)]
    raise ValueError("unsupported width")


def words_per_board(W: int) -> int:
    return 1 if W <= 4 else 2


@dataclass
class Instance:
    W: int
    tiles: List[int]
    kind: str          # "walk" or "perm"
    seed: int
    walk_len: int = -1  # -1 for permutations


def make_walk(W: int, seed: int, length: int) -> Instance:
    return Instance(W, random_walk(W, length, Xoshiro256ss(seed)), "walk", seed, length)


def make_perm(W: int, seed: int) -> Instance:
    return Instance(W, random_permutation(W, Xoshiro256ss(seed)), "perm", seed)


# ---------------------------------------------------------------------------
# Named workloads (sizes and mixes of the paper's 15-puzzle experiments and
# their batched / 24-puzzle / serving extensions).
# ---------------------------------------------------------------------------

def walks15_16x40() -> List[Instance]:
    """16 fifteen-puzzle boards, each a 40-move walk (seeds 1..16)."""
    return [make_walk(4, s, 40) for s in range(1, 17)]


def perms15_100() -> List[Instance]:
    """100 uniformly random solvable fifteen-puzzle boards (seeds 1001..1100);
    stands in for the paper's 100-instance benchmark set."""
    return [make_perm(4, s) for s in range(1001, 1101)]


def mixed15_4096() -> List[Instance]:
    """4096 fifteen-puzzle boards: every 20th a random solvable permutation
    (205 in all), the rest walks of a length drawn from [20, 90]."""
    out = []
    for i in range(4096):
        seed = 100000 + i
        if i % 20 == 0:
            out.append(make_perm(4, seed))
        else:
            rng = Xoshiro256ss(seed)
            length = rng.uniform_int(20, 90)
            out.append(Instance(4, random_walk(4, length, rng), "walk", seed, length))
    return out


def walks24_1024() -> List[Instance]:
    """1024 twenty-four-puzzle boards, walks of a length drawn from [40, 100]."""
    out = []
    for i in range(1024):
        seed = 200000 + i
        rng = Xoshiro256ss(seed)
        length = rng.uniform_int(40, 100)
        out.append(Instance(5, random_walk(5, length, rng), "walk", seed, length))
    return out


def serving_stream(rate_per_s: float, count: int, seed: int = 300000):
    """Poisson request stream: (arrival time in s, Instance) pairs. 98% are
    walks of a length drawn from [30, 90], 2% random solvable permutations."""
    rng = Xoshiro256ss(seed)
    t = 0.0
    out = []
    for i in range(count):
        u = rng.uniform01()
        t += -math.log(1.0 - u) / rate_per_s
        iseed = seed + 1 + i
        if rng.below(50) == 0:
            inst = make_perm(4, iseed)
        else:
            r2 = Xoshiro256ss(iseed)
            length = r2.uniform_int(30, 90)
            inst = Instance(4, random_walk(4, length, r2), "walk", iseed, length)
        out.append((t, inst))
    return out


# Tile groups of the pattern-database heuristic used by the benchmarks (a
# configuration, not an algorithm: each group's table is built by the solver
# or by the oracle). 5-5-5: three 16 MB tables (L2-resident); 6-6-3: two
# 256 MB tables and a 64 KB one (beyond L2, read from HBM).
PDB_PARTITIONS = {
    "555": [[1, 2, 3, 4, 5], [6, 7, 8, 9, 10], [11, 12, 13, 14, 15]],
    "663": [[1, 2, 3, 4, 5, 6], [7, 8, 9, 10, 11, 12], [13, 14, 15]],
}

WORKLOADS = {
    "walks15_16x40": walks15_16x40,
    "perms15_100": perms15_100,
    "mixed15_4096": mixed15_4096,
    "walks24_1024": walks24_1024,
}


def packed_array(instances: Sequence[Instance]):
    """numpy uint64 array of packed boards, shape (n,) for W<=4 or (n, 2)."""
    import numpy as np

    if not instances:
        return np.zeros((0,), dtype=np.uint64)
    W = instances[0].W
    rows = [pack(W, inst.tiles) for inst in instances]
    arr = np.array(rows, dtype=np.uint64)
    return arr.reshape(-1) if W <= 4 else arr.reshape(-1, 2)


def tiles_array(instances: Sequence[Instance]):
    """numpy uint8 array of shape (n, W*W)."""
    import numpy as np

    if not instances:
        return np.zeros((0, 0), dtype=np.uint8)
    return np.array([inst.tiles for inst in instances], dtype=np.uint8)
