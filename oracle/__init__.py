"""CPU oracle for Block-Parallel IDA*: plain sequential IDA* in C.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product path
(``paper_1705_02843_gb300``) never imports it. It shares no code with the
CUDA path.

What the C code computes is documented at the top of ``ida_oracle.c``
(Algorithms 1 and 2 of the paper without load balancing, Section 3's
sequential Solver C, Section 6's all-optimal-solutions mode).

Parity status: pinned (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ida_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, INVALID, BUDGET, LIMIT, BADARG = 0, 1, 4, 7, 8

# Caps for the tables the oracle fills (generous: 80 is the 15-puzzle
# diameter; 24-puzzle walks in this project are at most 100 moves).
MAX_LEN = {3: 40, 4: 96, 5: 208}
MAX_ITERS = {3: 24, 4: 49, 5: 105}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lpthread"]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_ida_batch.argtypes = [
            ctypes.c_int, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, i32p, u8p, u64p, i32p, i32p, u64p, i32p, i32p,
        ]
        lib.oracle_ida_batch.restype = ctypes.c_int
        lib.oracle_is_solvable.argtypes = [ctypes.c_int, u8p]
        lib.oracle_is_solvable.restype = ctypes.c_int
        lib.oracle_manhattan.argtypes = [ctypes.c_int, u8p]
        lib.oracle_manhattan.restype = ctypes.c_int
        lib.oracle_manhattan_batch.argtypes = [ctypes.c_int, u8p, ctypes.c_int, i32p]
        lib.oracle_manhattan_batch.restype = None
        lib.oracle_is_solvable_batch.argtypes = [ctypes.c_int, u8p, ctypes.c_int, i32p]
        lib.oracle_is_solvable_batch.restype = None
        lib.oracle_pdb_table_bytes.argtypes = [ctypes.c_int]
        lib.oracle_pdb_table_bytes.restype = ctypes.c_uint64
        lib.oracle_pdb_build.argtypes = [ctypes.c_int, i32p, ctypes.c_int, u8p, ctypes.c_uint64, i32p]
        lib.oracle_pdb_build.restype = ctypes.c_int
        lib.oracle_pdb_h_batch.argtypes = [ctypes.c_int, i32p, u8p, u8p, ctypes.c_int, i32p]
        lib.oracle_pdb_h_batch.restype = ctypes.c_int
        lib.oracle_ida_pdb_batch.argtypes = [
            ctypes.c_int, i32p, u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, i32p, u8p, u64p, i32p, i32p, u64p, i32p, i32p,
        ]
        lib.oracle_ida_pdb_batch.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class OracleResult:
    status: int
    length: int
    moves: List[int]
    nodes: List[int]          # nodes popped per iteration
    limits: List[int]         # f-limit of each iteration
    iters: int
    solutions: int            # optimal solutions counted (count-all mode)
    h0: int
    extra: dict = field(default_factory=dict)

    @property
    def total_nodes(self) -> int:
        return int(sum(self.nodes))


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def solve_batch(W: int, tiles, count_all: bool = True, node_budget: int = 0,
                nthreads: int = 0, pdb: "PatternDb" = None) -> List[OracleResult]:
    """Solve every board (rows of ``tiles``, shape (n, W*W)) independently,
    with the Manhattan distance or, given ``pdb``, its pattern databases."""
    lib = _load()
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint8).reshape(-1, W * W))
    n = t.shape[0]
    ml, mi = MAX_LEN[W], MAX_ITERS[W]
    out_len = np.zeros(n, np.int32)
    out_moves = np.zeros((n, ml), np.uint8)
    out_nodes = np.zeros((n, mi), np.uint64)
    out_limits = np.zeros((n, mi), np.int32)
    out_iters = np.zeros(n, np.int32)
    out_sol = np.zeros(n, np.uint64)
    out_h0 = np.zeros(n, np.int32)
    out_status = np.zeros(n, np.int32)
    if nthreads <= 0:
        nthreads = os.cpu_count() or 1
    outs = (_ptr(out_len, ctypes.c_int), _ptr(out_moves, ctypes.c_uint8),
            _ptr(out_nodes, ctypes.c_uint64), _ptr(out_limits, ctypes.c_int),
            _ptr(out_iters, ctypes.c_int), _ptr(out_sol, ctypes.c_uint64),
            _ptr(out_h0, ctypes.c_int), _ptr(out_status, ctypes.c_int))
    if n and pdb is None:
        rc = lib.oracle_ida_batch(
            W, _ptr(t, ctypes.c_uint8), n, 1 if count_all else 0, node_budget, mi, ml, nthreads, *outs)
        if rc != OK:
            raise ValueError("oracle_ida_batch rejected its arguments (code %d)" % rc)
    elif n:
        if pdb.W != W:
            raise ValueError("pattern databases built for width %d" % pdb.W)
        rc = lib.oracle_ida_pdb_batch(
            W, _ptr(pdb.group_of_tile, ctypes.c_int), _ptr(pdb.concatenated, ctypes.c_uint8),
            _ptr(t, ctypes.c_uint8), n, 1 if count_all else 0, node_budget, mi, ml, nthreads, *outs)
        if rc != OK:
            raise ValueError("oracle_ida_pdb_batch rejected its arguments (code %d)" % rc)
    res = []
    for i in range(n):
        it = int(out_iters[i])
        L = int(out_len[i])
        res.append(OracleResult(
            status=int(out_status[i]), length=L,
            moves=[int(x) for x in out_moves[i, :max(L, 0)]],
            nodes=[int(x) for x in out_nodes[i, :it]],
            limits=[int(x) for x in out_limits[i, :it]],
            iters=it, solutions=int(out_sol[i]), h0=int(out_h0[i])))
    return res


def solve(W: int, tiles: Sequence[int], count_all: bool = True, node_budget: int = 0,
          pdb: "PatternDb" = None) -> OracleResult:
    return solve_batch(W, [list(tiles)], count_all, node_budget, nthreads=1, pdb=pdb)[0]


def is_solvable(W: int, tiles: Sequence[int]) -> bool:
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint8))
    return bool(_load().oracle_is_solvable(W, _ptr(t, ctypes.c_uint8)))


def manhattan(W: int, tiles: Sequence[int]) -> int:
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint8))
    return int(_load().oracle_manhattan(W, _ptr(t, ctypes.c_uint8)))


def manhattan_batch(W: int, tiles) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint8).reshape(-1, W * W))
    out = np.zeros(t.shape[0], np.int32)
    _load().oracle_manhattan_batch(W, _ptr(t, ctypes.c_uint8), t.shape[0], _ptr(out, ctypes.c_int))
    return out


def is_solvable_batch(W: int, tiles) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint8).reshape(-1, W * W))
    out = np.zeros(t.shape[0], np.int32)
    _load().oracle_is_solvable_batch(W, _ptr(t, ctypes.c_uint8), t.shape[0], _ptr(out, ctypes.c_int))
    return out.astype(bool)


class PatternDb:
    """Additive disjoint pattern databases built by the oracle (see the
    "pattern databases" section of ``ida_oracle.c``): ``groups`` lists the
    tiles of each group; every tile 1..W*W-1 belongs to exactly one group of
    1 to 6 tiles. ``tables[g]`` holds d_G at index
    sum_j pos(t_j) << 4j | blank << 4k (tiles of the group in increasing
    order), 255 where no abstract state has that index."""

    def __init__(self, W: int, groups: Sequence[Sequence[int]]):
        lib = _load()
        self.W = W
        self.groups = [sorted(int(t) for t in g) for g in groups]
        got = np.full(W * W, -1, np.int32)
        for gi, g in enumerate(self.groups):
            for t in g:
                if not 1 <= t < W * W or got[t] != -1:
                    raise ValueError("tile %d is out of range or in two groups" % t)
                got[t] = gi
        if (got[1:] < 0).any():
            raise ValueError("every tile must belong to a group")
        got[0] = 0
        self.group_of_tile = got
        self.tables = []
        self.max_values = []
        for gi, g in enumerate(self.groups):
            size = int(lib.oracle_pdb_table_bytes(len(g)))
            if size == 0:
                raise ValueError("groups hold 1 to 6 tiles")
            tab = np.empty(size, np.uint8)
            mx = np.zeros(1, np.int32)
            rc = lib.oracle_pdb_build(W, _ptr(got, ctypes.c_int), gi, _ptr(tab, ctypes.c_uint8), size,
                                      _ptr(mx, ctypes.c_int))
            if rc != OK:
                raise ValueError("oracle_pdb_build failed (code %d)" % rc)
            self.tables.append(tab)
            self.max_values.append(int(mx[0]))
        self.concatenated = np.ascontiguousarray(np.concatenate(self.tables))

    def h_batch(self, tiles) -> np.ndarray:
        """The heuristic value of every board (rows of W*W tiles)."""
        t = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint8).reshape(-1, self.W * self.W))
        out = np.zeros(t.shape[0], np.int32)
        rc = _load().oracle_pdb_h_batch(self.W, _ptr(self.group_of_tile, ctypes.c_int),
                                        _ptr(self.concatenated, ctypes.c_uint8), _ptr(t, ctypes.c_uint8),
                                        t.shape[0], _ptr(out, ctypes.c_int))
        if rc != OK:
            raise ValueError("oracle_pdb_h_batch failed (code %d)" % rc)
        return out
