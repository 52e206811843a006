"""Python binding of the bpida C ABI (``include/bpida.h``).

Argument marshalling only: every step of the search runs in the CUDA
kernels of ``libbpida.so``. PyTorch supplies device memory and the stream.
There is no CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbpida.so")

OK, EINVAL, ENOMEM, ESTACK, EBUDGET, ETIMEOUT, ECUDA, ELIMIT, EINTERNAL = range(9)
# bpida_config.variant values
BLOCK_PARALLEL, PAPER_KERNEL, PSIMPLE, PSTATICLB, PFULLLB, BPSTATIC, BLOCK_MODE = range(7)

EXPORTS = (
    "bpida_max_len", "bpida_max_iters", "bpida_solve", "bpida_solve_ex", "bpida_set_timing",
    "bpida_set_fuse_nodes",
    "bpida_get_stats", "bpida_get_launch_log", "bpida_release_workspace", "bpida_status_str", "bpida_solve_noalloc",
    "bpida_server_create", "bpida_server_submit", "bpida_server_poll", "bpida_server_in_flight",
    "bpida_server_get_stats", "bpida_server_clock", "bpida_server_set_time_slice", "bpida_server_destroy",
    "bpida_pdb_create", "bpida_pdb_destroy", "bpida_pdb_groups", "bpida_pdb_table_bytes",
    "bpida_pdb_max_value", "bpida_pdb_copy_table", "bpida_solve_pdb",
)
NOALLOC_MAX_BOARDS = 256


class Config(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int),
        ("count_all", ctypes.c_int),
        ("split_target", ctypes.c_int),
        ("warps_per_block", ctypes.c_int),
        ("stack_entries", ctypes.c_int),
        ("exit_fraction_pct", ctypes.c_int),
        ("min_rounds", ctypes.c_int),
        ("node_budget", ctypes.c_uint64),
        ("driver", ctypes.c_int),
        ("min_pass_us", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int),
        ("passes", ctypes.c_int),
        ("records", ctypes.c_uint64),
        ("handed_back", ctypes.c_uint64),
        ("search_nodes", ctypes.c_uint64),
        ("search_ms", ctypes.c_double),
        ("grid_blocks", ctypes.c_int),
        ("block_threads", ctypes.c_int),
        ("sm_count", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("spills", ctypes.c_uint64),
        ("max_handed_back", ctypes.c_int),
        ("search_ms_device", ctypes.c_double),
        ("tp_threads", ctypes.c_int),
        ("tp_pad", ctypes.c_int),
        ("lb_ratio", ctypes.c_double),
        ("lb_ratio_last", ctypes.c_double),
        ("tp_roots", ctypes.c_uint64),
        ("tp_balances", ctypes.c_uint64),
        ("tp_steals", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [
        ("req_id", ctypes.c_uint64),
        ("status", ctypes.c_int),
        ("length", ctypes.c_int),
        ("num_iters", ctypes.c_int),
        ("pad", ctypes.c_int),
        ("submit_time_s", ctypes.c_double),
        ("done_time_s", ctypes.c_double),
        ("moves", ctypes.c_uint8 * 80),
        ("nodes_per_iter", ctypes.c_uint64 * 41),
        ("solutions", ctypes.c_uint64),
    ]

    def as_dict(self):
        L = self.length
        return {"req_id": self.req_id, "status": self.status, "length": L,
                "moves": list(self.moves[:max(L, 0)]), "iters": self.num_iters,
                "nodes": list(self.nodes_per_iter[:self.num_iters]),
                "solutions": self.solutions,
                "latency_s": self.done_time_s - self.submit_time_s}


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int),
        ("max_active", ctypes.c_int),
        ("submitted", ctypes.c_uint64),
        ("admitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("steps", ctypes.c_uint64),
        ("passes", ctypes.c_uint64),
        ("sliced_steps", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load():
    """Load libbpida.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libbpida.so is not built (run `python -c 'import __graft_entry__ as g; g.build()'`)")
        lib = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        lib.bpida_max_len.argtypes = [ctypes.c_int]
        lib.bpida_max_len.restype = ctypes.c_int
        lib.bpida_max_iters.argtypes = [ctypes.c_int]
        lib.bpida_max_iters.restype = ctypes.c_int
        lib.bpida_solve.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp]
        lib.bpida_solve.restype = ctypes.c_int
        lib.bpida_solve_ex.argtypes = [ctypes.POINTER(Config), vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.bpida_solve_ex.restype = ctypes.c_int
        lib.bpida_set_timing.argtypes = [ctypes.c_int]
        lib.bpida_set_timing.restype = None
        lib.bpida_set_fuse_nodes.argtypes = [ctypes.c_uint64]
        lib.bpida_set_fuse_nodes.restype = None
        lib.bpida_get_stats.argtypes = [ctypes.POINTER(Stats)]
        lib.bpida_get_stats.restype = None
        lib.bpida_get_launch_log.argtypes = [vp, vp, ctypes.c_int]
        lib.bpida_get_launch_log.restype = ctypes.c_int
        lib.bpida_release_workspace.argtypes = []
        lib.bpida_release_workspace.restype = None
        lib.bpida_solve_noalloc.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp]
        lib.bpida_solve_noalloc.restype = ctypes.c_int
        lib.bpida_server_create.argtypes = [ctypes.POINTER(Config), ctypes.c_size_t, ctypes.c_int]
        lib.bpida_server_create.restype = vp
        lib.bpida_server_submit.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64]
        lib.bpida_server_submit.restype = ctypes.c_int
        lib.bpida_server_poll.argtypes = [vp, ctypes.POINTER(Result), ctypes.c_int]
        lib.bpida_server_poll.restype = ctypes.c_int
        lib.bpida_server_in_flight.argtypes = [vp]
        lib.bpida_server_in_flight.restype = ctypes.c_int
        lib.bpida_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.bpida_server_get_stats.restype = None
        lib.bpida_server_clock.argtypes = []
        lib.bpida_server_clock.restype = ctypes.c_double
        lib.bpida_server_set_time_slice.argtypes = [vp, ctypes.c_int]
        lib.bpida_server_set_time_slice.restype = None
        lib.bpida_server_destroy.argtypes = [vp]
        lib.bpida_server_destroy.restype = None
        lib.bpida_status_str.argtypes = [ctypes.c_int]
        lib.bpida_status_str.restype = ctypes.c_char_p
        lib.bpida_pdb_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp), vp]
        lib.bpida_pdb_create.restype = ctypes.c_int
        lib.bpida_pdb_destroy.argtypes = [vp]
        lib.bpida_pdb_destroy.restype = None
        lib.bpida_pdb_groups.argtypes = [vp]
        lib.bpida_pdb_groups.restype = ctypes.c_int
        lib.bpida_pdb_table_bytes.argtypes = [vp, ctypes.c_int]
        lib.bpida_pdb_table_bytes.restype = ctypes.c_uint64
        lib.bpida_pdb_max_value.argtypes = [vp, ctypes.c_int]
        lib.bpida_pdb_max_value.restype = ctypes.c_int
        lib.bpida_pdb_copy_table.argtypes = [vp, ctypes.c_int, vp, ctypes.c_uint64, vp]
        lib.bpida_pdb_copy_table.restype = ctypes.c_int
        lib.bpida_solve_pdb.argtypes = [ctypes.POINTER(Config), vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.bpida_solve_pdb.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_len(width: int) -> int:
    return load().bpida_max_len(width)


def max_iters(width: int) -> int:
    return load().bpida_max_iters(width)


def status_str(code: int) -> str:
    return load().bpida_status_str(code).decode()


def set_timing(on: bool) -> None:
    load().bpida_set_timing(1 if on else 0)


def set_fuse_nodes(nodes: int) -> None:
    """Node cap of a fused step's top threshold (0: the defaults); see bpida.h."""
    load().bpida_set_fuse_nodes(int(nodes))


def last_stats() -> dict:
    s = Stats()
    load().bpida_get_stats(ctypes.byref(s))
    return s.as_dict()


def launch_log():
    """[(ms, nodes)] of every search launch of this thread's last host-driven
    call made with timing on (``set_timing(True)``, ``driver=1``)."""
    lib = load()
    k = lib.bpida_get_launch_log(None, None, 0)
    ms = (ctypes.c_double * max(k, 1))()
    nodes = (ctypes.c_uint64 * max(k, 1))()
    lib.bpida_get_launch_log(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(nodes, ctypes.c_void_p), k)
    return [(ms[i], int(nodes[i])) for i in range(k)]


def release_workspace() -> None:
    load().bpida_release_workspace()


@dataclass
class Solution:
    """The outputs of one solve call. The call is asynchronous: ``status`` is
    whether it was issued, and the tensors hold the results once ``stream``
    has reached the end of its work (``synchronize()``; ``to_host()`` does)."""
    status: int                    # call status
    length: torch.Tensor           # int32 (n,)
    moves: torch.Tensor            # uint8 (n, max_len)
    nodes: torch.Tensor            # int64 (n, max_iters) (uint64 bit pattern)
    iters: torch.Tensor            # int32 (n,)
    inst_status: torch.Tensor      # int32 (n,)
    solutions: Optional[torch.Tensor] = None  # int64 (n,): optimal solutions (count-all mode)
    stream: Optional[torch.cuda.Stream] = None  # the stream the call was issued on

    def synchronize(self) -> None:
        if self.stream is not None:
            self.stream.synchronize()

    def to_host(self):
        """Per-instance dicts with Python ints (moves trimmed to the length),
        after waiting for the call's stream."""
        self.synchronize()
        L = self.length.cpu().tolist()
        mv = self.moves.cpu().numpy()
        nd = self.nodes.cpu().numpy().view("uint64")
        it = self.iters.cpu().tolist()
        stt = self.inst_status.cpu().tolist()
        sol = self.solutions.cpu().tolist() if self.solutions is not None else [None] * len(L)
        out = []
        for i in range(len(L)):
            out.append({
                "status": stt[i], "length": L[i],
                "moves": [int(x) for x in mv[i, :max(L[i], 0)]],
                "nodes": [int(x) for x in nd[i, :it[i]]],
                "iters": it[i],
                "solutions": sol[i],
            })
        return out


# Configuration fields the autotuner caches (bpida_config names; the search
# mode is `variant`, 0 = a warp and 6 = a block per subtree group).
TUNE_FIELDS = ("variant", "split_target", "warps_per_block", "stack_entries", "exit_fraction_pct", "min_rounds")
_tune = {"path": None, "mtime": None, "doc": {}}


def tune_cache_path() -> str:
    """The autotuner's cache file: BPIDA_TUNE_CACHE, else ~/.cache/bpida/tune.json."""
    return os.environ.get("BPIDA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bpida", "tune.json"))


def tune_key(width: int, form: str, device=None) -> str:
    """Cache key: GPU name, SM count, board width, form ("plain": calls of at
    most 8 boards, "batched": larger calls)."""
    p = torch.cuda.get_device_properties(device if device is not None else torch.cuda.current_device())
    return "%s|%d|w%d|%s" % (p.name, p.multi_processor_count, width, form)


def tuned_knobs(width: int, form: str, path: Optional[str] = None, device=None) -> dict:
    """The cached knobs for this GPU, width and form ({} without an entry)."""
    import json

    path = path or tune_cache_path()
    if not path or not os.path.exists(path):
        return {}
    mtime = os.path.getmtime(path)
    if _tune["path"] != path or _tune["mtime"] != mtime:
        with open(path) as f:
            _tune.update(path=path, mtime=mtime, doc=json.load(f))
    return {k: int(v) for k, v in _tune["doc"].get(tune_key(width, form, device), {}).items() if k in TUNE_FIELDS}


def resolve_config(cfg: "Config", width: int, n: int, device=None) -> "Config":
    """A copy of cfg whose fields left at 0 take the autotuner's cached values
    for this GPU, width and call size (variant 0 takes the tuned search
    mode); cfg itself without a cache entry."""
    knobs = tuned_knobs(width, "plain" if n <= 8 else "batched", device=device)
    if not knobs:
        return cfg
    out = Config()
    ctypes.memmove(ctypes.byref(out), ctypes.byref(cfg), ctypes.sizeof(Config))
    for k, v in knobs.items():
        if getattr(out, k) == 0:
            setattr(out, k, v)
    return out


def make_config(width: int = 4, split_target: int = 0, warps_per_block: int = 0,
                stack_entries: int = 0, exit_fraction_pct: int = 0, min_rounds: int = 0,
                node_budget: int = 0, driver: int = 0, min_pass_us: int = 0,
                count_all: bool = True, variant: int = 0) -> Config:
    return Config(width, 1 if count_all else 0, split_target, warps_per_block, stack_entries,
                  exit_fraction_pct, min_rounds, node_budget, driver, min_pass_us, variant, 0)


def solve(boards: torch.Tensor, width: int = 4, config: Optional[Config] = None,
          stream: Optional[torch.cuda.Stream] = None, pdb: Optional["PatternDb"] = None,
          tuned: bool = True) -> Solution:
    """Solve packed boards already on the GPU.

    ``boards``: CUDA int64 tensor, shape (n,) for width 3/4, (n, 2) for 5,
    holding the packed words (bit pattern of the uint64 layout in bpida.h).
    Outputs are allocated on the same device; the call is issued on
    ``stream`` (default: the current stream) and returns without waiting
    (graph driver): the outputs are valid once that stream has reached the
    end of the call. With ``pdb`` the heuristic is that pattern database
    (bpida_solve_pdb), else the Manhattan distance. With ``tuned`` (and the
    Manhattan distance) the configuration fields left at 0 take the
    autotuner's cached values for this GPU (resolve_config).
    """
    lib = load()
    if not boards.is_cuda:
        raise ValueError("boards must be a CUDA tensor")
    if boards.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise ValueError("boards must be a 64-bit integer tensor")
    boards = boards.contiguous()
    n = boards.shape[0]
    if width == 5 and (boards.dim() != 2 or boards.shape[1] != 2):
        raise ValueError("width-5 boards must have shape (n, 2)")
    cfg = config if config is not None else make_config(width)
    cfg.width = width
    dev = boards.device
    if tuned and pdb is None:
        cfg = resolve_config(cfg, width, n, dev)
    ml, mi = lib.bpida_max_len(width), lib.bpida_max_iters(width)
    out_len = torch.empty(n, dtype=torch.int32, device=dev)
    out_moves = torch.empty((n, ml), dtype=torch.uint8, device=dev)
    out_nodes = torch.empty((n, mi), dtype=torch.int64, device=dev)
    out_iters = torch.empty(n, dtype=torch.int32, device=dev)
    out_status = torch.empty(n, dtype=torch.int32, device=dev)
    out_sol = torch.empty(n, dtype=torch.int64, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    outs = (out_len.data_ptr(), out_moves.data_ptr(), out_nodes.data_ptr(), out_iters.data_ptr(),
            out_status.data_ptr(), out_sol.data_ptr(), s.cuda_stream)
    with torch.cuda.device(dev):
        if pdb is None:
            rc = lib.bpida_solve_ex(ctypes.byref(cfg), boards.data_ptr(), n, *outs)
        else:
            rc = lib.bpida_solve_pdb(ctypes.byref(cfg), pdb.handle, boards.data_ptr(), n, *outs)
    return Solution(rc, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, s)


def solve_packed_host(packed, width: int = 4, config: Optional[Config] = None,
                      device: str = "cuda") -> List[dict]:
    """Convenience: numpy/list of packed words on the host -> host results."""
    import numpy as np

    arr = np.ascontiguousarray(np.asarray(packed, dtype=np.uint64)).view(np.int64)
    t = torch.from_numpy(arr).to(device)
    sol = solve(t, width, config)
    torch.cuda.synchronize()
    res = sol.to_host()
    for r in res:
        r["call_status"] = sol.status
    return res


def solve_noalloc(boards: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> Solution:
    """15-puzzle solve through bpida_solve_noalloc (no device allocation inside
    the library; the output tensors here are allocated by the caller side of
    this binding). At most NOALLOC_MAX_BOARDS boards."""
    lib = load()
    if not boards.is_cuda:
        raise ValueError("boards must be a CUDA tensor")
    boards = boards.contiguous()
    n = boards.shape[0]
    dev = boards.device
    ml, mi = lib.bpida_max_len(4), lib.bpida_max_iters(4)
    out_len = torch.empty(n, dtype=torch.int32, device=dev)
    out_moves = torch.empty((n, ml), dtype=torch.uint8, device=dev)
    out_nodes = torch.empty((n, mi), dtype=torch.int64, device=dev)
    out_iters = torch.empty(n, dtype=torch.int32, device=dev)
    out_status = torch.empty(n, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        rc = lib.bpida_solve_noalloc(boards.data_ptr(), n, out_len.data_ptr(), out_moves.data_ptr(),
                                     out_nodes.data_ptr(), out_iters.data_ptr(), out_status.data_ptr(),
                                     s.cuda_stream)
    return Solution(rc, out_len, out_moves, out_nodes, out_iters, out_status, None, s)


class PatternDb:
    """Pattern databases built on the GPU by bpida_pdb_create (see bpida.h):
    ``groups`` lists the tiles of each group (every tile 1..W*W-1 in exactly
    one group; at most 6 groups of 1 to 6 tiles)."""

    def __init__(self, width: int, groups, device: Optional[torch.device] = None):
        lib = load()
        self.width = width
        self.groups = [sorted(int(t) for t in g) for g in groups]
        got = (ctypes.c_int * (width * width))()
        seen = set()
        for gi, g in enumerate(self.groups):
            for t in g:
                if not 1 <= t < width * width or t in seen:
                    raise ValueError("tile %d is out of range or in two groups" % t)
                seen.add(t)
                got[t] = gi
        if len(seen) != width * width - 1:
            raise ValueError("every tile must belong to a group")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.bpida_pdb_create(width, got, ctypes.byref(h), torch.cuda.current_stream(self.device).cuda_stream)
        if rc != OK:
            raise RuntimeError("bpida_pdb_create failed: %s" % status_str(rc))
        self.handle = h.value

    def table_bytes(self, group: int) -> int:
        return int(load().bpida_pdb_table_bytes(self.handle, group))

    def max_value(self, group: int) -> int:
        return int(load().bpida_pdb_max_value(self.handle, group))

    def table(self, group: int) -> torch.Tensor:
        """Group ``group``'s table copied to a host uint8 tensor."""
        out = torch.empty(self.table_bytes(group), dtype=torch.uint8)
        with torch.cuda.device(self.device):
            rc = load().bpida_pdb_copy_table(self.handle, group, out.data_ptr(), out.numel(),
                                             torch.cuda.current_stream(self.device).cuda_stream)
        if rc != OK:
            raise RuntimeError("bpida_pdb_copy_table failed: %s" % status_str(rc))
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            with torch.cuda.device(self.device):
                load().bpida_pdb_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching 15-puzzle solve service (bpida_server_* calls)."""

    def __init__(self, frontier_bytes: int = 1 << 30, max_slots: int = 4096,
                 config: Optional[Config] = None, time_slice_us: Optional[int] = None):
        lib = load()
        cfg = config if config is not None else make_config(4)
        self._lib = lib
        self._h = lib.bpida_server_create(ctypes.byref(cfg), frontier_bytes, max_slots)
        if not self._h:
            raise RuntimeError("bpida_server_create failed")
        if time_slice_us is not None:
            lib.bpida_server_set_time_slice(self._h, time_slice_us)
        self._buf = (Result * 256)()

    def submit(self, packed_board: int, req_id: int) -> None:
        w = ctypes.c_uint64(packed_board)
        rc = self._lib.bpida_server_submit(self._h, ctypes.byref(w), req_id)
        if rc != OK:
            raise RuntimeError("submit failed: " + status_str(rc))

    def poll(self) -> List[dict]:
        out = []
        while True:
            k = self._lib.bpida_server_poll(self._h, self._buf, len(self._buf))
            out.extend(self._buf[i].as_dict() for i in range(k))
            if k < len(self._buf):
                return out

    def in_flight(self) -> int:
        return self._lib.bpida_server_in_flight(self._h)

    def stats(self) -> dict:
        s = ServerStats()
        self._lib.bpida_server_get_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    @staticmethod
    def clock() -> float:
        return load().bpida_server_clock()

    def close(self) -> None:
        if self._h:
            self._lib.bpida_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
