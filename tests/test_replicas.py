"""Multi-GPU runs: instances do not interact, so each rank solves its own
instance range with no collective on the data path, and the results are
gathered at the end (or, with --replicas, every rank solves the whole
workload). The bench's collectives are the max-over-ranks timing, sums of
counts and the final gather. Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r took (r + 1) seconds for the same 100 boards
    v = bench.replica_throughput(100, float(rank + 1), world, dist)
    m = bench.max_over_ranks(rank * 10.0, dist)
    # instance ranges of 4097 boards, each rank's rows gathered in order
    lo, hi = bench.shard_range(4097, world, rank)
    rows = bench.gather_rows([{"index": i, "rank": rank} for i in range(lo, hi)], dist)
    total = bench.sum_over_ranks(hi - lo, dist)
    q.put((rank, v, m, (lo, hi), [r["index"] for r in rows], [r["rank"] for r in rows], total))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # job throughput = 2 ranks x 100 boards / slowest rank's 2 s
    assert [round(o[1], 6) for o in out] == [100.0, 100.0]
    assert [o[2] for o in out] == [10.0, 10.0]
    # the ranges cover 0..4096 once, in order; every rank sees every row
    assert [o[3] for o in out] == [(0, 2049), (2049, 4097)]
    for o in out:
        assert o[4] == list(range(4097))
        assert o[5] == [0] * 2049 + [1] * 2048
        assert o[6] == 4097


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(100, 2.0, 1) == 50.0
    assert bench.shard_range(10, 1, 0) == (0, 10)
    assert bench.gather_rows([1, 2]) == [1, 2] and bench.sum_over_ranks(7) == 7


@pytest.mark.parametrize("n,world", [(4096, 8), (4096, 3), (5, 8), (100, 7)])
def test_instance_ranges_partition_the_workload(n, world):
    import bench

    rs = [bench.shard_range(n, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    sizes = [hi - lo for lo, hi in rs]
    assert max(sizes) - min(sizes) <= 1


def test_bench_pattern_database_constants_cover_every_partition():
    """Every tile partition the --pdb leg accepts has its measured
    instructions per expansion (DRAM bytes and ALU share only where measured
    on the bench's own launches), and the command line offers exactly those
    partitions."""
    import subprocess
    import sys

    import bench
    from paper_1705_02843_gb300 import inputs as I

    parts = set(I.PDB_PARTITIONS)
    assert set(bench.INSTR_PER_EXPANSION_PDB) == parts
    for table in (bench.INSTR_PER_EXPANSION_PDB, bench.TRAFFIC_PER_LAUNCH_PDB, bench.ALU_PIPE_SHARE_PDB):
        assert set(table) <= parts
        assert all(v is not None and v > 0 for v in table.values())
    for form in ("batched", "plain"):
        k = bench.KERNEL_COUNTERS[form]
        assert 0.0 < k["alu_pipe_share"] < 1.0 and k["instr_per_expansion"] > 1.0
    out = subprocess.run([sys.executable, bench.__file__, "--help"], capture_output=True, text=True, check=True).stdout
    assert "--pdb {%s}" % ",".join(sorted(parts)) in out
