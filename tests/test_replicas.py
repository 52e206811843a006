"""Multi-GPU runs are independent replicas (instances do not interact), so
the only collective is the benchmark's max-over-ranks timing. Checked with two
gloo ranks on the CPU."""
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
    q.put((rank, v, m))
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
    assert [round(v, 6) for _, v, _ in out] == [100.0, 100.0]
    assert [m for _, _, m in out] == [10.0, 10.0]


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(100, 2.0, 1) == 50.0


def test_bench_pattern_database_constants_cover_every_partition():
    """Every tile partition the --pdb leg accepts has its measured kernel
    figures, and the command line offers exactly those partitions."""
    import subprocess
    import sys

    import bench
    from paper_1705_02843_gb300 import inputs as I

    parts = set(I.PDB_PARTITIONS)
    for table in (bench.INSTR_PER_EXPANSION_PDB, bench.TRAFFIC_PER_LAUNCH_PDB, bench.ALU_PIPE_SHARE_PDB):
        assert set(table) == parts
        assert all(v is not None and v > 0 for v in table.values())
    for form in ("batched", "plain"):
        k = bench.KERNEL_COUNTERS[form]
        assert 0.0 < k["alu_pipe_share"] < 1.0 and k["instr_per_expansion"] > 1.0
    out = subprocess.run([sys.executable, bench.__file__, "--help"], capture_output=True, text=True, check=True).stdout
    assert "--pdb {%s}" % ",".join(sorted(parts)) in out
