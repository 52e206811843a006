"""Autotuner: every candidate it accepts must reproduce the oracle's results
exactly; the chosen configuration round-trips through the cache."""
import numpy as np
import pytest
import torch

import oracle
from paper_1705_02843_gb300 import autotune, bpida
from paper_1705_02843_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_tune_keeps_results_exact(tmp_path, monkeypatch):
    monkeypatch.setenv("BPIDA_TUNE_CACHE", str(tmp_path / "tune.json"))
    insts = I.walks15_16x40()
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64)).cuda()
    ref = oracle.solve_batch(4, I.tiles_array(insts))
    expected = [{"status": r.status, "length": r.length, "nodes": r.nodes, "moves": r.moves} for r in ref]
    best = autotune.tune(boards, 4, "batched", expected, repeats=1, rounds=1, log=lambda *a: None)
    assert set(best) == set(autotune.DEFAULT)
    autotune.save(4, "batched", best)
    cfg = autotune.load_config(4, "batched")
    assert cfg is not None and cfg.split_target == best["split_target"]
    sol = bpida.solve(boards, 4, cfg)
    torch.cuda.synchronize()
    got = sol.to_host()
    for g, e in zip(got, expected):
        assert (g["length"], g["nodes"], g["moves"]) == (e["length"], e["nodes"], e["moves"])


def test_tune_rejects_a_wrong_reference():
    insts = I.walks15_16x40()[:4]
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64)).cuda()
    ref = oracle.solve_batch(4, I.tiles_array(insts))
    wrong = [{"status": r.status, "length": r.length, "nodes": r.nodes[:-1] + [r.nodes[-1] + 1],
              "moves": r.moves} for r in ref]
    with pytest.raises(RuntimeError):
        autotune.tune(boards, 4, "batched", wrong, repeats=1, rounds=1, log=lambda *a: None)


def test_cached_configuration_is_picked_up(tmp_path, monkeypatch):
    """bpida.solve fills the configuration fields a caller leaves at 0 from
    the autotuner's cache entry for this GPU, width and call size (here a
    block-per-subtree search with 2-warp blocks for batched calls and 8-warp
    blocks for one-board calls); explicit fields and tuned=False keep the
    library's values; every result stays the oracle's."""
    monkeypatch.setenv("BPIDA_TUNE_CACHE", str(tmp_path / "tune.json"))
    autotune.save(4, "batched", {"variant": bpida.BLOCK_MODE, "warps_per_block": 2, "stack_entries": 384,
                                 "split_target": 1024, "exit_fraction_pct": 5, "min_rounds": 32})
    autotune.save(4, "plain", {"variant": 0, "warps_per_block": 8, "stack_entries": 512,
                               "split_target": 2048, "exit_fraction_pct": 10, "min_rounds": 64})
    insts = I.walks15_16x40()
    boards = torch.from_numpy(I.packed_array(insts).view(np.int64)).cuda()
    ref = oracle.solve_batch(4, I.tiles_array(insts))

    def check(sol, rows):
        for g, r in zip(sol.to_host(), rows):
            assert (g["length"], g["nodes"], g["moves"]) == (r.length, r.nodes, r.moves)

    sol = bpida.solve(boards, 4)
    check(sol, ref)
    assert bpida.last_stats()["block_threads"] == 64
    sol = bpida.solve(boards, 4, bpida.make_config(4, warps_per_block=4))
    check(sol, ref)
    assert bpida.last_stats()["block_threads"] == 128
    sol = bpida.solve(boards, 4, tuned=False)
    check(sol, ref)
    assert bpida.last_stats()["block_threads"] == 128
    sol = bpida.solve(boards[:1], 4)
    check(sol, ref[:1])
    assert bpida.last_stats()["block_threads"] == 256
    cfg = autotune.load_config(4, "batched")
    assert cfg.variant == bpida.BLOCK_MODE and cfg.stack_entries == 384
