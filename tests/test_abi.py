"""The C ABI library builds, loads and exports every function that
include/bpida.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1705_02843_gb300 import bpida
from paper_1705_02843_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bpida.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bpida_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return ctypes.CDLL(bpida.LIB_PATH)


def test_header_declares_the_expected_calls():
    names = declared_functions()
    assert "bpida_solve" in names and "bpida_solve_ex" in names
    assert set(names) == set(bpida.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    b = bpida.load()
    assert b.bpida_max_len(4) == 80 and b.bpida_max_iters(4) == 41
    assert b.bpida_max_len(3) >= 31 and b.bpida_max_len(5) >= 100
    assert b.bpida_max_len(7) == 0
    assert bpida.status_str(bpida.EBUDGET) == "node budget exhausted"


def test_config_struct_layout():
    assert ctypes.sizeof(bpida.Config) == 7 * 4 + 4 + 8 + 16


def test_variant_arguments_are_checked_before_any_work(lib):
    """Unknown variants, and the ablation variants 2-5 with a 24-puzzle
    width, first-solution mode or a node budget, are rejected on the host."""
    b = bpida.load()
    bad = [dict(variant=7), dict(variant=-1), dict(variant=bpida.BLOCK_MODE, width=5), dict(variant=bpida.PSIMPLE, width=5),
           dict(variant=bpida.PSTATICLB, count_all=False), dict(variant=bpida.PFULLLB, node_budget=10),
           dict(variant=bpida.BPSTATIC, width=5), dict(variant=bpida.BPSTATIC, count_all=False)]
    for kw in bad:
        width = kw.pop("width", 4)
        cfg = bpida.make_config(width, **kw)
        rc = b.bpida_solve_ex(ctypes.byref(cfg), None, 0, None, None, None, None, None, None, None)
        assert rc == bpida.EINVAL, kw
    for v in (bpida.PSIMPLE, bpida.PSTATICLB, bpida.PFULLLB, bpida.BPSTATIC):
        cfg = bpida.make_config(4, variant=v)
        assert b.bpida_solve_ex(ctypes.byref(cfg), None, 0, None, None, None, None, None, None, None) == bpida.OK


def test_pattern_database_arguments_are_checked_before_any_work(lib):
    """Bad widths and groupings, a null table set and null outputs are
    rejected on the host, before any device call."""
    b = bpida.load()
    h = ctypes.c_void_p()
    ok15 = [0] + [0] * 5 + [1] * 5 + [2] * 5
    cases = [
        (5, ok15 + [0] * 9),                       # 24-puzzle: not supported
        (2, [0, 0, 0, 0]),                         # width out of range
        (4, [0] + [0] * 7 + [1] * 8),              # a group of 8 tiles
        (4, [0] + [0] * 5 + [2] * 10),             # group 1 empty
        (4, [0] + [6] * 3 + [0] * 12),             # group index 6
        (4, [0] + [-1] + [0] * 14),                # negative group
    ]
    for width, groups in cases:
        arr = (ctypes.c_int * len(groups))(*groups)
        assert b.bpida_pdb_create(width, arr, ctypes.byref(h), None) == bpida.EINVAL, (width, groups)
        assert h.value is None
    assert b.bpida_pdb_create(4, None, ctypes.byref(h), None) == bpida.EINVAL
    assert b.bpida_pdb_create(4, (ctypes.c_int * 16)(*ok15), None, None) == bpida.EINVAL
    cfg = bpida.make_config(4)
    assert b.bpida_solve_pdb(ctypes.byref(cfg), None, None, 0, None, None, None, None, None, None,
                             None) == bpida.EINVAL
    assert b.bpida_pdb_groups(None) == 0
    assert b.bpida_pdb_table_bytes(None, 0) == 0
    assert b.bpida_pdb_max_value(None, 0) == -1
    assert b.bpida_pdb_copy_table(None, 0, None, 0, None) == bpida.EINVAL
