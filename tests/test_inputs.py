"""Seeded input generators: determinism, board validity, packing."""
import numpy as np

from paper_1705_02843_gb300 import inputs as I
from tests import puzzle_ref as P


def test_splitmix64_reference_value():
    # first SplitMix64 output for state 0, as published with the generator
    assert I.splitmix64(0)[1] == 0xE220A8397B1DCDAF


def test_xoshiro_deterministic_and_bounded():
    a, b = I.Xoshiro256ss(5), I.Xoshiro256ss(5)
    xs = [a.next_u64() for _ in range(100)]
    assert xs == [b.next_u64() for _ in range(100)]
    assert len(set(xs)) == 100
    r = I.Xoshiro256ss(6)
    v = [r.below(7) for _ in range(7000)]
    assert set(v) == set(range(7))
    assert all(600 < v.count(k) < 1400 for k in range(7))


def test_walks_are_boards_and_reversal_free():
    for W in (3, 4, 5):
        for s in range(20):
            t = I.random_walk(W, 30, I.Xoshiro256ss(s))
            assert sorted(t) == list(range(W * W))


def test_pack_roundtrip():
    for W in (3, 4, 5):
        rng = I.Xoshiro256ss(W)
        for _ in range(50):
            t = I.random_permutation(W, rng)
            assert I.unpack(W, I.pack(W, t)) == t
    assert I.pack(4, list(range(16))) == [0xFEDCBA9876543210]


def test_named_workloads_shapes():
    w = I.walks15_16x40()
    assert len(w) == 16 and all(x.walk_len == 40 for x in w)
    p = I.perms15_100()
    assert len(p) == 100 and len({tuple(x.tiles) for x in p}) == 100
    m = I.mixed15_4096()
    assert len(m) == 4096 and sum(x.kind == "perm" for x in m) == 205
    assert all(20 <= x.walk_len <= 90 for x in m if x.kind == "walk")
    arr = I.packed_array(m)
    assert arr.dtype == np.uint64 and arr.shape == (4096,)


def test_permutations_in_goal_class_8puzzle():
    dist, _, _ = P.bfs8()
    rng = I.Xoshiro256ss(11)
    for _ in range(200):
        assert tuple(I.random_permutation(3, rng)) in dist


def test_pattern_database_partitions_are_well_formed():
    for name, groups in I.PDB_PARTITIONS.items():
        tiles = sorted(t for g in groups for t in g)
        assert tiles == list(range(1, 16)), name
        assert 1 <= len(groups) <= 6 and all(1 <= len(g) <= 6 for g in groups), name


def test_stored_pattern_database_results_match_the_oracle():
    """The stored oracle results the --pdb bench checks against: the ten
    cheapest boards of the 5-5-5 file re-solved by the oracle now, and the
    6-6-3 file's lengths and first solutions equal the Manhattan file's (any
    admissible heuristic returns the same length, solution count and first
    optimal path)."""
    import json
    import os

    import oracle

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    md = {r["index"]: r for r in json.load(open(os.path.join(here, "perms15_100.json")))["instances"]}
    insts = I.perms15_100()
    for part in ("555", "663"):
        doc = json.load(open(os.path.join(here, "perms15_100_pdb%s.json" % part)))
        recs = {r["index"]: r for r in doc["instances"]}
        assert sorted(recs) == list(range(100))
        for i, r in recs.items():
            assert r["status"] == 0 and r["seed"] == insts[i].seed
            assert (r["length"], r["moves"], r["solutions"]) == (md[i]["length"], md[i]["moves"], md[i]["solutions"])
            assert sum(r["nodes"]) < sum(md[i]["nodes"])
    pdb = oracle.PatternDb(4, I.PDB_PARTITIONS["555"])
    recs = json.load(open(os.path.join(here, "perms15_100_pdb555.json")))["instances"]
    cheap = sorted(recs, key=lambda r: sum(r["nodes"]))[:10]
    res = oracle.solve_batch(4, np.array([insts[r["index"]].tiles for r in cheap], dtype=np.uint8), pdb=pdb)
    for r, o in zip(cheap, res):
        assert o.nodes == r["nodes"] and o.limits == r["limits"] and o.h0 == r["h0"]
