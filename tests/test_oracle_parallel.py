"""The root-partitioned oracle harness (the all-cores CPU baseline and the full-size golden
script): the oracle run on root parts in spawned processes gives the same row counts and
count-sink digests as one run over the whole root sample, and the golden script's rooted,
oriented rules give the whole relations' digests on a small graph."""
import os
import sys
import tempfile

import numpy as np

import oracle
from oracle.parallel import run_rooted, split_roots
from paper_2604_20073_gb300 import datagen as dg

RELS = {"E": 2, "Root": 1, "Tri": 3}
TRI_ROOTED = [(("Tri", ["x", "y", "z"]), [("Root", ["x"]), ("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"])])]


def test_root_parts_add_up_to_the_whole_sample():
    e = dg.rmat_edges(1 << 9, 4000, 17, symmetric=True)
    roots = np.unique(e[:, 0])[::3].astype(np.uint32).reshape(-1, 1)
    whole = oracle.evaluate(RELS, {"E": e, "Root": roots}, TRI_ROOTED)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "E.npy")
        np.save(path, e)
        run = run_rooted({"E": path}, RELS, TRI_ROOTED, roots, 3, timeout=120)
        sunk = run_rooted({"E": path}, RELS, TRI_ROOTED, roots, 2, timeout=120, sinks=("Tri",), nparts=5,
                          weight=np.arange(len(roots)))
    assert run.counts["Tri"] == len(whole.relations["Tri"]) > 0
    assert run.counts["Root"] == len(roots)
    assert run.wall > 0 and len(run.join_s) == 3
    assert sunk.digests["Tri"] == oracle.tuple_digest(whole.relations["Tri"])
    assert len(sunk.join_s) == 5


def test_split_roots_deals_heaviest_first():
    parts = split_roots(np.arange(10), 3, weight=np.arange(10))
    assert [p.reshape(-1).tolist() for p in parts] == [[0, 3, 6, 9], [2, 5, 8], [1, 4, 7]]
    assert sorted(np.concatenate(parts).reshape(-1).tolist()) == list(range(10))


def test_golden_script_rules_match_the_whole_relations():
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_fullsize_cliques as m
    got = m.compute(10, 2, 6, log=lambda *a: None)
    n = 1 << 10
    e = dg.rmat_edges(n, 16 * n, 1001, symmetric=True)
    rels = {"E": 2, "TriLt": 3, "Q4Lt": 4, "Tri": 3}
    rules = [(("TriLt", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"]),
                                           ("<", "x", "y"), ("<", "y", "z")]),
             (("Q4Lt", ["w", "x", "y", "z"]), [("E", ["w", "x"]), ("E", ["w", "y"]), ("E", ["w", "z"]),
                                               ("E", ["x", "y"]), ("E", ["x", "z"]), ("E", ["y", "z"]),
                                               ("<", "w", "x"), ("<", "x", "y"), ("<", "y", "z")]),
             (("Tri", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"])])]
    whole = oracle.evaluate(rels, {"E": e}, rules)
    for name in ("TriLt", "Q4Lt", "Tri"):
        g = got[name]
        assert (g["count"], g["sum"], g["xor"]) == oracle.tuple_digest(whole.relations[name]), name
        assert g["count"] > 0
    assert got["Tri"]["count"] == 6 * got["TriLt"]["count"]
