"""The all-cores CPU baseline harness: the oracle run on root parts in spawned processes
gives the same row counts as one run over the whole root sample."""
import os
import tempfile

import numpy as np

import oracle
from oracle.parallel import run_rooted
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
        counts, wall = run_rooted({"E": path}, RELS, TRI_ROOTED, roots, 3, timeout=120)
    assert counts["Tri"] == len(whole.relations["Tri"]) > 0
    assert counts["Root"] == len(roots)
    assert wall > 0
