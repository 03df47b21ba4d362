"""Parity at the full size of the skewed cyclic workload (symmetrised R-MAT scale 20,
16,777,216 rows), in the launch configuration bench.py times.

* whole relations against the oracle: the count and order-independent digest of the
  oriented triangles (TriLt) and 4-cliques (Q4Lt, count sink) and of the symmetric
  triangles (Tri), from tests/golden/cliques_rmat20.json (written by
  tests/golden/make_fullsize_cliques.py, which runs only the oracle); the symmetric 4-clique
  count is 24 x the oracle's oriented count and the symmetric triangle count 6 x (each
  clique in every order);
* sampled outputs: Tri and Q4 rows rooted at sampled vertices (the heaviest hubs for Tri,
  random vertices plus heavy keys with bitmaps for Q4), computed by the GPU and by the
  oracle as root-restricted programs (Root(x) is one more body atom), compared tuple for
  tuple;
* properties that hold at any size, between independent GPU runs: |Tri| on the symmetric
  graph = 6 x |Tri| on the id-oriented graph, |Q4| = 24 x, and the AGM bounds
  |Tri| <= |E|^1.5, |Q4| <= |E|^2 (paper Section 2).
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu

TRI_R = [(("TriR", ["x", "y", "z"]), [("Root", ["x"]), ("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"])],
          ["x", "y", "z"])]
Q4_R = [(("Q4R", ["w", "x", "y", "z"]),
         [("Root4", ["w"]), ("E", ["w", "x"]), ("E", ["w", "y"]), ("E", ["x", "y"]), ("E", ["w", "z"]),
          ("E", ["x", "z"]), ("E", ["y", "z"])], ["w", "x", "y", "z"])]


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cliques_rmat20.json")
TRI_LT = [(("TriLt", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"]),
                                       ("<", "x", "y"), ("<", "y", "z")], ["x", "y", "z"])]
Q4_LT = [(("Q4Lt", ["w", "x", "y", "z"]), [("E", ["w", "x"]), ("E", ["w", "y"]), ("E", ["w", "z"]),
                                          ("E", ["x", "y"]), ("E", ["x", "z"]), ("E", ["y", "z"]),
                                          ("<", "w", "x"), ("<", "x", "y"), ("<", "y", "z")], ["w", "x", "y", "z"])]


@pytest.fixture(scope="module")
def edges():
    return dg.rmat_edges(1 << 20, 1 << 24, 1001, symmetric=True)


def test_whole_relations_match_oracle_goldens(edges):
    gold = json.load(open(GOLDEN))
    assert gold["graph"] == "rmat_edges(1048576, 16777216, 1001, symmetric=True)"
    want = {k: (gold[k]["count"], gold[k]["sum"], gold[k]["xor"]) for k in ("TriLt", "Q4Lt", "Tri")}
    # the oriented rules (comparison filters) and the symmetric ones, as bench.py runs them
    with pkg.Engine(flags=pkg.DL_FLAG_PROFILE) as eng:
        pkg.build_program(eng, {"E": 2, "TriLt": 3, "Q4Lt": 4}, TRI_LT + Q4_LT, {"Q4Lt": pkg.DL_SINK_COUNT})
        eng.load("E", edges)
        eng.fixpoint()
        assert eng.digest("TriLt") == want["TriLt"]
        assert eng.digest("Q4Lt") == want["Q4Lt"]
    with pkg.Engine(flags=pkg.DL_FLAG_PROFILE) as eng:
        pkg.build_program(eng, {"E": 2, "Tri": 3, "Q4": 4}, P.TRI + P.Q4, {"Q4": pkg.DL_SINK_COUNT})
        eng.load("E", edges)
        eng.fixpoint()
        assert eng.digest("Tri") == want["Tri"]
        assert eng.size("Tri") == 6 * want["TriLt"][0]
        assert eng.size("Q4") == 24 * want["Q4Lt"][0]


def test_sampled_roots_match_oracle(edges):
    e = edges
    deg = np.bincount(e[:, 0], minlength=1 << 20)
    order = np.argsort(-deg, kind="stable")
    rng = np.random.default_rng(2024)
    tri_roots = np.unique(np.concatenate([order[:4], rng.choice(order[:200000], 60, replace=False)]))
    q4_roots = np.unique(rng.choice(order[2000:300000], 48, replace=False))
    rels = {"E": 2, "Root": 1, "Root4": 1, "TriR": 3, "Q4R": 4}
    facts = {"E": e, "Root": tri_roots.astype(np.uint32).reshape(-1, 1),
             "Root4": q4_roots.astype(np.uint32).reshape(-1, 1)}
    got, strata, _ = pkg.run_program(rels, facts, TRI_R + Q4_R)
    ref = oracle.evaluate(rels, facts, TRI_R + Q4_R)
    for name in ("TriR", "Q4R"):
        assert np.array_equal(got[name], ref.relations[name]), name
    assert len(got["TriR"]) > 1000 and len(got["Q4R"]) > 100


def test_heavy_key_q4_roots_match_oracle(edges):
    """4-cliques rooted at eight heavy keys (degree ranks 1200-1900, about 700-900 rows each:
    keys with membership bitmaps, whose candidate ranges are split across warps and CTAs),
    compared by count and digest (count sinks on both sides)."""
    e = edges
    deg = np.bincount(e[:, 0], minlength=1 << 20)
    order = np.argsort(-deg, kind="stable")
    roots = np.sort(order[1200:2000:100]).astype(np.uint32).reshape(-1, 1)
    assert deg[roots.reshape(-1)].min() >= 512
    rels = {"E": 2, "Root4": 1, "Q4R": 4}
    facts = {"E": e, "Root4": roots}
    got, _, _ = pkg.run_program(rels, facts, Q4_R, {"Q4R": pkg.DL_SINK_COUNT})
    ref = oracle.evaluate(rels, facts, Q4_R, sinks=["Q4R"])
    assert got["Q4R"] == ref.digests["Q4R"]
    assert ref.digests["Q4R"][0] > 1_000_000


def test_orientation_invariants_and_agm(edges):
    e = edges
    eo = e[e[:, 0] < e[:, 1]]
    sinks = {"Q4": pkg.DL_SINK_COUNT}
    rels = {"E": 2, "Tri": 3, "Q4": 4}
    counts = []
    for g in (e, eo):
        with pkg.Engine() as eng:
            pkg.build_program(eng, rels, P.TRI + P.Q4, sinks)
            eng.load("E", g)
            eng.fixpoint()
            counts.append((eng.size("Tri"), eng.size("Q4")))
    (tri, q4), (tri_o, q4_o) = counts
    assert tri == 6 * tri_o and q4 == 24 * q4_o
    assert tri <= len(e) ** 1.5 and q4 <= len(e) ** 2
    assert tri > 0 and q4 > 0
