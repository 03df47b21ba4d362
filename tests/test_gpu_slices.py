"""Bounded-memory joins: a join level whose next frontier would exceed dl_config.frontier_bytes
processes its input prefixes in slices, each carried through the remaining levels before the
next.  With a tiny frontier cap every multi-level join is sliced (down to single prefixes when
needed); the results and round counts must equal the oracle's, including the levels that read
an entry's sibling run (candidate reuse), filtered rules and recursive programs."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cap", [256, 4096, 1 << 16])
def test_sliced_cliques_match_oracle(cap):
    e = dg.rmat_edges(1 << 10, 12_000, 31, symmetric=True)
    rels = {"E": 2, "Tri": 3, "Q4": 4}
    ref = oracle.evaluate(rels, {"E": e}, P.TRI + P.Q4, sinks=["Q4"])
    got, strata, st = pkg.run_program(rels, {"E": e}, P.TRI + P.Q4, {"Q4": pkg.DL_SINK_COUNT},
                                      frontier_bytes=cap)
    assert np.array_equal(got["Tri"], ref.relations["Tri"])
    assert got["Q4"] == ref.digests["Q4"]
    assert st["join_slices"] > 0


def test_sliced_recursive_programs_match_oracle():
    e = dg.rmat_edges(512, 4000, 1000)
    ref = oracle.evaluate(P.TC_TRI_RELS, {"E": e}, P.TC_TRI)
    got, strata, st = pkg.run_program(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, frontier_bytes=1024)
    for name in P.TC_TRI_RELS:
        assert np.array_equal(got[name], ref.relations[name]), name
    assert sorted(strata) == sorted(ref.strata)
    assert st["join_slices"] > 0
    facts = {k: v for k, v in dg.points_to_facts(1 / 4096, 1002).items() if k != "domains"}
    ref = oracle.evaluate(P.POINTS_TO_RELS, facts, P.POINTS_TO)
    got, strata, st = pkg.run_program(P.POINTS_TO_RELS, facts, P.POINTS_TO, frontier_bytes=4096)
    for name in P.POINTS_TO_RELS:
        assert np.array_equal(got[name], ref.relations[name]), name
    assert sorted(strata) == sorted(ref.strata)
    assert st["join_slices"] > 0


def test_sliced_filtered_rules_match_oracle():
    e = dg.rmat_edges(1 << 9, 6000, 77, symmetric=True)
    rels = {"E": 2, "Q4Lt": 4}
    rule = [(("Q4Lt", ["w", "x", "y", "z"]), [("E", ["w", "x"]), ("E", ["w", "y"]), ("E", ["w", "z"]),
                                             ("E", ["x", "y"]), ("E", ["x", "z"]), ("E", ["y", "z"]),
                                             ("<", "w", "x"), ("<", "x", "y"), ("<", "y", "z")],
             ["w", "x", "y", "z"])]
    ref = oracle.evaluate(rels, {"E": e}, rule)
    got, _, st = pkg.run_program(rels, {"E": e}, rule, frontier_bytes=512)
    assert np.array_equal(got["Q4Lt"], ref.relations["Q4Lt"])
    assert st["join_slices"] > 0
