"""Dense relation bitmaps (dl_config.dense_bytes): during a recursive stratum's rounds, a
relation whose column domains are small gets one bit per possible row, and a round's new rows
are found by one test-and-set per derived row instead of probing the relation's index and a
deduplicating sort (the paper's Section 4 Compute Delta).  By default the join's last level
sets the bits itself (the dense sink: no rule output is written) and the round's delta is read
back from the bits set since the previous round; DL_FLAG_NO_DENSE_SINK writes the rows and
filters them.  Results and round counts equal the oracle's with the sink, without it, and
without bitmaps (dense_bytes = 1), for recursive programs with binary and ternary relations,
several variants per rule, comparisons, constants and a repeated variable in the head,
chunked rule output, head/body flushes, both kernel shapes (the autotuner times each, so the
sink runs more than once on the same round) and the batched form."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


# a recursive relation with constants and a repeated variable in its heads, and a recursive
# rule with a comparison (the filtered kernels with the sink)
HEADS = [
    (("R3", ["x", "y", 1]), [("E", ["x", "y"])], ["x", "y"]),
    (("R3", ["x", "z", 1]), [("R3", ["x", "y", "c"]), ("E", ["y", "z"]), ("!=", "x", "z")], ["x", "y", "c", "z"]),
    (("R3", ["z", "z", 2]), [("R3", ["x", "z", "c"]), ("E", ["z", "x"])], ["c", "x", "z"]),
]
HEADS_RELS = {"E": 2, "R3": 3}


def cases():
    pt = {k: v for k, v in dg.points_to_facts(1 / 2048, 1002).items() if k != "domains"}
    return [(P.TC_TRI_RELS, {"E": dg.rmat_edges(1024, 9000, 1000)}, P.TC_TRI),
            (P.POINTS_TO_RELS, pt, P.POINTS_TO),
            (P.SG_RELS, {"Edge": dg.rmat_edges(300, 1500, 11)}, P.SG),
            (HEADS_RELS, {"E": dg.rmat_edges(400, 2400, 12)}, HEADS)]


NO_SINK = pkg.DL_FLAG_NO_DENSE_SINK


@pytest.mark.parametrize("cfg", [{}, {"dense_bytes": 1}, {"chunk_rows": 5000, "head_percent": 1},
                                 {"flags": NO_SINK}, {"flags": NO_SINK, "chunk_rows": 5000, "head_percent": 1},
                                 {"flags": pkg.DL_FLAG_AUTOTUNE}, {"tile_units": 4096}])
def test_dense_bitmaps_match_oracle(cfg):
    for rels, facts, rules in cases():
        ref = oracle.evaluate(rels, facts, rules)
        got, strata, st = pkg.run_program(rels, facts, rules, **cfg)
        for name in rels:
            assert np.array_equal(got[name], ref.relations[name]), (cfg, name)
        assert sorted(strata) == sorted(ref.strata)
        assert (st["dense_relations"] > 0) == (cfg.get("dense_bytes") != 1)


def test_dense_sink_writes_no_rule_output():
    """With the sink, a recursive round's rule rows never pass through the write pass: the
    delta kernels see only the extraction, and the join's raw row count is still reported."""
    rels, facts, rules = cases()[1]
    got, _, st = pkg.run_program(rels, facts, rules, flags=pkg.DL_FLAG_PROFILE)
    got2, _, st2 = pkg.run_program(rels, facts, rules, flags=pkg.DL_FLAG_PROFILE | NO_SINK)
    for name in rels:
        assert np.array_equal(got[name], got2[name])
    assert st["join_rows"] == st2["join_rows"] > 0
    assert st["kernels"]["sort"]["launches"] < st2["kernels"]["sort"]["launches"]


@pytest.mark.parametrize("flags", [0, NO_SINK])
def test_dense_bitmaps_batched_form(flags):
    insts = [{"E": dg.rmat_edges(150 + 40 * i, 800 + 250 * i, 120 + i)} for i in range(6)]
    outs, rounds, st = pkg.run_batched(P.TC_TRI_RELS, insts, P.TC_TRI, flags=flags)
    assert st["dense_relations"] > 0
    for i, facts in enumerate(insts):
        ref = oracle.evaluate(P.TC_TRI_RELS, facts, P.TC_TRI)
        for name in P.TC_TRI_RELS:
            assert np.array_equal(outs[i][name], ref.relations[name]), (i, name)
        assert sorted(rounds[i]) == sorted(ref.strata)
