"""Dense relation bitmaps (dl_config.dense_bytes): during a recursive stratum's rounds, a
relation whose column domains are small gets one bit per possible row, and a round's new rows
are found by one test-and-set per derived row instead of probing the relation's index and a
deduplicating sort (the paper's Section 4 Compute Delta).  Results and round counts equal the
oracle's with the bitmaps and without them (dense_bytes = 1), for recursive programs with
binary and ternary relations, several variants per rule, chunked rule output, head/body
flushes and the batched form."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


def cases():
    pt = {k: v for k, v in dg.points_to_facts(1 / 2048, 1002).items() if k != "domains"}
    return [(P.TC_TRI_RELS, {"E": dg.rmat_edges(1024, 9000, 1000)}, P.TC_TRI),
            (P.POINTS_TO_RELS, pt, P.POINTS_TO),
            (P.SG_RELS, {"Edge": dg.rmat_edges(300, 1500, 11)}, P.SG)]


@pytest.mark.parametrize("cfg", [{}, {"dense_bytes": 1}, {"chunk_rows": 5000, "head_percent": 1}])
def test_dense_bitmaps_match_oracle(cfg):
    for rels, facts, rules in cases():
        ref = oracle.evaluate(rels, facts, rules)
        got, strata, st = pkg.run_program(rels, facts, rules, **cfg)
        for name in rels:
            assert np.array_equal(got[name], ref.relations[name]), (cfg, name)
        assert sorted(strata) == sorted(ref.strata)
        assert (st["dense_relations"] > 0) == (cfg.get("dense_bytes") != 1)


def test_dense_bitmaps_batched_form():
    insts = [{"E": dg.rmat_edges(150 + 40 * i, 800 + 250 * i, 120 + i)} for i in range(6)]
    outs, rounds, st = pkg.run_batched(P.TC_TRI_RELS, insts, P.TC_TRI)
    assert st["dense_relations"] > 0
    for i, facts in enumerate(insts):
        ref = oracle.evaluate(P.TC_TRI_RELS, facts, P.TC_TRI)
        for name in P.TC_TRI_RELS:
            assert np.array_equal(outs[i][name], ref.relations[name]), (i, name)
        assert sorted(rounds[i]) == sorted(ref.strata)
