"""Head/body relations (the paper's Section 4, Merge): during a recursive stratum's rounds a
round's new rows go into a small head that is merged into the body above
dl_config.head_percent of it, and joins read body and head as one relation.  Results and
round counts must equal the oracle's whatever the threshold: flushing every round, at 25%,
or only at the stratum's end."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu

NEVER = 0xFFFFFFFF


@pytest.mark.parametrize("pct", [1, 25, 400, NEVER])
def test_head_body_recursive_programs_match_oracle(pct):
    cases = [(P.TC_TRI_RELS, {"E": dg.rmat_edges(1024, 8000, 1000)}, P.TC_TRI),
             (P.POINTS_TO_RELS, {k: v for k, v in dg.points_to_facts(1 / 4096, 1002).items() if k != "domains"},
              P.POINTS_TO)]
    for rels, facts, rules in cases:
        ref = oracle.evaluate(rels, facts, rules)
        got, strata, st = pkg.run_program(rels, facts, rules, head_percent=pct)
        for name in rels:
            assert np.array_equal(got[name], ref.relations[name]), (pct, name)
        assert sorted(strata) == sorted(ref.strata)
        if pct == 1:
            assert st["head_flushes"] > 0


def test_head_body_batched_form_matches_alone():
    insts = [{"E": dg.rmat_edges(200 + 50 * i, 900 + 300 * i, 40 + i)} for i in range(6)]
    outs, rounds, st = pkg.run_batched(P.TC_TRI_RELS, insts, P.TC_TRI, head_percent=5)
    for i, facts in enumerate(insts):
        ref = oracle.evaluate(P.TC_TRI_RELS, facts, P.TC_TRI)
        for name in P.TC_TRI_RELS:
            assert np.array_equal(outs[i][name], ref.relations[name]), (i, name)
        assert sorted(rounds[i]) == sorted(ref.strata)
