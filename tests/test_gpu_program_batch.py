"""Batches of different programs (dl_program_* + dl_fixpoint_batch): TC + Tri, 4-clique
(count sink) and points-to programs of different sizes evaluated in one batch; programs of
the same shape share each stage's launches.  Every program's relations, count-sink digests
and round counts equal the oracle's and those of the program run alone."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu
SINK = {"Q4": pkg.DL_SINK_COUNT}


def mixed_programs():
    progs = []
    for i in range(5):
        m = 300 + 700 * i
        progs.append(("tc", P.TC_TRI_RELS, {"E": dg.rmat_edges(max(2, m // 8), m, 60 + i)}, P.TC_TRI, None))
    for i in range(4):
        m = 2000 + 3000 * i
        progs.append(("q4", P.Q4_RELS, {"E": dg.rmat_edges(max(16, m // 16), m, 70 + i, symmetric=True)}, P.Q4, SINK))
    for i in range(2):
        f = {k: v for k, v in dg.points_to_facts(1 / 8192, 80 + i).items() if k != "domains"}
        progs.append(("pt", P.POINTS_TO_RELS, f, P.POINTS_TO, None))
    return progs


def test_mixed_program_batch_matches_oracle_and_alone():
    progs = mixed_programs()
    with pkg.Engine() as eng:
        handles = []
        for kind, rels, facts, rules, sinks in progs:
            p = pkg.Program(eng, rels, rules, sinks)
            for name, rows in facts.items():
                p.load(name, rows)
            handles.append(p)
        stats = pkg.fixpoint_batch(eng, handles)
        assert len(stats) == len(progs)
        for (kind, rels, facts, rules, sinks), p in zip(progs, handles):
            got = p.result()
            ref = oracle.evaluate(rels, facts, rules, sinks=[n for n in (sinks or {})])
            alone, alone_strata, _ = pkg.run_program(rels, facts, rules, sinks)
            for name in rels:
                if (sinks or {}).get(name) == pkg.DL_SINK_COUNT:
                    assert got[name] == ref.digests[name] == alone[name], (kind, name)
                else:
                    assert np.array_equal(got[name], ref.relations[name]), (kind, name)
                    assert np.array_equal(got[name], alone[name]), (kind, name)
            assert sorted(p.strata()) == sorted(ref.strata) == sorted(alone_strata), kind
        for p in handles:
            p.close()


def test_batched_count_sink_per_instance():
    insts = [{"E": dg.rmat_edges(64 + 32 * i, 900 + 400 * i, 90 + i, symmetric=True)} for i in range(5)]
    outs, rounds, st = pkg.run_batched(P.Q4_RELS, insts, P.Q4, sinks=SINK)
    for i, facts in enumerate(insts):
        ref = oracle.evaluate(P.Q4_RELS, facts, P.Q4, sinks=["Q4"])
        assert outs[i]["Q4"] == ref.digests["Q4"], i
        assert np.array_equal(outs[i]["E"], ref.relations["E"])


def test_program_errors_are_reported():
    with pkg.Engine() as eng:
        p = pkg.Program(eng, {"E": 2, "R": 2}, [(("R", ["x", "y"]), [("E", ["x", "y"])], ["x", "y"])])
        with pytest.raises(pkg.DatalogError):
            p.fetch("R")          # not evaluated yet
        # a variable order that leaves out a body variable is rejected when the batch runs
        bad = pkg.Program(eng, {"E": 2, "R": 1}, [(("R", ["x"]), [("E", ["x", "y"])], ["x"])])
        bad.load("E", np.array([[1, 2]], dtype=np.uint32))
        with pytest.raises(pkg.DatalogError):
            pkg.fixpoint_batch(eng, [bad])
        p.close()
        bad.close()
