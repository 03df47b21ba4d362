"""Helper-relation splitting on the GPU (dl_rule_add_split): the split rule gives the same
tuples as the unsplit rule and as the oracle, its helper relation holds the oracle's helper
rows, and a split over lower-stratum atoms keeps every round count."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


def run_split(rels, facts, rules, split, helper, **cfg):
    """rules[split[0]] is added split (atoms split[1] factored out into `helper`)."""
    with pkg.Engine(**cfg) as eng:
        for name, a in rels.items():
            eng.relation(name, a)
        for k, r in enumerate(rules):
            if k == split[0]:
                cols, _, _ = eng.rule_split(r[0], r[1], r[2], split[1], helper)
            else:
                eng.rule(r[0], r[1], r[2])
        for name, rows in facts.items():
            eng.load(name, rows)
        st = eng.fixpoint()
        out = {name: eng.fetch(name) for name in list(rels) + [helper]}
        return out, eng.strata(), cols, st


@pytest.mark.parametrize("scale", [0.05, 0.3])
def test_call_graph_edge_split_equals_unsplit_and_oracle(scale):
    f = dg.call_graph_facts(scale, 1007)
    ref = oracle.evaluate(dict(P.CGE_RELS, HelpNT=4), f, P.CGE_HELPER)
    mono, _, _ = pkg.run_program(P.CGE_RELS, f, P.CGE)
    split, _, cols, _ = run_split(P.CGE_RELS, f, P.CGE, (0, P.CGE_SPLIT), "HelpNT")
    assert cols == ["sn", "dsc", "h", "m"]
    assert len(ref.relations["CallGraphEdge"]) > 0
    assert np.array_equal(mono["CallGraphEdge"], ref.relations["CallGraphEdge"])
    assert np.array_equal(split["CallGraphEdge"], ref.relations["CallGraphEdge"])
    assert np.array_equal(split["HelpNT"], ref.relations["HelpNT"])


REACH3 = [
    (("R", ["x", "z"]), [("E", ["x", "z"])], ["x", "z"]),
    (("R", ["x", "z"]), [("R", ["x", "y"]), ("E", ["y", "w"]), ("E", ["w", "z"])], ["x", "y", "w", "z"]),
]


def test_split_of_a_recursive_rule():
    e = dg.rmat_edges(300, 1500, 1008)
    ref = oracle.evaluate({"E": 2, "R": 2}, {"E": e}, REACH3)
    # factoring the two edge atoms: the helper is a lower stratum, round counts unchanged
    got, strata, cols, _ = run_split({"E": 2, "R": 2}, {"E": e}, REACH3, (1, (1, 2)), "H")
    assert cols == ["y", "z"]
    assert np.array_equal(got["R"], ref.relations["R"])
    assert [r for names, r in strata if "R" in names] == [r for names, r in ref.strata if "R" in names]
    # factoring the recursive atom: same tuples (the helper joins the recursive stratum)
    got2, strata2, cols2, _ = run_split({"E": 2, "R": 2}, {"E": e}, REACH3, (1, (0, 1)), "H")
    assert cols2 == ["x", "w"]
    assert np.array_equal(got2["R"], ref.relations["R"])
    assert any("H" in names and "R" in names for names, _ in strata2)


def test_split_in_the_batched_form():
    facts = [dg.call_graph_facts(0.02, 1100 + k) for k in range(3)]
    with pkg.Engine(instances=3) as eng:
        for name, a in P.CGE_RELS.items():
            eng.relation(name, a)
        head, body, order = P.CGE[0]
        eng.rule_split(head, body, order, P.CGE_SPLIT, "HelpNT")
        for k, f in enumerate(facts):
            for name, rows in f.items():
                eng.load_instance(name, k, rows)
        eng.fixpoint()
        for k, f in enumerate(facts):
            ref = oracle.evaluate(P.CGE_RELS, f, P.CGE)
            assert np.array_equal(eng.fetch_instance("CallGraphEdge", k), ref.relations["CallGraphEdge"])


def test_bad_split_adds_nothing():
    with pkg.Engine() as eng:
        for name, a in P.CGE_RELS.items():
            eng.relation(name, a)
        head, body, order = P.CGE[0]
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule_split(head, body, order, P.CGE_SPLIT, "MethodLookup")   # name taken
        assert ex.value.code == pkg.DL_ERR_ARG
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule_split(head, body, order[:-1], P.CGE_SPLIT, "HelpNT")    # bad order
        assert ex.value.code == pkg.DL_ERR_ARG
        n = pkg.ctypes.c_uint64()
        assert eng.lib.dl_relation_size(eng.h, len(P.CGE_RELS), pkg.ctypes.byref(n)) != pkg.DL_OK
        eng.rule_split(head, body, order, P.CGE_SPLIT, "HelpNT")
        f = dg.call_graph_facts(0.02, 1200)
        for name, rows in f.items():
            eng.load(name, rows)
        eng.fixpoint()
        ref = oracle.evaluate(P.CGE_RELS, f, P.CGE)
        assert np.array_equal(eng.fetch("CallGraphEdge"), ref.relations["CallGraphEdge"])
