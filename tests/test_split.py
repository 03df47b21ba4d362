"""Helper-relation splitting (Section 5): the helper columns a split creates (host logic of
the C ABI, no GPU), and the oracle's result for the CallGraphEdge rule pinned to a direct
evaluation of the rule's definition."""
import itertools

import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P


def test_split_columns_of_the_call_graph_rule():
    head, body, order = P.CGE[0]
    # the factored atoms bind h, t, sn, dsc, m; t is used nowhere else
    assert pkg.split_columns(head, body, order, P.CGE_SPLIT) == ["sn", "dsc", "h", "m"]
    assert pkg.split_columns(head, body, order, (0, 1)) == ["i"]
    assert pkg.split_columns(head, body, order, (2,)) == ["i", "b", "sn", "dsc"]


def test_split_columns_follow_the_variable_order():
    head, body = ("R", ["x", "z"]), [("A", ["x", "y"]), ("B", ["y", "w"]), ("C", ["w", "z"])]
    assert pkg.split_columns(head, body, ["x", "y", "w", "z"], (1, 2)) == ["y", "z"]
    assert pkg.split_columns(head, body, ["z", "w", "y", "x"], (1, 2)) == ["z", "y"]


@pytest.mark.parametrize("factored,code", [((), pkg.DL_ERR_ARG), ((0, 1, 2), pkg.DL_ERR_ARG), ((5,), pkg.DL_ERR_ARG)])
def test_bad_splits_are_rejected(factored, code):
    head, body = ("R", ["x", "z"]), [("A", ["x", "y"]), ("B", ["y", "w"]), ("C", ["w", "z"])]
    with pytest.raises(pkg.DatalogError) as ex:
        pkg.split_columns(head, body, ["x", "y", "w", "z"], factored)
    assert ex.value.code == code


def test_split_sharing_nothing_is_unsupported():
    with pytest.raises(pkg.DatalogError) as ex:
        pkg.split_columns(("R", ["x"]), [("A", ["x"]), ("B", ["y"])], ["x", "y"], (1,))
    assert ex.value.code == pkg.DL_ERR_UNSUPPORTED


def _direct_cge(f):
    """CallGraphEdge written out from its definition: for every binding of the body's
    variables that satisfies all six atoms, the pair (i, m)."""
    reach = {r[0] for r in f["Reachable"].tolist()}
    im = {}
    for i, j in f["InstructionMethod"].tolist():
        im.setdefault(i, []).append(j)
    vpt = {}
    for h, b in f["VarPointsTo"].tolist():
        vpt.setdefault(b, []).append(h)
    hat = {}
    for h, t in f["HeapAllocationType"].tolist():
        hat.setdefault(h, []).append(t)
    ml = {}
    for sn, dsc, t, m in f["MethodLookup"].tolist():
        ml.setdefault((sn, dsc, t), []).append(m)
    out = set()
    for i, b, sn, dsc in f["VirtualMethodInvoc"].tolist():
        if not any(j in reach for j in im.get(i, [])):
            continue
        for h in vpt.get(b, []):
            for t in hat.get(h, []):
                for m in ml.get((sn, dsc, t), []):
                    out.add((i, m))
    return np.array(sorted(out), dtype=np.uint32).reshape(-1, 2)


def test_oracle_call_graph_edge_matches_its_definition():
    f = dg.call_graph_facts(0.05, 1005)
    ref = oracle.evaluate(P.CGE_RELS, f, P.CGE)
    want = _direct_cge(f)
    assert len(want) > 100
    assert np.array_equal(ref.relations["CallGraphEdge"], want)


def test_oracle_split_by_hand_equals_unsplit():
    f = dg.call_graph_facts(0.05, 1006)
    a = oracle.evaluate(P.CGE_RELS, f, P.CGE)
    b = oracle.evaluate(dict(P.CGE_RELS, HelpNT=4), f, P.CGE_HELPER)
    assert np.array_equal(a.relations["CallGraphEdge"], b.relations["CallGraphEdge"])
    # the helper holds the join of its two atoms projected on (sn, dsc, h, m)
    hat, ml = f["HeapAllocationType"].tolist(), f["MethodLookup"].tolist()
    by_t = {}
    for sn, dsc, t, m in ml:
        by_t.setdefault(t, []).append((sn, dsc, m))
    help_rows = sorted({(sn, dsc, h, m) for h, t in hat for sn, dsc, m in by_t.get(t, [])})
    assert np.array_equal(b.relations["HelpNT"], np.array(help_rows, dtype=np.uint32).reshape(-1, 4))
