"""Pins for the oracle's comparisons and stratified negation: closed forms, dense numpy
counts and an independent reachability routine; random programs with filters against the
brute-force evaluator."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P


def run(rels, facts, rules, mode="seminaive"):
    return oracle.evaluate(rels, facts, rules, mode)


@pytest.mark.parametrize("n", [3, 5, 9])
def test_oriented_cliques_on_complete_graphs(n):
    e = dg.complete_sym(n)
    r = run({"E": 2, "TriLt": 3, "Q4Lt": 4}, {"E": e}, P.TRI_LT + P.Q4_LT)
    assert len(r.relations["TriLt"]) == math.comb(n, 3)
    assert len(r.relations["Q4Lt"]) == math.comb(n, 4)
    assert all(a < b < c for a, b, c in r.relations["TriLt"].tolist())


@pytest.mark.parametrize("seed", range(3))
def test_oriented_triangles_match_dense_count(seed):
    e = dg.random_graph(40, 300, 70 + seed)
    e = dg.unique_rows(np.concatenate([e, e[:, ::-1]]))
    A = np.zeros((40, 40), dtype=np.int64)
    A[e[:, 0], e[:, 1]] = 1
    r = run({"E": 2, "TriLt": 3}, {"E": e}, P.TRI_LT)
    assert len(r.relations["TriLt"]) == np.trace(A @ A @ A) // 6


@pytest.mark.parametrize("op,count", [("<", lambda n: n * (n - 1) // 2), ("<=", lambda n: n * (n + 1) // 2),
                                      (">", lambda n: n * (n - 1) // 2), (">=", lambda n: n * (n + 1) // 2),
                                      ("!=", lambda n: n * (n - 1))])
def test_comparison_pairs_closed_forms(op, count):
    n = 11
    nodes = np.arange(n, dtype=np.uint32).reshape(-1, 1)
    rules = [(("Pair", ["x", "y"]), [("N", ["x"]), ("N", ["y"]), (op, "x", "y")])]
    r = run({"N": 1, "Pair": 2}, {"N": nodes}, rules)
    assert len(r.relations["Pair"]) == count(n)
    py_op = {"<": np.less, "<=": np.less_equal, ">": np.greater, ">=": np.greater_equal, "!=": np.not_equal}[op]
    assert all(py_op(x, y) for x, y in r.relations["Pair"].tolist())


def test_comparisons_with_constants():
    nodes = np.arange(30, dtype=np.uint32).reshape(-1, 1)
    rules = [(("Mid", ["x"]), [("N", ["x"]), (">=", "x", 10), ("<", "x", 20), ("!=", "x", 15)])]
    r = run({"N": 1, "Mid": 1}, {"N": nodes}, rules)
    assert r.relations["Mid"][:, 0].tolist() == [x for x in range(10, 20) if x != 15]


def test_common_neighbours_without_self_pairs():
    e = dg.random_graph(30, 120, 5)
    A = np.zeros((30, 30), dtype=np.int64)
    A[e[:, 0], e[:, 1]] = 1
    rules = [(("CN", ["x", "y"]), [("E", ["x", "z"]), ("E", ["y", "z"]), ("!=", "x", "y")])]
    r = run({"E": 2, "CN": 2}, {"E": e}, rules)
    want = (A @ A.T) > 0
    np.fill_diagonal(want, False)
    assert r.relations["CN"].tolist() == np.argwhere(want).tolist()


@pytest.mark.parametrize("n", [2, 5, 12])
def test_unreachable_pairs_on_paths_and_cycles(n):
    r = run(P.UNREACH_RELS, {"E": dg.path_graph(n)}, P.UNREACH)
    assert len(r.relations["Unreach"]) == n * (n + 1) // 2
    c = run(P.UNREACH_RELS, {"E": dg.cycle_graph(n)}, P.UNREACH)
    assert len(c.relations["Unreach"]) == 0


def test_unreachable_pairs_match_an_independent_closure():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    e = dg.random_graph(60, 90, 9)
    n = 60
    g = sp.csr_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    d = csgraph.shortest_path(g, unweighted=True)
    reach = np.isfinite(d) & (d > 0)
    # x reaches itself only through a cycle
    _, lab = csgraph.connected_components(g, directed=True, connection="strong")
    for v in range(n):
        reach[v, v] = bool(((lab == lab[v]).sum() > 1) or g[v, v])
    nodes = np.unique(e)
    want = [[x, y] for x in nodes for y in nodes if not reach[x, y]]
    r = run(P.UNREACH_RELS, {"E": e}, P.UNREACH)
    assert r.relations["Unreach"].tolist() == want
    # the negated relation is complete first: Reach's stratum precedes Unreach's
    names = [s for s, _ in r.strata]
    assert names.index(["Reach"]) < names.index(["Unreach"])


def test_negated_atom_with_a_constant():
    e = dg.random_graph(20, 60, 3)
    rules = [(("N", ["y"]), [("E", ["x", "y"])]),
             (("NotFrom0", ["y"]), [("N", ["y"]), ("not", ("E", [0, "y"]))])]
    r = run({"E": 2, "N": 1, "NotFrom0": 1}, {"E": e}, rules)
    from0 = set(e[e[:, 0] == 0][:, 1].tolist())
    assert r.relations["NotFrom0"][:, 0].tolist() == sorted(set(e[:, 1].tolist()) - from0)


def test_unstratifiable_and_unsafe_programs_are_rejected():
    nodes = np.arange(4, dtype=np.uint32).reshape(-1, 1)
    rels = {"N": 1, "P": 1, "Q": 1}
    cyc = [(("P", ["x"]), [("N", ["x"]), ("not", ("Q", ["x"]))]),
           (("Q", ["x"]), [("N", ["x"]), ("not", ("P", ["x"]))])]
    with pytest.raises(oracle.OracleError, match="stratifiable"):
        run(rels, {"N": nodes}, cyc)
    with pytest.raises(oracle.OracleError, match="not bound"):
        run(rels, {"N": nodes}, [(("P", ["x"]), [("N", ["x"]), ("not", ("Q", ["y"]))])])
    with pytest.raises(oracle.OracleError, match="not bound"):
        run(rels, {"N": nodes}, [(("P", ["x"]), [("N", ["x"]), ("<", "x", "y")])])
    with pytest.raises(oracle.OracleError, match="undefined for negation"):
        run(rels, {"N": nodes}, [(("P", ["x"]), [("N", ["x"]), ("not", ("Q", ["x"]))])], "naive_global")


def _random_filtered_program(rng):
    """Relations R0..: EDB first; each IDB relation's rules negate only relations of lower
    index (stratifiable by construction) and add random comparisons."""
    nrel = int(rng.integers(3, 6))
    arity = {f"R{i}": int(rng.integers(1, 3)) for i in range(nrel)}
    names = list(arity)
    n_edb = int(rng.integers(1, nrel - 1))
    D = int(rng.integers(2, 6))
    facts = {r: rng.integers(0, D, size=(int(rng.integers(0, 10)), arity[r])).astype(np.uint32)
             for r in names[:n_edb]}
    rules = []
    for hi in range(n_edb, nrel):
        head = names[hi]
        for _ in range(int(rng.integers(1, 3))):
            nv = int(rng.integers(1, 4))
            vs = [f"v{i}" for i in range(nv)]
            body = []
            for _ in range(int(rng.integers(1, 3))):
                rel = names[int(rng.integers(0, hi + 1))]        # positive: lower or itself
                body.append((rel, [vs[int(rng.integers(0, nv))] for _ in range(arity[rel])]))
            bound = sorted({t for _, ts in body for t in ts})
            for _ in range(int(rng.integers(0, 2))):
                rel = names[int(rng.integers(0, hi))]            # negated: strictly lower
                body.append(("not", (rel, [bound[int(rng.integers(0, len(bound)))] for _ in range(arity[rel])])))
            for _ in range(int(rng.integers(0, 3))):
                op = ["<", "<=", ">", ">=", "!="][int(rng.integers(0, 5))]
                a = bound[int(rng.integers(0, len(bound)))]
                b = bound[int(rng.integers(0, len(bound)))] if rng.random() < 0.7 else int(rng.integers(0, D))
                body.append((op, a, b))
            rules.append(((head, [bound[int(rng.integers(0, len(bound)))] for _ in range(arity[head])]), body))
    return arity, facts, rules


@pytest.mark.parametrize("chunk", range(3))
def test_filtered_programs_match_brute_force(chunk):
    rng = np.random.default_rng(4321 + chunk)
    checked = 0
    for _ in range(300):
        arity, facts, rules = _random_filtered_program(rng)
        semi = run(arity, facts, rules)
        strat = run(arity, facts, rules, "naive_strata")
        for name in arity:
            assert np.array_equal(semi.relations[name], strat.relations[name]), (rules, name)
        checked += 1
    assert checked == 300
