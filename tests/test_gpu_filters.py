"""Comparisons and stratified negation on the GPU (dl_rule_add_ex) against the oracle:
oriented cliques under several variable orders and launch shapes, count-sink digests,
constants, negated atoms of one to three columns, random stratifiable programs, the batched
form, and the unstratifiable case."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


def check(rels, facts, rules, sinks=None, **cfg):
    got, strata, stats = pkg.run_program(rels, facts, rules, sinks, **cfg)
    ref = oracle.evaluate(rels, facts, rules)
    for name in rels:
        if (sinks or {}).get(name) == pkg.DL_SINK_COUNT:
            assert got[name] == oracle.tuple_digest(ref.relations[name]), name
        else:
            assert np.array_equal(got[name], ref.relations[name]), name
    assert sorted(strata) == sorted(ref.strata)
    return got, ref


def reorder(rules, order):
    return [(h, b, order) for h, b, _ in rules]


@pytest.mark.parametrize("order", [["x", "y", "z"], ["z", "y", "x"], ["y", "x", "z"]])
def test_oriented_triangles(order):
    e = dg.rmat_edges(1 << 10, 12000, 2101, symmetric=True)
    got, ref = check({"E": 2, "TriLt": 3}, {"E": e}, reorder(P.TRI_LT, order))
    assert len(got["TriLt"]) > 0
    assert all(a < b < c for a, b, c in got["TriLt"][:1000].tolist())


@pytest.mark.parametrize("cfg", [{}, {"flags": pkg.DL_FLAG_NAIVE_ROOTS}, {"tile_units": 64}, {"hub_rows": 8}])
def test_oriented_four_cliques(cfg):
    e = dg.rmat_edges(1 << 9, 8000, 2102, symmetric=True)
    got, ref = check({"E": 2, "Q4Lt": 4}, {"E": e}, P.Q4_LT, **cfg)
    sym = oracle.evaluate({"E": 2, "Q4": 4}, {"E": e}, P.Q4)
    assert 24 * len(got["Q4Lt"]) == len(sym.relations["Q4"])


def test_oriented_cliques_count_sink():
    e = dg.rmat_edges(1 << 10, 12000, 2103, symmetric=True)
    check({"E": 2, "Q4Lt": 4}, {"E": e}, P.Q4_LT, {"Q4Lt": pkg.DL_SINK_COUNT})


def test_comparisons_with_constants_and_all_operators():
    e = dg.random_graph(200, 3000, 2104)
    rules = [
        (("A", ["x", "y"]), [("E", ["x", "y"]), (">=", "x", 50), ("<", "y", 120), ("!=", "x", 77)], ["x", "y"]),
        (("B", ["x", "y"]), [("E", ["x", "y"]), ("<=", "y", "x")], ["y", "x"]),
        (("C", ["x", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("!=", "x", "z"), (">", "z", "y")], ["x", "y", "z"]),
        (("D", ["x"]), [("E", ["x", "y"]), ("<", 5, 3)], ["x", "y"]),          # never holds
        (("F", ["x"]), [("E", ["x", "y"]), ("<=", "x", "x")], ["x", "y"]),     # always holds
    ]
    got, _ = check({"E": 2, "A": 2, "B": 2, "C": 2, "D": 1, "F": 1}, {"E": e}, rules)
    assert len(got["A"]) and len(got["B"]) and len(got["C"]) and not len(got["D"]) and len(got["F"])


def test_negation_unreachable_pairs():
    for e in (dg.path_graph(40), dg.cycle_graph(30), dg.rmat_edges(400, 900, 2105)):
        got, _ = check(P.UNREACH_RELS, {"E": e}, P.UNREACH)


def test_negated_atoms_of_one_two_and_three_columns():
    e = dg.rmat_edges(1 << 9, 5000, 2106, symmetric=True)
    rules = [
        (("Tri", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"])], ["x", "y", "z"]),
        (("Hub", ["x"]), [("E", ["x", "y"]), ("<", "y", 20)], ["x", "y"]),
        # open wedges: a path x-y-z whose ends are not adjacent
        (("Open", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("!=", "x", "z"),
                                     ("not", ("E", ["x", "z"]))], ["y", "x", "z"]),
        # wedges closed into no triangle through a hub: three-column negation
        (("W", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["z", "x"]),
                                  ("not", ("Tri", ["z", "y", "x"])), ("not", ("Hub", ["y"]))], ["x", "y", "z"]),
    ]
    got, ref = check({"E": 2, "Tri": 3, "Hub": 1, "Open": 3, "W": 3}, {"E": e}, rules)
    assert len(got["Open"]) > 0


def _random_filtered_gpu_program(rng):
    nrel = int(rng.integers(3, 6))
    arity = {f"R{i}": int(rng.integers(1, 3)) for i in range(nrel)}
    names = list(arity)
    n_edb = int(rng.integers(1, nrel - 1))
    D = int(rng.integers(2, 7))
    facts = {r: rng.integers(0, D, size=(int(rng.integers(0, 14)), arity[r])).astype(np.uint32) for r in names[:n_edb]}
    rules = []
    for hi in range(n_edb, nrel):
        for _ in range(int(rng.integers(1, 3))):
            nv = int(rng.integers(1, 5))
            pool = [f"v{i}" for i in range(nv)]
            body = []
            for _ in range(int(rng.integers(1, 4))):
                rel = names[int(rng.integers(0, hi + 1))]
                if arity[rel] > nv:
                    continue
                body.append((rel, [str(t) for t in rng.choice(pool, size=arity[rel], replace=False)]))
            if not body:
                continue
            bound = sorted({t for _, ts in body for t in ts})
            for _ in range(int(rng.integers(0, 2))):
                rel = names[int(rng.integers(0, hi))]
                if arity[rel] > len(bound):
                    continue
                body.append(("not", (rel, [str(t) for t in rng.choice(bound, size=arity[rel], replace=False)])))
            for _ in range(int(rng.integers(0, 3))):
                op = ["<", "<=", ">", ">=", "!="][int(rng.integers(0, 5))]
                a = bound[int(rng.integers(0, len(bound)))]
                b = bound[int(rng.integers(0, len(bound)))] if rng.random() < 0.7 else int(rng.integers(0, D))
                body.append((op, a, b))
            head = (names[hi], [bound[int(rng.integers(0, len(bound)))] for _ in range(arity[names[hi]])])
            rules.append((head, body, [str(v) for v in rng.permutation(bound)]))
    return arity, facts, rules


@pytest.mark.parametrize("seed", range(2))
def test_random_filtered_programs(seed):
    rng = np.random.default_rng(2200 + seed)
    done = 0
    for _ in range(60):
        arity, facts, rules = _random_filtered_gpu_program(rng)
        if not rules:
            continue
        check(arity, facts, rules)
        done += 1
    assert done > 40


def test_filters_in_the_batched_form():
    edges = [dg.rmat_edges(300, 1500 + 100 * k, 2300 + k) for k in range(4)]
    outs, rounds, _ = pkg.run_batched(P.UNREACH_RELS, [{"E": e} for e in edges], P.UNREACH)
    for k, e in enumerate(edges):
        ref = oracle.evaluate(P.UNREACH_RELS, {"E": e}, P.UNREACH)
        for name in P.UNREACH_RELS:
            assert np.array_equal(outs[k][name], ref.relations[name]), (k, name)


def test_unstratifiable_program_is_rejected():
    rules = [(("P", ["x"]), [("N", ["x"]), ("not", ("Q", ["x"]))], ["x"]),
             (("Q", ["x"]), [("N", ["x"]), ("not", ("P", ["x"]))], ["x"])]
    with pkg.Engine() as eng:
        pkg.build_program(eng, {"N": 1, "P": 1, "Q": 1}, rules)
        eng.load("N", np.arange(4, dtype=np.uint32).reshape(-1, 1))
        with pytest.raises(pkg.DatalogError) as ex:
            eng.fixpoint()
        assert ex.value.code == pkg.DL_ERR_UNSUPPORTED
    with pkg.Engine() as eng:
        pkg.build_program(eng, {"N": 1, "P": 1, "Q": 1}, [])
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule(("P", ["x"]), [("N", ["x"]), ("not", ("Q", ["y"]))], ["x"])
        assert ex.value.code == pkg.DL_ERR_ARG
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule(("P", ["x"]), [("N", ["x"]), ("not", ("Q", [3]))], ["x"])
        assert ex.value.code == pkg.DL_ERR_UNSUPPORTED
