"""GPU path vs the oracle: identical sorted, deduplicated tuple sets per relation and identical
round counts per stratum (integer work: bit-exact).  Every case runs through the C ABI."""
import math

import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


def gpu(rels, facts, rules, sinks=None, **cfg):
    return pkg.run_program(rels, facts, rules, sinks, **cfg)


def check(rels, facts, rules, **cfg):
    got, strata, stats = gpu(rels, facts, rules, **cfg)
    ref = oracle.evaluate(rels, facts, rules)
    for name in rels:
        assert got[name].shape == ref.relations[name].shape, (name, got[name].shape, ref.relations[name].shape)
        assert np.array_equal(got[name], ref.relations[name]), name
    assert sorted(strata) == sorted(ref.strata)
    return got, strata, stats


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 3, 17, 64, 300])
def test_tc_path(n):
    got, strata, _ = check(P.TC_RELS, {"E": dg.path_graph(n)}, P.TC)
    assert len(got["Reach"]) == n * (n - 1) // 2
    assert strata == [(["Reach"], n)]


@pytest.mark.parametrize("n", [2, 5, 40])
def test_tc_cycle(n):
    got, strata, _ = check(P.TC_RELS, {"E": dg.cycle_graph(n)}, P.TC)
    assert len(got["Reach"]) == n * n and strata == [(["Reach"], n + 1)]


@pytest.mark.parametrize("n", [3, 8, 30])
def test_complete_graph_cliques(n):
    rels = {"E": 2, "Tri": 3, "Q4": 4}
    got, _, _ = check(rels, {"E": dg.complete_dag(n)}, P.TRI + P.Q4)
    assert len(got["Tri"]) == math.comb(n, 3) and len(got["Q4"]) == math.comb(n, 4)
    got, _, _ = check(rels, {"E": dg.complete_sym(n)}, P.TRI + P.Q4)
    assert len(got["Tri"]) == n * (n - 1) * (n - 2)
    assert len(got["Q4"]) == n * (n - 1) * (n - 2) * (n - 3)


def test_bipartite_no_cliques():
    e = dg.random_bipartite(200, 300, 5000, 3)
    got, _, _ = check({"E": 2, "Tri": 3, "Q4": 4}, {"E": e}, P.TRI + P.Q4)
    assert len(got["Tri"]) == 0 and len(got["Q4"]) == 0


def test_points_to_chain():
    k = 25
    assign = np.array([[i, i + 1] for i in range(k)], dtype=np.uint32)
    new = np.array([[k, 0], [k, 3]], dtype=np.uint32)
    e3 = np.zeros((0, 3), dtype=np.uint32)
    got, strata, _ = check(P.POINTS_TO_RELS, {"New": new, "Assign": assign, "Load": e3, "Store": e3}, P.POINTS_TO)
    assert len(got["VPT"]) == 2 * (k + 1)
    assert dict((tuple(r), c) for r, c in strata)[("FPT", "VPT")] == k + 2


# ---------------------------------------------------------------- workloads

def test_tc_tri_small_rmat():
    e = dg.rmat_edges(4096, 32768, 1000)
    got, strata, stats = check(P.TC_TRI_RELS, {"E": e}, P.TC_TRI)
    assert stats["kernel_launches"] > 0 and stats["join_rows"] > 0


@pytest.mark.parametrize("scale,m", [(9, 6000), (11, 40000)])
def test_skewed_cliques(scale, m):
    e = dg.rmat_edges(1 << scale, m, 2000 + scale, symmetric=True)
    rels = {"E": 2, "Tri": 3, "Q4": 4}
    ref = oracle.evaluate(rels, {"E": e}, P.TRI + P.Q4)
    for cfg in [dict(), dict(flags=pkg.DL_FLAG_NAIVE_ROOTS), dict(tile_units=64), dict(tile_units=100003)]:
        got, strata, _ = gpu(rels, {"E": e}, P.TRI + P.Q4, **cfg)
        for name in ("Tri", "Q4"):
            assert np.array_equal(got[name], ref.relations[name]), (name, cfg)


@pytest.mark.parametrize("f", [1 / 2048, 1 / 512])
def test_points_to_synthetic(f):
    facts = dg.points_to_facts(f, 1002)
    facts = {k: v for k, v in facts.items() if k != "domains"}
    check(P.POINTS_TO_RELS, facts, P.POINTS_TO)


@pytest.mark.parametrize("chunk_rows", [1, 997, 50000])
def test_chunked_rule_output(chunk_rows):
    # rule outputs larger than chunk_rows are written, deduplicated and anti-joined in chunks
    facts = dg.points_to_facts(1 / 4096, 1002)
    facts = {k: v for k, v in facts.items() if k != "domains"}
    check(P.POINTS_TO_RELS, facts, P.POINTS_TO, chunk_rows=chunk_rows)
    e = dg.rmat_edges(2048, 16000, 6)
    check(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, chunk_rows=chunk_rows)


@pytest.mark.parametrize("seed", [1, 2])
def test_same_generation(seed):
    e = dg.rmat_edges(1500, 3000, 700 + seed)
    got, strata, _ = check(P.SG_RELS, {"Edge": e}, P.SG)
    assert len(got["SG"]) > len(e)


def test_same_generation_tree_closed_form():
    from tests.test_oracle_pins import kary_tree
    got, strata, _ = check(P.SG_RELS, {"Edge": kary_tree(3, 5)}, P.SG)
    assert len(got["SG"]) == sum(3 ** (2 * d) for d in range(1, 6)) and strata == [(["SG"], 6)]


# ------------------------------------------------------- metamorphic checks

@pytest.mark.parametrize("order", [["x", "y", "z"], ["y", "x", "z"], ["z", "y", "x"], ["y", "z", "x"]])
def test_variable_order_does_not_change_results(order):
    e = dg.rmat_edges(1024, 8000, 77)
    tc = [P.TC[0], (P.TC[1][0], P.TC[1][1], order)]
    tri = [(P.TRI[0][0], P.TRI[0][1], order)]
    check(P.TC_TRI_RELS, {"E": e}, tc + tri)


# 5-clique; atoms listed so that the oracle's left-deep plan closes each triangle early
Q5 = [(("Q5", ["a", "b", "c", "d", "e"]),
       [("E", [u, v]) for j, v in enumerate("abcde") for u in "abcde"[:j]], ["a", "b", "c", "d", "e"])]
# same rule on a directed graph, where deferring a depth-0 check changes which prefixes survive
DQ4 = [(("DQ4", ["w", "x", "y", "z"]), P.Q4[0][1], ["w", "x", "y", "z"])]


@pytest.mark.parametrize("order", [["w", "x", "y", "z"], ["x", "w", "z", "y"], ["z", "y", "x", "w"]])
def test_clique_orders_and_candidate_reuse(order):
    e = dg.rmat_edges(1 << 8, 3000, 404, symmetric=True)
    rels = {"E": 2, "Q4": 4, "Q5": 5}
    q4 = [(P.Q4[0][0], P.Q4[0][1], order)]
    got = check(rels, {"E": e}, q4 + Q5)[0]
    assert len(got["Q5"]) > 0 and len(got["Q4"]) > 0


def test_directed_cliques_with_deferred_checks():
    e = dg.rmat_edges(1 << 9, 6000, 405)
    got = check({"E": 2, "DQ4": 4, "Tri": 3}, {"E": e}, DQ4 + P.TRI)[0]
    assert len(got["DQ4"]) > 0


@pytest.mark.parametrize("hub_rows", [1, 16, 300])
def test_heavy_key_bitmaps(hub_rows):
    # probes into keys with >= hub_rows rows test a bitmap of the key's values; the results
    # must not depend on which keys have one (hub_rows = UINT32_MAX: none)
    e = dg.hub_graph(3, 420, 1500, 91)
    rels = {"E": 2, "Tri": 3, "Q4": 4, "Q5": 5}
    rules = P.TRI + P.Q4 + Q5
    ref = oracle.evaluate(rels, {"E": e}, rules)
    d = dg.rmat_edges(1 << 9, 6000, 406)
    dref = oracle.evaluate({"E": 2, "DQ4": 4}, {"E": d}, DQ4)
    for order in (["w", "x", "y", "z"], ["z", "y", "x", "w"]):
        q4 = [(P.Q4[0][0], P.Q4[0][1], order)]
        got, _, st = gpu(rels, {"E": e}, P.TRI + q4 + Q5, hub_rows=hub_rows)
        assert st["hub_keys"] > 0
        for name in ("Tri", "Q4", "Q5"):
            assert np.array_equal(got[name], ref.relations[name]), (name, order)
    got, _, st = gpu({"E": 2, "DQ4": 4}, {"E": d}, DQ4, hub_rows=hub_rows, tile_units=64)
    assert np.array_equal(got["DQ4"], dref.relations["DQ4"])
    got, _, st = gpu(rels, {"E": e}, rules, hub_rows=0xFFFFFFFF)
    assert st["hub_keys"] == 0 and np.array_equal(got["Q4"], ref.relations["Q4"])


def test_heavy_key_bitmaps_in_recursive_and_random_programs():
    # a stratum reading relations of lower strata gets bitmaps for them; its own relations
    # (which change every round) get none
    rng = np.random.default_rng(77)
    done = 0
    for _ in range(40):
        arity, facts, rules = _random_gpu_program(rng)
        if not rules:
            continue
        got, strata, _ = gpu(arity, facts, rules, hub_rows=2)
        ref = oracle.evaluate(arity, facts, rules)
        for name in arity:
            assert np.array_equal(got[name], ref.relations[name]), name
        assert sorted(strata) == sorted(ref.strata)
        done += 1
    assert done > 25
    e = dg.hub_graph(2, 300, 600, 5)
    got, _, st = gpu(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, hub_rows=8)
    ref = oracle.evaluate(P.TC_TRI_RELS, {"E": e}, P.TC_TRI)
    assert st["hub_keys"] > 0
    for name in P.TC_TRI_RELS:
        assert np.array_equal(got[name], ref.relations[name]), name


def test_rerun_is_deterministic_and_debug_checks_pass():
    e = dg.rmat_edges(2048, 16000, 5)
    a = gpu(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, flags=pkg.DL_FLAG_DEBUG_CHECKS)
    b = gpu(P.TC_TRI_RELS, {"E": e}, P.TC_TRI)
    for name in P.TC_TRI_RELS:
        assert np.array_equal(a[0][name], b[0][name])
    assert a[1] == b[1]


def test_torch_allocator_backing():
    e = dg.rmat_edges(1024, 6000, 9)
    check(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, use_torch_allocator=True)


# ------------------------------------------------------ random programs

def _random_gpu_program(rng):
    nrel = int(rng.integers(2, 5))
    arity = {f"R{i}": int(rng.integers(1, 4)) for i in range(nrel)}
    names = list(arity)
    n_edb = int(rng.integers(1, nrel))
    edb, idb = names[:n_edb], names[n_edb:]
    D = int(rng.integers(2, 7))
    facts = {r: rng.integers(0, D, size=(int(rng.integers(0, 15)), arity[r])).astype(np.uint32) for r in edb}
    rules = []
    for _ in range(int(rng.integers(1, 5))):
        head = idb[int(rng.integers(0, len(idb)))]
        nvars = int(rng.integers(1, 6))
        pool = [f"v{i}" for i in range(nvars)]
        body = []
        for _ in range(int(rng.integers(1, 4))):
            rel = names[int(rng.integers(0, nrel))]
            if arity[rel] > nvars:
                continue
            terms = list(rng.choice(pool, size=arity[rel], replace=False))
            body.append((rel, [str(t) for t in terms]))
        bvars = sorted({t for _, ts in body for t in ts})
        if not body:
            continue
        hterms = [int(rng.integers(0, D)) if rng.random() < 0.05 else bvars[int(rng.integers(0, len(bvars)))]
                  for _ in range(arity[head])]
        order = [str(v) for v in rng.permutation(bvars)]
        rules.append(((head, hterms), body, order))
    return arity, facts, rules


@pytest.mark.parametrize("seed", range(3))
def test_random_programs(seed):
    rng = np.random.default_rng(500 + seed)
    done = 0
    for _ in range(80):
        arity, facts, rules = _random_gpu_program(rng)
        if not rules:
            continue
        check(arity, facts, rules)
        done += 1
    assert done > 50


# ------------------------------------------------------------ sinks & edges

def test_count_sink_matches_oracle_digest():
    e = dg.rmat_edges(1 << 10, 12000, 31, symmetric=True)
    rels = {"E": 2, "Q4": 4}
    got, _, stats = gpu(rels, {"E": e}, P.Q4, sinks={"Q4": pkg.DL_SINK_COUNT})
    ref = oracle.evaluate(rels, {"E": e}, P.Q4)
    assert got["Q4"] == oracle.tuple_digest(ref.relations["Q4"])
    assert stats["count_rows"] == len(ref.relations["Q4"])


def test_empty_and_tiny_inputs():
    e0 = np.zeros((0, 2), dtype=np.uint32)
    got, strata, _ = gpu(P.TC_TRI_RELS, {"E": e0}, P.TC_TRI)
    assert len(got["Reach"]) == 0 and len(got["Tri"]) == 0
    assert sorted(strata) == [(["Reach"], 1), (["Tri"], 1)]
    check(P.TC_TRI_RELS, {"E": np.array([[5, 5]], dtype=np.uint32)}, P.TC_TRI)
    check(P.TC_TRI_RELS, {"E": np.array([[0, 4294967294], [4294967294, 0]], dtype=np.uint32)}, P.TC_TRI)


def test_duplicate_and_preloaded_facts():
    e = np.array([[0, 1], [0, 1], [1, 2], [2, 0], [1, 2]], dtype=np.uint32)
    pre = np.array([[9, 0], [9, 0]], dtype=np.uint32)
    check(P.TC_RELS, {"E": e, "Reach": pre}, P.TC)


# Body constants and a variable repeated within an atom (the oracle evaluates them as filters;
# the GPU path rewrites each into a fresh variable equal to the constant or to the first
# occurrence): selections, self loops, reachability from a constant source, a triangle
# through a fixed vertex, and a constant in a recursive rule.
BODY_TERMS = [
    (("Sel", ["x"]), [("E", ["x", 5])], ["x"]),
    (("Loop", ["x"]), [("E", ["x", "x"])], ["x"]),
    (("LoopOut", ["x", "y"]), [("E", ["x", "x"]), ("E", ["x", "y"])], ["x", "y"]),
    (("From0", ["y"]), [("E", [0, "y"])], ["y"]),
    (("From0", ["z"]), [("From0", ["y"]), ("E", ["y", "z"])], ["y", "z"]),
    (("Via7", ["y", "z"]), [("E", [7, "y"]), ("E", ["y", "z"]), ("E", [7, "z"])], ["y", "z"]),
    (("Back", ["x"]), [("From0", ["x"]), ("E", ["x", 0]), ("E", ["x", "x"])], ["x"]),
]
BODY_TERMS_RELS = {"E": 2, "Sel": 1, "Loop": 1, "LoopOut": 2, "From0": 1, "Via7": 2, "Back": 1}


@pytest.mark.parametrize("seed", [1, 2])
def test_body_constants_and_repeated_variables(seed):
    e = dg.rmat_edges(200, 1500, 40 + seed)
    loops = np.stack([np.arange(0, 200, 7), np.arange(0, 200, 7)], axis=1).astype(np.uint32)
    e = np.concatenate([e, loops, np.array([[0, 5], [7, 5], [5, 0], [7, 7]], dtype=np.uint32)])
    got, _, _ = check(BODY_TERMS_RELS, {"E": e}, BODY_TERMS)
    assert len(got["Loop"]) > 0 and len(got["Sel"]) > 0 and len(got["From0"]) > 0


def test_errors_are_reported_not_raised_across_the_abi():
    with pkg.Engine() as eng:
        eng.relation("E", 2)
        eng.relation("R", 2)
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule(("R", ["x", "y"]), [("E", ["x", "x"])], ["x"])
        assert ex.value.code == pkg.DL_ERR_ARG
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule(("R", ["x", "y"]), [("E", ["x", "y"])], ["x"])
        assert ex.value.code == pkg.DL_ERR_ARG
        with pytest.raises(pkg.DatalogError) as ex:
            eng.rule(("R", ["x", "q"]), [("E", ["x", "y"])], ["x", "y"])
        assert ex.value.code == pkg.DL_ERR_ARG
        with pytest.raises(pkg.DatalogError) as ex:
            eng.relation("E", 2)
        assert ex.value.code == pkg.DL_ERR_ARG


def test_capacity_error_is_clean():
    e = dg.rmat_edges(4096, 32768, 1000)
    with pkg.Engine(arena_bytes=3 << 20) as eng:
        pkg.build_program(eng, P.TC_TRI_RELS, P.TC_TRI)
        eng.load("E", e)
        with pytest.raises(pkg.DatalogError) as ex:
            eng.fixpoint()
        assert ex.value.code == pkg.DL_ERR_CAPACITY
        assert np.array_equal(eng.fetch("E"), e)
