"""Pins for the oracle: closed forms, brute force, independent library routines and the
paper's worked example.  None of these re-types the oracle's own code: each expected
value comes from mathematics, from a textbook routine in scipy/numpy, or from the
paper's printed example."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import partition
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run(rels, facts, rules, mode="seminaive"):
    return oracle.evaluate(rels, facts, rules, mode)


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 3, 5, 9, 16])
def test_tc_path(n):
    r = run(P.TC_RELS, {"E": dg.path_graph(n)}, P.TC)
    assert len(r.relations["Reach"]) == n * (n - 1) // 2
    assert r.rounds_of("Reach") == n
    i, j = np.triu_indices(n, 1)
    assert np.array_equal(r.relations["Reach"], np.stack([i, j], 1).astype(np.uint32))


@pytest.mark.parametrize("n", [1, 2, 3, 7, 12])
def test_tc_cycle(n):
    e = dg.cycle_graph(n) if n > 1 else np.array([[0, 0]], dtype=np.uint32)
    r = run(P.TC_RELS, {"E": e}, P.TC)
    assert len(r.relations["Reach"]) == n * n
    assert r.rounds_of("Reach") == (n + 1 if n > 1 else 2)


@pytest.mark.parametrize("n", [3, 6, 10])
def test_tc_complete_dag(n):
    r = run(P.TC_RELS, {"E": dg.complete_dag(n)}, P.TC)
    assert len(r.relations["Reach"]) == math.comb(n, 2)
    assert r.rounds_of("Reach") == 2


@pytest.mark.parametrize("n", [3, 4, 7, 10])
def test_cliques_closed_form(n):
    r = run({"E": 2, "Tri": 3, "Q4": 4}, {"E": dg.complete_dag(n)}, P.TRI + P.Q4)
    assert len(r.relations["Tri"]) == math.comb(n, 3)
    assert len(r.relations["Q4"]) == math.comb(n, 4)
    assert r.rounds_of("Tri") == 1 and r.rounds_of("Q4") == 1
    r = run({"E": 2, "Tri": 3, "Q4": 4}, {"E": dg.complete_sym(n)}, P.TRI + P.Q4)
    assert len(r.relations["Tri"]) == n * (n - 1) * (n - 2)
    assert len(r.relations["Q4"]) == n * (n - 1) * (n - 2) * (n - 3)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bipartite_has_no_cliques(seed):
    e = dg.random_bipartite(20, 30, 300, seed)
    r = run({"E": 2, "Tri": 3, "Q4": 4}, {"E": e}, P.TRI + P.Q4)
    assert len(r.relations["Tri"]) == 0 and len(r.relations["Q4"]) == 0


@pytest.mark.parametrize("k", [0, 1, 4, 9])
def test_points_to_assign_chain(k):
    # Assign(v_i, v_{i+1}) copies v_{i+1}'s points-to set into v_i; New(v_k, h0).
    assign = np.array([[i, i + 1] for i in range(k)], dtype=np.uint32).reshape(-1, 2)
    new = np.array([[k, 0]], dtype=np.uint32)
    empty3 = np.zeros((0, 3), dtype=np.uint32)
    r = run(P.POINTS_TO_RELS, {"New": new, "Assign": assign, "Load": empty3, "Store": empty3}, P.POINTS_TO)
    assert len(r.relations["VPT"]) == k + 1
    assert r.rounds_of("VPT") == k + 2
    assert len(r.relations["FPT"]) == 0


def test_points_to_two_heaps_by_hand():
    # p = new h0; q = new h1; p.f = q (Store(p, f, q)); r = p.f (Load(r, p, f)); s = r.
    p, q, r_, s = 0, 1, 2, 3
    h0, h1, f = 0, 1, 7
    facts = {
        "New": np.array([[p, h0], [q, h1]], dtype=np.uint32),
        "Assign": np.array([[s, r_]], dtype=np.uint32),
        "Store": np.array([[p, f, q]], dtype=np.uint32),
        "Load": np.array([[r_, p, f]], dtype=np.uint32),
    }
    res = run(P.POINTS_TO_RELS, facts, P.POINTS_TO)
    # VPT: p->h0, q->h1 (round 1); FPT(h0, f, h1) (round 2); r->h1 (round 3); s->h1 (round 4)
    assert res.relations["VPT"].tolist() == [[p, h0], [q, h1], [r_, h1], [s, h1]]
    assert res.relations["FPT"].tolist() == [[h0, f, h1]]
    assert res.rounds_of("VPT") == 5


def kary_tree(k, depth):
    edges, frontier, nxt = [], [0], 1
    for _ in range(depth):
        new = []
        for u in frontier:
            for _ in range(k):
                edges.append((u, nxt))
                new.append(nxt)
                nxt += 1
        frontier = new
    return np.array(edges, dtype=np.uint32).reshape(-1, 2)


@pytest.mark.parametrize("k,depth", [(2, 1), (2, 4), (3, 3), (1, 5)])
def test_same_generation_on_trees(k, depth):
    # SG holds exactly for pairs at the same depth >= 1.  A pair whose lowest common ancestor
    # is t >= 1 levels up appears in round t (a node paired with itself: t = 1, through its
    # parent), so the last productive round is `depth` when k >= 2 and 1 on a path.
    r = run(P.SG_RELS, {"Edge": kary_tree(k, depth)}, P.SG)
    assert len(r.relations["SG"]) == sum(k ** (2 * d) for d in range(1, depth + 1))
    assert r.rounds_of("SG") == (depth if k >= 2 else 1) + 1


# ------------------------------------------------------- independent routines

def test_reach_equals_graph_reachability():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    n = 600
    e = dg.rmat_edges(n, 3000, 7)
    r = run(P.TC_RELS, {"E": e}, P.TC)
    g = sp.csr_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    dist = csgraph.shortest_path(g, unweighted=True, directed=True)
    reach = np.isfinite(dist)
    np.fill_diagonal(reach, False)
    ncomp, lab = csgraph.connected_components(g, directed=True, connection="strong")
    sizes = np.bincount(lab, minlength=ncomp)
    on_cycle = sizes[lab] > 1
    reach[np.arange(n), np.arange(n)] = on_cycle
    expect = np.argwhere(reach).astype(np.uint32)
    assert np.array_equal(r.relations["Reach"], expect)
    # round count = 1 + the longest shortest path among reachable pairs (plus the empty round)
    finite = dist[np.isfinite(dist)]
    diam = int(finite.max())
    cyc_extra = 0
    if on_cycle.any():
        # (x, x) appears at the length of x's shortest cycle
        succ = [e[e[:, 0] == x, 1] for x in range(n)]
        cyc = [1 + min(dist[s, x] for s in succ[x]) for x in range(n) if on_cycle[x]]
        cyc_extra = int(max(cyc))
    assert r.rounds_of("Reach") == max(diam, cyc_extra) + 1


@pytest.mark.parametrize("seed", [11, 12])
def test_tri_q4_dense_brute_force(seed):
    n = 40
    e = dg.random_graph(n, 500, seed)
    e = dg.unique_rows(np.concatenate([e, e[:, ::-1]]))
    A = np.zeros((n, n), dtype=bool)
    A[e[:, 0], e[:, 1]] = True
    tri = np.argwhere(A[:, :, None] & A[None, :, :] & A[:, None, :]).astype(np.uint32)
    q4 = np.argwhere(A[:, :, None, None] & A[:, None, :, None] & A[:, None, None, :]
                     & A[None, :, :, None] & A[None, :, None, :] & A[None, None, :, :]).astype(np.uint32)
    r = run({"E": 2, "Tri": 3, "Q4": 4}, {"E": e}, P.TRI + P.Q4)
    assert np.array_equal(r.relations["Tri"], tri)
    assert np.array_equal(r.relations["Q4"], q4)
    # invariants: symmetric counts are 6x / 24x the oriented ones; AGM bounds
    eo = e[e[:, 0] < e[:, 1]]
    ro = run({"E": 2, "Tri": 3, "Q4": 4}, {"E": eo}, P.TRI + P.Q4)
    assert len(tri) == 6 * len(ro.relations["Tri"])
    assert len(q4) == 24 * len(ro.relations["Q4"])
    assert len(tri) <= len(e) ** 1.5 and len(q4) <= len(e) ** 2


# ------------------------------------------------ brute-force property test

def _random_program(rng):
    nrel = int(rng.integers(2, 5))
    arity = {f"R{i}": int(rng.integers(1, 4)) for i in range(nrel)}
    names = list(arity)
    n_edb = int(rng.integers(1, nrel))
    edb, idb = names[:n_edb], names[n_edb:]
    D = int(rng.integers(2, 6))
    facts = {}
    for r in edb:
        m = int(rng.integers(0, 12))
        facts[r] = rng.integers(0, D, size=(m, arity[r])).astype(np.uint32)
    rules = []
    for _ in range(int(rng.integers(1, 5))):
        head = idb[int(rng.integers(0, len(idb)))]
        nvars = int(rng.integers(1, 5))
        vars_ = [f"v{i}" for i in range(nvars)]
        body = []
        for _ in range(int(rng.integers(1, 4))):
            rel = names[int(rng.integers(0, nrel))]
            terms = [int(rng.integers(0, D)) if rng.random() < 0.1 else vars_[int(rng.integers(0, nvars))]
                     for _ in range(arity[rel])]
            body.append((rel, terms))
        bvars = sorted({t for _, ts in body for t in ts if isinstance(t, str)})
        if not bvars:
            continue
        hterms = [int(rng.integers(0, D)) if rng.random() < 0.05 else bvars[int(rng.integers(0, len(bvars)))]
                  for _ in range(arity[head])]
        rules.append(((head, hterms), body))
    return arity, facts, rules, set(edb)


def _recursive_strata(rules, strata):
    out = set()
    for rels, _ in strata:
        for (h, _), body in rules:
            if h in rels and any(b in rels for b, _ in body):
                out.add(tuple(rels))
    return out


@pytest.mark.parametrize("chunk", range(4))
def test_seminaive_matches_brute_force(chunk):
    rng = np.random.default_rng(1234 + chunk)
    checked = 0
    for _ in range(600):
        arity, facts, rules, edb = _random_program(rng)
        if not rules:
            continue
        semi = run(arity, facts, rules)
        glob = run(arity, facts, rules, "naive_global")
        strat = run(arity, facts, rules, "naive_strata")
        for name in arity:
            assert np.array_equal(semi.relations[name], glob.relations[name]), (rules, name)
            assert np.array_equal(semi.relations[name], strat.relations[name]), (rules, name)
        rec = _recursive_strata(rules, semi.strata)
        assert [s for s, _ in semi.strata] == [s for s, _ in strat.strata]
        for (rels, r1), (_, r2) in zip(semi.strata, strat.strata):
            if tuple(rels) in rec:
                assert r1 == r2, (rules, rels)
        checked += 1
    assert checked > 500


def test_preloaded_idb_facts_join_round_one():
    # Facts loaded into an IDB relation are part of round 1's delta.
    e = dg.path_graph(5)
    pre = np.array([[10, 0]], dtype=np.uint32)
    r = run(P.TC_RELS, {"E": e, "Reach": pre}, P.TC)
    naive = run(P.TC_RELS, {"E": e, "Reach": pre}, P.TC, "naive_global")
    assert np.array_equal(r.relations["Reach"], naive.relations["Reach"])
    assert [10, 4] in r.relations["Reach"].tolist()


def test_strata_order_and_duplicate_facts():
    e = np.array([[0, 1], [0, 1], [1, 2], [1, 2]], dtype=np.uint32)
    rels = {"E": 2, "Reach": 2, "Tri": 3, "Top": 1}
    rules = P.TC + P.TRI + [(("Top", ["x"]), [("Reach", ["x", "y"]), ("Tri", ["x", "y", "z"])])]
    r = run(rels, {"E": e}, rules)
    assert len(r.relations["E"]) == 2
    assert [s for s, _ in r.strata] == [["Reach"], ["Tri"], ["Top"]]


# -------------------------------------------------- worked example (Figure 2)

def test_worked_example_partition():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_partition.json")))
    C = list(np.cumsum(g["fanout"]))
    assert C == g["prefix_inclusive"] and C[-1] == g["total"]
    assert -(-C[-1] // g["groups"]) == g["slice"]
    got = partition.work_slices(C, g["groups"])
    keys = g["keys"]
    assert [[[keys[k], a, b] for k, a, b in grp] for grp in got] == g["expected_pieces"]
    b_groups = sorted({i for i, grp in enumerate(got) for k, _, _ in grp if keys[k] == "B"})
    assert b_groups == g["prose_checks"]["heavy_key_B_split_across_groups"]


@pytest.mark.parametrize("seed", range(5))
def test_decode_matches_enumeration(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 30))
    d1 = rng.integers(0, 6, size=K)
    d2 = rng.integers(1, 6, size=K)
    W = d1 * d2
    C = list(np.cumsum(W))
    enum = [(k, i1, i2) for k in range(K) for i1 in range(d1[k]) for i2 in range(d2[k])]
    assert [partition.decode_unit(C, list(d2), g) for g in range(int(C[-1]))] == enum
    for p in (1, 2, 3, 7, 64):
        pieces = [(k, a, b) for grp in partition.work_slices(C, p) for k, a, b in grp]
        cover = [(k, u) for k, a, b in pieces for u in range(a, b)]
        assert cover == [(k, u) for k in range(K) for u in range(W[k])]
