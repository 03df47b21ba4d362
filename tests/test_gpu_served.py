"""Serving loop: a mix of requests (TC + Tri, 4-clique counts, points-to) submitted together
to a server with few slots and a small memory budget (so requests queue, are admitted as
slots and memory free up, and run concurrently on separate streams).  Every result equals
the oracle's and the same request evaluated alone; a request that outgrows its share fails
alone with DL_ERR_CAPACITY, or, with grow_retries, is evaluated again with a doubled share."""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu

SINK = {"Q4": pkg.DL_SINK_COUNT}


def make_requests(k, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(k):
        kind = rng.choice(["tc", "q4", "pt"], p=[0.6, 0.3, 0.1])
        s = dg.instance_seed(seed, i)
        if kind == "tc":
            m = int(np.exp(rng.uniform(np.log(200), np.log(6000))))
            e = dg.rmat_edges(max(2, m // 8), m, s)
            reqs.append(("tc", P.TC_TRI_RELS, {"E": e}, P.TC_TRI, None))
        elif kind == "q4":
            m = int(np.exp(rng.uniform(np.log(2000), np.log(20000))))
            e = dg.rmat_edges(max(16, m // 16), m, s, symmetric=True)
            reqs.append(("q4", P.Q4_RELS, {"E": e}, P.Q4, SINK))
        else:
            f = {k2: v for k2, v in dg.points_to_facts(1 / 8192, s & 0xFFFF).items() if k2 != "domains"}
            reqs.append(("pt", P.POINTS_TO_RELS, f, P.POINTS_TO, None))
    return reqs


def test_mixed_requests_match_alone_and_oracle():
    reqs = make_requests(24, 4004)
    with pkg.Server(budget_bytes=3 << 30, max_slots=4, default_share=512 << 20) as srv:
        tickets = [None] * len(reqs)

        def submit(lo, hi):      # two client threads submitting concurrently
            for i in range(lo, hi):
                kind, rels, facts, rules, sinks = reqs[i]
                tickets[i] = srv.submit(rels, facts, rules, sinks)
        th = [threading.Thread(target=submit, args=(0, 12)), threading.Thread(target=submit, args=(12, 24))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        # handle requests in completion order: a finished request keeps its memory share until
        # released, so waiting in submission order could stall admission
        left = set(range(len(reqs)))
        deadline = time.time() + 600
        order = []
        max_running = 0
        while left:
            assert time.time() < deadline, srv.stats()
            max_running = max(max_running, srv.stats()["running"])
            ready = [i for i in sorted(left) if srv.poll(tickets[i])[0] == pkg.DL_REQ_DONE]
            if not ready:
                time.sleep(0.005)
                continue
            i = ready[0]
            left.discard(i)
            order.append(i)
            kind, rels, facts, rules, sinks = reqs[i]
            assert srv.wait(tickets[i]) == pkg.DL_OK
            eng = srv.result(tickets[i])
            alone, alone_strata, _ = pkg.run_program(rels, facts, rules, sinks)
            ref = oracle.evaluate(rels, facts, rules)
            for name in rels:
                if (sinks or {}).get(name) == pkg.DL_SINK_COUNT:
                    got = eng.digest(name)
                    assert got == alone[name] == oracle.tuple_digest(ref.relations[name])
                else:
                    got = eng.fetch(name)
                    assert np.array_equal(got, alone[name]) and np.array_equal(got, ref.relations[name])
            assert sorted(eng.strata()) == sorted(alone_strata) == sorted(ref.strata)
            srv.release(tickets[i])
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["peak_reserved_bytes"] <= 3 << 30
        # continuous batching, not a queue alone: several requests held memory at once and
        # several were evaluated at the same time on their slots' streams
        assert st["peak_reserved_bytes"] >= 2 * (512 << 20)
        assert max_running >= 2
        assert st["reserved_bytes"] == 0


def test_over_share_request_fails_alone():
    e = dg.rmat_edges(4096, 32768, 1000)
    small = dg.rmat_edges(256, 2000, 3)
    with pkg.Server(budget_bytes=2 << 30, max_slots=2) as srv:
        big = srv.submit(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, share=8 << 20)
        ok = srv.submit(P.TC_TRI_RELS, {"E": small}, P.TC_TRI, share=256 << 20)
        assert srv.wait(big) == pkg.DL_ERR_CAPACITY
        assert srv.wait(ok) == pkg.DL_OK
        ref = oracle.evaluate(P.TC_TRI_RELS, {"E": small}, P.TC_TRI)
        eng = srv.result(ok)
        assert np.array_equal(eng.fetch("Reach"), ref.relations["Reach"])
        srv.release(big)
        srv.release(ok)
        with pytest.raises(pkg.DatalogError):
            srv.submit(P.TC_TRI_RELS, {"E": small}, P.TC_TRI, share=4 << 30)


def test_share_grows_until_the_request_fits():
    """Final sizes unknown up front: with grow_retries the request that fails at an 8 MiB share
    is evaluated again with twice the share until it fits, while another request runs; both
    equal the oracle, and the doubled shares are returned to the budget."""
    e = dg.rmat_edges(4096, 32768, 1000)
    small = dg.rmat_edges(256, 2000, 3)
    with pkg.Server(budget_bytes=2 << 30, max_slots=2, grow_retries=12) as srv:
        big = srv.submit(P.TC_TRI_RELS, {"E": e}, P.TC_TRI, share=8 << 20)
        ok = srv.submit(P.TC_TRI_RELS, {"E": small}, P.TC_TRI, share=256 << 20)
        assert srv.wait(big) == pkg.DL_OK
        assert srv.wait(ok) == pkg.DL_OK
        for t, facts in ((big, {"E": e}), (ok, {"E": small})):
            ref = oracle.evaluate(P.TC_TRI_RELS, facts, P.TC_TRI)
            eng = srv.result(t)
            for name in P.TC_TRI_RELS:
                assert np.array_equal(eng.fetch(name), ref.relations[name]), name
            assert sorted(eng.strata()) == sorted(ref.strata)
        st = srv.stats()
        assert st["regrown"] >= 1 and st["failed"] == 0 and st["completed"] == 2
        srv.release(big)
        srv.release(ok)
        assert srv.stats()["reserved_bytes"] == 0


def test_served_rules_with_negation_and_comparisons():
    """Requests carry negated atoms and comparisons (dl_rule_spec.neg / .cmps)."""
    tri_lt = [(("TriLt", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"]),
                                           ("<", "x", "y"), ("<", "y", "z")], ["x", "y", "z"])]
    unreach = P.TC + [(("V", ["x"]), [("E", ["x", "y"])], ["x", "y"]),
                      (("NR", ["x", "y"]), [("V", ["x"]), ("V", ["y"]), ("not", ("Reach", ["x", "y"])),
                                            ("!=", "x", "y")], ["x", "y"])]
    cases = [({"E": 2, "TriLt": 3}, {"E": dg.rmat_edges(300, 2500, 5, symmetric=True)}, tri_lt),
             ({"E": 2, "Reach": 2, "V": 1, "NR": 2}, {"E": dg.rmat_edges(200, 600, 6)}, unreach)]
    with pkg.Server(budget_bytes=2 << 30, max_slots=2) as srv:
        tickets = [srv.submit(rels, facts, rules) for rels, facts, rules in cases]
        for (rels, facts, rules), t in zip(cases, tickets):
            assert srv.wait(t) == pkg.DL_OK
            eng = srv.result(t)
            ref = oracle.evaluate(rels, facts, rules)
            for name in rels:
                assert np.array_equal(eng.fetch(name), ref.relations[name]), name
            srv.release(t)
