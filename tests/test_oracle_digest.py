"""Pins for the order-independent digest (count, sum mod 2^64, xor of a 64-bit row hash) and
for the oracle's count-sink mode, which the full-size clique checks rest on.

* The mixing function is splitmix64's finaliser; its outputs for the generator seeded with 0
  are published with the reference implementation (Steele, Lea and Flood, OOPSLA 2014; the
  splitmix64.c of the xoshiro family): 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
  0x06C45D188009454F, 0xF88BB8A8724C81EC -- outputs k = 1..4 are mix(k * 0x9E3779B97F4A7C15).
* Two independent implementations of the digest -- the C oracle's count sink (64-bit
  wrap-around) and oracle.tuple_digest (Python big integers and explicit masks) -- agree on
  stored examples (tests/golden/digest_examples.json, written by a script that calls only the
  oracle) and on random relations.
* Properties any correct digest has: row order does not matter, disjoint unions combine,
  and a changed value, a swapped column pair or a missing row changes it.
* The count sink gives the count and digest of the relation the same rule stores, also for
  rules with comparisons (checked as soon as their variables are bound), and it refuses the
  programs for which that would not hold."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mix_is_splitmix64():
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    for k, want in enumerate(published, start=1):
        assert oracle.splitmix64_mix((k * 0x9E3779B97F4A7C15) % (1 << 64)) == want


def test_stored_examples_match_python_definition():
    ex = json.load(open(os.path.join(GOLDEN, "digest_examples.json")))
    assert len(ex) >= 4
    for name, case in ex.items():
        rows = np.asarray(case["rows"], dtype=np.uint32)
        assert list(oracle.tuple_digest(rows)) == case["digest"], name
        if len(rows) == 1:   # one row: sum and xor are its hash
            assert case["digest"][1] == case["digest"][2] == oracle.row_hash(rows[0].tolist())


def test_digest_properties():
    rng = np.random.default_rng(3)
    rows = np.unique(rng.integers(0, 50, size=(300, 3), dtype=np.uint64).astype(np.uint32), axis=0)
    d = oracle.tuple_digest(rows)
    assert d[0] == len(rows)
    assert oracle.tuple_digest(rows[rng.permutation(len(rows))]) == d
    a, b = rows[: len(rows) // 3], rows[len(rows) // 3:]
    assert oracle.combine_digests([oracle.tuple_digest(a), oracle.tuple_digest(b)]) == d
    changed = rows.copy()
    changed[17, 1] += 1000
    assert oracle.tuple_digest(changed)[1:] != d[1:]
    swapped = rows.copy()
    swapped[5, [0, 2]] = swapped[5, [2, 0]]
    if swapped[5, 0] != swapped[5, 2]:
        assert oracle.tuple_digest(swapped)[1:] != d[1:]
    assert oracle.tuple_digest(rows[1:])[1:] != d[1:]
    # column position enters the hash: (1, 2) and (2, 1) differ
    assert oracle.row_hash([1, 2]) != oracle.row_hash([2, 1])


@pytest.mark.parametrize("seed", range(6))
def test_count_sink_equals_stored_relation(seed):
    e = dg.rmat_edges(128, 1200, 500 + seed, symmetric=True)
    rels = {"E": 2, "Tri": 3, "Q4": 4, "TriLt": 3}
    tri_lt = [(("TriLt", ["x", "y", "z"]),
               [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"]), ("<", "x", "y"), ("<", "y", "z")])]
    rules = P.TRI + P.Q4 + tri_lt
    stored = oracle.evaluate(rels, {"E": e}, rules)
    sunk = oracle.evaluate(rels, {"E": e}, rules, sinks=["Tri", "Q4", "TriLt"])
    for name in ("Tri", "Q4", "TriLt"):
        assert sunk.digests[name] == oracle.tuple_digest(stored.relations[name])
        assert len(sunk.relations[name]) == 0
    assert sunk.digests["Tri"][0] == 6 * sunk.digests["TriLt"][0]


def test_count_sink_refuses_programs_it_would_miscount():
    e = dg.rmat_edges(64, 300, 9)
    # a projection: two bindings can give one tuple
    with pytest.raises(oracle.OracleError):
        oracle.evaluate({"E": 2, "S": 1}, {"E": e}, [(("S", ["x"]), [("E", ["x", "y"])])], sinks=["S"])
    # two rules deriving the sink
    two = [(("S", ["x", "y"]), [("E", ["x", "y"])]), (("S", ["y", "x"]), [("E", ["x", "y"])])]
    with pytest.raises(oracle.OracleError):
        oracle.evaluate({"E": 2, "S": 2}, {"E": e}, two, sinks=["S"])
    # read by another rule
    rd = [(("S", ["x", "y"]), [("E", ["x", "y"])]), (("T", ["x", "y"]), [("S", ["x", "y"])])]
    with pytest.raises(oracle.OracleError):
        oracle.evaluate({"E": 2, "S": 2, "T": 2}, {"E": e}, rd, sinks=["S"])
    # facts loaded into it, and the naive modes
    with pytest.raises(oracle.OracleError):
        oracle.evaluate({"E": 2, "S": 2}, {"E": e, "S": e}, [(("S", ["x", "y"]), [("E", ["x", "y"])])], sinks=["S"])
    with pytest.raises(oracle.OracleError):
        oracle.evaluate({"E": 2, "S": 2}, {"E": e}, [(("S", ["x", "y"]), [("E", ["x", "y"])])], mode="naive_strata",
                        sinks=["S"])


def test_planted_digest_mistake_is_caught():
    """A digest that dropped the column index from the row hash would collide on (1, 2) and
    (2, 1); the stored two-row example separates them."""
    def wrong_row_hash(row):
        h = 0x243F6A8885A308D3
        for v in row:
            h = oracle.splitmix64_mix(h ^ ((int(v) + 0x9E3779B97F4A7C15) % (1 << 64)))
        return h
    ex = json.load(open(os.path.join(GOLDEN, "digest_examples.json")))["two rows (1, 2), (2, 1)"]
    hs = [wrong_row_hash(r) for r in ex["rows"]]
    assert [2, sum(hs) % (1 << 64), hs[0] ^ hs[1]] != ex["digest"]
