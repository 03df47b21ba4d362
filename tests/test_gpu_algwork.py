"""The algorithmic work the join reports, checked against a CPU count that does not use the
GPU path, and the heavy-key bitmaps and tile sizes checked not to change any result.

Algorithmic work of a join level (the paper's Section 2 intersection cost): every candidate
of each frontier entry's smallest source.  At the 4-clique rule's last level (order
w < x < y < z) the frontier entries are the triangles (w, x, y) of the symmetric graph, and
the sources of z are the common neighbours of w and x (the entry's siblings) and the
neighbours of y, so the work is sum over triangles of min(|N(w) & N(x)|, |N(y)|).  The
CPU side gets the triangles from the oracle and the rest from numpy."""
import numpy as np
import pytest

import oracle
import paper_2604_20073_gb300 as pkg
from paper_2604_20073_gb300 import datagen as dg
from tests import programs as P

pytestmark = pytest.mark.gpu


def cpu_last_level_work(e, n):
    tri = oracle.evaluate(P.TRI_RELS, {"E": e}, P.TRI).relations["Tri"]     # (w, x, y) rows
    deg = np.bincount(e[:, 0].astype(np.int64), minlength=n)
    key = tri[:, 0].astype(np.int64) * n + tri[:, 1].astype(np.int64)
    _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    common = cnt[inv]                                   # |N(w) & N(x)| for each row's (w, x)
    return int(np.minimum(common, deg[tri[:, 2].astype(np.int64)]).sum()), len(tri)


def test_q4_last_level_work_matches_cpu_count():
    n = 1 << 16
    e = dg.rmat_edges(n, 16 * n, 1001, symmetric=True)
    work, entries = cpu_last_level_work(e, n)
    with pkg.Engine(flags=pkg.DL_FLAG_PROFILE) as eng:
        pkg.build_program(eng, P.Q4_RELS, P.Q4, {"Q4": pkg.DL_SINK_COUNT})
        eng.load("E", e)
        st = eng.fixpoint()
    top = st["top"]
    assert top["kind"] == "join_count"
    assert top["units"] == work and top["entries"] == entries
    # algorithmic bytes: 4 per candidate plus each entry's state (values and sibling run)
    assert top["alg_bytes"] >= 4 * work + 12 * entries
    assert (top["alg_bytes"] - 4 * work) % entries == 0


@pytest.fixture(scope="module")
def hub_case():
    e = dg.hub_graph(3, 2000, 12000, 71)
    rels = {"E": 2, "Tri": 3, "Q4": 4}
    return e, rels, oracle.evaluate(rels, {"E": e}, P.TRI + P.Q4, sinks=["Q4"])


@pytest.mark.parametrize("hub_rows,tile_units", [(0, 0), (0xFFFFFFFF, 0), (16, 0), (0, 4096), (16, 65536)])
def test_probe_structures_and_tiles_do_not_change_results(hub_case, hub_rows, tile_units):
    e, rels, ref = hub_case
    got, strata, st = pkg.run_program(rels, {"E": e}, P.TRI + P.Q4, {"Q4": pkg.DL_SINK_COUNT},
                                      hub_rows=hub_rows, tile_units=tile_units)
    assert np.array_equal(got["Tri"], ref.relations["Tri"])
    assert got["Q4"] == ref.digests["Q4"] and ref.digests["Q4"][0] > 0
    assert (st["hub_keys"] > 0) == (hub_rows != 0xFFFFFFFF)


def test_autotuner_choices_are_cached_and_do_not_change_results(hub_case, tmp_path):
    e, rels, ref = hub_case
    cache = str(tmp_path / "tune.txt")
    flags = pkg.DL_FLAG_AUTOTUNE
    got, _, st = pkg.run_program(rels, {"E": e}, P.TRI + P.Q4, {"Q4": pkg.DL_SINK_COUNT}, flags=flags,
                                 tune_cache=cache)
    assert np.array_equal(got["Tri"], ref.relations["Tri"]) and got["Q4"] == ref.digests["Q4"]
    assert st["tuned_levels"] > 0
    lines = open(cache).read().split("\n")
    assert len([x for x in lines if x.strip()]) == st["tuned_levels"]
    # a second engine reads the choices back: no level is tuned again
    got, _, st = pkg.run_program(rels, {"E": e}, P.TRI + P.Q4, {"Q4": pkg.DL_SINK_COUNT}, flags=flags,
                                 tune_cache=cache)
    assert np.array_equal(got["Tri"], ref.relations["Tri"]) and got["Q4"] == ref.digests["Q4"]
    assert st["tuned_levels"] == 0 and st["tune_hits"] > 0
