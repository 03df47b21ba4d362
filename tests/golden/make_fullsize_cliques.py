"""Writes cliques_rmat<scale>.json: the oracle's exact count and order-independent digest of
the triangle and 4-clique relations of the skewed cyclic workload's graph (symmetrised R-MAT,
a, b, c, d = 0.57, 0.19, 0.19, 0.05, seed 1001, 2^scale nodes, 16 * 2^scale rows):

* TriLt(x,y,z) :- E(x,y), E(y,z), E(x,z), x < y, y < z     (each triangle once)
* Q4Lt(w,x,y,z) :- the six edges of {w,x,y,z}, w < x < y < z (each 4-clique once)
* Tri(x,y,z) :- E(x,y), E(y,z), E(x,z)                       (every ordering)

The symmetric relations hold 6 (triangles) and 24 (4-cliques) orderings of each oriented
row, so |Tri| = 6 |TriLt| and |Q4| = 24 |Q4Lt| (the orientation invariants of the paper's
Section 2 cliques); the symmetric 4-clique relation is too large for the oracle, so only its
count follows from Q4Lt's.

Calls only the seeded generator and oracle/: every rule is evaluated by the unchanged oracle
as count sinks, restricted to a part of the z values by a unary Root(z) atom, on every host
core (oracle/parallel.py); the parts' rows are disjoint and cover the whole relation, so
their counts and digests combine into the relation's.  Body atoms are listed so that the
oracle's left-deep plan starts from z, the largest vertex id of an oriented row (R-MAT puts
its hubs at the low ids, so z is usually the lighter end).  About an hour on 8 cores at
scale 20.

    python tests/golden/make_fullsize_cliques.py [--scale 20] [--processes N]
"""
import argparse
import json
import os
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle.parallel import run_rooted  # noqa: E402
from paper_2604_20073_gb300 import datagen as dg  # noqa: E402

RELS = {"E": 2, "Root": 1, "TriLt": 3, "Q4Lt": 4, "Tri": 3}
TRI_LT = (("TriLt", ["x", "y", "z"]),
          [("Root", ["z"]), ("E", ["y", "z"]), ("<", "y", "z"), ("E", ["x", "z"]), ("<", "x", "y"),
           ("E", ["x", "y"])])
Q4_LT = (("Q4Lt", ["w", "x", "y", "z"]),
         [("Root", ["z"]), ("E", ["y", "z"]), ("<", "y", "z"), ("E", ["x", "z"]), ("<", "x", "y"),
          ("E", ["x", "y"]), ("E", ["w", "z"]), ("<", "w", "x"), ("E", ["w", "x"]), ("E", ["w", "y"])])
TRI = (("Tri", ["x", "y", "z"]), [("Root", ["z"]), ("E", ["y", "z"]), ("E", ["x", "z"]), ("E", ["x", "y"])])


def golden_path(scale: int) -> str:
    return os.path.join(HERE, f"cliques_rmat{scale}.json")


def compute(scale: int, processes: int, nparts: int, rules=(TRI_LT, Q4_LT, TRI), log=print) -> dict:
    n = 1 << scale
    e = dg.rmat_edges(n, 16 * n, 1001, symmetric=True)
    deg = np.bincount(e[:, 1].astype(np.int64), minlength=n).astype(np.float64)
    roots = np.arange(n, dtype=np.uint32)
    out = {"graph": f"rmat_edges({n}, {16 * n}, 1001, symmetric=True)", "rows_E": int(len(e)),
           "how": "oracle count sinks over Root(z) parts, combined (count, sum mod 2^64, xor)"}
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "E.npy")
        np.save(path, e)
        for rule in rules:
            name = rule[0][0]
            t0 = time.time()
            run = run_rooted({"E": path}, RELS, [rule], roots, processes, timeout=24 * 3600.0,
                             sinks=(name,), nparts=nparts, weight=deg * deg)
            c, s, x = run.digests[name]
            out[name] = {"count": c, "sum": s, "xor": x, "seconds": round(time.time() - t0, 1)}
            log(f"{name}: {c} rows in {time.time() - t0:.0f} s")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--processes", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--parts", type=int, default=0, help="root parts (default: 8 per process)")
    a = ap.parse_args()
    out = compute(a.scale, a.processes, a.parts or 8 * a.processes)
    out["command"] = f"python tests/golden/make_fullsize_cliques.py --scale {a.scale}"
    with open(golden_path(a.scale), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
