"""Writes datagen_digests.json: SHA-256 digests of small outputs of the seeded input
generators, so that a change to a generator (which would silently change every workload and
its measured numbers) shows up as a test failure.  Calls only the generators."""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2604_20073_gb300 import datagen as dg  # noqa: E402

CASES = {
    "rmat_edges(4096, 32768, 1000)": lambda: dg.rmat_edges(4096, 32768, 1000),
    "rmat_edges(1024, 8192, 1001, symmetric=True)": lambda: dg.rmat_edges(1024, 8192, 1001, symmetric=True),
    "points_to_facts(1/4096, 1002)": lambda: dg.points_to_facts(1 / 4096, 1002),
    "call_graph_facts(0.05, 1005)": lambda: dg.call_graph_facts(0.05, 1005),
    "batched_instances(8, 1003, 100, 2000)": lambda: dg.batched_instances(8, 1003, 100, 2000),
    "hub_graph(3, 420, 1500, 91)": lambda: dg.hub_graph(3, 420, 1500, 91),
}


def digest(obj) -> str:
    h = hashlib.sha256()

    def feed(x):
        if isinstance(x, dict):
            for k in sorted(x):
                h.update(str(k).encode())
                feed(x[k])
        elif isinstance(x, (list, tuple)):
            for y in x:
                feed(y)
        elif hasattr(x, "tobytes"):
            h.update(str(x.shape).encode())
            h.update(x.astype("<u4").tobytes())
        else:
            h.update(repr(x).encode())
    feed(obj)
    return h.hexdigest()


if __name__ == "__main__":
    out = {name: digest(fn()) for name, fn in CASES.items()}
    with open(os.path.join(HERE, "datagen_digests.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))
