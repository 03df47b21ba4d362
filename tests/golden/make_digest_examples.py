"""Writes digest_examples.json: the count and order-independent digest of a few tiny row sets,
as the C oracle's count sink computes them (a copy rule Out(..) :- In(..) whose head is a
count sink).  Calls only oracle/.  The tests check the Python definition (oracle.tuple_digest)
against these values, so the two independent implementations of the digest -- C with 64-bit
wrap-around, Python with big integers and explicit masks -- have to agree on them."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

CASES = {
    "one row (0)": [[0]],
    "one row (1, 2)": [[1, 2]],
    "two rows (1, 2), (2, 1)": [[1, 2], [2, 1]],
    "two rows (0, 0, 0), (4294967294, 7, 123456789)": [[0, 0, 0], [4294967294, 7, 123456789]],
}


def sink_digest(rows):
    rows = np.asarray(rows, dtype=np.uint32)
    a = rows.shape[1]
    v = [f"v{i}" for i in range(a)]
    r = oracle.evaluate({"In": a, "Out": a}, {"In": rows}, [(("Out", v), [("In", v)])], sinks=["Out"])
    return list(r.digests["Out"])


def main():
    out = {name: {"rows": rows, "digest": sink_digest(rows)} for name, rows in CASES.items()}
    with open(os.path.join(HERE, "digest_examples.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
