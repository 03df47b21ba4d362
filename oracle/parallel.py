"""Root-partitioned runs of the oracle on several host cores.

Test and timing infrastructure only (the CPU baseline of the benchmark and the committed
script that writes the full-size golden digests): it splits a set of root values into parts
and evaluates, in separate processes, the same root-restricted program on each part with
the unchanged oracle.  The rows of a root-restricted rule are disjoint across roots, so the
parts' row counts, digest sums and digest xors combine into the whole sample's.  Processes
are started with the spawn method (safe after a CUDA context exists in the parent)."""
from __future__ import annotations

import multiprocessing as mp
import time
from dataclasses import dataclass, field

import numpy as np

_FACTS = None


def _init(paths):
    global _FACTS
    _FACTS = {name: np.load(p) for name, p in paths.items()}


def _ready(_):
    return _FACTS is not None


def _run(job):
    relations, rules, roots, sinks = job
    from oracle import evaluate
    facts = dict(_FACTS)
    facts["Root"] = roots
    r = evaluate(relations, facts, rules, sinks=sinks)
    return {"counts": {name: len(rows) for name, rows in r.relations.items()}, "digests": r.digests,
            "join_s": r.join_seconds}


@dataclass
class RootedRun:
    counts: dict                      # rows per stored relation, summed over the parts
    digests: dict                     # count sinks: (count, sum, xor) of the union of the parts
    wall: float                       # wall seconds of the evaluation (start-up and fact loading excluded)
    join_s: list = field(default_factory=list)   # per part: seconds in the oracle's nested loops


def split_roots(roots: np.ndarray, nparts: int, weight: np.ndarray | None = None) -> list:
    """Deal the roots to nparts parts: heaviest first (by weight, when given), round robin,
    so that hubs are spread over the parts."""
    r = np.asarray(roots, dtype=np.uint32).reshape(-1)
    if weight is not None:
        r = r[np.argsort(-np.asarray(weight, dtype=np.float64).reshape(-1), kind="stable")]
    return [np.sort(r[i::nparts]).reshape(-1, 1) for i in range(nparts) if len(r[i::nparts])]


def run_rooted(fact_paths: dict, relations: dict, rules: list, roots: np.ndarray, processes: int,
               timeout: float = 600.0, sinks: tuple = (), nparts: int | None = None,
               weight: np.ndarray | None = None) -> RootedRun:
    """Evaluate `rules` (which read a unary relation Root) for `roots` split into `nparts`
    parts (default: one per process) on `processes` spawned workers; facts are read by each
    worker from the .npy files in `fact_paths`.  Raises multiprocessing.TimeoutError after
    `timeout` seconds."""
    from oracle import combine_digests
    parts = split_roots(roots, nparts or processes, weight)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(processes, len(parts)), initializer=_init, initargs=(fact_paths,)) as pool:
        assert all(pool.map_async(_ready, range(min(processes, len(parts))), chunksize=1).get(timeout))
        t0 = time.perf_counter()
        outs = pool.map_async(_run, [(relations, rules, p, tuple(sinks)) for p in parts], chunksize=1).get(timeout)
        wall = time.perf_counter() - t0
    total = {}
    for o in outs:
        for k, v in o["counts"].items():
            total[k] = total.get(k, 0) + v
    digests = {name: combine_digests([o["digests"][name] for o in outs]) for name in sinks}
    return RootedRun(total, digests, wall, [o["join_s"] for o in outs])
