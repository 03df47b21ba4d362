"""Root-partitioned runs of the oracle on several host cores.

Test and timing infrastructure only (the CPU baseline of the benchmark): it splits a set of
root values into parts and evaluates, in separate processes, the same root-restricted
program on each part with the unchanged oracle.  The rows of a root-restricted rule are
disjoint across roots, so the parts' row counts add up to the whole sample's.  Processes
are started with the spawn method (safe after a CUDA context exists in the parent)."""
from __future__ import annotations

import multiprocessing as mp
import time

import numpy as np

_FACTS = None


def _init(paths):
    global _FACTS
    _FACTS = {name: np.load(p) for name, p in paths.items()}


def _ready(_):
    return _FACTS is not None


def _run(job):
    relations, rules, roots = job
    from oracle import evaluate
    facts = dict(_FACTS)
    facts["Root"] = roots
    r = evaluate(relations, facts, rules)
    return {name: len(rows) for name, rows in r.relations.items()}


def run_rooted(fact_paths: dict, relations: dict, rules: list, roots: np.ndarray, processes: int,
               timeout: float = 600.0):
    """Evaluate `rules` (which read a unary relation Root) for `roots` split over `processes`
    spawned workers; facts are read by each worker from the .npy files in `fact_paths`.
    Returns (summed row counts per relation, wall seconds of the evaluation, excluding
    worker start-up and fact loading).  Raises multiprocessing.TimeoutError after `timeout`
    seconds per stage."""
    r = np.asarray(roots, dtype=np.uint32).reshape(-1, 1)
    parts = [r[i::processes] for i in range(processes) if len(r[i::processes])]   # interleaved: spreads hubs
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(parts), initializer=_init, initargs=(fact_paths,)) as pool:
        assert all(pool.map_async(_ready, range(len(parts)), chunksize=1).get(timeout))
        t0 = time.perf_counter()
        outs = pool.map_async(_run, [(relations, rules, p) for p in parts], chunksize=1).get(timeout)
        wall = time.perf_counter() - t0
    total = {}
    for o in outs:
        for k, v in o.items():
            total[k] = total.get(k, 0) + v
    return total, wall
