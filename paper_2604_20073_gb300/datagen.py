"""Seeded synthetic fact generators shared by the GPU path's tests/bench and the oracle.

This module holds no Datalog arithmetic: it only draws facts.  Both sides of every
parity test receive the arrays produced here.  Randomness comes from one
counter-based generator, splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i of a stream with seed s is
mix(s + (i + 1) * GAMMA), so any slice of a stream can be drawn without drawing what
precedes it, identically on every platform (numpy uint64 arithmetic wraps mod 2^64).

Workload shapes (the paper's graph and program-analysis workloads are not available,
so these synthetic stand-ins take their place):

* ``rmat_edges``: R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004) directed or
  symmetrised graphs; quadrant probabilities a, b, c, d; bits chosen MSB first; self
  loops, out-of-range ids and duplicates rejected; sampling repeats until exactly
  ``m`` distinct rows exist (the first ``m`` distinct rows in sample order).  Hubs sit
  at low ids (no vertex permutation).
* ``points_to_facts``: Andersen-style New / Assign / Load / Store facts with Zipf(1.1)
  Assign endpoints, every domain and row count scaled by a factor ``f``.
* ``batched_instances``: many independent R-MAT instances with log-uniform sizes.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_scalar(x: int) -> int:
    """One splitmix64 output for state ``x`` (Python int in, Python int out)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_u64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the splitmix64 stream seeded by ``seed``."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    state = np.uint64(seed & _MASK64) + idx * GAMMA
    return _mix(state)


def stream_uniform(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) built from the top 53 bits of each stream output."""
    return (stream_u64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def instance_seed(base: int, i: int) -> int:
    """Seed of instance/request ``i`` of a family whose base seed is ``base``."""
    return splitmix64_scalar((base ^ i) & _MASK64)


def rmat_edges(n: int, m: int, seed: int, a=0.57, b=0.19, c=0.19, symmetric=False,
               batch: int | None = None) -> np.ndarray:
    """R-MAT edge list as an (rows, 2) uint32 array, rows sorted ascending.

    Directed: exactly ``m`` distinct (u, v), u != v.  Symmetrised: exactly ``m`` rows made
    of ``m // 2`` distinct unordered pairs {u < v}, both directions emitted.
    """
    if n < 2:
        raise ValueError("need at least two nodes")
    scale = max(1, math.ceil(math.log2(n)))
    target = m // 2 if symmetric else m
    if target > (n * (n - 1)) // (2 if symmetric else 1):
        raise ValueError("more distinct edges requested than the graph can hold")
    ab, abc = a + b, a + b + c
    if batch is None:
        batch = min(max(2 * target, 4096), 1 << 22)
    seen = np.zeros(0, dtype=np.uint64)      # sorted distinct keys accepted so far
    ordered: list[np.ndarray] = []           # the same keys in first-occurrence order
    drawn = 0
    have = 0
    while have < target:
        r = stream_uniform(seed, drawn * scale, batch * scale).reshape(batch, scale)
        drawn += batch
        u = np.zeros(batch, dtype=np.uint64)
        v = np.zeros(batch, dtype=np.uint64)
        for lvl in range(scale):
            x = r[:, lvl]
            # quadrant q: 0 = a (0,0), 1 = b (0,1), 2 = c (1,0), 3 = d (1,1)
            q = (x >= a).astype(np.uint64) + (x >= ab) + (x >= abc)
            sh = np.uint64(scale - 1 - lvl)
            u |= (q >> np.uint64(1)) << sh
            v |= (q & np.uint64(1)) << sh
        ok = (u < n) & (v < n) & (u != v)
        u, v = u[ok], v[ok]
        if symmetric:
            u, v = np.minimum(u, v), np.maximum(u, v)
        k = (u << np.uint64(32)) | v
        order = np.argsort(k, kind="stable")
        ks = k[order]
        firstmask = np.ones(ks.size, dtype=bool)
        firstmask[1:] = ks[1:] != ks[:-1]
        uk, first = ks[firstmask], order[firstmask]      # distinct keys, first sample index
        pos = np.searchsorted(seen, uk)
        present = np.zeros(uk.size, dtype=bool)
        inb = pos < seen.size
        present[inb] = seen[pos[inb]] == uk[inb]
        fresh, fidx = uk[~present], first[~present]
        ordered.append(fresh[np.argsort(fidx, kind="stable")])
        seen = np.insert(seen, np.searchsorted(seen, fresh), fresh)
        have = seen.size
    chosen = np.sort(np.concatenate(ordered)[:target])
    src = (chosen >> np.uint64(32)).astype(np.uint32)
    dst = (chosen & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    if symmetric:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    e = np.stack([src, dst], axis=1)
    return sort_rows(e)


def sort_rows(rows: np.ndarray) -> np.ndarray:
    """Rows sorted ascending lexicographically (column 0 most significant)."""
    if rows.shape[0] == 0:
        return rows
    keys = [rows[:, j] for j in range(rows.shape[1] - 1, -1, -1)]
    return rows[np.lexsort(keys)]


def unique_rows(rows: np.ndarray) -> np.ndarray:
    """Sorted distinct rows."""
    if rows.shape[0] == 0:
        return rows
    return np.unique(rows, axis=0)


def _zipf_ranks(seed: int, start: int, count: int, domain: int, s: float) -> np.ndarray:
    w = np.arange(1, domain + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = stream_uniform(seed, start, count)
    return np.minimum(np.searchsorted(cdf, u, side="right"), domain - 1).astype(np.uint32)


def _uniform_ids(seed: int, start: int, count: int, domain: int) -> np.ndarray:
    return (stream_u64(seed, start, count) % np.uint64(domain)).astype(np.uint32)


def points_to_facts(f: float, seed: int, zipf_s: float = 1.1) -> dict:
    """Andersen-style facts at scale ``f`` of 2M variables, 500k heaps, 2k fields,
    New 1M rows, Assign 6M rows (Zipf endpoints), Load / Store 1.5M rows each.

    Returns dict name -> (rows, arity) uint32 arrays, each deduplicated and sorted, plus
    the domain sizes.  Load is (v, w, f); Store is (v, f, w).
    """
    V = max(1, int(round(2_000_000 * f)))
    H = max(1, int(round(500_000 * f)))
    F = max(1, int(round(2_000 * f)))
    n_new = max(1, int(round(1_000_000 * f)))
    n_asg = max(1, int(round(6_000_000 * f)))
    n_ls = max(1, int(round(1_500_000 * f)))
    pos = 0

    def take(cnt):
        nonlocal pos
        s = pos
        pos += cnt
        return s

    new = np.stack([_uniform_ids(seed, take(n_new), n_new, V),
                    _uniform_ids(seed, take(n_new), n_new, H)], axis=1)
    asg = np.stack([_zipf_ranks(seed, take(n_asg), n_asg, V, zipf_s),
                    _zipf_ranks(seed, take(n_asg), n_asg, V, zipf_s)], axis=1)
    load = np.stack([_uniform_ids(seed, take(n_ls), n_ls, V),
                     _uniform_ids(seed, take(n_ls), n_ls, V),
                     _uniform_ids(seed, take(n_ls), n_ls, F)], axis=1)
    store = np.stack([_uniform_ids(seed, take(n_ls), n_ls, V),
                      _uniform_ids(seed, take(n_ls), n_ls, F),
                      _uniform_ids(seed, take(n_ls), n_ls, V)], axis=1)
    return {
        "New": unique_rows(new), "Assign": unique_rows(asg),
        "Load": unique_rows(load), "Store": unique_rows(store),
        "domains": {"V": V, "H": H, "F": F},
    }


def batched_sizes(count: int, base_seed: int, lo: int = 100, hi: int = 50_000) -> list:
    """Per-instance (edges, nodes, seed): edges log-uniform in [lo, hi], nodes = max(2, edges // 8)."""
    out = []
    for i in range(count):
        s = instance_seed(base_seed, i)
        u = float(stream_uniform(s, 0, 1)[0])
        m = int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))
        n = max(2, m // 8)
        m = min(m, n * (n - 1))
        out.append((m, n, s))
    return out


def batched_instances(count: int, base_seed: int, lo: int = 100, hi: int = 50_000) -> list:
    """Edge arrays of ``count`` independent R-MAT instances (sizes from ``batched_sizes``)."""
    return [rmat_edges(n, m, s ^ 0x5DEECE66D)
            for (m, n, s) in batched_sizes(count, base_seed, lo, hi)]


# ----- small deterministic shapes used by closed-form tests -----

def path_graph(n: int) -> np.ndarray:
    return np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.uint32)


def cycle_graph(n: int) -> np.ndarray:
    return np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).astype(np.uint32)


def complete_dag(n: int) -> np.ndarray:
    i, j = np.triu_indices(n, 1)
    return np.stack([i, j], axis=1).astype(np.uint32)


def complete_sym(n: int) -> np.ndarray:
    i, j = np.nonzero(~np.eye(n, dtype=bool))
    return np.stack([i, j], axis=1).astype(np.uint32)


def random_bipartite(n_left: int, n_right: int, m: int, seed: int, symmetric=True) -> np.ndarray:
    u = _uniform_ids(seed, 0, m, n_left)
    v = (_uniform_ids(seed, m, m, n_right) + np.uint32(n_left)).astype(np.uint32)
    e = np.stack([u, v], axis=1)
    if symmetric:
        e = np.concatenate([e, e[:, ::-1]])
    return unique_rows(e)


def random_graph(n: int, m: int, seed: int) -> np.ndarray:
    """Uniform random directed graph without self loops (duplicates removed)."""
    u = _uniform_ids(seed, 0, m, n)
    v = _uniform_ids(seed, m, m, n)
    ok = u != v
    return unique_rows(np.stack([u[ok], v[ok]], axis=1))


def hub_graph(hubs: int, n: int, m: int, seed: int) -> np.ndarray:
    """Symmetric graph on n vertices: vertices 0..hubs-1 are adjacent to every other vertex,
    plus about m uniform random edges among the rest (both directions, no self loops)."""
    h = np.arange(hubs, dtype=np.uint32)
    rest = np.arange(hubs, n, dtype=np.uint32)
    star = np.stack([np.repeat(h, len(rest)), np.tile(rest, hubs)], axis=1)
    hh = np.array([(a, b) for a in range(hubs) for b in range(hubs) if a != b], dtype=np.uint32).reshape(-1, 2)
    r = random_graph(n - hubs, m, seed) + np.uint32(hubs)
    rows = np.concatenate([star, star[:, ::-1], hh, r, r[:, ::-1]])
    return unique_rows(rows)


def call_graph_facts(scale: float, seed: int) -> dict:
    """Facts shaped like the virtual-call resolution step of a Java points-to analysis (the
    CallGraphEdge rule): methods, invocation sites, variables, heap objects and types, with
    Zipf-skewed heaps, method names, descriptors and types so that a few types (the
    java.lang.Object-like base classes) own most heap objects and answer most method lookups.

    Sizes at scale 1: 2,000 methods (60% reachable), 20,000 invocations, 10,000 variables,
    20,000 heaps, 500 types, 200 simple names x 20 descriptors.  Returns name -> rows:
    Reachable(j), InstructionMethod(i, j), VirtualMethodInvoc(i, b, sn, dsc),
    VarPointsTo(h, b), HeapAllocationType(h, t), MethodLookup(sn, dsc, t, m); every
    relation deduplicated and sorted."""
    M = max(2, int(round(2_000 * scale)))
    I = max(2, int(round(20_000 * scale)))
    B = max(2, int(round(10_000 * scale)))
    H = max(2, int(round(20_000 * scale)))
    T, NS, ND = 500, 200, 20
    pos = 0

    def take(cnt):
        nonlocal pos
        s = pos
        pos += cnt
        return s

    reach = _uniform_ids(seed, take(int(0.6 * M)), int(0.6 * M), M).reshape(-1, 1)
    im = np.stack([np.arange(I, dtype=np.uint32), _uniform_ids(seed, take(I), I, M)], axis=1)
    vmi = np.stack([np.arange(I, dtype=np.uint32), _uniform_ids(seed, take(I), I, B),
                    _zipf_ranks(seed, take(I), I, NS, 1.1), _zipf_ranks(seed, take(I), I, ND, 1.1)], axis=1)
    n_vpt = 3 * B
    vpt = np.stack([_zipf_ranks(seed, take(n_vpt), n_vpt, H, 1.1), _uniform_ids(seed, take(n_vpt), n_vpt, B)], axis=1)
    hat = np.stack([np.arange(H, dtype=np.uint32), _zipf_ranks(seed, take(H), H, T, 1.3)], axis=1)
    # each type answers 20 lookups, the 5 most common types 320 more (their methods are
    # inherited everywhere); the resolved method is a hash of (sn, dsc, t)
    per = np.full(T, 20, dtype=np.int64)
    per[:5] += 300
    t_col = np.repeat(np.arange(T, dtype=np.uint32), per)
    n_ml = len(t_col)
    sn = _zipf_ranks(seed, take(n_ml), n_ml, NS, 1.1)
    dsc = _zipf_ranks(seed, take(n_ml), n_ml, ND, 1.1)
    key = (sn.astype(np.uint64) << np.uint64(40)) | (dsc.astype(np.uint64) << np.uint64(20)) | t_col.astype(np.uint64)
    m = (_mix(key ^ np.uint64(seed & 0xFFFFFFFF)) % np.uint64(M)).astype(np.uint32)
    ml = np.stack([sn, dsc, t_col, m], axis=1)
    return {"Reachable": unique_rows(reach), "InstructionMethod": unique_rows(im),
            "VirtualMethodInvoc": unique_rows(vmi), "VarPointsTo": unique_rows(vpt),
            "HeapAllocationType": unique_rows(hat), "MethodLookup": unique_rows(ml)}
