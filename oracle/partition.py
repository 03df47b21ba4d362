"""Oracle for the root-level work partition of the paper's Section 5 (Algorithm 1 and
Algorithm 2 and the worked example with keys A, B, C, D of Figure 2).

Test infrastructure only (see the package docstring).

Definitions followed here, written out plainly:

* The per-key fan-outs W[0..K) are prefix-summed into C (inclusive), so key k owns the
  flat work units [C[k-1], C[k]) with C[-1] = 0, and T = C[K-1] (Algorithm 1, Phase 1).
* With p groups, group b takes the contiguous slice [b * ceil(T/p), min((b+1) * ceil(T/p), T))
  (Algorithm 2, first step); its first key is the one whose range holds the slice start,
  i.e. the first k with C[k] > start (Algorithm 2's binary search on C; C is inclusive,
  hence an upper bound).
* A flat unit g decodes to (key, i1, i2) by local = g - C[key-1], i1 = local div d2(key),
  i2 = local mod d2(key) (Section 5, the decode formula), d2 being the inner degree under
  the key.
"""
from __future__ import annotations

import bisect


def owner(C: list, g: int) -> int:
    """Key whose unit range holds flat unit g (first k with C[k] > g)."""
    return bisect.bisect_right(C, g)


def work_slices(C: list, p: int) -> list:
    """For each of p groups: a list of (key, first_local_unit, end_local_unit) pieces."""
    T = C[-1] if C else 0
    if T == 0:
        return [[] for _ in range(p)]
    step = -(-T // p)
    groups = []
    for b in range(p):
        s, e = b * step, min((b + 1) * step, T)
        pieces = []
        g = s
        while g < e:
            k = owner(C, g)
            base = C[k - 1] if k > 0 else 0
            end = min(e, C[k])
            pieces.append((k, g - base, end - base))
            g = end
        groups.append(pieces)
    return groups


def decode_unit(C: list, d2: list, g: int) -> tuple:
    """(key, i1, i2) of flat unit g."""
    k = owner(C, g)
    local = g - (C[k - 1] if k > 0 else 0)
    return k, local // d2[k], local % d2[k]
