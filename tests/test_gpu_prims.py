"""The delta primitives through the C ABI, against numpy: loading facts in two steps sorts,
deduplicates and anti-joins the second load against the relation and merges it in (radix
sort on packed keys or on all columns, the staged scatter, the shared-memory merge path),
at arities 1-8, sizes around the sort and merge tile boundaries, narrow and full 32-bit
value ranges, and heavy duplication."""
import numpy as np
import pytest

import paper_2604_20073_gb300 as pkg

pytestmark = pytest.mark.gpu


def _rows(rng, n, arity, vmax):
    return rng.integers(0, vmax, size=(n, arity), dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("arity", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("vmax", [7, 5000, 0xFFFFFFFF])
def test_two_step_load_equals_numpy_union(arity, vmax):
    rng = np.random.default_rng(arity * 1000 + (vmax % 997))
    for n1, n2 in [(0, 5), (1, 1), (2047, 2049), (4096, 4095), (100_003, 37_001)]:
        a, b = _rows(rng, n1, arity, vmax), _rows(rng, n2, arity, vmax)
        if n1 and n2:
            b[: n2 // 3] = a[rng.integers(0, n1, n2 // 3)]      # overlap with the first load
        with pkg.Engine() as eng:
            eng.relation("R", arity)
            if n1:
                eng.load("R", a)
                first = eng.fetch("R")
                assert np.array_equal(first, np.unique(a, axis=0))
            eng.load("R", b)
            got = eng.fetch("R")
        want = np.unique(np.concatenate([a, b]).reshape(-1, arity), axis=0)
        assert np.array_equal(got, want), (arity, vmax, n1, n2)
