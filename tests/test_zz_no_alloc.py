"""The allocation-free sort + dedup entry point (dl_sort_unique_noalloc) gives the same rows
as the engine's own path (dl_load_facts_device + dl_fetch_device) and as a host numpy
sort + unique of the same rows, on two calls in a row.

It exists for callers that may not allocate device memory while they run (a plugin whose
host application's allocator owns the device budget, or a latency-bound loop that bans
cudaMalloc/cudaFree); its scratch is one static device array shared by every call.  This
file is collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import paper_2604_20073_gb300 as pkg

pytestmark = pytest.mark.gpu


def _noalloc(lib, cols_dev, out_dev, stream):
    import torch
    n = ctypes.c_uint64()
    ins = (ctypes.c_void_p * len(cols_dev))(*[c.data_ptr() for c in cols_dev])
    outs = (ctypes.c_void_p * len(out_dev))(*[c.data_ptr() for c in out_dev])
    rc = lib.dl_sort_unique_noalloc(ins, len(cols_dev), cols_dev[0].numel(), outs, ctypes.byref(n),
                                    ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, n.value


def _engine_sort_unique(rows_dev, arity):
    import torch
    with pkg.Engine() as eng:
        eng.relation("R", arity)
        eng.load("R", rows_dev)
        n = eng.size("R")
        cols = [torch.empty(max(n, 1), dtype=torch.int32, device="cuda") for _ in range(arity)]
        eng.fetch_device("R", cols)
        torch.cuda.synchronize()
        return n, [c[:n].cpu().numpy().view(np.uint32) for c in cols]


def _host_sort_unique(host):
    """Sorted distinct rows computed on the host (numpy), independent of every GPU kernel."""
    rows = np.unique(host.T, axis=0)          # lexicographic over columns 0..arity-1, unsigned
    return [np.ascontiguousarray(rows[:, c]) for c in range(host.shape[0])]


def test_noalloc_sort_unique_matches_engine_twice():
    import torch
    lib = pkg.load_library()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(77)
    cases = [(3, 200_000, 300), (2, 70_001, 1 << 31)]     # (arity, rows, value range): many / few duplicates
    for arity, n, vmax in cases:
        host = rng.integers(0, vmax, size=(arity, n), dtype=np.uint64).astype(np.uint32)
        rows_dev = torch.from_numpy(host.view(np.int32)).cuda()
        cols_dev = [rows_dev[c].contiguous() for c in range(arity)]
        out_dev = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(arity)]
        rc, m = _noalloc(lib, cols_dev, out_dev, stream)
        assert rc == pkg.DL_OK
        n_ref, ref = _engine_sort_unique(rows_dev, arity)
        host_ref = _host_sort_unique(host)
        assert m == n_ref == len(host_ref[0])
        for c in range(arity):
            got = out_dev[c][:m].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref[c])
            assert np.array_equal(got, host_ref[c])
        # the input columns are left untouched
        for c in range(arity):
            assert np.array_equal(cols_dev[c].cpu().numpy().view(np.uint32), host[c])


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    lib = pkg.load_library()
    big = 262_145
    col = torch.zeros(big, dtype=torch.int32, device="cuda")
    rc, _ = _noalloc(lib, [col], [torch.zeros(big, dtype=torch.int32, device="cuda")], torch.cuda.current_stream())
    assert rc == pkg.DL_ERR_CAPACITY
    five = [torch.zeros(8, dtype=torch.int32, device="cuda") for _ in range(5)]
    rc, _ = _noalloc(lib, five, five, torch.cuda.current_stream())
    assert rc == pkg.DL_ERR_CAPACITY
