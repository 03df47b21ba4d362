"""The C-ABI library loads and exports every symbol include/dl.h declares; the host-side
partition helpers (the same routine the join kernels use to map work units to keys) agree
with the oracle's partition and with the paper's worked example.  No GPU needed."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import oracle.partition as opart
import paper_2604_20073_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dl.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2604_20073_gb300.build import build_library
        build_library()
    return pkg.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dl_[a-z_0-9]+)\s*\(", text)) - {"dl_alloc_fn", "dl_free_fn"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["dl_engine_create", "dl_engine_destroy", "dl_last_error", "dl_relation_create",
                 "dl_load_facts", "dl_rule_add", "dl_fixpoint", "dl_fetch", "dl_fetch_digest"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(pkg.exported_symbols())


def test_version(lib):
    assert lib.dl_version().decode().count(".") == 2


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def lib_slices(lib, C, p):
    C = _u64(C)
    fk = np.zeros(p, dtype=np.uint64)
    su = np.zeros(p, dtype=np.uint64)
    assert lib.dl_partition_slices(_p(C), len(C), p, _p(fk), _p(su)) == 0
    return fk.tolist(), su.tolist()


def test_partition_worked_example(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_example_partition.json")))
    fk, su = lib_slices(lib, g["prefix_inclusive"], g["groups"])
    expect = opart.work_slices(g["prefix_inclusive"], g["groups"])
    assert su == [0, 5, 10, 15]
    assert fk == [grp[0][0] for grp in expect]          # A, B, B, D
    assert [g["keys"][k] for k in fk] == ["A", "B", "B", "D"]


@pytest.mark.parametrize("seed", range(6))
def test_partition_and_decode_match_oracle(lib, seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 40))
    d1 = rng.integers(0, 7, size=K)
    d2 = rng.integers(1, 7, size=K)
    C = np.cumsum(d1 * d2)
    if C[-1] == 0:
        return
    for p in (1, 3, 8, 100):
        fk, su = lib_slices(lib, C, p)
        ex = opart.work_slices(list(C), p)
        for b in range(p):
            if ex[b]:
                assert fk[b] == ex[b][0][0]
    key, i1, i2 = (ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64())
    Cu, d2u = _u64(C), _u64(d2)
    for gidx in range(int(C[-1])):
        assert lib.dl_decode_unit(_p(Cu), _p(d2u), K, gidx, ctypes.byref(key), ctypes.byref(i1), ctypes.byref(i2)) == 0
        assert (key.value, i1.value, i2.value) == opart.decode_unit(list(C), list(d2), gidx)
    assert lib.dl_decode_unit(_p(Cu), _p(d2u), K, int(C[-1]), ctypes.byref(key), ctypes.byref(i1),
                              ctypes.byref(i2)) == pkg.DL_ERR_ARG


def test_engine_create_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.dl_engine_create(None, ctypes.byref(h))
    assert rc == pkg.DL_ERR_CUDA and not h.value
    with pytest.raises(RuntimeError):
        pkg.Engine()


STRUCTS = ["dl_config", "dl_term", "dl_cmp", "dl_atom", "dl_kernel_stat", "dl_stats", "dl_server_config",
           "dl_rule_spec", "dl_fact_spec", "dl_request", "dl_server_stats"]


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the ctypes binding mirrors has the header's size and field offsets (a C
    program built here against include/dl.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dl.h"', "int main(void) {"]
    for name in STRUCTS:
        st = getattr(pkg, name)
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = {}
    for line in out:
        if line.strip():
            name, field, value = line.split()
            want[(name, field)] = int(value)
    for name in STRUCTS:
        st = getattr(pkg, name)
        assert ctypes.sizeof(st) == want[(name, "sizeof")], name
        for field, _ in st._fields_:
            assert getattr(st, field).offset == want[(name, field)], (name, field)
