"""CPU oracle for Datalog with stratified negation and comparisons (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the GPU library; the product never
loads it.

The evaluator itself is plain C (``oracle.c``): a semi-naive engine with left-deep,
hash-indexed nested-loop joins (paper Section 2), and a brute-force naive T_P used to
pin it.  This module compiles it with gcc, loads it with ctypes and converts between
numpy arrays and the C calls.

Program format (plain data, built by the caller):

* ``relations``: ``{name: arity}``
* ``facts``: ``{name: (rows, arity) uint32 array}``
* ``rules``: list of ``(head, body)`` where ``head`` is an atom and ``body`` a list of
  items; an atom is ``(relation_name, [term, ...])``; a term is a ``str`` (variable)
  or an ``int`` (constant).  A body item is an atom, a negated atom ``("not", atom)``
  or a comparison ``(op, term, term)`` with op one of ``<  <=  >  >=  !=`` (unsigned
  32-bit order).  A rule may carry a third item, a variable order, which is ignored: the
  oracle's result does not depend on one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .partition import decode_unit, work_slices  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"seminaive": 0, "naive_strata": 1, "naive_global": 2}


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_error.restype = ctypes.c_char_p
            lib.orc_error.argtypes = [ctypes.c_void_p]
            lib.orc_relation.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
            lib.orc_add_facts.argtypes = [ctypes.c_void_p, ctypes.c_int, u32p, ctypes.c_uint64]
            lib.orc_add_rule.argtypes = [ctypes.c_void_p, ctypes.c_int, u32p, u32p, ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_int32), u32p, u32p]
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.orc_add_rule_ex.argtypes = [ctypes.c_void_p, ctypes.c_int, u32p, u32p, ctypes.c_uint32, i32p, u32p,
                                            u32p, ctypes.c_uint32, i32p, u32p, u32p, ctypes.c_uint32, u32p, u32p,
                                            u32p]
            lib.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_count.restype = ctypes.c_uint64
            lib.orc_count.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_fetch.argtypes = [ctypes.c_void_p, ctypes.c_int, u32p]
            lib.orc_num_strata.restype = ctypes.c_uint32
            lib.orc_num_strata.argtypes = [ctypes.c_void_p]
            lib.orc_stratum.argtypes = [ctypes.c_void_p, ctypes.c_uint32, u32p, u32p, u32p]
            lib.orc_set_count_sink.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_sink_digest.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
            lib.orc_join_seconds.restype = ctypes.c_double
            lib.orc_join_seconds.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _u32(a) -> ctypes.POINTER(ctypes.c_uint32):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class OracleError(RuntimeError):
    pass


class Result:
    """Per-relation sorted distinct rows and the strata with their round counts."""

    def __init__(self, relations: dict, strata: list, digests: dict | None = None, join_seconds: float = 0.0):
        self.relations = relations          # name -> (rows, arity) uint32, sorted, distinct
        self.strata = strata                # [(sorted relation names, rounds), ...] in evaluation order
        self.digests = digests or {}        # count sinks: name -> (count, sum, xor), as tuple_digest
        self.join_seconds = join_seconds    # time in the nested loops (hash index builds excluded)

    def rounds_of(self, name: str) -> int:
        for rels, r in self.strata:
            if name in rels:
                return r
        raise KeyError(name)


def evaluate(relations: dict, facts: dict, rules: list, mode: str = "seminaive",
             sinks: tuple | list | set = ()) -> Result:
    """Run a program to its least fixpoint and return every relation.  Relations named in
    `sinks` are count sinks: they keep no rows (an empty array is returned for them) and
    their count and digest, as tuple_digest defines it, go to Result.digests."""
    lib = _load()
    h = lib.orc_create()
    try:
        names = list(relations)
        rid = {}
        for name in names:
            r = lib.orc_relation(h, int(relations[name]))
            if r < 0:
                raise OracleError(lib.orc_error(h).decode())
            rid[name] = r
        for name in sinks:
            if lib.orc_set_count_sink(h, rid[name]) != 0:
                raise OracleError(lib.orc_error(h).decode())
        for name, rows in facts.items():
            rows = np.ascontiguousarray(rows, dtype=np.uint32).reshape(-1, relations[name])
            if lib.orc_add_facts(h, rid[name], _u32(rows), rows.shape[0]) != 0:
                raise OracleError(lib.orc_error(h).decode())
        for rule in rules:
            head, body = rule[0], rule[1]   # a third item (a variable order) is ignored
            def enc(terms, rel):
                if len(terms) != relations[rel]:
                    raise OracleError(f"arity mismatch in atom {rel}{tuple(terms)}")
                kinds, vals = [], []
                for t in terms:
                    if isinstance(t, str):
                        kinds.append(0)
                        vals.append(var_ids.setdefault(t, len(var_ids)))
                    else:
                        kinds.append(1)
                        vals.append(int(t))
                return kinds, vals
            var_ids: dict = {}
            pos, neg, cmps = [], [], []
            for item in body:
                if len(item) == 3:
                    cmps.append(item)
                elif item[0] == "not":
                    neg.append(item[1])
                else:
                    pos.append(item)
            bk, bv, brels = [], [], []
            for rel, terms in pos:
                k, v = enc(terms, rel)
                bk += k
                bv += v
                brels.append(rid[rel])
            nk, nv, nrels = [], [], []
            for rel, terms in neg:
                k, v = enc(terms, rel)
                nk += k
                nv += v
                nrels.append(rid[rel])
            ops, ck, cv = [], [], []
            for op, a, b in cmps:
                if op in (">", ">="):
                    op, a, b = ("<" if op == ">" else "<="), b, a
                ops.append({"<": 0, "<=": 1, "!=": 2}[op])
                for t in (a, b):
                    if isinstance(t, str):
                        if t not in var_ids:
                            raise OracleError(f"comparison variable {t} not bound by a positive atom")
                        ck.append(0)
                        cv.append(var_ids[t])
                    else:
                        ck.append(1)
                        cv.append(int(t))
            hk, hv = enc(head[1], head[0])
            arr = lambda x: np.asarray(x if len(x) else [0], dtype=np.uint32)  # noqa: E731
            arr_i = lambda x: np.asarray(x if len(x) else [0], dtype=np.int32)  # noqa: E731
            hk_a, hv_a, bk_a, bv_a, nk_a, nv_a = arr(hk), arr(hv), arr(bk), arr(bv), arr(nk), arr(nv)
            ops_a, ck_a, cv_a = arr(ops), arr(ck), arr(cv)
            br_a, nr_a = arr_i(brels), arr_i(nrels)
            i32 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
            ok = lib.orc_add_rule_ex(h, rid[head[0]], _u32(hk_a), _u32(hv_a), len(pos), i32(br_a),
                                     _u32(bk_a), _u32(bv_a), len(neg), i32(nr_a), _u32(nk_a), _u32(nv_a),
                                     len(cmps), _u32(ops_a), _u32(ck_a), _u32(cv_a))
            if ok < 0:
                raise OracleError(lib.orc_error(h).decode())
        if lib.orc_run(h, MODES[mode]) != 0:
            raise OracleError(lib.orc_error(h).decode())
        out = {}
        for name in names:
            n = lib.orc_count(h, rid[name])
            rows = np.empty((n, relations[name]), dtype=np.uint32)
            if n:
                lib.orc_fetch(h, rid[name], _u32(rows))
            out[name] = rows
        strata = []
        for s in range(lib.orc_num_strata(h)):
            rounds = ctypes.c_uint32()
            nrels = ctypes.c_uint32()
            rels = np.empty(len(names), dtype=np.uint32)
            lib.orc_stratum(h, s, ctypes.byref(rounds), _u32(rels), ctypes.byref(nrels))
            strata.append((sorted(names[i] for i in rels[: nrels.value]), rounds.value))
        digests = {}
        for name in sinks:
            d = (ctypes.c_uint64 * 3)()
            if lib.orc_sink_digest(h, rid[name], d) != 0:
                raise OracleError(lib.orc_error(h).decode())
            digests[name] = (int(d[0]), int(d[1]), int(d[2]))
        return Result(out, strata, digests, float(lib.orc_join_seconds(h)))
    finally:
        lib.orc_destroy(h)


_M64 = (1 << 64) - 1


def splitmix64_mix(z: int) -> int:
    """The splitmix64 output finaliser (Steele, Lea and Flood, 2014), on Python integers."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def row_hash(row) -> int:
    """64-bit hash of one row: h = 0x243F6A8885A308D3; for column j with value v,
    h = mix(h ^ (v + 0x9E3779B97F4A7C15 * (j + 1)))."""
    h = 0x243F6A8885A308D3
    for j, v in enumerate(row):
        h = splitmix64_mix((h ^ ((int(v) + 0x9E3779B97F4A7C15 * (j + 1)) & _M64)) & _M64)
    return h


def tuple_digest(rows: np.ndarray) -> tuple:
    """Order-independent digest of a set of rows: (count, sum mod 2^64, xor) of row_hash
    over the rows.  Written here from that definition with Python integers, row by row."""
    s = 0
    x = 0
    rows = np.asarray(rows, dtype=np.uint64)
    for row in rows.tolist():
        h = row_hash(row)
        s = (s + h) & _M64
        x ^= h
    return (len(rows), s, x)


def combine_digests(parts) -> tuple:
    """Digest of the union of disjoint row sets from their digests."""
    c = s = x = 0
    for pc, ps, px in parts:
        c += pc
        s = (s + ps) & _M64
        x ^= px
    return (c, s, x)
