"""Python binding of libdlgpu.so, the GB300 semi-naive WCOJ Datalog library.

The ``dl_*`` functions below carry the same names and arguments as the C ABI in
``include/dl.h`` and only marshal arguments (ctypes).  Every step of the evaluation runs
in the library's CUDA kernels; there is no Python or CPU fallback: if the library is
missing or no GPU is present, creating an engine raises.

PyTorch is used only as plumbing: the current CUDA stream (and, optionally, the caching
allocator) is handed to the engine.  ``Engine`` wraps one engine handle with numpy-based
convenience methods; ``run_program`` evaluates a whole program given as plain data:

* ``relations``: ``{name: arity}``
* ``facts``: ``{name: (rows, arity) uint32 array}``
* ``rules``: list of ``(head, body, var_order)``; an atom is ``(relation, [terms])``, a term
  is a ``str`` (variable) or an ``int`` (constant).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdlgpu.so")

DL_OK, DL_ERR_ARG, DL_ERR_UNSUPPORTED, DL_ERR_CAPACITY, DL_ERR_CUDA, DL_ERR_TIMEOUT, DL_ERR_STATE = range(7)
ERR_NAMES = {1: "DL_ERR_ARG", 2: "DL_ERR_UNSUPPORTED", 3: "DL_ERR_CAPACITY", 4: "DL_ERR_CUDA",
             5: "DL_ERR_TIMEOUT", 6: "DL_ERR_STATE"}
DL_FLAG_NAIVE_ROOTS = 0x1
DL_FLAG_DEBUG_CHECKS = 0x2
DL_FLAG_PROFILE = 0x4
DL_FLAG_AUTOTUNE = 0x8
DL_FLAG_NO_DENSE_SINK = 0x10
KERNEL_KINDS = ["join_hist", "join_count", "join_write", "scan", "sort", "delta", "merge", "other"]
DL_SINK_STORE, DL_SINK_COUNT = 0, 1
DL_TERM_VAR, DL_TERM_CONST = 0, 1
DL_CMP_LT, DL_CMP_LE, DL_CMP_NE = 0, 1, 2
DL_MAX_STRATA = 64

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)

DL_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)
DL_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)


class dl_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64),
                ("alloc", DL_ALLOC_FN), ("free", DL_FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("flags", ctypes.c_uint32), ("tile_units", ctypes.c_uint32), ("instances", ctypes.c_uint32),
                ("chunk_rows", ctypes.c_uint64), ("hub_rows", ctypes.c_uint32),
                ("frontier_bytes", ctypes.c_uint64), ("head_percent", ctypes.c_uint32),
                ("dense_bytes", ctypes.c_uint64), ("tune_cache", ctypes.c_char_p)]


class dl_term(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("id", ctypes.c_uint32)]


class dl_cmp(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint32), ("a", dl_term), ("b", dl_term)]


class dl_atom(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_uint32), ("arity", ctypes.c_uint32), ("terms", ctypes.POINTER(dl_term))]


class dl_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("ms", ctypes.c_double), ("alg_bytes", ctypes.c_uint64),
                ("units", ctypes.c_uint64), ("entries", ctypes.c_uint64)]


class dl_stats(ctypes.Structure):
    _fields_ = [("nstrata", ctypes.c_uint32), ("rounds", ctypes.c_uint32 * DL_MAX_STRATA),
                ("stratum_first_rel", ctypes.c_uint32 * DL_MAX_STRATA), ("total_rounds", ctypes.c_uint32),
                ("join_rows", ctypes.c_uint64), ("count_rows", ctypes.c_uint64), ("delta_rows", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("ms_total", ctypes.c_double), ("ms_join", ctypes.c_double), ("ms_sort", ctypes.c_double),
                ("ms_dedup", ctypes.c_double), ("ms_merge", ctypes.c_double),
                ("kernels", dl_kernel_stat * len(KERNEL_KINDS)), ("top_kind", ctypes.c_uint32),
                ("top", dl_kernel_stat), ("hub_keys", ctypes.c_uint32),
                ("join_slices", ctypes.c_uint32), ("tuned_levels", ctypes.c_uint32), ("tune_hits", ctypes.c_uint32),
                ("head_flushes", ctypes.c_uint32), ("dense_relations", ctypes.c_uint32)]


class dl_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("default_share", ctypes.c_uint64), ("grow_retries", ctypes.c_uint32)]


class dl_rule_spec(ctypes.Structure):
    _fields_ = [("head", dl_atom), ("body", ctypes.POINTER(dl_atom)), ("nbody", ctypes.c_uint32),
                ("var_order", _u32p), ("nvars", ctypes.c_uint32), ("neg", ctypes.POINTER(dl_atom)),
                ("nneg", ctypes.c_uint32), ("cmps", ctypes.POINTER(dl_cmp)), ("ncmp", ctypes.c_uint32)]


class dl_fact_spec(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_uint32), ("rows", _u32p), ("nrows", ctypes.c_uint64)]


class dl_request(ctypes.Structure):
    _fields_ = [("nrel", ctypes.c_uint32), ("rel_names", ctypes.POINTER(ctypes.c_char_p)),
                ("rel_arity", _u32p), ("rel_sink", _u32p), ("nrules", ctypes.c_uint32),
                ("rules", ctypes.POINTER(dl_rule_spec)), ("nfacts", ctypes.c_uint32),
                ("facts", ctypes.POINTER(dl_fact_spec)), ("share_bytes", ctypes.c_uint64)]


class dl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("reserved_bytes", ctypes.c_uint64),
                ("peak_reserved_bytes", ctypes.c_uint64), ("running", ctypes.c_uint32), ("queued", ctypes.c_uint32),
                ("regrown", ctypes.c_uint64)]


DL_REQ_QUEUED, DL_REQ_RUNNING, DL_REQ_DONE = 0, 1, 2

_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); mirrors include/dl.h
_SIGS = {
    "dl_version": (ctypes.c_char_p, []),
    "dl_engine_create": (ctypes.c_int, [ctypes.POINTER(dl_config), ctypes.POINTER(ctypes.c_void_p)]),
    "dl_engine_destroy": (None, [ctypes.c_void_p]),
    "dl_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "dl_relation_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_uint32, _u32p]),
    "dl_relation_set_sink": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32]),
    "dl_load_facts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(_u32p), ctypes.c_uint64]),
    "dl_load_facts_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u32p, ctypes.c_uint64]),
    "dl_load_facts_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_uint64]),
    "dl_relation_clear": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "dl_rule_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_atom), ctypes.POINTER(dl_atom),
                                   ctypes.c_uint32, _u32p, ctypes.c_uint32, _u32p]),
    "dl_rule_add_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_atom), ctypes.POINTER(dl_atom),
                                      ctypes.c_uint32, ctypes.POINTER(dl_atom), ctypes.c_uint32,
                                      ctypes.POINTER(dl_cmp), ctypes.c_uint32, _u32p, ctypes.c_uint32, _u32p]),
    "dl_rule_add_split": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_atom), ctypes.POINTER(dl_atom),
                                         ctypes.c_uint32, _u32p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_char_p,
                                         _u32p, _u32p, _u32p]),
    "dl_split_columns": (ctypes.c_int, [ctypes.POINTER(dl_atom), ctypes.POINTER(dl_atom), ctypes.c_uint32, _u32p,
                                        ctypes.c_uint32, ctypes.c_uint64, _u32p, ctypes.c_uint32, _u32p]),
    "dl_fixpoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_stats)]),
    "dl_stratum_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u32p, ctypes.c_uint32, _u32p, _u32p]),
    "dl_relation_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p]),
    "dl_fetch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(_u32p), ctypes.c_uint64, _u64p]),
    "dl_fetch_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.c_uint64, _u64p]),
    "dl_fetch_digest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p]),
    "dl_partition_slices": (ctypes.c_int, [_u64p, ctypes.c_uint64, ctypes.c_uint32, _u64p, _u64p]),
    "dl_decode_unit": (ctypes.c_int, [_u64p, _u64p, ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p]),
    "dl_load_facts_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_u32p),
                                              ctypes.c_uint64]),
    "dl_fetch_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_u32p),
                                         ctypes.c_uint64, _u64p]),
    "dl_instance_rounds": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u32p, ctypes.c_uint32, _u32p]),
    "dl_instance_digest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p]),
    "dl_server_create": (ctypes.c_int, [ctypes.POINTER(dl_server_config), ctypes.POINTER(ctypes.c_void_p)]),
    "dl_server_destroy": (None, [ctypes.c_void_p]),
    "dl_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_request), _u64p]),
    "dl_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "dl_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "dl_server_result": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]),
    "dl_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "dl_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_server_stats)]),
    "dl_tune_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "dl_engine_set_flags": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "dl_program_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "dl_program_destroy": (None, [ctypes.c_void_p]),
    "dl_program_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "dl_program_relation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32, _u32p]),
    "dl_program_rule": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dl_atom), ctypes.POINTER(dl_atom), ctypes.c_uint32,
                                       ctypes.POINTER(dl_atom), ctypes.c_uint32, ctypes.POINTER(dl_cmp), ctypes.c_uint32,
                                       _u32p, ctypes.c_uint32]),
    "dl_program_load_facts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(_u32p), ctypes.c_uint64]),
    "dl_fixpoint_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32,
                                         ctypes.POINTER(dl_stats)]),
    "dl_program_fetch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(_u32p), ctypes.c_uint64, _u64p]),
    "dl_program_digest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p]),
    "dl_program_rounds": (ctypes.c_int, [ctypes.c_void_p, _u32p, ctypes.c_uint32, _u32p]),
    "dl_program_stratum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u32p, ctypes.c_uint32, _u32p]),
    "dl_sort_unique_noalloc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32, ctypes.c_uint64,
                                              ctypes.POINTER(ctypes.c_void_p), _u64p, ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH):
    """Load libdlgpu.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list:
    return list(_SIGS)


class DatalogError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def __getattr__(name):  # module-level dl_* access: paper_2604_20073_gb300.dl_fixpoint(...)
    if name in _SIGS:
        return getattr(load_library(), name)
    raise AttributeError(name)


def _cols_ptrs(arrs):
    arr = (_u32p * len(arrs))()
    for i, a in enumerate(arrs):
        arr[i] = a.ctypes.data_as(_u32p)
    return arr


def _encode_atom(rel_ids, atom, var_ids, keep):
    rel, terms = atom
    ts = (dl_term * len(terms))()
    for i, t in enumerate(terms):
        if isinstance(t, str):
            ts[i].kind, ts[i].id = DL_TERM_VAR, var_ids.setdefault(t, len(var_ids))
        else:
            ts[i].kind, ts[i].id = DL_TERM_CONST, int(t)
    keep.append(ts)
    a = dl_atom()
    a.rel, a.arity, a.terms = rel_ids[rel], len(terms), ts
    return a


def _encode_rule(rel_ids, head, body, order):
    """ctypes arguments of a rule: body items are atoms (rel, [terms]), negated atoms
    ("not", atom) and comparisons (op, term, term) with op in < <= > >= !=."""
    var_ids: dict = {}
    keep: list = []
    pos = [b for b in body if len(b) == 2 and b[0] != "not"]
    neg = [b[1] for b in body if len(b) == 2 and b[0] == "not"]
    cmps = [b for b in body if len(b) == 3]
    batoms = (dl_atom * len(pos))()
    for i, b in enumerate(pos):
        batoms[i] = _encode_atom(rel_ids, b, var_ids, keep)
    natoms = (dl_atom * max(1, len(neg)))()
    for i, b in enumerate(neg):
        natoms[i] = _encode_atom(rel_ids, b, var_ids, keep)
    carr = (dl_cmp * max(1, len(cmps)))()
    for i, (op, a, b) in enumerate(cmps):
        if op in (">", ">="):
            op, a, b = ("<" if op == ">" else "<="), b, a
        carr[i].op = {"<": DL_CMP_LT, "<=": DL_CMP_LE, "!=": DL_CMP_NE}[op]
        for t, dst in ((a, carr[i].a), (b, carr[i].b)):
            if isinstance(t, str):
                dst.kind, dst.id = DL_TERM_VAR, var_ids.get(t, 1023)
            else:
                dst.kind, dst.id = DL_TERM_CONST, int(t)
    h = _encode_atom(rel_ids, head, var_ids, keep)
    ordr = (ctypes.c_uint32 * len(order))(*[var_ids.get(v, 1023) for v in order])
    keep += [batoms, natoms, carr, ordr]
    return h, batoms, len(pos), natoms, len(neg), carr, len(cmps), ordr, len(order), keep


class Engine:
    """One engine handle (owns all of its device memory)."""

    def __init__(self, device: int = 0, stream=None, arena_bytes: int = 0, flags: int = 0, tile_units: int = 0,
                 use_torch_allocator: bool = False, instances: int = 0, chunk_rows: int = 0, hub_rows: int = 0,
                 frontier_bytes: int = 0, tune_cache: str | None = None, head_percent: int = 0,
                 dense_bytes: int = 0):
        import torch  # plumbing only: stream handle and (optionally) the caching allocator
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the Datalog engine runs only on the GPU")
        torch.cuda.set_device(device)
        cfg = dl_config()
        cfg.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._torch_stream = stream
        cfg.stream = ctypes.c_void_p(stream.cuda_stream)
        cfg.arena_bytes = arena_bytes
        cfg.flags = flags
        cfg.tile_units = tile_units
        cfg.instances = instances
        cfg.chunk_rows = chunk_rows
        cfg.hub_rows = hub_rows
        cfg.frontier_bytes = frontier_bytes
        cfg.head_percent = head_percent
        cfg.dense_bytes = dense_bytes
        self._tune_cache = tune_cache.encode() if tune_cache else None   # kept alive for the engine
        cfg.tune_cache = self._tune_cache
        self.instances = instances
        self._cb = None
        if use_torch_allocator:
            def _alloc(nbytes, strm, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, strm)
                except Exception:
                    return None

            def _free(ptr, nbytes, strm, user):
                torch.cuda.caching_allocator_delete(ptr)
            self._cb = (DL_ALLOC_FN(_alloc), DL_FREE_FN(_free))
            cfg.alloc, cfg.free = self._cb
        h = ctypes.c_void_p()
        rc = self.lib.dl_engine_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_engine_create failed")
        self.h = h
        self.rel_ids: dict = {}
        self.arity: dict = {}
        self.names: list = []

    def _check(self, rc):
        if rc != DL_OK:
            raise DatalogError(rc, self.lib.dl_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.dl_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def relation(self, name: str, arity: int) -> int:
        rid = ctypes.c_uint32()
        self._check(self.lib.dl_relation_create(self.h, name.encode(), arity, ctypes.byref(rid)))
        self.rel_ids[name] = rid.value
        self.arity[name] = arity
        self.names.append(name)
        return rid.value

    def set_sink(self, name: str, sink: int):
        self._check(self.lib.dl_relation_set_sink(self.h, self.rel_ids[name], sink))

    def load(self, name: str, rows):
        """rows: (n, arity) uint32 numpy array on the host, or a torch CUDA tensor of shape (arity, n)."""
        if hasattr(rows, "is_cuda") and rows.is_cuda:
            cols = [rows[c].contiguous() for c in range(rows.shape[0])]
            ptrs = (ctypes.c_void_p * len(cols))(*[c.data_ptr() for c in cols])
            self._check(self.lib.dl_load_facts_device(self.h, self.rel_ids[name], ptrs, cols[0].numel()))
            return
        rows = np.asarray(rows, dtype=np.uint32).reshape(-1, self.arity[name])
        cols = [np.ascontiguousarray(rows[:, c]) for c in range(rows.shape[1])]
        self._check(self.lib.dl_load_facts(self.h, self.rel_ids[name], _cols_ptrs(cols), rows.shape[0]))

    def load_instance(self, name: str, inst: int, rows):
        """Batched form: add (n, arity) uint32 host rows to instance `inst` of a relation."""
        rows = np.asarray(rows, dtype=np.uint32).reshape(-1, self.arity[name])
        cols = [np.ascontiguousarray(rows[:, c]) for c in range(rows.shape[1])]
        self._check(self.lib.dl_load_facts_instance(self.h, self.rel_ids[name], inst, _cols_ptrs(cols), rows.shape[0]))

    def size_instance(self, name: str, inst: int) -> int:
        """Batched form: rows of one instance's relation."""
        n = ctypes.c_uint64()
        self._check(self.lib.dl_fetch_instance(self.h, self.rel_ids[name], inst, None, 0, ctypes.byref(n)))
        return n.value

    def fetch_instance(self, name: str, inst: int) -> np.ndarray:
        n = ctypes.c_uint64()
        rid = self.rel_ids[name]
        self._check(self.lib.dl_fetch_instance(self.h, rid, inst, None, 0, ctypes.byref(n)))
        a = self.arity[name]
        cols = [np.empty(n.value, dtype=np.uint32) for _ in range(a)]
        self._check(self.lib.dl_fetch_instance(self.h, rid, inst, _cols_ptrs(cols), n.value, ctypes.byref(n)))
        return np.stack(cols, axis=1)

    def instance_digest(self, name: str, inst: int) -> tuple:
        """Batched form: (count, sum, xor) digest of one instance's relation (count sinks too)."""
        c = ctypes.c_uint64()
        d = (ctypes.c_uint64 * 2)()
        self._check(self.lib.dl_instance_digest(self.h, self.rel_ids[name], inst, ctypes.byref(c), d))
        return (c.value, d[0], d[1])

    def instance_rounds(self, inst: int) -> list:
        r = (ctypes.c_uint32 * DL_MAX_STRATA)()
        ns = ctypes.c_uint32()
        self._check(self.lib.dl_instance_rounds(self.h, inst, r, DL_MAX_STRATA, ctypes.byref(ns)))
        return list(r[: ns.value])

    def clear(self, name: str):
        self._check(self.lib.dl_relation_clear(self.h, self.rel_ids[name]))

    def _atom(self, atom, var_ids, keep):
        return _encode_atom(self.rel_ids, atom, var_ids, keep)

    def rule(self, head, body, order):
        """Add a rule.  body items: atoms (rel, [terms]), negated atoms ("not", atom) and
        comparisons (op, term, term) with op in < <= > >= != (dl_rule_add_ex)."""
        h, batoms, npos, natoms, nneg, carr, ncmp, ordr, norder, keep = _encode_rule(self.rel_ids, head, body, order)
        rid = ctypes.c_uint32()
        if nneg or ncmp:
            self._check(self.lib.dl_rule_add_ex(self.h, ctypes.byref(h), batoms, npos, natoms, nneg, carr, ncmp, ordr,
                                                norder, ctypes.byref(rid)))
        else:
            self._check(self.lib.dl_rule_add(self.h, ctypes.byref(h), batoms, npos, ordr, norder, ctypes.byref(rid)))
        return rid.value

    def rule_split(self, head, body, order, factored, helper: str):
        """Add a rule split in two (dl_rule_add_split): the body atoms at the positions in
        `factored` go into a helper rule whose head is relation `helper`; returns
        (helper columns as variable names, helper rule id, consumer rule id)."""
        var_ids: dict = {}
        keep: list = []
        batoms = (dl_atom * len(body))()
        for i, b in enumerate(body):
            batoms[i] = self._atom(b, var_ids, keep)
        h = self._atom(head, var_ids, keep)
        ordr = (ctypes.c_uint32 * len(order))(*[var_ids.get(v, 1023) for v in order])
        mask = sum(1 << i for i in set(factored))
        cols = (ctypes.c_uint32 * 8)()
        k = ctypes.c_uint32()
        rc = self.lib.dl_split_columns(ctypes.byref(h), batoms, len(body), ordr, len(order), mask, cols, 8,
                                       ctypes.byref(k))
        hrel, hr, cr = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        self._check(self.lib.dl_rule_add_split(self.h, ctypes.byref(h), batoms, len(body), ordr, len(order), mask,
                                               helper.encode(), ctypes.byref(hrel), ctypes.byref(hr), ctypes.byref(cr)))
        assert rc == DL_OK
        names = {v: n for n, v in var_ids.items()}
        self.rel_ids[helper] = hrel.value
        self.arity[helper] = k.value
        self.names.append(helper)
        return [names[c] for c in cols[: k.value]], hr.value, cr.value

    def fixpoint(self) -> dict:
        st = dl_stats()
        self._check(self.lib.dl_fixpoint(self.h, ctypes.byref(st)))
        out = {f: getattr(st, f) for f, _ in dl_stats._fields_
               if f not in ("rounds", "stratum_first_rel", "kernels", "top", "top_kind")}
        out["top"] = {"kind": KERNEL_KINDS[st.top_kind], "ms": st.top.ms, "alg_bytes": st.top.alg_bytes,
                      "units": st.top.units, "entries": st.top.entries}
        out["rounds"] = list(st.rounds[: min(st.nstrata, DL_MAX_STRATA)])
        out["kernels"] = {k: {"launches": st.kernels[i].launches, "ms": st.kernels[i].ms,
                              "alg_bytes": st.kernels[i].alg_bytes, "units": st.kernels[i].units,
                              "entries": st.kernels[i].entries} for i, k in enumerate(KERNEL_KINDS)}
        return out

    def set_flags(self, flags: int):
        """Replace the engine's DL_FLAG_* flags for its later calls."""
        self._check(self.lib.dl_engine_set_flags(self.h, flags))

    def tune_choices(self) -> list:
        """The autotuner's choices so far: [{key, tile, warp_major, ms}]."""
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            p = os.path.join(td, "tune.txt")
            self.tune_save(p)
            out = []
            for line in open(p):
                k, tile, wm, ms = line.split()
                out.append({"key": k, "tile": int(tile), "warp_major": wm == "1", "ms": float(ms)})
            return out

    def tune_save(self, path: str):
        """Write the autotuner's choices (DL_FLAG_AUTOTUNE) to a text file."""
        self._check(self.lib.dl_tune_save(self.h, path.encode()))

    def strata(self) -> list:
        out = []
        s = 0
        while True:
            rels = (ctypes.c_uint32 * 256)()
            n = ctypes.c_uint32()
            r = ctypes.c_uint32()
            rc = self.lib.dl_stratum_info(self.h, s, rels, 256, ctypes.byref(n), ctypes.byref(r))
            if rc != DL_OK:
                break
            out.append((sorted(self.names[i] for i in rels[: n.value]), r.value))
            s += 1
        return out

    def size(self, name: str) -> int:
        n = ctypes.c_uint64()
        self._check(self.lib.dl_relation_size(self.h, self.rel_ids[name], ctypes.byref(n)))
        return n.value

    def fetch(self, name: str) -> np.ndarray:
        n = ctypes.c_uint64()
        rid = self.rel_ids[name]
        self._check(self.lib.dl_fetch(self.h, rid, None, 0, ctypes.byref(n)))
        a = self.arity[name]
        cols = [np.empty(n.value, dtype=np.uint32) for _ in range(a)]
        self._check(self.lib.dl_fetch(self.h, rid, _cols_ptrs(cols), n.value, ctypes.byref(n)))
        return np.stack(cols, axis=1) if a else np.zeros((0, 0), np.uint32)

    def fetch_into(self, name: str, cols: list) -> int:
        """Fetch into caller-provided host column buffers (e.g. pinned); returns the row count."""
        n = ctypes.c_uint64()
        cap = min(c.size for c in cols)
        self._check(self.lib.dl_fetch(self.h, self.rel_ids[name], _cols_ptrs(cols), cap, ctypes.byref(n)))
        return n.value

    def fetch_device(self, name: str, cols: list) -> int:
        """Fetch into torch CUDA tensors (one per column); returns the row count."""
        n = ctypes.c_uint64()
        ptrs = (ctypes.c_void_p * len(cols))(*[c.data_ptr() for c in cols])
        cap = min(c.numel() for c in cols)
        self._check(self.lib.dl_fetch_device(self.h, self.rel_ids[name], ptrs, cap, ctypes.byref(n)))
        return n.value

    def digest(self, name: str) -> tuple:
        c = ctypes.c_uint64()
        d = (ctypes.c_uint64 * 2)()
        self._check(self.lib.dl_fetch_digest(self.h, self.rel_ids[name], ctypes.byref(c), d))
        return (c.value, d[0], d[1])


class _Borrowed(Engine):
    """A finished request's engine, owned by the server (never destroyed from here)."""

    def __init__(self, lib, h, relations: dict):
        self.lib = lib
        self.h = h
        self.instances = 0
        self.names = list(relations)
        self.rel_ids = {n: i for i, n in enumerate(self.names)}
        self.arity = dict(relations)

    def close(self):
        self.h = None


class Server:
    """Request loop (dl_server_*): submit programs from any thread; results stay on the GPU
    until released."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, max_slots: int = 8, flags: int = 0,
                 default_share: int = 0, grow_retries: int = 0):
        import torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the Datalog server runs only on the GPU")
        cfg = dl_server_config(device, budget_bytes, max_slots, flags, default_share, grow_retries)
        h = ctypes.c_void_p()
        rc = self.lib.dl_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_server_create failed")
        self.h = h
        self.req_relations: dict = {}

    def submit(self, relations: dict, facts: dict, rules: list, sinks: dict | None = None, share: int = 0) -> int:
        names = list(relations)
        rid = {n: i for i, n in enumerate(names)}
        keep = []
        cnames = (ctypes.c_char_p * len(names))(*[n.encode() for n in names])
        arity = (ctypes.c_uint32 * len(names))(*[relations[n] for n in names])
        sink = (ctypes.c_uint32 * len(names))(*[(sinks or {}).get(n, DL_SINK_STORE) for n in names])
        rs = (dl_rule_spec * len(rules))()
        for k, r in enumerate(rules):
            # body items: atoms, negated atoms ("not", atom) and comparisons (op, a, b)
            head, batoms, npos, natoms, nneg, carr, ncmp, order, norder, kp = _encode_rule(rid, r[0], r[1], r[2])
            keep += kp
            rs[k].head, rs[k].body, rs[k].nbody = head, batoms, npos
            rs[k].var_order, rs[k].nvars = order, norder
            rs[k].neg, rs[k].nneg = natoms, nneg
            rs[k].cmps, rs[k].ncmp = carr, ncmp
        fs = (dl_fact_spec * len(facts))()
        for k, (name, rows) in enumerate(facts.items()):
            rows = np.ascontiguousarray(np.asarray(rows, dtype=np.uint32).reshape(-1, relations[name]))
            keep.append(rows)
            fs[k].rel, fs[k].rows, fs[k].nrows = rid[name], rows.ctypes.data_as(_u32p), rows.shape[0]
        req = dl_request(len(names), cnames, arity, sink, len(rules), rs, len(facts), fs, share)
        t = ctypes.c_uint64()
        rc = self.lib.dl_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_server_submit failed")
        self.req_relations[t.value] = dict(relations)
        return t.value

    def poll(self, ticket: int) -> tuple:
        st, status = ctypes.c_int(), ctypes.c_int()
        rc = self.lib.dl_server_poll(self.h, ticket, ctypes.byref(st), ctypes.byref(status))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_server_poll failed")
        return st.value, status.value

    def wait(self, ticket: int) -> int:
        status = ctypes.c_int()
        rc = self.lib.dl_server_wait(self.h, ticket, ctypes.byref(status))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_server_wait failed")
        return status.value

    def result(self, ticket: int) -> Engine:
        e = ctypes.c_void_p()
        rc = self.lib.dl_server_result(self.h, ticket, ctypes.byref(e))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_server_result failed")
        return _Borrowed(self.lib, e, self.req_relations[ticket])

    def release(self, ticket: int):
        rc = self.lib.dl_server_release(self.h, ticket)
        if rc != DL_OK:
            raise DatalogError(rc, "dl_server_release failed")
        self.req_relations.pop(ticket, None)

    def stats(self) -> dict:
        st = dl_server_stats()
        self.lib.dl_server_get_stats(self.h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in dl_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.dl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def split_columns(head, body, order, factored) -> list:
    """The helper columns (variable names) that splitting `factored` out of the rule would
    create (dl_split_columns; host only, no GPU needed).  Raises DatalogError on a bad split."""
    lib = load_library()
    var_ids: dict = {}
    keep: list = []

    def atom(a):
        rel, terms = a
        ts = (dl_term * len(terms))()
        for i, t in enumerate(terms):
            if isinstance(t, str):
                ts[i].kind, ts[i].id = DL_TERM_VAR, var_ids.setdefault(t, len(var_ids))
            else:
                ts[i].kind, ts[i].id = DL_TERM_CONST, int(t)
        keep.append(ts)
        x = dl_atom()
        x.rel, x.arity, x.terms = 0, len(terms), ts
        return x
    batoms = (dl_atom * len(body))()
    for i, b in enumerate(body):
        batoms[i] = atom(b)
    h = atom(head)
    ordr = (ctypes.c_uint32 * len(order))(*[var_ids.get(v, 1023) for v in order])
    cols = (ctypes.c_uint32 * 16)()
    k = ctypes.c_uint32()
    rc = lib.dl_split_columns(ctypes.byref(h), batoms, len(body), ordr, len(order),
                              sum(1 << i for i in set(factored)), cols, 16, ctypes.byref(k))
    if rc != DL_OK:
        raise DatalogError(rc, "dl_split_columns failed")
    names = {v: n for n, v in var_ids.items()}
    return [names[c] for c in cols[: k.value]]


class Program:
    """A program for dl_fixpoint_batch (dl_program_*): relations, rules and host facts; after
    fixpoint_batch its results are read with fetch / digest / strata."""

    def __init__(self, engine: Engine, relations: dict, rules: list, sinks: dict | None = None):
        self.lib = engine.lib
        self.engine = engine
        h = ctypes.c_void_p()
        rc = self.lib.dl_program_create(engine.h, ctypes.byref(h))
        if rc != DL_OK:
            raise DatalogError(rc, "dl_program_create failed")
        self.h = h
        self.rel_ids, self.arity, self.names = {}, {}, list(relations)
        for name, a in relations.items():
            rid = ctypes.c_uint32()
            self._check(self.lib.dl_program_relation(self.h, name.encode(), a, (sinks or {}).get(name, DL_SINK_STORE),
                                                     ctypes.byref(rid)))
            self.rel_ids[name] = rid.value
            self.arity[name] = a
        self.sinks = dict(sinks or {})
        for r in rules:
            h_, batoms, npos, natoms, nneg, carr, ncmp, ordr, norder, keep = _encode_rule(self.rel_ids, r[0], r[1], r[2])
            self._check(self.lib.dl_program_rule(self.h, ctypes.byref(h_), batoms, npos, natoms, nneg, carr, ncmp, ordr,
                                                 norder))

    def _check(self, rc):
        if rc != DL_OK:
            raise DatalogError(rc, self.lib.dl_program_last_error(self.h).decode())

    def load(self, name: str, rows):
        rows = np.asarray(rows, dtype=np.uint32).reshape(-1, self.arity[name])
        cols = [np.ascontiguousarray(rows[:, c]) for c in range(rows.shape[1])]
        self._check(self.lib.dl_program_load_facts(self.h, self.rel_ids[name], _cols_ptrs(cols), rows.shape[0]))

    def fetch(self, name: str) -> np.ndarray:
        n = ctypes.c_uint64()
        rid = self.rel_ids[name]
        self._check(self.lib.dl_program_fetch(self.h, rid, None, 0, ctypes.byref(n)))
        cols = [np.empty(n.value, dtype=np.uint32) for _ in range(self.arity[name])]
        self._check(self.lib.dl_program_fetch(self.h, rid, _cols_ptrs(cols), n.value, ctypes.byref(n)))
        return np.stack(cols, axis=1)

    def digest(self, name: str) -> tuple:
        c = ctypes.c_uint64()
        d = (ctypes.c_uint64 * 2)()
        self._check(self.lib.dl_program_digest(self.h, self.rel_ids[name], ctypes.byref(c), d))
        return (c.value, d[0], d[1])

    def strata(self) -> list:
        r = (ctypes.c_uint32 * DL_MAX_STRATA)()
        ns = ctypes.c_uint32()
        self._check(self.lib.dl_program_rounds(self.h, r, DL_MAX_STRATA, ctypes.byref(ns)))
        out = []
        for s in range(ns.value):
            rels = (ctypes.c_uint32 * 256)()
            n = ctypes.c_uint32()
            self._check(self.lib.dl_program_stratum(self.h, s, rels, 256, ctypes.byref(n)))
            out.append((sorted(self.names[i] for i in rels[: n.value]), r[s]))
        return out

    def result(self) -> dict:
        return {name: (self.digest(name) if self.sinks.get(name) == DL_SINK_COUNT else self.fetch(name))
                for name in self.names}

    def close(self):
        if getattr(self, "h", None):
            self.lib.dl_program_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fixpoint_batch(engine: Engine, programs: list) -> list:
    """Evaluate programs together (dl_fixpoint_batch); returns each program's group stats."""
    arr = (ctypes.c_void_p * len(programs))(*[p.h.value for p in programs])
    st = (dl_stats * len(programs))()
    rc = engine.lib.dl_fixpoint_batch(engine.h, arr, len(programs), st)
    if rc != DL_OK:
        msgs = [p.lib.dl_program_last_error(p.h).decode() for p in programs]
        raise DatalogError(rc, "dl_fixpoint_batch failed: " + next((m for m in msgs if m), ""))
    return [{"rounds": list(s.rounds[: min(s.nstrata, DL_MAX_STRATA)]), "kernel_launches": s.kernel_launches,
             "peak_bytes": s.peak_bytes} for s in st]


def build_program(eng: Engine, relations: dict, rules: list, sinks: dict | None = None):
    for name, a in relations.items():
        eng.relation(name, a)
    for name, s in (sinks or {}).items():
        eng.set_sink(name, s)
    for r in rules:
        eng.rule(r[0], r[1], r[2])


def run_batched(relations: dict, facts_per_instance: list, rules: list, sinks: dict | None = None, **cfg):
    """Evaluate independent instances of one program together (batched form); returns
    (per-instance relations dicts, per-instance [(stratum relation names, rounds)], stats).
    Count sinks give their per-instance (count, sum, xor) digest instead of rows."""
    n = len(facts_per_instance)
    with Engine(instances=n, **cfg) as eng:
        build_program(eng, relations, rules, sinks)
        for i, facts in enumerate(facts_per_instance):
            for name, rows in facts.items():
                if len(rows):
                    eng.load_instance(name, i, rows)
        stats = eng.fixpoint()
        strata = eng.strata()
        outs, rounds = [], []
        for i in range(n):
            outs.append({name: (eng.instance_digest(name, i) if (sinks or {}).get(name) == DL_SINK_COUNT
                                else eng.fetch_instance(name, i)) for name in relations})
            r = eng.instance_rounds(i)
            rounds.append([(rels, r[k]) for k, (rels, _) in enumerate(strata)])
        return outs, rounds, stats


def run_program(relations: dict, facts: dict, rules: list, sinks: dict | None = None, **cfg):
    """Evaluate a program on the GPU; returns (relations dict, strata list, stats dict)."""
    with Engine(**cfg) as eng:
        build_program(eng, relations, rules, sinks)
        for name, rows in facts.items():
            eng.load(name, rows)
        stats = eng.fixpoint()
        out = {}
        for name in relations:
            if (sinks or {}).get(name, DL_SINK_STORE) == DL_SINK_COUNT:
                out[name] = eng.digest(name)
            else:
                out[name] = eng.fetch(name)
        return out, eng.strata(), stats
