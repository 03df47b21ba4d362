/*
 * dl.h -- C ABI of the GB300 semi-naive WCOJ Datalog library (libdlgpu.so).
 *
 * The library evaluates positive Datalog programs (Horn clauses
 * Head(...) <- Body1(...), ..., Bodyn(...), paper Section 2 "Datalog") to their least
 * fixpoint by semi-naive evaluation (Section 2, Delta_{i+1} = pi(Delta_i |x| ...) \ Full),
 * stratum by stratum (Section 2: SCCs of the relation dependency graph, each run to its
 * own fixpoint and then read-only).  Every rule body is joined attribute at a time, a
 * worst-case-optimal join in the sense of Section 2 "Join Processing and Worst-Case
 * Optimal Join": under a variable order (x1..xm) the candidates of x_i are the
 * intersection of the sorted projections of every atom that mentions x_i, restricted by
 * the prefix bound so far.  Relations are flat, lexicographically sorted uint32 column
 * arrays (Section 4, flat SoA storage); join output is allocated by a count pass, a device
 * prefix scan and a write pass (Section 4, imperative 1; Algorithm 1).
 *
 * Conventions for every call:
 *  - Every function returns an int status; DL_OK (0) means success.  On failure the
 *    engine keeps a one-line description, readable through dl_last_error().  No C++
 *    exception crosses this boundary.
 *  - An engine handle is single-threaded: calls on one handle must not overlap.
 *  - Values are uint32.  Row counts, offsets and sizes are uint64.
 *  - Host pointers are only read during the call (the library copies what it keeps);
 *    device pointers returned by the library stay owned by the engine.
 *  - All device work is issued on the engine's stream (dl_config.stream).  Calls that
 *    return host-visible results synchronise that stream before returning.
 */
#ifndef DL_H
#define DL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define DL_OK 0
#define DL_ERR_ARG 1          /* an argument is invalid (bad id, arity mismatch, unsafe rule, ...) */
#define DL_ERR_UNSUPPORTED 2  /* valid Datalog that this GPU path does not evaluate (see dl_rule_add) */
#define DL_ERR_CAPACITY 3     /* the device-memory budget would be exceeded; state is unchanged */
#define DL_ERR_CUDA 4         /* a CUDA runtime call failed; the engine must be destroyed */
#define DL_ERR_TIMEOUT 5      /* reserved: a bounded device-side wait gave up */
#define DL_ERR_STATE 6        /* the call is not valid in the engine's current state */

/* ------------------------------------------------------------------ limits */
#define DL_MAX_ARITY 8        /* columns per relation */
#define DL_MAX_VARS 12        /* distinct variables per rule */
#define DL_MAX_BODY 12        /* atoms per rule body; at most 8 of them may mention one variable */
#define DL_MAX_NEG 4          /* negated atoms per rule (dl_rule_add_ex) */
#define DL_MAX_CMP 8          /* comparisons per rule (dl_rule_add_ex) */
#define DL_MAX_STRATA 64      /* strata reported in dl_stats (more may exist) */

/* dl_config.flags */
#define DL_FLAG_NAIVE_ROOTS 0x1u  /* A/B baseline: one root key per work group, no histogram split
                                     (the naive assignment ablated in Section 7.3) */
#define DL_FLAG_DEBUG_CHECKS 0x2u /* re-verify sortedness/uniqueness of every index after each round */
#define DL_FLAG_PROFILE 0x4u      /* time every kernel launch with CUDA events (dl_stats.kernels) */
#define DL_FLAG_AUTOTUNE 0x8u     /* autotuner: the first time a join level of a given rule and size
                                     bucket (log2 of its work units and of its frontier entries)
                                     runs, its count pass is timed with every candidate tile size
                                     (4096, 16384, 65536 units per CTA) and kernel shape (a thread per
                                     unit, or a warp per entry range), and the fastest is kept for
                                     every later run of that bucket (dl_config.tune_cache keeps the
                                     choices across engines); ignored when dl_config.tile_units is
                                     set.  Results never depend on the choice */
#define DL_FLAG_NO_DENSE_SINK 0x10u /* A/B baseline: rules deriving a relation that has a dense
                                     bitmap (dl_config.dense_bytes) write their rows out, which are
                                     then test-and-set and compacted, instead of the join's last
                                     level test-and-setting them in the bitmap directly (the dense
                                     sink, whose round delta is read back from the bits set since
                                     the previous round).  Results never depend on it */

typedef struct dl_engine dl_engine;
typedef uint32_t dl_rel_id;
typedef uint32_t dl_rule_id;

/* Optional allocator: when alloc is set, every device buffer of the engine comes from
 * alloc(bytes, stream, user) and is returned through free(ptr, bytes, stream, user).
 * Returned pointers must be 256-byte aligned device memory.  NULL from alloc means out of
 * memory (reported as DL_ERR_CAPACITY). */
typedef void* (*dl_alloc_fn)(uint64_t bytes, void* stream, void* user);
typedef void (*dl_free_fn)(void* ptr, uint64_t bytes, void* stream, void* user);

typedef struct dl_config {
    int device;               /* CUDA device ordinal; -1 = the calling thread's current device */
    void* stream;             /* cudaStream_t to issue all work on; NULL = engine-owned stream */
    uint64_t arena_bytes;     /* device-memory budget; 0 = 90% of free memory at creation */
    dl_alloc_fn alloc;        /* optional, see above (both or neither of alloc/free) */
    dl_free_fn free;
    void* alloc_user;
    uint32_t flags;           /* DL_FLAG_* */
    uint32_t tile_units;      /* join work units per CTA tile; 0 = chosen per join level: the
                                 largest power of two in [4096, 2^16] that still leaves eight
                                 waves of resident CTAs */
    uint32_t instances;       /* 0: one program.  N >= 1: batched form, see below */
    uint64_t chunk_rows;      /* a rule's raw output per round above this many rows is written and
                                 reduced (sorted, deduplicated, anti-joined) in chunks of at most
                                 this size; 0 = default (2^30) */
    uint32_t hub_rows;        /* a key with at least this many rows in an index that stays fixed
                                 during dl_fixpoint gets a bitmap of its second-column values, so
                                 that a join probe into its rows that needs no narrowed range is
                                 one bit test; 0 = default (512), UINT32_MAX = never.  Bitmaps
                                 take at most 1 GiB per index and a quarter of the budget left */
    uint64_t frontier_bytes;  /* a join level whose next frontier (the surviving prefixes and
                                 their carried ranges) would take more than this many bytes
                                 processes its input prefixes in slices, each carried through
                                 the remaining levels before the next, so that memory follows
                                 one slice's frontier; 0 = default (a third of the budget left
                                 at that point, at least 64 MiB) */
    uint32_t head_percent;    /* head/body relations (paper Section 4, Merge): during a recursive
                                 stratum's rounds each relation is a large body plus a small head
                                 holding the rows added since the last flush; a round's new rows
                                 are merged into the head only, and the head is merged into the
                                 body (one merge-path pass per index, root offsets rebuilt) once
                                 it exceeds this percentage of the body, and at the stratum's end.
                                 Joins read body and head as one relation.  0 = default (25),
                                 UINT32_MAX = flush only at the stratum's end */
    uint64_t dense_bytes;     /* dense relation bitmaps: during a recursive stratum's rounds, a
                                 relation whose column domains (largest value + 1 per column, over
                                 its rows and all rows the rules can derive) multiply to at most
                                 8 x this many bits gets one bit per possible row; a round's new
                                 rows are then found by one test-and-set per derived row (paper
                                 Section 4, Compute Delta), replacing the probe of the relation's
                                 index and the deduplicating sort.  By default the join sets the
                                 bits itself and the round's delta is read back from them (see
                                 DL_FLAG_NO_DENSE_SINK), which keeps a second copy of the bitmap:
                                 then at most an eighth of the budget left, else a quarter.
                                 0 = default (8 GiB), 1 = never */
    const char* tune_cache;   /* DL_FLAG_AUTOTUNE: text file of tuned choices, read when the
                                 engine is created (if it exists) and rewritten when it is
                                 destroyed or by dl_tune_save; NULL = choices kept in memory */
} dl_config;

/* Batched form (dl_config.instances = N >= 1).  The engine holds N independent instances
 * of one program: every relation and rule is declared once, facts are loaded per instance
 * (dl_load_facts_instance) and results read per instance (dl_fetch_instance,
 * dl_instance_rounds).  One dl_fixpoint call evaluates all instances together, each
 * evaluation stage being one launch over all of them (the instance id is an extra leading
 * join variable shared by every atom, so instances never join with each other and the
 * work histogram balances uneven instances across the GPU).  Results and per-instance round
 * counts equal those of evaluating each instance alone.  In this form relations have at
 * most DL_MAX_ARITY - 1 columns and rules at most DL_MAX_VARS - 1 variables; count sinks
 * count and digest per instance (dl_instance_digest); dl_load_facts*, dl_fetch and
 * dl_fetch_device are not available (DL_ERR_STATE); every
 * relation, summed over its instances, holds fewer than 2^32 rows. */

/* ------------------------------------------------------------------ engine */

/* Create an engine.  cfg may be NULL (all defaults).  *out receives the handle.
 * Errors: DL_ERR_ARG (bad config), DL_ERR_CUDA (no device / context creation failed). */
int dl_engine_create(const dl_config* cfg, dl_engine** out);

/* Replace the engine's DL_FLAG_* flags for its later calls (e.g. switch the autotuner or
 * profiling on between fixpoints).  Errors: DL_ERR_ARG (NULL engine). */
int dl_engine_set_flags(dl_engine* e, uint32_t flags);

/* Destroy an engine and free every device buffer it owns.  NULL is ignored. */
void dl_engine_destroy(dl_engine* e);

/* Description of the last failure on this engine ("" if none).  The string is owned by
 * the engine and valid until its next call. */
const char* dl_last_error(const dl_engine* e);

/* Library version string, e.g. "1.0.0". */
const char* dl_version(void);

/* ---------------------------------------------------------------- relations */

/* Declare a relation of the given arity (1..DL_MAX_ARITY); all columns are uint32
 * (Section 4: flat sorted uint32 columns).  Names are unique per engine.
 * Errors: DL_ERR_ARG (arity out of range, duplicate or empty name), DL_ERR_STATE (after
 * dl_fixpoint has begun using the relation set). */
int dl_relation_create(dl_engine* e, const char* name, uint32_t arity, dl_rel_id* out);

/* Relation sinks.  DL_SINK_STORE (default) materialises the relation.  DL_SINK_COUNT keeps
 * only the number of distinct derived tuples and an order-independent digest of them
 * (dl_fetch_digest); it is for outputs too large to hold (e.g. 4-cliques of a large
 * graph).  A count sink must not appear in any rule body, and must be derived by exactly
 * one rule whose head lists each body variable exactly once (then every binding the join
 * enumerates is a distinct tuple and no deduplication is needed).
 * Errors: DL_ERR_ARG (bad id or sink), DL_ERR_UNSUPPORTED (rules violate the above; checked
 * at dl_fixpoint). */
#define DL_SINK_STORE 0u
#define DL_SINK_COUNT 1u
int dl_relation_set_sink(dl_engine* e, dl_rel_id rel, uint32_t sink);

/* Add facts to a relation from HOST memory.  cols[j] points to nrows uint32 values of
 * column j (column-major, one pointer per column).  Set semantics: duplicates, also
 * against facts already loaded, are dropped (Section 2: relations are sets).  Facts may be
 * loaded into any relation before dl_fixpoint; facts loaded into a derived relation are
 * part of its stratum's first-round delta.  The caller keeps ownership of the buffers.
 * Errors: DL_ERR_ARG (bad id, NULL column with nrows > 0), DL_ERR_CAPACITY, DL_ERR_STATE
 * (the relation is a count sink). */
int dl_load_facts(dl_engine* e, dl_rel_id rel, const uint32_t* const* cols, uint64_t nrows);

/* Same, from one HOST row-major buffer of nrows * arity values. */
int dl_load_facts_rows(dl_engine* e, dl_rel_id rel, const uint32_t* rows, uint64_t nrows);

/* Same, from DEVICE memory (column pointers on the engine's device); the data are copied,
 * the caller keeps ownership.  The copy is ordered on the engine's stream. */
int dl_load_facts_device(dl_engine* e, dl_rel_id rel, const uint32_t* const* dcols, uint64_t nrows);

/* Remove every tuple of a relation (facts and derived tuples).  Rules are kept. */
int dl_relation_clear(dl_engine* e, dl_rel_id rel);

/* ------------------------------------------------------------------- rules */

#define DL_TERM_VAR 0u
#define DL_TERM_CONST 1u
typedef struct dl_term {
    uint32_t kind;            /* DL_TERM_VAR or DL_TERM_CONST */
    uint32_t id;              /* variable id (any uint32 < 1024) or the constant value */
} dl_term;

typedef struct dl_atom {
    dl_rel_id rel;
    uint32_t arity;           /* must equal the relation's arity */
    const dl_term* terms;     /* arity terms */
} dl_atom;

/* Add the rule head <- body[0], ..., body[nbody-1] (Section 2, Horn clause) with the join
 * variable order var_order[0..nvars) (Section 2, WCOJ: "fix a global variable order
 * (x1..xm)"; it fixes the attribute order of the join, not a filter on values).
 * var_order must be a permutation of the distinct body variables.  Every head variable
 * must occur in the body (range restriction).
 * A constant in a body atom, or a variable repeated within one body atom, selects the rows
 * whose column equals it: each such term becomes a fresh variable with two comparisons that
 * make it equal to the constant or to the variable's first occurrence (the fresh variable of
 * a constant leads the variable order, a repeat's follows its variable), so each one takes
 * one of DL_MAX_VARS and two of DL_MAX_CMP (DL_ERR_UNSUPPORTED beyond).  Head constants are
 * allowed.  A count sink's rule takes no body constants or repeats.
 * Errors: DL_ERR_ARG (bad ids, arity mismatch, unsafe head, bad order, nbody == 0 or
 * > DL_MAX_BODY, more than DL_MAX_VARS variables), DL_ERR_UNSUPPORTED, DL_ERR_STATE. */
int dl_rule_add(dl_engine* e, const dl_atom* head, const dl_atom* body, uint32_t nbody,
                const uint32_t* var_order, uint32_t nvars, dl_rule_id* out);

/* Comparison filter "a op b" over unsigned 32-bit values; a and b are variables of the rule
 * or constants (dl_term). */
#define DL_CMP_LT 0u          /* a <  b */
#define DL_CMP_LE 1u          /* a <= b */
#define DL_CMP_NE 2u          /* a != b */
typedef struct dl_cmp {
    uint32_t op;              /* DL_CMP_* */
    dl_term a, b;
} dl_cmp;

/* dl_rule_add with negated atoms and comparisons (stratified negation and comparison
 * filters, the extension listed in Table 1; the paper leaves their semantics open, the
 * reading here): a binding of the positive atoms body[0..nbody) yields the head tuple iff
 * every comparison cmps[0..ncmp) holds and no negated atom neg[0..nneg) has its tuple in
 * its relation.  Every variable of a negated atom or comparison must occur in a positive
 * atom (safety); var_order lists the positive atoms' variables.  A negated relation is
 * read complete: dl_fixpoint stratifies with negated atoms as dependency edges and
 * evaluates a negated relation's stratum first; a negated relation in the head's own
 * recursive component makes dl_fixpoint fail with DL_ERR_UNSUPPORTED (not stratifiable).
 * A filter is applied in the join at the level of its last variable in var_order.
 * GPU path limits: negated atoms take distinct variables only (constants or a repeated
 * variable: DL_ERR_UNSUPPORTED).
 * Errors: as dl_rule_add; DL_ERR_ARG (nneg > DL_MAX_NEG, ncmp > DL_MAX_CMP, bad op, an
 * unbound filter variable, a negated count sink). */
int dl_rule_add_ex(dl_engine* e, const dl_atom* head, const dl_atom* body, uint32_t nbody,
                   const dl_atom* neg, uint32_t nneg, const dl_cmp* cmps, uint32_t ncmp,
                   const uint32_t* var_order, uint32_t nvars, dl_rule_id* out);

/* Helper-relation splitting (Section 5, the CallGraphEdge example): add a rule in two parts.
 * The body atoms selected by `mask` (bit b = body[b]) are factored out into a helper rule
 *     helper_name(c1, ..., ck) <- the selected atoms
 * and the rest becomes the consumer rule
 *     head <- the other atoms, helper_name(c1, ..., ck),
 * where c1..ck are the variables the selected atoms share with the other atoms or the head,
 * in var_order's order (dl_split_columns returns them).  Each part's variable order is
 * var_order restricted to its body's variables.  A new relation helper_name of arity k is
 * created.  The split changes no result: the consumer's bindings are exactly the original
 * rule's, projected through the helper.  It moves skewed inner variables of a deep rule to
 * the top levels of two shallower joins, where the histogram balancing reaches them.  Round
 * counts are unchanged when the selected atoms read only relations of lower strata; when a
 * selected atom is recursive, the helper joins the recursive stratum and derived tuples may
 * take extra rounds.
 * Errors: everything dl_rule_add reports for the unsplit rule; DL_ERR_ARG (mask empty, all
 * atoms, or beyond nbody; empty or duplicate helper_name); DL_ERR_UNSUPPORTED (the selected
 * atoms share no variable with the rest, or k > DL_MAX_ARITY).  On error nothing is added. */
int dl_rule_add_split(dl_engine* e, const dl_atom* head, const dl_atom* body, uint32_t nbody,
                      const uint32_t* var_order, uint32_t nvars, uint64_t mask, const char* helper_name,
                      dl_rel_id* helper_rel, dl_rule_id* helper_rule, dl_rule_id* consumer_rule);

/* The helper columns dl_rule_add_split would create (host only; needs no engine or GPU):
 * *ncols receives k; cols (may be NULL) receives the k variable ids if cap >= k, else
 * DL_ERR_ARG.  Errors as dl_rule_add_split for the mask; the rule itself is not checked. */
int dl_split_columns(const dl_atom* head, const dl_atom* body, uint32_t nbody, const uint32_t* var_order,
                     uint32_t nvars, uint64_t mask, uint32_t* cols, uint32_t cap, uint32_t* ncols);

/* ------------------------------------------------------------------ fixpoint */

/* Kernel kinds reported in dl_stats.kernels (filled when DL_FLAG_PROFILE is set). */
#define DL_K_JOIN_HIST 0      /* per-level work histogram (Algorithm 1, Phase 1) */
#define DL_K_JOIN_COUNT 1     /* count pass (Algorithm 1, Phase 2) */
#define DL_K_JOIN_WRITE 2     /* write pass (Algorithm 1, Phase 3) */
#define DL_K_SCAN 3           /* device prefix scans */
#define DL_K_SORT 4           /* radix-sort histogram + scatter passes (Build Index) */
#define DL_K_DELTA 5          /* dedup + anti-join against the full relation (Compute Delta) */
#define DL_K_MERGE 6          /* merge path (Merge) */
#define DL_K_OTHER 7          /* root offsets, digests, reductions */
#define DL_KERNEL_KINDS 8

typedef struct dl_kernel_stat {
    uint64_t launches;        /* launches of this kind during the call */
    double ms;                /* summed device time (CUDA events on the engine's stream) */
    uint64_t alg_bytes;       /* algorithmic bytes the launches had to move: for a join
                               * count or write pass 4*T + (entry bytes + 9)*F, T being the
                               * candidates examined (each element of the smaller candidate
                               * range, read once) and F the frontier entries, plus
                               * 4*columns*rows written; for a merge 8*arity*(N + |delta|);
                               * for a radix pass 4*n (histogram) or (4 + 8*arity)*n
                               * (scatter); for dedup / anti-join 4*arity*n read (twice for
                               * dedup) plus 4*arity*kept rows written */
    uint64_t units;           /* join passes: candidates of the smallest source of every frontier
                               * entry (T above), summed over the launches */
    uint64_t entries;         /* join passes: frontier entries (F above), summed */
} dl_kernel_stat;

typedef struct dl_stats {
    uint32_t nstrata;                        /* strata evaluated (relations derived by rules) */
    uint32_t rounds[DL_MAX_STRATA];          /* rounds of each stratum, in evaluation order */
    uint32_t stratum_first_rel[DL_MAX_STRATA]; /* smallest relation id of each stratum */
    uint32_t total_rounds;
    uint64_t join_rows;        /* rows written by the join materialize passes (before dedup) */
    uint64_t count_rows;       /* bindings counted into DL_SINK_COUNT relations */
    uint64_t delta_rows;       /* new tuples merged over all rounds */
    uint64_t peak_bytes;       /* peak device bytes held by the engine during the call */
    uint64_t kernel_launches;  /* kernels launched by the call */
    double ms_total;           /* wall time of the call */
    double ms_join;            /* device time of histogram + count + scan + materialize */
    double ms_sort;            /* device time of delta radix sorts */
    double ms_dedup;           /* device time of dedup + anti-join (compute delta) */
    double ms_merge;           /* device time of merges and index rebuilds */
    dl_kernel_stat kernels[DL_KERNEL_KINDS];  /* per kernel kind; zero unless DL_FLAG_PROFILE */
    uint32_t top_kind;         /* DL_FLAG_PROFILE: kind of the single longest launch */
    dl_kernel_stat top;        /* that launch (launches = 1) */
    uint32_t hub_keys;         /* keys given a membership bitmap by the call: index keys with
                                  >= dl_config.hub_rows rows, so that a join probe into them that needs
                                  no narrowed range is one bit test (implementation detail,
                                  reported for tests and tuning) */
    uint32_t join_slices;      /* join levels whose input prefixes were processed in slices
                                  (dl_config.frontier_bytes) */
    uint32_t tuned_levels;     /* DL_FLAG_AUTOTUNE: join levels tuned by this call (new buckets) */
    uint32_t tune_hits;        /* DL_FLAG_AUTOTUNE: join levels that used a cached choice */
    uint32_t head_flushes;     /* heads merged into their bodies (dl_config.head_percent) */
    uint32_t dense_relations;  /* relations given a dense bitmap for their rounds (dl_config.dense_bytes) */
} dl_stats;

/* Evaluate all rules to the least fixpoint (semi-naive, Jacobi rounds: every rule of a
 * round reads the state at the round's start).  Round 1 of a stratum evaluates its
 * non-recursive rules; rounds t >= 2 evaluate one delta variant per recursive body atom;
 * a stratum stops at the first round with an empty delta, and its round count includes
 * that round (a stratum without recursive rules takes 1 round).  stats may be NULL.
 * May be called again after more facts are loaded; it then continues from the current
 * contents (all relations are treated as loaded facts).
 * Errors: DL_ERR_CAPACITY (the budget would be exceeded; relations keep the state of the
 * last completed round), DL_ERR_UNSUPPORTED, DL_ERR_CUDA. */
int dl_fixpoint(dl_engine* e, dl_stats* stats);

/* Stratum details after dl_fixpoint: relation ids of stratum s (ascending) into
 * rels[0..cap), their number in *nrels, and its round count. */
int dl_stratum_info(dl_engine* e, uint32_t s, dl_rel_id* rels, uint32_t cap, uint32_t* nrels,
                    uint32_t* rounds);

/* --------------------------------------------------------------------- fetch */

/* Batched form: add facts to instance `inst` (< dl_config.instances) of a relation from
 * HOST column pointers, as dl_load_facts does for a single program.  Loads are merged into
 * the relation lazily (at the next dl_fixpoint or fetch), so loading many instances costs
 * one sort and merge in total.  Errors: DL_ERR_ARG (bad id or instance), DL_ERR_STATE (not
 * a batched engine), DL_ERR_CAPACITY. */
int dl_load_facts_instance(dl_engine* e, dl_rel_id rel, uint32_t inst, const uint32_t* const* cols,
                           uint64_t nrows);

/* Batched form: copy instance `inst` of a relation to HOST memory, column-major, rows
 * distinct and sorted as dl_fetch does; NULL cols_out returns only *nrows_out. */
int dl_fetch_instance(dl_engine* e, dl_rel_id rel, uint32_t inst, uint32_t* const* cols_out, uint64_t cap_rows,
                      uint64_t* nrows_out);

/* Batched form: count and order-independent digest (as dl_fetch_digest defines it, over the
 * instance's own columns) of one instance's relation; for a count sink, the counts and
 * digests its rule derived for that instance.  Equals dl_fetch_digest of the instance run
 * alone.  Errors: DL_ERR_STATE (not a batched engine), DL_ERR_ARG (bad ids). */
int dl_instance_digest(dl_engine* e, dl_rel_id rel, uint32_t inst, uint64_t* count, uint64_t digest[2]);

/* Batched form, after dl_fixpoint: round count of instance `inst` in each stratum (the
 * count it would have alone, same definition as dl_stats.rounds) into rounds[0..cap);
 * *nstrata receives the number of strata. */
int dl_instance_rounds(dl_engine* e, uint32_t inst, uint32_t* rounds, uint32_t cap, uint32_t* nstrata);

/* Number of tuples currently in a relation (DL_SINK_COUNT: the counted tuples; batched
 * form: summed over instances). */
int dl_relation_size(dl_engine* e, dl_rel_id rel, uint64_t* nrows);

/* Copy a relation to HOST memory, column-major: cols_out[j] receives column j.  Rows are
 * distinct and sorted ascending lexicographically over columns 0..arity-1 (unsigned).
 * Two-call pattern: with cols_out == NULL only *nrows_out is written.  cap_rows is the
 * capacity of each column buffer.
 * Errors: DL_ERR_ARG (cap_rows < size), DL_ERR_STATE (count sink). */
int dl_fetch(dl_engine* e, dl_rel_id rel, uint32_t* const* cols_out, uint64_t cap_rows,
             uint64_t* nrows_out);

/* Same into DEVICE buffers on the engine's device (ordered on the engine's stream). */
int dl_fetch_device(dl_engine* e, dl_rel_id rel, uint32_t* const* dcols_out, uint64_t cap_rows,
                    uint64_t* nrows_out);

/* Order-independent digest of a relation: *count = number of tuples, digest[0] = sum mod
 * 2^64 and digest[1] = xor of a 64-bit hash of every tuple.  Tuple hash: h starts at
 * 0x243F6A8885A308D3; for column j with value v, h = mix(h ^ (v + 0x9E3779B97F4A7C15*(j+1)))
 * where mix is the splitmix64 finaliser.  Works for stored relations and count sinks. */
int dl_fetch_digest(dl_engine* e, dl_rel_id rel, uint64_t* count, uint64_t digest[2]);

/* ------------------------------------------------------------- host helpers */

/* Root-level work partition of Algorithm 2 / Figure 2, the same routine the join kernels
 * run: given the inclusive prefix sums C[0..K) of per-key work, group b of p takes flat
 * units [b*ceil(T/p), min((b+1)*ceil(T/p), T)) with T = C[K-1]; its first key is the first
 * k with C[k] > start.  Writes first_key[b] and start_unit[b] (global unit index) for every
 * b < p.  Host-callable; needs no GPU. */
int dl_partition_slices(const uint64_t* C, uint64_t K, uint32_t p, uint64_t* first_key,
                        uint64_t* start_unit);

/* Decode one flat unit g into (key, i1, i2) with local = g - C[key-1],
 * i1 = local / d2[key], i2 = local % d2[key] (Section 5, the decode formula). Host-callable. */
int dl_decode_unit(const uint64_t* C, const uint64_t* d2, uint64_t K, uint64_t g, uint64_t* key,
                   uint64_t* i1, uint64_t* i2);

/* ---------------------------------------------------------------- serving */

/* A request loop over one GPU: requests (a program plus its facts) are submitted from any
 * thread, admitted in arrival order as soon as a worker slot is free and their device-
 * memory share fits in the server's budget, evaluated on the slot's own CUDA stream (so the
 * work of concurrent requests overlaps on the device, in the spirit of the stream-parallel
 * rule schedule of Section 6), and keep their relations resident on the device until the
 * client releases them.  A request that outgrows its share fails alone with
 * DL_ERR_CAPACITY; others are not disturbed.  With dl_server_config.grow_retries the server
 * instead re-runs it with a doubled share, so callers need not know final sizes up front.  The paper evaluates one program at a time;
 * this loop is an addition for serving many programs. */
typedef struct dl_server dl_server;

typedef struct dl_server_config {
    int device;               /* CUDA device ordinal; -1 = current */
    uint64_t budget_bytes;    /* device memory all admitted requests may hold together; 0 = 90% free */
    uint32_t max_slots;       /* concurrent requests (worker threads / streams); 0 = 8 */
    uint32_t flags;           /* DL_FLAG_* for every request's engine */
    uint64_t default_share;   /* share of a request that states none; 0 = 1 GiB */
    uint32_t grow_retries;    /* final sizes unknown up front: a request that fails with
                                 DL_ERR_CAPACITY is evaluated again from scratch with twice its
                                 share (at most the whole budget), re-queued ahead of later
                                 arrivals, up to this many times; 0 = never (it fails alone) */
} dl_server_config;

typedef struct dl_rule_spec {  /* a rule of a request, as dl_rule_add_ex takes it */
    dl_atom head;
    const dl_atom* body;
    uint32_t nbody;
    const uint32_t* var_order;
    uint32_t nvars;
    const dl_atom* neg;           /* negated atoms (stratified negation), or NULL */
    uint32_t nneg;
    const dl_cmp* cmps;           /* comparisons, or NULL */
    uint32_t ncmp;
} dl_rule_spec;

typedef struct dl_fact_spec {
    dl_rel_id rel;            /* index into the request's relation list */
    const uint32_t* rows;     /* HOST, row-major, nrows * arity values */
    uint64_t nrows;
} dl_fact_spec;

typedef struct dl_request {
    uint32_t nrel;
    const char* const* rel_names;   /* relation i has id i inside the request */
    const uint32_t* rel_arity;
    const uint32_t* rel_sink;       /* DL_SINK_* per relation, or NULL (all stored) */
    uint32_t nrules;
    const dl_rule_spec* rules;
    uint32_t nfacts;
    const dl_fact_spec* facts;
    uint64_t share_bytes;           /* device memory the request may use; 0 = server default */
} dl_request;

#define DL_REQ_QUEUED 0
#define DL_REQ_RUNNING 1
#define DL_REQ_DONE 2

typedef struct dl_server_stats {
    uint64_t submitted, admitted, completed, failed;
    uint64_t reserved_bytes, peak_reserved_bytes;
    uint32_t running, queued;
    uint64_t regrown;         /* re-evaluations with a doubled share (dl_server_config.grow_retries) */
} dl_server_stats;

/* Create / destroy a server (destroy waits for running requests and frees everything). */
int dl_server_create(const dl_server_config* cfg, dl_server** out);
void dl_server_destroy(dl_server* s);

/* Submit a request (thread-safe).  Everything the request points to is copied before the
 * call returns.  *ticket identifies it.  Errors: DL_ERR_ARG (malformed request, share above
 * the whole budget). */
int dl_server_submit(dl_server* s, const dl_request* req, uint64_t* ticket);

/* State of a request: *state = DL_REQ_QUEUED / RUNNING / DONE; once DONE, *status is the
 * dl_* status of its evaluation (thread-safe). */
int dl_server_poll(dl_server* s, uint64_t ticket, int* state, int* status);

/* Block until the request is DONE; *status as in dl_server_poll (thread-safe). */
int dl_server_wait(dl_server* s, uint64_t ticket, int* status);

/* Borrow the finished request's engine (relation ids as in the request) for dl_fetch,
 * dl_fetch_digest, dl_relation_size and dl_stratum_info; valid until dl_server_release.
 * Errors: DL_ERR_STATE (not DONE). */
int dl_server_result(dl_server* s, uint64_t ticket, dl_engine** engine);

/* Free a request's device memory and its ticket (after DONE).  A finished request keeps its
 * share of the budget until it is released, so a client that waits for requests in
 * submission order should release finished ones as it goes, or admission can stall. */
int dl_server_release(dl_server* s, uint64_t ticket);

int dl_server_get_stats(dl_server* s, dl_server_stats* out);

/* ------------------------------------------------------- batches of programs */

/* Programs evaluated in batches (the paper's problem statement, Section 2, for many
 * independent programs at once).  A dl_program describes relations, rules and host facts of
 * one program without touching the device; dl_fixpoint_batch evaluates many programs:
 * programs of the same shape (equal relations, sinks and rules; facts may differ) form a group
 * that runs in the batched form of the engine (see dl_config.instances), so each evaluation
 * stage of a group is one launch over all of its programs; groups run one after another on
 * the engine's stream, with the engine's configuration.  Results and round counts equal
 * those of each program run alone.  A group's results stay in device memory (taken from the
 * engine's budget left when the batch ran) until its last program is destroyed.
 * Relations have at most DL_MAX_ARITY - 1 columns and rules at most DL_MAX_VARS - 1
 * variables.  The rule and relation calls have the semantics of dl_relation_create,
 * dl_relation_set_sink and dl_rule_add_ex; they are checked when the batch runs. */
typedef struct dl_program dl_program;
int dl_program_create(dl_engine* e, dl_program** out);
void dl_program_destroy(dl_program* p);
const char* dl_program_last_error(const dl_program* p);
int dl_program_relation(dl_program* p, const char* name, uint32_t arity, uint32_t sink, dl_rel_id* out);
int dl_program_rule(dl_program* p, const dl_atom* head, const dl_atom* body, uint32_t nbody, const dl_atom* neg,
                    uint32_t nneg, const dl_cmp* cmps, uint32_t ncmp, const uint32_t* var_order, uint32_t nvars);
/* Host facts, copied (cols[j] points to nrows values of column j). */
int dl_program_load_facts(dl_program* p, dl_rel_id rel, const uint32_t* const* cols, uint64_t nrows);
/* Evaluate n programs (all created on e); per_prog (NULL or n entries) receives each program's
 * group's statistics.  Errors: the first failing group's status (its programs keep the text in
 * dl_program_last_error and no result); DL_ERR_ARG (a program of another engine). */
int dl_fixpoint_batch(dl_engine* e, dl_program* const* progs, uint32_t n, dl_stats* per_prog);
/* Results of an evaluated program: rows (as dl_fetch: two-call pattern, sorted columns to
 * HOST buffers), digest (as dl_fetch_digest; count sinks too), rounds per stratum and the
 * relations of each stratum.  DL_ERR_STATE before the program has been evaluated. */
int dl_program_fetch(dl_program* p, dl_rel_id rel, uint32_t* const* cols_out, uint64_t cap_rows, uint64_t* nrows_out);
int dl_program_digest(dl_program* p, dl_rel_id rel, uint64_t* count, uint64_t digest[2]);
int dl_program_rounds(dl_program* p, uint32_t* rounds, uint32_t cap, uint32_t* nstrata);
int dl_program_stratum(dl_program* p, uint32_t s, dl_rel_id* rels, uint32_t cap, uint32_t* nrels);

/* Write the autotuner's choices (DL_FLAG_AUTOTUNE) to a text file, one per line: the key
 * (rule shape hash, level, log2 of units and entries, sources, filters), the tile size, the
 * kernel shape (1 = a warp per entry range) and the count pass's time in ms when chosen.
 * Errors: DL_ERR_ARG (NULL path), DL_ERR_STATE (the file cannot be written). */
int dl_tune_save(dl_engine* e, const char* path);

/* ------------------------------------------------- allocation-free sort + dedup */

/* The paper has no counterpart to this call.  It serves callers that must not allocate
 * device memory while they run: for example a plugin inside a host application whose own
 * allocator owns the whole device budget (an extra cudaMalloc would fail or fragment it), or
 * a latency-bound service loop where cudaMalloc/cudaFree are banned because they can stall
 * or synchronise the device.  Such callers cannot create an engine per request, so this
 * call performs the library's sort + deduplicate step on their own buffers instead.
 *
 * It reads nrows rows from the DEVICE columns dcols_in[0..arity) (a host array of device
 * pointers, one column each) and writes the distinct rows, sorted ascending
 * lexicographically over columns 0..arity-1 (unsigned), to the DEVICE columns
 * dcols_out[0..arity), each of which must hold nrows values; *nrows_out (host) receives the
 * number of distinct rows.  The result equals what dl_load_facts_device followed by
 * dl_fetch_device returns for an empty relation of that arity.  Inputs are not modified.
 * Work is issued on `stream` (a cudaStream_t; NULL = the default stream).  The call reads
 * the number of distinct rows back to the host, so it waits for `stream` to finish before it
 * returns.  A launch error still pending on the calling thread from earlier work is cleared
 * at entry, so that DL_ERR_CUDA reports only this call's own failures.
 *
 * Memory: no allocation at all.  Scratch is one fixed static device array of about 8.1 MiB
 * (two DL_NOALLOC_MAX_ARITY x DL_NOALLOC_MAX_ROWS uint32 buffers plus counters), which every
 * GPU that loads the library's device code holds until the process exits.
 * Limits: arity 1..DL_NOALLOC_MAX_ARITY, nrows <= DL_NOALLOC_MAX_ROWS; larger inputs are
 * rejected with DL_ERR_CAPACITY before any work is issued.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for later calls.
 * Sharing: all calls on a device use the same array, which keeps the previous call's
 * contents (every counter the call reads is rewritten by the call first).  Calls whose
 * work overlaps on the GPU -- on different streams or threads without ordering between
 * them -- race on the array and corrupt each other's results; order such calls.
 * Errors: DL_ERR_ARG (NULL pointers, arity 0), DL_ERR_CAPACITY (limits above), DL_ERR_CUDA. */
#define DL_NOALLOC_MAX_ROWS 262144u
#define DL_NOALLOC_MAX_ARITY 4u
int dl_sort_unique_noalloc(const uint32_t* const* dcols_in, uint32_t arity, uint64_t nrows,
                           uint32_t* const* dcols_out, uint64_t* nrows_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DL_H */
