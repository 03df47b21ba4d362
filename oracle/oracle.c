/*
 * Oracle: a plain, slow, obviously-correct CPU evaluator of Datalog with stratified
 * negation and comparison filters.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or helper with the
 * GPU library; the two meet only at the seeded fact arrays the tests hand to both.
 *
 * What it computes (paper Section 2, "Datalog"): the least model of a set of Horn
 * clauses Head <- Body1,...,Bodyn over finite uint32 relations, evaluated stratum by
 * stratum (relation dependency graph -> strongly connected components, each SCC run
 * to its own fixpoint and then frozen).  Shared variables are equality constraints;
 * constants and a variable repeated inside one atom act as filters.
 *
 * Negation and comparisons (the extension the paper lists in Table 1 and leaves
 * unspecified; the reading used here): a rule may carry negated atoms "not R(...)" and
 * comparisons "a < b", "a <= b", "a != b" between variables or constants (unsigned 32-bit
 * order).  Every variable of a negated atom or comparison must occur in a positive body
 * atom (safety).  A binding of the positive atoms yields the head tuple iff every
 * comparison holds and no negated atom's tuple is present.  A negated relation must be
 * complete before the rule runs: the program is stratified with negated atoms as
 * dependency edges, and a negated relation in the head's own component is an error (not
 * stratifiable).  Negated relations are read in full in every round.
 *
 * Three evaluators:
 *  - ORC_SEMINAIVE: semi-naive evaluation (Section 2, the differential rule
 *    Delta_{i+1} = pi(Delta_i |x| ...) \ Full).  Jacobi rounds: every rule of a round
 *    reads the state at the start of the round.  For a recursive rule each body
 *    position j whose relation is in the stratum yields one variant in which atom j
 *    reads the previous round's delta and every other atom reads the full relation
 *    (which already contains that delta).  Join per variant: left-deep, in body order,
 *    index nested loops over a hash index on the columns already bound.  This is the
 *    binary-join pipeline of Section 2/3, deliberately not the WCOJ under test.
 *  - ORC_NAIVE_STRATA: naive iteration I_t = I_{t-1} U T_P(I_{t-1}) per stratum,
 *    where T_P is computed by brute force: every assignment of the rule's variables
 *    over the active domain is tried and kept if every body tuple is present.
 *  - ORC_NAIVE_GLOBAL: the same brute-force T_P iterated over all rules at once, with
 *    no stratification at all (the least model of a positive program does not depend
 *    on stratification).  Refused for programs with negation, whose meaning needs the
 *    strata.
 *
 * Comparisons are checked in the nested loops as soon as all their variables are bound
 * (and once more on the complete binding): a conjunction holds whatever order its terms are
 * checked in, so this prunes work without changing which bindings pass.
 *
 * Count sinks (outputs too large to store, e.g. the 4-clique relation of a large graph): a
 * relation marked with orc_set_count_sink keeps no tuples; every derived tuple instead adds
 * to the relation's count and to its order-independent digest (sum mod 2^64 and xor of a
 * 64-bit row hash; the row hash is h = 0x243F6A8885A308D3 and, for column j with value v,
 * h = mix(h ^ (v + 0x9E3779B97F4A7C15 * (j + 1))), mix being the splitmix64 finaliser).
 * This equals the digest of the stored relation only when every binding yields a distinct
 * tuple, so a count sink must be the head of exactly one rule, whose head lists each of the
 * rule's variables exactly once, and must appear in no body; orc_run checks this.
 *
 * Readings of points the paper leaves open (each stated again where used):
 *  - Rounds of a stratum: round 1 evaluates the non-recursive rules of the stratum;
 *    the facts loaded into the stratum's relations join round 1's delta; round t >= 2
 *    evaluates the delta variants; the count stops at the first round whose delta is
 *    empty and includes that round.  A stratum without recursive rules takes 1 round.
 *  - Results are sets: duplicate facts are dropped; output rows are sorted ascending,
 *    lexicographically over columns 0..arity-1, as unsigned 32-bit values.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define ORC_MAX_ARITY 8
#define ORC_MAX_VARS 16
#define ORC_MAX_BODY 16
#define ORC_MAX_NEG 8
#define ORC_MAX_CMP 16

enum { ORC_SEMINAIVE = 0, ORC_NAIVE_STRATA = 1, ORC_NAIVE_GLOBAL = 2 };
enum { T_VAR = 0, T_CONST = 1 };
enum { CMP_LT = 0, CMP_LE = 1, CMP_NE = 2 };

/* ------------------------------------------------------------------ tables */

typedef struct {
    uint32_t arity;
    uint64_t n, cap;
    uint32_t* rows;      /* row-major, n * arity */
    uint64_t* slots;     /* open-addressing set: row index + 1, 0 = empty */
    uint64_t nslots;
} table;

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t hash_vals(const uint32_t* v, uint32_t k) {
    uint64_t h = 0x243F6A8885A308D3ULL;
    for (uint32_t i = 0; i < k; i++) h = mix64(h ^ ((uint64_t)v[i] + 0x9E3779B97F4A7C15ULL * (i + 1)));
    return h;
}

static void* xmalloc(size_t n) {
    void* p = malloc(n ? n : 1);
    if (!p) { fprintf(stderr, "oracle: out of host memory (%zu bytes)\n", n); abort(); }
    return p;
}

static void* xcalloc(size_t n, size_t s) {
    void* p = calloc(n ? n : 1, s ? s : 1);
    if (!p) { fprintf(stderr, "oracle: out of host memory\n"); abort(); }
    return p;
}

static void table_init(table* t, uint32_t arity) {
    memset(t, 0, sizeof(*t));
    t->arity = arity;
}

static void table_free(table* t) {
    free(t->rows);
    free(t->slots);
    memset(t, 0, sizeof(*t));
}

static void table_clear(table* t) {
    uint32_t a = t->arity;
    table_free(t);
    table_init(t, a);
}

static const uint32_t* row_at(const table* t, uint64_t i) { return t->rows + i * t->arity; }

static void set_rehash(table* t, uint64_t nslots) {
    free(t->slots);
    t->slots = (uint64_t*)xcalloc(nslots, sizeof(uint64_t));
    t->nslots = nslots;
    for (uint64_t i = 0; i < t->n; i++) {
        uint64_t h = hash_vals(row_at(t, i), t->arity) & (nslots - 1);
        while (t->slots[h]) h = (h + 1) & (nslots - 1);
        t->slots[h] = i + 1;
    }
}

static int table_contains(const table* t, const uint32_t* v) {
    if (!t->nslots) return 0;
    uint64_t h = hash_vals(v, t->arity) & (t->nslots - 1);
    while (t->slots[h]) {
        if (memcmp(row_at(t, t->slots[h] - 1), v, t->arity * sizeof(uint32_t)) == 0) return 1;
        h = (h + 1) & (t->nslots - 1);
    }
    return 0;
}

/* Insert a tuple; returns 1 if it was new. */
static int table_insert(table* t, const uint32_t* v) {
    if ((t->n + 1) * 2 > t->nslots) set_rehash(t, t->nslots ? t->nslots * 2 : 64);
    uint64_t h = hash_vals(v, t->arity) & (t->nslots - 1);
    while (t->slots[h]) {
        if (memcmp(row_at(t, t->slots[h] - 1), v, t->arity * sizeof(uint32_t)) == 0) return 0;
        h = (h + 1) & (t->nslots - 1);
    }
    if (t->n == t->cap) {
        t->cap = t->cap ? t->cap * 2 : 64;
        uint32_t* r = (uint32_t*)xmalloc(t->cap * (t->arity ? t->arity : 1) * sizeof(uint32_t));
        if (t->n) memcpy(r, t->rows, t->n * t->arity * sizeof(uint32_t));
        free(t->rows);
        t->rows = r;
    }
    memcpy(t->rows + t->n * t->arity, v, t->arity * sizeof(uint32_t));
    t->slots[h] = ++t->n;
    return 1;
}

/* ------------------------------------------------------------------ program */

typedef struct { uint32_t kind, val; } term;
typedef struct { int32_t rel; uint32_t arity; term t[ORC_MAX_ARITY]; } atom;
typedef struct { uint32_t op; term a, b; } comparison;
typedef struct {
    atom head;
    uint32_t nbody;
    atom body[ORC_MAX_BODY];
    uint32_t nneg;
    atom neg[ORC_MAX_NEG];          /* negated atoms */
    uint32_t ncmp;
    comparison cmp[ORC_MAX_CMP];
    uint32_t nvars;                 /* variables are renumbered 0..nvars-1 */
} rule;

typedef struct {
    uint32_t nrel;
    uint32_t* arity;
    table* full;                    /* current contents (facts + derived) */
    table* delta;
    table* fresh;                   /* per-round collector */
    uint32_t nrule, caprule;
    rule* rules;
    /* stratification result */
    uint32_t nstrata;
    uint32_t* stratum_of_rel;       /* UINT32_MAX for relations not in any stratum */
    uint32_t* strata_rels;          /* relations of stratum s at [strata_off[s], strata_off[s+1]) */
    uint32_t* strata_off;
    uint32_t* rounds;
    uint8_t* sink;                  /* 1: count sink (count + digest, no tuples kept) */
    uint64_t* sink_acc;             /* per relation: count, sum, xor of the row hashes */
    double join_seconds;            /* time spent in the nested loops (index builds excluded) */
    char err[256];
} program;

static int fail(program* p, const char* msg) {
    snprintf(p->err, sizeof(p->err), "%s", msg);
    return -1;
}

void* orc_create(void) {
    program* p = (program*)xcalloc(1, sizeof(program));
    return p;
}

static void free_strata(program* p) {
    free(p->stratum_of_rel); free(p->strata_rels); free(p->strata_off); free(p->rounds);
    p->stratum_of_rel = p->strata_rels = p->strata_off = p->rounds = NULL;
    p->nstrata = 0;
}

void orc_destroy(void* h) {
    program* p = (program*)h;
    if (!p) return;
    for (uint32_t r = 0; r < p->nrel; r++) {
        table_free(&p->full[r]); table_free(&p->delta[r]); table_free(&p->fresh[r]);
    }
    free(p->full); free(p->delta); free(p->fresh); free(p->arity); free(p->rules);
    free(p->sink); free(p->sink_acc);
    free_strata(p);
    free(p);
}

const char* orc_error(void* h) { return ((program*)h)->err; }

int orc_relation(void* h, uint32_t arity) {
    program* p = (program*)h;
    if (arity < 1 || arity > ORC_MAX_ARITY) return fail(p, "arity out of range");
    uint32_t r = p->nrel++;
    p->arity = (uint32_t*)realloc(p->arity, p->nrel * sizeof(uint32_t));
    p->full = (table*)realloc(p->full, p->nrel * sizeof(table));
    p->delta = (table*)realloc(p->delta, p->nrel * sizeof(table));
    p->fresh = (table*)realloc(p->fresh, p->nrel * sizeof(table));
    p->sink = (uint8_t*)realloc(p->sink, p->nrel);
    p->sink_acc = (uint64_t*)realloc(p->sink_acc, p->nrel * 3 * sizeof(uint64_t));
    p->sink[r] = 0;
    p->sink_acc[3 * r] = p->sink_acc[3 * r + 1] = p->sink_acc[3 * r + 2] = 0;
    p->arity[r] = arity;
    table_init(&p->full[r], arity);
    table_init(&p->delta[r], arity);
    table_init(&p->fresh[r], arity);
    return (int)r;
}

/* Mark a relation as a count sink (see the header comment). */
int orc_set_count_sink(void* h, int rel) {
    program* p = (program*)h;
    if (rel < 0 || (uint32_t)rel >= p->nrel) return fail(p, "bad relation");
    if (p->full[rel].n) return fail(p, "a count sink holds no facts");
    p->sink[rel] = 1;
    return 0;
}

/* Count and digest (sum, xor) of a count sink after orc_run. */
int orc_sink_digest(void* h, int rel, uint64_t* out3) {
    program* p = (program*)h;
    if (rel < 0 || (uint32_t)rel >= p->nrel || !p->sink[rel]) return fail(p, "not a count sink");
    memcpy(out3, p->sink_acc + 3 * rel, 3 * sizeof(uint64_t));
    return 0;
}

double orc_join_seconds(void* h) { return ((program*)h)->join_seconds; }

int orc_add_facts(void* h, int rel, const uint32_t* rows, uint64_t n) {
    program* p = (program*)h;
    if (rel < 0 || (uint32_t)rel >= p->nrel) return fail(p, "bad relation");
    if (p->sink[rel] && n) return fail(p, "a count sink holds no facts");
    for (uint64_t i = 0; i < n; i++) table_insert(&p->full[rel], rows + i * p->arity[rel]);
    return 0;
}

static int read_atom(program* p, atom* a, int32_t rel, const uint32_t* kinds, const uint32_t* vals,
                     uint32_t* var_map, uint32_t* nvars) {
    if (rel < 0 || (uint32_t)rel >= p->nrel) return fail(p, "bad relation in rule");
    a->rel = rel;
    a->arity = p->arity[rel];
    for (uint32_t c = 0; c < a->arity; c++) {
        if (kinds[c] == T_CONST) { a->t[c].kind = T_CONST; a->t[c].val = vals[c]; continue; }
        if (kinds[c] != T_VAR) return fail(p, "bad term kind");
        if (vals[c] >= 1024) return fail(p, "variable id too large");
        if (var_map[vals[c]] == UINT32_MAX) {
            if (*nvars >= ORC_MAX_VARS) return fail(p, "too many variables");
            var_map[vals[c]] = (*nvars)++;
        }
        a->t[c].kind = T_VAR;
        a->t[c].val = var_map[vals[c]];
    }
    return 0;
}

/* body_kinds / body_vals hold the terms of all body atoms back to back; the same for the
 * negated atoms.  Comparison c is "term 2c  op[c]  term 2c+1" over cmp_kinds / cmp_vals. */
int orc_add_rule_ex(void* h, int head_rel, const uint32_t* head_kinds, const uint32_t* head_vals,
                    uint32_t nbody, const int32_t* body_rels, const uint32_t* body_kinds,
                    const uint32_t* body_vals, uint32_t nneg, const int32_t* neg_rels,
                    const uint32_t* neg_kinds, const uint32_t* neg_vals, uint32_t ncmp,
                    const uint32_t* cmp_ops, const uint32_t* cmp_kinds, const uint32_t* cmp_vals) {
    program* p = (program*)h;
    if (nbody < 1 || nbody > ORC_MAX_BODY) return fail(p, "body size out of range");
    if (nneg > ORC_MAX_NEG || ncmp > ORC_MAX_CMP) return fail(p, "too many negated atoms or comparisons");
    rule r;
    memset(&r, 0, sizeof(r));
    uint32_t var_map[1024];
    for (int i = 0; i < 1024; i++) var_map[i] = UINT32_MAX;
    uint32_t nv = 0, off = 0;
    for (uint32_t b = 0; b < nbody; b++) {
        if (body_rels[b] < 0 || (uint32_t)body_rels[b] >= p->nrel) return fail(p, "bad relation in rule");
        if (read_atom(p, &r.body[b], body_rels[b], body_kinds + off, body_vals + off, var_map, &nv)) return -1;
        off += p->arity[body_rels[b]];
    }
    uint32_t nbody_vars = nv;
    off = 0;
    for (uint32_t b = 0; b < nneg; b++) {
        if (neg_rels[b] < 0 || (uint32_t)neg_rels[b] >= p->nrel) return fail(p, "bad relation in rule");
        if (read_atom(p, &r.neg[b], neg_rels[b], neg_kinds + off, neg_vals + off, var_map, &nv)) return -1;
        off += p->arity[neg_rels[b]];
    }
    for (uint32_t c = 0; c < ncmp; c++) {
        if (cmp_ops[c] > CMP_NE) return fail(p, "bad comparison");
        r.cmp[c].op = cmp_ops[c];
        term* t[2] = {&r.cmp[c].a, &r.cmp[c].b};
        for (int s = 0; s < 2; s++) {
            const uint32_t k = cmp_kinds[2 * c + s], v = cmp_vals[2 * c + s];
            if (k == T_CONST) { t[s]->kind = T_CONST; t[s]->val = v; continue; }
            if (k != T_VAR || v >= 1024) return fail(p, "bad term in comparison");
            if (var_map[v] == UINT32_MAX) return fail(p, "comparison variable not bound by a positive atom");
            t[s]->kind = T_VAR;
            t[s]->val = var_map[v];
        }
    }
    if (nv != nbody_vars) return fail(p, "negated atom variable not bound by a positive atom");
    if (read_atom(p, &r.head, head_rel, head_kinds, head_vals, var_map, &nv)) return -1;
    if (nv != nbody_vars) return fail(p, "head variable not bound by the body");
    r.nbody = nbody;
    r.nneg = nneg;
    r.ncmp = ncmp;
    r.nvars = nv;
    if (p->nrule == p->caprule) {
        p->caprule = p->caprule ? p->caprule * 2 : 8;
        p->rules = (rule*)realloc(p->rules, p->caprule * sizeof(rule));
    }
    p->rules[p->nrule++] = r;
    return (int)(p->nrule - 1);
}

int orc_add_rule(void* h, int head_rel, const uint32_t* head_kinds, const uint32_t* head_vals,
                 uint32_t nbody, const int32_t* body_rels, const uint32_t* body_kinds,
                 const uint32_t* body_vals) {
    return orc_add_rule_ex(h, head_rel, head_kinds, head_vals, nbody, body_rels, body_kinds, body_vals, 0, NULL,
                           NULL, NULL, 0, NULL, NULL, NULL);
}

/* The rule's filters for one binding of its variables: every comparison holds and no
 * negated atom's tuple is in its (complete, lower-stratum) relation. */
static int filters_hold(const program* p, const rule* r, const uint32_t* vals) {
    for (uint32_t c = 0; c < r->ncmp; c++) {
        const comparison* q = &r->cmp[c];
        const uint32_t a = q->a.kind == T_CONST ? q->a.val : vals[q->a.val];
        const uint32_t b = q->b.kind == T_CONST ? q->b.val : vals[q->b.val];
        if (q->op == CMP_LT && !(a < b)) return 0;
        if (q->op == CMP_LE && !(a <= b)) return 0;
        if (q->op == CMP_NE && !(a != b)) return 0;
    }
    for (uint32_t n = 0; n < r->nneg; n++) {
        const atom* a = &r->neg[n];
        uint32_t tup[ORC_MAX_ARITY];
        for (uint32_t c = 0; c < a->arity; c++) tup[c] = a->t[c].kind == T_CONST ? a->t[c].val : vals[a->t[c].val];
        if (table_contains(&p->full[a->rel], tup)) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------ stratification */

/* Tarjan's strongly connected components over relations, edge body rel -> head rel. */
typedef struct {
    uint32_t n, *adj_off, *adj, *index, *low, *stack, *comp;
    uint8_t* on;
    uint32_t next_index, sp, ncomp;
} tarjan_state;

static void tarjan_visit(tarjan_state* s, uint32_t v) {
    s->index[v] = s->low[v] = s->next_index++;
    s->stack[s->sp++] = v;
    s->on[v] = 1;
    for (uint32_t e = s->adj_off[v]; e < s->adj_off[v + 1]; e++) {
        uint32_t w = s->adj[e];
        if (s->index[w] == UINT32_MAX) {
            tarjan_visit(s, w);
            if (s->low[w] < s->low[v]) s->low[v] = s->low[w];
        } else if (s->on[w] && s->index[w] < s->low[v]) {
            s->low[v] = s->index[w];
        }
    }
    if (s->low[v] == s->index[v]) {
        uint32_t w;
        do { w = s->stack[--s->sp]; s->on[w] = 0; s->comp[w] = s->ncomp; } while (w != v);
        s->ncomp++;
    }
}

static int stratify(program* p) {
    free_strata(p);
    uint32_t n = p->nrel;
    tarjan_state s;
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.adj_off = (uint32_t*)xcalloc(n + 1, sizeof(uint32_t));
    uint32_t ne = 0;
    for (uint32_t i = 0; i < p->nrule; i++) ne += p->rules[i].nbody + p->rules[i].nneg;
    s.adj = (uint32_t*)xcalloc(ne, sizeof(uint32_t));
    for (uint32_t i = 0; i < p->nrule; i++) {
        for (uint32_t b = 0; b < p->rules[i].nbody; b++) s.adj_off[p->rules[i].body[b].rel + 1]++;
        for (uint32_t b = 0; b < p->rules[i].nneg; b++) s.adj_off[p->rules[i].neg[b].rel + 1]++;
    }
    for (uint32_t v = 0; v < n; v++) s.adj_off[v + 1] += s.adj_off[v];
    uint32_t* fill = (uint32_t*)xcalloc(n, sizeof(uint32_t));
    for (uint32_t i = 0; i < p->nrule; i++)
        for (uint32_t b = 0; b < p->rules[i].nbody + p->rules[i].nneg; b++) {
            const atom* a = b < p->rules[i].nbody ? &p->rules[i].body[b] : &p->rules[i].neg[b - p->rules[i].nbody];
            uint32_t u = (uint32_t)a->rel;
            s.adj[s.adj_off[u] + fill[u]++] = (uint32_t)p->rules[i].head.rel;
        }
    s.index = (uint32_t*)xmalloc(n * sizeof(uint32_t));
    s.low = (uint32_t*)xmalloc(n * sizeof(uint32_t));
    s.stack = (uint32_t*)xmalloc(n * sizeof(uint32_t));
    s.comp = (uint32_t*)xmalloc(n * sizeof(uint32_t));
    s.on = (uint8_t*)xcalloc(n, 1);
    for (uint32_t v = 0; v < n; v++) s.index[v] = UINT32_MAX;
    for (uint32_t v = 0; v < n; v++) if (s.index[v] == UINT32_MAX) tarjan_visit(&s, v);

    /* Topological order of the components (Kahn), ties broken by smallest relation id. */
    uint32_t nc = s.ncomp;
    uint32_t* minrel = (uint32_t*)xmalloc(nc * sizeof(uint32_t));
    uint32_t* indeg = (uint32_t*)xcalloc(nc, sizeof(uint32_t));
    uint8_t* has_rule = (uint8_t*)xcalloc(nc, 1);
    uint8_t* done = (uint8_t*)xcalloc(nc, 1);
    for (uint32_t c = 0; c < nc; c++) minrel[c] = UINT32_MAX;
    for (uint32_t v = 0; v < n; v++) if (v < minrel[s.comp[v]]) minrel[s.comp[v]] = v;
    for (uint32_t i = 0; i < p->nrule; i++) has_rule[s.comp[p->rules[i].head.rel]] = 1;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t e = s.adj_off[u]; e < s.adj_off[u + 1]; e++)
            if (s.comp[u] != s.comp[s.adj[e]]) indeg[s.comp[s.adj[e]]]++;
    uint32_t* order = (uint32_t*)xmalloc(nc * sizeof(uint32_t));
    for (uint32_t k = 0; k < nc; k++) {
        uint32_t best = UINT32_MAX;
        for (uint32_t c = 0; c < nc; c++)
            if (!done[c] && indeg[c] == 0 && (best == UINT32_MAX || minrel[c] < minrel[best])) best = c;
        done[best] = 1;
        order[k] = best;
        for (uint32_t u = 0; u < n; u++)
            if (s.comp[u] == best)
                for (uint32_t e = s.adj_off[u]; e < s.adj_off[u + 1]; e++)
                    if (s.comp[s.adj[e]] != best) indeg[s.comp[s.adj[e]]]--;
    }
    p->stratum_of_rel = (uint32_t*)xmalloc(n * sizeof(uint32_t));
    for (uint32_t v = 0; v < n; v++) p->stratum_of_rel[v] = UINT32_MAX;
    p->strata_off = (uint32_t*)xcalloc(nc + 1, sizeof(uint32_t));
    p->strata_rels = (uint32_t*)xcalloc(n, sizeof(uint32_t));
    uint32_t ns = 0, nr = 0;
    for (uint32_t k = 0; k < nc; k++) {
        uint32_t c = order[k];
        if (!has_rule[c]) continue;
        p->strata_off[ns] = nr;
        for (uint32_t v = 0; v < n; v++)
            if (s.comp[v] == c) { p->strata_rels[nr++] = v; p->stratum_of_rel[v] = ns; }
        ns++;
    }
    p->strata_off[ns] = nr;
    p->nstrata = ns;
    p->rounds = (uint32_t*)xcalloc(ns ? ns : 1, sizeof(uint32_t));
    int stratifiable = 1;
    for (uint32_t i = 0; i < p->nrule; i++)
        for (uint32_t b = 0; b < p->rules[i].nneg; b++)
            if (s.comp[p->rules[i].neg[b].rel] == s.comp[p->rules[i].head.rel]) stratifiable = 0;
    free(s.adj_off); free(s.adj); free(fill); free(s.index); free(s.low); free(s.stack);
    free(s.comp); free(s.on); free(minrel); free(indeg); free(has_rule); free(done); free(order);
    return stratifiable ? 0 : fail(p, "negation inside a recursive component: the program is not stratifiable");
}

/* ------------------------------------------------- hash-indexed nested loops */

typedef struct {
    const table* t;
    uint32_t ncols, cols[ORC_MAX_ARITY];    /* the columns the key is made of */
    uint64_t nb;
    int64_t* head;
    int64_t* next;
} hindex;

static void hindex_build(hindex* x, const table* t, const uint32_t* cols, uint32_t ncols) {
    x->t = t;
    x->ncols = ncols;
    memcpy(x->cols, cols, ncols * sizeof(uint32_t));
    x->nb = 64;
    while (x->nb < t->n * 2) x->nb <<= 1;
    x->head = (int64_t*)xmalloc(x->nb * sizeof(int64_t));
    x->next = (int64_t*)xmalloc((t->n ? t->n : 1) * sizeof(int64_t));
    for (uint64_t b = 0; b < x->nb; b++) x->head[b] = -1;
    uint32_t key[ORC_MAX_ARITY];
    /* insert in reverse so that each chain lists rows in ascending row order */
    for (uint64_t i = t->n; i-- > 0;) {
        const uint32_t* r = row_at(t, i);
        for (uint32_t k = 0; k < ncols; k++) key[k] = r[cols[k]];
        uint64_t h = hash_vals(key, ncols) & (x->nb - 1);
        x->next[i] = x->head[h];
        x->head[h] = (int64_t)i;
    }
}

static void hindex_free(hindex* x) { free(x->head); free(x->next); }

typedef struct {
    program* p;
    const rule* r;
    const table* src[ORC_MAX_BODY];           /* table each body atom reads */
    hindex idx[ORC_MAX_BODY];
    uint32_t bound_at[ORC_MAX_BODY][ORC_MAX_ARITY];  /* 1 if column is a lookup key */
    uint32_t vals[ORC_MAX_VARS];
    uint32_t ncheck[ORC_MAX_BODY];                   /* comparisons first fully bound at atom k */
    uint32_t check[ORC_MAX_BODY][ORC_MAX_CMP];
    table* out;
    uint64_t* sink_acc;                              /* non-NULL: count sink accumulators */
} join_ctx;

/* Does comparison c hold for the current values (all its variables bound)? */
static int cmp_holds(const comparison* q, const uint32_t* vals) {
    const uint32_t a = q->a.kind == T_CONST ? q->a.val : vals[q->a.val];
    const uint32_t b = q->b.kind == T_CONST ? q->b.val : vals[q->b.val];
    if (q->op == CMP_LT) return a < b;
    if (q->op == CMP_LE) return a <= b;
    return a != b;
}

static void emit_head(join_ctx* j) {
    uint32_t tup[ORC_MAX_ARITY];
    const atom* h = &j->r->head;
    if (!filters_hold(j->p, j->r, j->vals)) return;
    for (uint32_t c = 0; c < h->arity; c++) tup[c] = h->t[c].kind == T_CONST ? h->t[c].val : j->vals[h->t[c].val];
    if (j->sink_acc) {
        /* count sink: every binding is a distinct tuple (checked in orc_run) */
        const uint64_t x = hash_vals(tup, h->arity);
        j->sink_acc[0] += 1;
        j->sink_acc[1] += x;
        j->sink_acc[2] ^= x;
        return;
    }
    table_insert(j->out, tup);
}

static void join_rec(join_ctx* j, uint32_t k, uint8_t* bound) {
    if (k == j->r->nbody) { emit_head(j); return; }
    const atom* a = &j->r->body[k];
    const hindex* x = &j->idx[k];
    uint32_t key[ORC_MAX_ARITY];
    for (uint32_t q = 0; q < x->ncols; q++) {
        const term* t = &a->t[x->cols[q]];
        key[q] = t->kind == T_CONST ? t->val : j->vals[t->val];
    }
    uint64_t h = hash_vals(key, x->ncols) & (x->nb - 1);
    for (int64_t i = x->head[h]; i >= 0; i = x->next[i]) {
        const uint32_t* row = row_at(x->t, (uint64_t)i);
        int ok = 1;
        for (uint32_t q = 0; q < x->ncols && ok; q++) ok = row[x->cols[q]] == key[q];
        if (!ok) continue;
        /* bind the atom's new variables; a variable repeated inside the atom must agree */
        uint32_t newly[ORC_MAX_ARITY], nnew = 0;
        for (uint32_t c = 0; c < a->arity && ok; c++) {
            if (a->t[c].kind != T_VAR || j->bound_at[k][c]) continue;
            uint32_t v = a->t[c].val;
            if (bound[v]) { ok = j->vals[v] == row[c]; continue; }
            bound[v] = 1;
            j->vals[v] = row[c];
            newly[nnew++] = v;
        }
        /* comparisons whose last variable this atom binds are checked here already */
        for (uint32_t q = 0; q < j->ncheck[k] && ok; q++) ok = cmp_holds(&j->r->cmp[j->check[k][q]], j->vals);
        if (ok) join_rec(j, k + 1, bound);
        for (uint32_t q = 0; q < nnew; q++) bound[newly[q]] = 0;
    }
}

static double now_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Evaluate one rule: atom k reads srcs[k]; every derived head tuple goes into out (or into
 * the head's count-sink accumulators). */
static void eval_rule(program* p, const rule* r, const table* const* srcs, table* out) {
    join_ctx j;
    memset(&j, 0, sizeof(j));
    j.p = p;
    j.r = r;
    j.out = out;
    if (p->sink[r->head.rel]) j.sink_acc = p->sink_acc + 3 * r->head.rel;
    uint8_t bound_before[ORC_MAX_VARS] = {0};
    for (uint32_t k = 0; k < r->nbody; k++) {
        const atom* a = &r->body[k];
        uint32_t cols[ORC_MAX_ARITY], nc = 0;
        for (uint32_t c = 0; c < a->arity; c++) {
            const term* t = &a->t[c];
            /* a lookup key column: a constant, or a variable bound by an earlier atom */
            int key = t->kind == T_CONST || bound_before[t->val];
            j.bound_at[k][c] = (uint32_t)key;
            if (key) cols[nc++] = c;
        }
        for (uint32_t c = 0; c < a->arity; c++)
            if (a->t[c].kind == T_VAR) bound_before[a->t[c].val] = 1;
        j.src[k] = srcs[k];
        hindex_build(&j.idx[k], srcs[k], cols, nc);
    }
    /* comparison c is checked at the first atom after which all its variables are bound */
    for (uint32_t c = 0; c < r->ncmp; c++) {
        uint8_t seen[ORC_MAX_VARS] = {0};
        for (uint32_t k = 0; k < r->nbody; k++) {
            for (uint32_t q = 0; q < r->body[k].arity; q++)
                if (r->body[k].t[q].kind == T_VAR) seen[r->body[k].t[q].val] = 1;
            const term* a = &r->cmp[c].a;
            const term* b = &r->cmp[c].b;
            if ((a->kind == T_CONST || seen[a->val]) && (b->kind == T_CONST || seen[b->val])) {
                j.check[k][j.ncheck[k]++] = c;
                break;
            }
        }
    }
    uint8_t bound[ORC_MAX_VARS] = {0};
    const double t0 = now_seconds();
    join_rec(&j, 0, bound);
    p->join_seconds += now_seconds() - t0;
    for (uint32_t k = 0; k < r->nbody; k++) hindex_free(&j.idx[k]);
}

static int rule_is_recursive(const program* p, const rule* r, uint32_t s) {
    for (uint32_t b = 0; b < r->nbody; b++)
        if (p->stratum_of_rel[r->body[b].rel] == s) return 1;
    return 0;
}

static void seminaive_stratum(program* p, uint32_t s) {
    const uint32_t *rels = p->strata_rels + p->strata_off[s], nrels = p->strata_off[s + 1] - p->strata_off[s];
    int any_rec = 0;
    for (uint32_t i = 0; i < p->nrule; i++)
        if (p->stratum_of_rel[p->rules[i].head.rel] == s && rule_is_recursive(p, &p->rules[i], s)) any_rec = 1;

    /* Round 1: the non-recursive rules over full relations.  Facts loaded into the
     * stratum's relations are part of round 1's delta. */
    for (uint32_t q = 0; q < nrels; q++) {
        uint32_t R = rels[q];
        table_clear(&p->fresh[R]);
        for (uint64_t i = 0; i < p->full[R].n; i++) table_insert(&p->fresh[R], row_at(&p->full[R], i));
    }
    for (uint32_t i = 0; i < p->nrule; i++) {
        const rule* r = &p->rules[i];
        if (p->stratum_of_rel[r->head.rel] != s || rule_is_recursive(p, r, s)) continue;
        const table* srcs[ORC_MAX_BODY];
        for (uint32_t b = 0; b < r->nbody; b++) srcs[b] = &p->full[r->body[b].rel];
        eval_rule(p, r, srcs, &p->fresh[r->head.rel]);
    }
    int any_new = 0;
    for (uint32_t q = 0; q < nrels; q++) {
        uint32_t R = rels[q];
        table_clear(&p->delta[R]);
        for (uint64_t i = 0; i < p->fresh[R].n; i++) {
            table_insert(&p->delta[R], row_at(&p->fresh[R], i));
            table_insert(&p->full[R], row_at(&p->fresh[R], i));
        }
        if (p->delta[R].n) any_new = 1;
        table_clear(&p->fresh[R]);
    }
    uint32_t t = 1;
    if (!any_rec || !any_new) { p->rounds[s] = 1; goto done; }

    /* Rounds t >= 2 (Jacobi): every delta variant reads the state at the round's start. */
    for (;;) {
        t++;
        for (uint32_t i = 0; i < p->nrule; i++) {
            const rule* r = &p->rules[i];
            if (p->stratum_of_rel[r->head.rel] != s || !rule_is_recursive(p, r, s)) continue;
            for (uint32_t j = 0; j < r->nbody; j++) {
                if (p->stratum_of_rel[r->body[j].rel] != s) continue;
                const table* srcs[ORC_MAX_BODY];
                for (uint32_t b = 0; b < r->nbody; b++) srcs[b] = &p->full[r->body[b].rel];
                srcs[j] = &p->delta[r->body[j].rel];
                eval_rule(p, r, srcs, &p->fresh[r->head.rel]);
            }
        }
        any_new = 0;
        for (uint32_t q = 0; q < nrels; q++) {
            uint32_t R = rels[q];
            table_clear(&p->delta[R]);
            for (uint64_t i = 0; i < p->fresh[R].n; i++) {
                const uint32_t* row = row_at(&p->fresh[R], i);
                if (!table_contains(&p->full[R], row)) table_insert(&p->delta[R], row);
            }
            table_clear(&p->fresh[R]);
        }
        for (uint32_t q = 0; q < nrels; q++) {
            uint32_t R = rels[q];
            if (p->delta[R].n) any_new = 1;
            for (uint64_t i = 0; i < p->delta[R].n; i++) table_insert(&p->full[R], row_at(&p->delta[R], i));
        }
        if (!any_new) break;
    }
    p->rounds[s] = t;
done:
    for (uint32_t q = 0; q < nrels; q++) table_clear(&p->delta[rels[q]]);
}

/* ----------------------------------------------------- brute-force naive T_P */

typedef struct { uint32_t* v; uint64_t n; } domain;

static domain active_domain(const program* p) {
    uint64_t cap = 16, n = 0;
    uint32_t* v = (uint32_t*)xmalloc(cap * sizeof(uint32_t));
    table seen;
    table_init(&seen, 1);
    for (uint32_t r = 0; r < p->nrel; r++)
        for (uint64_t i = 0; i < p->full[r].n * p->arity[r]; i++) table_insert(&seen, &p->full[r].rows[i]);
    for (uint32_t i = 0; i < p->nrule; i++) {
        const rule* r = &p->rules[i];
        for (uint32_t b = 0; b <= r->nbody + r->nneg; b++) {
            const atom* a = b < r->nbody ? &r->body[b] : b < r->nbody + r->nneg ? &r->neg[b - r->nbody] : &r->head;
            for (uint32_t c = 0; c < a->arity; c++)
                if (a->t[c].kind == T_CONST) table_insert(&seen, &a->t[c].val);
        }
        for (uint32_t c = 0; c < r->ncmp; c++) {
            if (r->cmp[c].a.kind == T_CONST) table_insert(&seen, &r->cmp[c].a.val);
            if (r->cmp[c].b.kind == T_CONST) table_insert(&seen, &r->cmp[c].b.val);
        }
    }
    for (uint64_t i = 0; i < seen.n; i++) {
        if (n == cap) { cap *= 2; v = (uint32_t*)realloc(v, cap * sizeof(uint32_t)); }
        v[n++] = seen.rows[i];
    }
    table_free(&seen);
    domain d = {v, n};
    return d;
}

/* T_P for one rule by enumerating every assignment of its variables over the domain. */
static void brute_rule(const program* p, const rule* r, const domain* d, table* out) {
    uint64_t idx[ORC_MAX_VARS] = {0};
    uint32_t vals[ORC_MAX_VARS];
    if (d->n == 0) return;
    for (;;) {
        for (uint32_t v = 0; v < r->nvars; v++) vals[v] = d->v[idx[v]];
        int ok = 1;
        for (uint32_t b = 0; b < r->nbody && ok; b++) {
            const atom* a = &r->body[b];
            uint32_t tup[ORC_MAX_ARITY];
            for (uint32_t c = 0; c < a->arity; c++) tup[c] = a->t[c].kind == T_CONST ? a->t[c].val : vals[a->t[c].val];
            ok = table_contains(&p->full[a->rel], tup);
        }
        if (ok) ok = filters_hold(p, r, vals);
        if (ok) {
            uint32_t tup[ORC_MAX_ARITY];
            for (uint32_t c = 0; c < r->head.arity; c++)
                tup[c] = r->head.t[c].kind == T_CONST ? r->head.t[c].val : vals[r->head.t[c].val];
            table_insert(out, tup);
        }
        uint32_t v = 0;
        while (v < r->nvars && ++idx[v] == d->n) idx[v++] = 0;
        if (v == r->nvars) break;
    }
}

/* Naive iteration of the brute-force T_P over the rules selected by `in_scope`;
 * returns the number of applications including the last one that changed nothing. */
static uint32_t naive_iterate(program* p, const domain* d, int32_t stratum) {
    uint32_t t = 0;
    for (;;) {
        t++;
        for (uint32_t i = 0; i < p->nrule; i++) {
            const rule* r = &p->rules[i];
            if (stratum >= 0 && p->stratum_of_rel[r->head.rel] != (uint32_t)stratum) continue;
            brute_rule(p, r, d, &p->fresh[r->head.rel]);
        }
        int changed = 0;
        for (uint32_t R = 0; R < p->nrel; R++) {
            for (uint64_t i = 0; i < p->fresh[R].n; i++) changed |= table_insert(&p->full[R], row_at(&p->fresh[R], i));
            table_clear(&p->fresh[R]);
        }
        if (!changed) return t;
    }
}

/* ------------------------------------------------------------------ driver */

/* A count sink must be the head of exactly one rule, whose head lists each of the rule's
 * variables exactly once, and must appear in no rule body. */
static int check_sinks(program* p) {
    for (uint32_t R = 0; R < p->nrel; R++) {
        if (!p->sink[R]) continue;
        uint32_t heads = 0;
        for (uint32_t i = 0; i < p->nrule; i++) {
            const rule* r = &p->rules[i];
            for (uint32_t b = 0; b < r->nbody + r->nneg; b++) {
                const atom* a = b < r->nbody ? &r->body[b] : &r->neg[b - r->nbody];
                if ((uint32_t)a->rel == R) return fail(p, "a count sink is read by a rule body");
            }
            if ((uint32_t)r->head.rel != R) continue;
            heads++;
            uint8_t seen[ORC_MAX_VARS] = {0};
            if (r->head.arity != r->nvars) return fail(p, "a count sink's head must list every rule variable once");
            for (uint32_t c = 0; c < r->head.arity; c++) {
                if (r->head.t[c].kind != T_VAR || seen[r->head.t[c].val])
                    return fail(p, "a count sink's head must list every rule variable once");
                seen[r->head.t[c].val] = 1;
            }
        }
        if (heads != 1) return fail(p, "a count sink needs exactly one rule");
        p->sink_acc[3 * R] = p->sink_acc[3 * R + 1] = p->sink_acc[3 * R + 2] = 0;
    }
    return 0;
}

int orc_run(void* h, int mode) {
    program* p = (program*)h;
    p->join_seconds = 0;
    if (check_sinks(p)) return -1;
    if (stratify(p)) return -1;
    if (mode != ORC_SEMINAIVE)
        for (uint32_t R = 0; R < p->nrel; R++)
            if (p->sink[R]) return fail(p, "count sinks need the semi-naive mode");
    if (mode == ORC_NAIVE_GLOBAL)
        for (uint32_t i = 0; i < p->nrule; i++)
            if (p->rules[i].nneg) return fail(p, "global naive iteration is undefined for negation");
    if (mode == ORC_SEMINAIVE) {
        for (uint32_t s = 0; s < p->nstrata; s++) seminaive_stratum(p, s);
        return 0;
    }
    domain d = active_domain(p);
    if (mode == ORC_NAIVE_STRATA) {
        for (uint32_t s = 0; s < p->nstrata; s++) p->rounds[s] = naive_iterate(p, &d, (int32_t)s);
    } else if (mode == ORC_NAIVE_GLOBAL) {
        uint32_t t = naive_iterate(p, &d, -1);
        for (uint32_t s = 0; s < p->nstrata; s++) p->rounds[s] = t;
    } else {
        free(d.v);
        return fail(p, "unknown mode");
    }
    free(d.v);
    return 0;
}

uint64_t orc_count(void* h, int rel) {
    program* p = (program*)h;
    if (rel < 0 || (uint32_t)rel >= p->nrel) return 0;
    return p->full[rel].n;
}

static uint32_t g_sort_arity;
static int cmp_rows(const void* a, const void* b) {
    const uint32_t *x = (const uint32_t*)a, *y = (const uint32_t*)b;
    for (uint32_t c = 0; c < g_sort_arity; c++) {
        if (x[c] < y[c]) return -1;
        if (x[c] > y[c]) return 1;
    }
    return 0;
}

/* Copy the relation out, row-major, sorted ascending lexicographically. */
int orc_fetch(void* h, int rel, uint32_t* out) {
    program* p = (program*)h;
    if (rel < 0 || (uint32_t)rel >= p->nrel) return fail(p, "bad relation");
    const table* t = &p->full[rel];
    memcpy(out, t->rows, t->n * t->arity * sizeof(uint32_t));
    g_sort_arity = t->arity;
    qsort(out, t->n, t->arity * sizeof(uint32_t), cmp_rows);
    return 0;
}

uint32_t orc_num_strata(void* h) { return ((program*)h)->nstrata; }

/* Relations (ascending ids) and round count of stratum s, in evaluation order. */
int orc_stratum(void* h, uint32_t s, uint32_t* rounds, uint32_t* rels, uint32_t* nrels) {
    program* p = (program*)h;
    if (s >= p->nstrata) return fail(p, "bad stratum");
    *rounds = p->rounds[s];
    *nrels = p->strata_off[s + 1] - p->strata_off[s];
    if (rels) memcpy(rels, p->strata_rels + p->strata_off[s], *nrels * sizeof(uint32_t));
    return 0;
}
