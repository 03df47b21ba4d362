// Host-side engine state (internal).
#pragma once

#include <array>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace dl {

using Perm = std::array<uint8_t, kMaxArity>;

inline Perm identity_perm() {
    Perm p{};
    for (int i = 0; i < kMaxArity; i++) p[i] = (uint8_t)i;
    return p;
}

struct Relation {
    std::string name;
    uint32_t arity = 0;               // stored columns (batched form: user columns + instance)
    uint32_t user_arity = 0;
    std::vector<std::pair<DevPtr, TableView>> pending;   // loaded rows not yet merged
    uint32_t sink = DL_SINK_STORE;
    std::vector<Perm> perms;          // perms[0] is the identity (canonical order)
    std::vector<Index> full;          // one index per perm; full[0] is always valid
    std::vector<Index> delta;         // one index per perm (valid during a stratum's rounds)
    // Head/body form during a recursive stratum's rounds: full[k] is the body and head[k] the
    // rows added since the last flush; the relation is their (disjoint) union.  Empty outside
    // the rounds: the stratum's end flushes every head into its body.
    std::vector<Index> head;
    // Dense bitmap of the relation's rows during a recursive stratum's rounds (when its column
    // domains are small enough): the round's delta is found by one test-and-set per raw row.
    DevPtr dense;
    uint32_t dense_dom[kMaxArity] = {0};
    // Dense sink (rule rows test-and-set straight into `dense` by the join): the bitmap as of
    // the last extraction, and one byte per kDenseBlockWords words marking blocks with bits set
    // since then.  Null when the rows are materialised and filtered instead.
    DevPtr dense_old, dense_dirty;
    uint64_t dense_words = 0;
    bool full_perms_built = false;    // full[k > 0] are up to date
    std::vector<bool> root_needed;    // per perm: build dense root offsets
    uint64_t sink_count = 0;
    unsigned long long sink_digest[2] = {0, 0};
    std::vector<uint64_t> sink_inst;  // batched count sink: per instance [count, sum, xor]
    int stratum = -1;
};

struct RuleAtom {
    uint32_t rel = 0;
    uint32_t arity = 0;
    dl_term terms[kMaxArity];
};

struct RuleCmp {
    uint32_t op = 0;                  // DL_CMP_*
    dl_term a{}, b{};
};

struct Rule {
    RuleAtom head;
    std::vector<RuleAtom> body;
    std::vector<RuleAtom> neg;        // negated atoms (relations of lower strata)
    std::vector<RuleCmp> cmps;        // comparison filters
    std::vector<uint32_t> order;      // user variable ids in join order
};

struct Stratum {
    std::vector<uint32_t> rels;       // ascending ids
    uint32_t rounds = 0;
};

struct PhaseEvents {                  // accumulated device time per phase kind
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
};

struct KernelEvent {
    int kind;
    cudaEvent_t a, b;
    uint64_t bytes;
    uint64_t units, entries;          // join passes: candidates of the smallest sources, frontier entries
};

struct TuneChoice {                   // autotuner: a join level's tile size and kernel shape
    uint32_t tile = 0;
    bool wm = false;
    float ms = 0;                     // the count pass's time when it was chosen
};

class Engine {
  public:
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t budget = 0, used = 0, peak = 0;
    cudaMemPool_t pool = nullptr;     // engine-owned stream-ordered pool (no user allocator)
    dl_alloc_fn ualloc = nullptr;
    dl_free_fn ufree = nullptr;
    void* uuser = nullptr;
    uint32_t flags = 0;
    uint32_t tile_units = 0;        // 0: chosen per join level (auto_tile)
    uint32_t sms = 152;             // multiprocessors of the device
    std::string err;
    std::vector<Relation> rels;
    std::vector<Rule> rules;
    std::vector<Stratum> strata;
    uint32_t V = 0;                   // values seen so far are < V
    uint32_t instances = 0;           // batched form: number of instances (0 = one program)
    uint64_t chunk_rows = 1ull << 30; // larger rule outputs are written and reduced in chunks
    std::vector<std::vector<uint32_t>> inst_rounds;   // batched form: [stratum][instance]
    uint64_t host_scratch[64] = {0};  // readback target (pageable: freeing pinned memory would
                                      // synchronise the whole device, stalling other engines)
    uint64_t launches = 0;
    uint64_t hub_keys = 0;          // heavy keys given membership bitmaps
    uint32_t hub_rows = kHubMinRows;  // rows that make a key heavy
    uint64_t join_rows = 0, count_rows = 0, delta_rows = 0;
    uint64_t frontier_bytes = 0;      // join frontier bytes before slicing (0: a third of the budget left)
    uint64_t join_slices = 0;         // levels whose input was processed in slices
    uint32_t head_percent = 25;       // flush a head into its body above this percentage of the body
    uint64_t dense_bytes = 8ull << 30;  // largest dense relation bitmap (and at most a quarter of the budget left)
    uint64_t dense_relations = 0;
    uint64_t head_flushes = 0;
    std::map<std::string, TuneChoice> tune;   // DL_FLAG_AUTOTUNE: choices by rule, level and size bucket
    std::string tune_path;            // file the choices are loaded from and saved to ("" = none)
    uint64_t tuned_levels = 0, tune_hits = 0;
    bool in_fixpoint = false;
    std::vector<cudaEvent_t> event_pool;
    size_t event_next = 0;
    PhaseEvents phases;
    std::vector<KernelEvent> kev;     // DL_FLAG_PROFILE: one entry per timed launch
    uint64_t klaunch[DL_KERNEL_KINDS] = {0};

    ~Engine();
    void* alloc(size_t bytes);
    void release(void* p, size_t bytes);
    DevPtr make(size_t bytes) { return std::make_shared<DevMem>(this, bytes); }
    template <class T>
    DArray<T> array(uint64_t n) {
        DArray<T> a;
        a.mem = make(sizeof(T) * (n ? n : 1));
        a.p = (T*)a.mem->ptr;
        a.n = n;
        return a;
    }
    // Copy `count` uint64 words from device to host scratch and wait.
    const uint64_t* readback(const void* dev, size_t words);
    void sync() { DL_CUDA(cudaStreamSynchronize(stream)); }
    cudaEvent_t next_event();
    void phase_begin(int kind);
    void phase_end(int kind);
};

// Times one kernel launch (or a short sequence) of a given kind when profiling is enabled,
// and counts launches of that kind in every case.
struct KernelScope {
    Engine& E;
    int kind;
    uint64_t bytes, units, entries;
    cudaEvent_t a = nullptr;
    KernelScope(Engine& e, int k, uint64_t b, int nlaunch = 1, uint64_t u = 0, uint64_t ent = 0)
        : E(e), kind(k), bytes(b), units(u), entries(ent) {
        E.launches += nlaunch;
        E.klaunch[k] += nlaunch;
        if (E.flags & DL_FLAG_PROFILE) {
            a = E.next_event();
            cudaEventRecord(a, E.stream);
        }
    }
    ~KernelScope() {
        if (a) {
            cudaEvent_t b = E.next_event();
            cudaEventRecord(b, E.stream);
            E.kev.push_back({kind, a, b, bytes, units, entries});
        }
    }
};

// Allocates an index of `n` rows, `arity` columns in permutation `perm`.
Index make_index(Engine& E, uint32_t arity, const Perm& perm, uint64_t n);
TableView table_of(const Index& ix);
AtomView atom_of(const Index& ix);

// ---- join (wcoj.cu)

struct RulePlan;
// Evaluate one variant of a rule; src_index[k] is the index body atom k reads.  For a stored
// head the output rows (head column order) are appended to `out_parts`; for a count sink the
// counts go to the relation's sink counters.
struct JoinOutput {
    std::vector<TableView> parts;     // each part: arity columns
    std::vector<DevPtr> owners;
    std::vector<Index> rparts;        // parts already sorted, deduplicated and anti-joined with full
    bool sorted_unique = true;        // a single unreduced part is sorted (canonical) and distinct
    bool dense_sunk = false;          // rows went to the head's dense bitmap (extracted at the round's end)
    uint64_t dense_rows = 0;          // raw rows those were
    // Receives an output chunk of a rule whose output exceeds the chunk size; it reduces the
    // chunk and appends it as a reduced part.
    std::function<void(DevPtr, TableView)> chunk_sink;
};
// src: the index each positive body atom reads; nsrc: each negated atom's (complete) index.
void run_join(Engine& E, const Rule& R, const std::vector<const Index*>& src, const std::vector<const Index*>& nsrc,
              Relation& head, JoinOutput& out);

}  // namespace dl
