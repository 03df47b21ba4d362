// C ABI entry points and the host runtime: relation store, stratification, semi-naive
// rounds (paper Sections 2 and 4), fetch.
#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <set>

#include "engine.h"

namespace dl {

Perm atom_perm(const Rule& R, uint32_t a);
Perm neg_perm(const Rule& R, uint32_t n);
bool head_is_order(const Rule& R);

// ------------------------------------------------------------------ memory

DevMem::DevMem(Engine* e, size_t b) : eng(e), bytes(b) { ptr = e->alloc(b); }
DevMem::~DevMem() {
    if (ptr) eng->release(ptr, bytes);
}

void* Engine::alloc(size_t bytes) {
    if (bytes == 0) bytes = 1;
    bytes = (bytes + 255) & ~size_t(255);
    if (used + bytes > budget)
        throw Error(DL_ERR_CAPACITY, "device budget exceeded: need " + std::to_string(bytes) + " more bytes, " +
                                         std::to_string(used) + " of " + std::to_string(budget) + " in use");
    void* p = nullptr;
    if (ualloc) {
        p = ualloc(bytes, stream, uuser);
        if (!p) throw Error(DL_ERR_CAPACITY, "user allocator returned NULL");
    } else {
        cudaError_t st = cudaMallocFromPoolAsync(&p, bytes, pool, stream);
        if (st == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            throw Error(DL_ERR_CAPACITY, "device out of memory");
        }
        if (st != cudaSuccess) throw Error(DL_ERR_CUDA, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(st));
    }
    used += bytes;
    peak = std::max(peak, used);
    return p;
}

void Engine::release(void* p, size_t bytes) {
    if (bytes == 0) bytes = 1;
    bytes = (bytes + 255) & ~size_t(255);
    if (ufree) ufree(p, bytes, stream, uuser);
    else cudaFreeAsync(p, stream);
    used -= bytes;
}

const uint64_t* Engine::readback(const void* dev, size_t words) {
    if (words > 64) throw Error(DL_ERR_ARG, "readback too large");
    DL_CUDA(cudaMemcpyAsync(host_scratch, dev, words * 8, cudaMemcpyDeviceToHost, stream));
    DL_CUDA(cudaStreamSynchronize(stream));
    return host_scratch;
}

cudaEvent_t Engine::next_event() {
    if (event_next == event_pool.size()) {
        cudaEvent_t ev;
        DL_CUDA(cudaEventCreate(&ev));
        event_pool.push_back(ev);
    }
    return event_pool[event_next++];
}

void Engine::phase_begin(int kind) {
    cudaEvent_t a = next_event();
    DL_CUDA(cudaEventRecord(a, stream));
    phases.ev[kind].push_back({a, nullptr});
}

void Engine::phase_end(int kind) {
    cudaEvent_t b = next_event();
    DL_CUDA(cudaEventRecord(b, stream));
    phases.ev[kind].back().second = b;
}

// Autotuner cache file: "key tile wm ms" per line.
void tune_load(Engine& E, const std::string& path) {
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return;
    char key[128];
    unsigned tile = 0;
    int wm = 0;
    float ms = 0;
    while (fscanf(f, "%127s %u %d %f", key, &tile, &wm, &ms) == 4)
        if (tile >= 32 && tile <= (1u << 24)) E.tune[key] = {tile, wm != 0, ms};
    fclose(f);
}

bool tune_write(const Engine& E, const std::string& path) {
    FILE* f = fopen(path.c_str(), "w");
    if (!f) return false;
    for (const auto& kv : E.tune) fprintf(f, "%s %u %d %.3f\n", kv.first.c_str(), kv.second.tile, kv.second.wm ? 1 : 0,
                                          kv.second.ms);
    return fclose(f) == 0;
}

Engine::~Engine() {
    if (!tune_path.empty() && tuned_levels) tune_write(*this, tune_path);
    rels.clear();                      // stream-ordered frees: no wait needed
    for (auto ev : event_pool) cudaEventDestroy(ev);
    if (pool) {
        cudaStreamSynchronize(stream);  // the pool's memory must be idle before it is destroyed
        cudaMemPoolDestroy(pool);
    }
    if (own_stream && stream) cudaStreamDestroy(stream);
}

// ------------------------------------------------------------------ indexes

Index make_index(Engine& E, uint32_t arity, const Perm& perm, uint64_t n) {
    if (n >= 0xFFFFFFFEull) throw Error(DL_ERR_CAPACITY, "index of 2^32 - 2 rows or more");
    Index ix;
    ix.arity = arity;
    for (int k = 0; k < kMaxArity; k++) ix.perm[k] = perm[k];
    ix.n = n;
    ix.cap = std::max<uint64_t>(n, 1);
    ix.cols = E.make(sizeof(uint32_t) * arity * ix.cap);
    return ix;
}

TableView table_of(const Index& ix) {
    TableView t;
    memset(&t, 0, sizeof(t));
    t.arity = ix.arity;
    t.n = ix.n;
    for (uint32_t k = 0; k < ix.arity; k++) t.col[k] = ix.col((int)k);
    return t;
}

AtomView atom_of(const Index& ix) {
    AtomView a;
    memset(&a, 0, sizeof(a));
    for (uint32_t k = 0; k < ix.arity; k++) a.col[k] = ix.col((int)k);
    a.root = ix.root_ptr();
    a.V = ix.rootV;
    a.hub = ix.hub ? (const int32_t*)ix.hub->ptr : nullptr;
    a.bits = ix.bits ? (const uint32_t*)ix.bits->ptr : nullptr;
    a.bmwords = ix.bmwords;
    a.hubmin = ix.hubmin;
    a.n = (uint32_t)ix.n;
    a.arity = ix.arity;
    return a;
}

namespace {

const char* kVersion = "1.0.0";

bool same_perm(const Perm& a, const Perm& b, uint32_t arity) {
    for (uint32_t k = 0; k < arity; k++)
        if (a[k] != b[k]) return false;
    return true;
}

Index empty_index(uint32_t arity, const Perm& perm) {
    Index ix;
    ix.arity = arity;
    for (int k = 0; k < kMaxArity; k++) ix.perm[k] = perm[k];
    return ix;
}

// Sort a table (canonical column order of its index) in place; returns an Index holding it.
// `buf` owns t's columns, which lie `stride` values apart (0: t.n apart); the result owns
// whichever buffer ends up holding the sorted rows.
Index sort_into_index(Engine& E, DevPtr buf, TableView t, const Perm& perm, uint32_t arity, uint64_t stride = 0) {
    if (!stride) stride = std::max<uint64_t>(t.n, 1);
    Index ix = empty_index(arity, perm);
    ix.n = t.n;
    ix.cap = stride;
    if (t.n <= 1) {
        ix.cols = buf;
        return ix;
    }
    const uint64_t tcap = std::max<uint64_t>(t.n, 1);
    DevPtr tmpbuf = E.make(sizeof(uint32_t) * arity * tcap);
    TableView tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.arity = arity;
    tmp.n = t.n;
    for (uint32_t c = 0; c < arity; c++) tmp.col[c] = (uint32_t*)tmpbuf->ptr + (size_t)c * tcap;
    uint32_t* orig0 = t.col[0];
    E.phase_begin(1);
    radix_sort_rows(E, t, tmp, nullptr);
    E.phase_end(1);
    if (t.col[0] != orig0) {
        ix.cols = tmpbuf;
        ix.cap = tcap;
    } else {
        ix.cols = buf;
    }
    return ix;
}

// Sorted distinct rows of a raw table as a new index: the packed-key path when the rows'
// varying bits fit in 64 bits, else sort + adjacent unique.
Index sort_unique_index(Engine& E, DevPtr buf, TableView t, const Perm& perm, uint32_t arity, uint64_t stride);

void build_roots(Engine& E, Index& ix, bool needed) {
    ix.root.reset();
    ix.rootV = 0;
    ix.hub.reset();
    ix.bits.reset();
    ix.bmwords = 0;
    ix.hubmin = 0;
    if (!needed || E.V == 0 || E.V > kDenseRootLimit || ix.n == 0) return;
    ix.root = E.make(sizeof(uint32_t) * ((size_t)E.V + 1));
    ix.rootV = E.V;
    build_root(E, ix.col(0), ix.n, (uint32_t*)ix.root->ptr, E.V);
}

// Heavy-key bitmaps for an index whose root offsets exist: a join probe into the range of a
// key with >= E.hub_rows rows becomes one bit test.  Built for indexes that stay fixed while
// the joins read them (a merge rebuilds the roots and drops the bitmaps).
void build_hubs(Engine& E, Index& ix) {
    if (!ix.root || ix.hub || ix.arity != 2 || ix.n < E.hub_rows) return;
    const uint32_t V = ix.rootV;
    std::vector<uint32_t> root((size_t)V + 1);
    DL_CUDA(cudaMemcpyAsync(root.data(), ix.root->ptr, sizeof(uint32_t) * root.size(), cudaMemcpyDeviceToHost,
                            E.stream));
    E.sync();
    std::vector<std::pair<uint32_t, uint32_t>> heavy;   // (degree, key)
    for (uint32_t k = 0; k < V; k++)
        if (root[k + 1] - root[k] >= E.hub_rows) heavy.push_back({root[k + 1] - root[k], k});
    if (heavy.empty()) return;
    std::sort(heavy.rbegin(), heavy.rend());
    const uint32_t bmwords = (V + 31) / 32;
    // at most kHubBitmapBytes, and at most a quarter of the budget left: the bitmaps only
    // speed probes up and must not turn a program that fits into one that does not
    const uint64_t room = std::min<uint64_t>(kHubBitmapBytes, E.budget > E.used ? (E.budget - E.used) / 4 : 0);
    const uint64_t slots = sizeof(int32_t) * (uint64_t)V;
    const uint64_t maxh = room > slots ? (room - slots) / (sizeof(uint32_t) * (uint64_t)bmwords) : 0;
    if (heavy.size() > maxh) heavy.resize(maxh);
    if (heavy.empty()) return;
    std::vector<int32_t> slot(V, -1);
    std::vector<uint32_t> keys(heavy.size());
    for (size_t i = 0; i < heavy.size(); i++) {
        keys[i] = heavy[i].second;
        slot[heavy[i].second] = (int32_t)i;
    }
    // the index takes the bitmaps only once they are complete (an allocation that fails
    // leaves it without any)
    DevPtr hub = E.make(sizeof(int32_t) * V);
    DevPtr bits = E.make(sizeof(uint32_t) * (uint64_t)bmwords * keys.size());
    auto dkeys = E.array<uint32_t>(keys.size());
    DL_CUDA(cudaMemcpyAsync(hub->ptr, slot.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice, E.stream));
    DL_CUDA(cudaMemcpyAsync(dkeys.p, keys.data(), sizeof(uint32_t) * keys.size(), cudaMemcpyHostToDevice, E.stream));
    build_hub_bits(E, (const uint32_t*)ix.root->ptr, ix.col(1), dkeys.p, (uint32_t)keys.size(),
                   (uint32_t*)bits->ptr, bmwords);
    E.sync();   // the host vectors above must outlive the copies
    ix.hub = hub;
    ix.bits = bits;
    ix.bmwords = bmwords;
    ix.hubmin = heavy.back().first;
    E.hub_keys += keys.size();
}

// Δ = unique(sorted new rows) \ full, written into a fresh index (canonical order).
Index compute_delta(Engine& E, const Index& sorted_new, const Index& full, const Perm& perm, uint32_t arity,
                    bool known_unique) {
    if (sorted_new.n == 0) return empty_index(arity, perm);
    if (full.n == 0 && known_unique) return sorted_new;
    Index d = make_index(E, arity, perm, sorted_new.n);
    AtomView fa = atom_of(full);
    E.phase_begin(2);
    d.n = unique_anti(E, table_of(sorted_new), full.n ? &fa : nullptr, table_of(d));
    E.phase_end(2);
    return d;
}

Index merge_into(Engine& E, const Index& full, const Index& delta) {
    if (delta.n == 0) return full;
    if (full.n == 0) return delta;
    if (full.n + delta.n >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "relation index of 2^32 rows or more");
    Index out = make_index(E, full.arity, [&] {
        Perm p;
        for (int k = 0; k < kMaxArity; k++) p[k] = full.perm[k];
        return p;
    }(), full.n + delta.n);
    E.phase_begin(3);
    merge_rows(E, table_of(full), table_of(delta), table_of(out));
    E.phase_end(3);
    return out;
}

Index permuted_sorted(Engine& E, const Index& canon, const Perm& perm) {
    const uint32_t a = canon.arity;
    Index ix = empty_index(a, perm);
    if (canon.n == 0) return ix;
    DevPtr buf = E.make(sizeof(uint32_t) * a * canon.n);
    TableView t;
    memset(&t, 0, sizeof(t));
    t.arity = a;
    t.n = canon.n;
    for (uint32_t c = 0; c < a; c++) t.col[c] = (uint32_t*)buf->ptr + (size_t)c * canon.n;
    permute_copy(E, table_of(canon), perm.data(), t);
    return sort_into_index(E, buf, t, perm, a);
}

void check_sorted(Engine& E, const Index& ix, const std::string& what) {
    if (!(E.flags & DL_FLAG_DEBUG_CHECKS)) return;
    uint64_t bad = count_order_violations(E, table_of(ix));
    if (bad) throw Error(DL_ERR_STATE, "debug check: " + what + " has " + std::to_string(bad) + " order violations");
}

// Add rows (canonical column order, any order, duplicates allowed) to a relation's full index.
void add_rows(Engine& E, Relation& R, DevPtr buf, TableView t) {
    if (t.n == 0) return;
    Index sorted = sort_into_index(E, buf, t, identity_perm(), R.arity);
    Index d = compute_delta(E, sorted, R.full[0], identity_perm(), R.arity, false);
    R.full[0] = merge_into(E, R.full[0], d);
    R.full_perms_built = false;
    check_sorted(E, R.full[0], R.name);
}

// Merge every pending load of a relation into its full index (one sort and merge in total).
void flush_pending(Engine& E, Relation& R) {
    if (R.pending.empty()) return;
    if (R.pending.size() == 1) {
        auto pr = R.pending[0];
        R.pending.clear();
        add_rows(E, R, pr.first, pr.second);
        return;
    }
    uint64_t tot = 0;
    for (auto& pr : R.pending) tot += pr.second.n;
    if (tot >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "2^32 or more pending rows in one relation");
    DevPtr buf = E.make(sizeof(uint32_t) * R.arity * tot);
    TableView t;
    memset(&t, 0, sizeof(t));
    t.arity = R.arity;
    t.n = tot;
    for (uint32_t c = 0; c < R.arity; c++) t.col[c] = (uint32_t*)buf->ptr + (size_t)c * tot;
    uint64_t off = 0;
    for (auto& pr : R.pending) {
        for (uint32_t c = 0; c < R.arity; c++)
            DL_CUDA(cudaMemcpyAsync(t.col[c] + off, pr.second.col[c], sizeof(uint32_t) * pr.second.n,
                                    cudaMemcpyDeviceToDevice, E.stream));
        off += pr.second.n;
    }
    R.pending.clear();
    add_rows(E, R, buf, t);
}

void update_max_value(Engine& E, const TableView& t) {
    if (!t.n) return;
    auto m = E.array<uint32_t>(2);
    DL_CUDA(cudaMemsetAsync(m.p, 0, 8, E.stream));
    for (uint32_t c = 0; c < t.arity; c++) column_max(E, t.col[c], t.n, m.p);
    uint32_t mx = (uint32_t)(E.readback(m.p, 1)[0] & 0xffffffffu);
    if (mx == 0xffffffffu) throw Error(DL_ERR_UNSUPPORTED, "value 0xFFFFFFFF is reserved");
    E.V = std::max(E.V, mx + 1);
}

uint32_t perm_slot(Relation& R, const Perm& p) {
    for (size_t k = 0; k < R.perms.size(); k++)
        if (same_perm(R.perms[k], p, R.arity)) return (uint32_t)k;
    R.perms.push_back(p);
    R.full.push_back(empty_index(R.arity, p));
    R.delta.push_back(empty_index(R.arity, p));
    R.root_needed.push_back(false);
    R.full_perms_built = false;
    return (uint32_t)(R.perms.size() - 1);
}

void ensure_full_perms(Engine& E, Relation& R) {
    if (!R.full_perms_built) {
        for (size_t k = 1; k < R.perms.size(); k++) R.full[k] = permuted_sorted(E, R.full[0], R.perms[k]);
        R.full_perms_built = true;
    }
    for (size_t k = 0; k < R.perms.size(); k++) build_roots(E, R.full[k], R.root_needed[k]);
}

// ------------------------------------------------------------------ strata

// Kosaraju's SCC over relations (edge: body relation -> head relation); components in
// topological order, ties broken by the smallest relation id.
std::vector<Stratum> stratify(const Engine& E) {
    const uint32_t n = (uint32_t)E.rels.size();
    std::vector<std::vector<uint32_t>> g(n), gr(n);
    std::vector<bool> derived(n, false);
    for (const Rule& r : E.rules) {
        derived[r.head.rel] = true;
        for (const RuleAtom& a : r.body) {
            g[a.rel].push_back(r.head.rel);
            gr[r.head.rel].push_back(a.rel);
        }
        for (const RuleAtom& a : r.neg) {     // a negated relation is computed first
            g[a.rel].push_back(r.head.rel);
            gr[r.head.rel].push_back(a.rel);
        }
    }
    std::vector<uint32_t> finish;
    std::vector<bool> seen(n, false);
    for (uint32_t s = 0; s < n; s++) {
        if (seen[s]) continue;
        std::vector<std::pair<uint32_t, size_t>> st{{s, 0}};
        seen[s] = true;
        while (!st.empty()) {
            auto& [v, i] = st.back();
            if (i < g[v].size()) {
                uint32_t w = g[v][i++];
                if (!seen[w]) {
                    seen[w] = true;
                    st.push_back({w, 0});
                }
            } else {
                finish.push_back(v);
                st.pop_back();
            }
        }
    }
    std::vector<int> comp(n, -1);
    int nc = 0;
    for (auto it = finish.rbegin(); it != finish.rend(); ++it) {
        if (comp[*it] >= 0) continue;
        std::vector<uint32_t> st{*it};
        comp[*it] = nc;
        while (!st.empty()) {
            uint32_t v = st.back();
            st.pop_back();
            for (uint32_t w : gr[v])
                if (comp[w] < 0) {
                    comp[w] = nc;
                    st.push_back(w);
                }
        }
        nc++;
    }
    for (const Rule& r : E.rules)
        for (const RuleAtom& a : r.neg)
            if (comp[a.rel] == comp[r.head.rel])
                throw Error(DL_ERR_UNSUPPORTED, "relation '" + E.rels[a.rel].name +
                                                    "' is negated inside its own recursive component: the program is "
                                                    "not stratifiable");
    std::vector<std::set<int>> succ(nc);
    std::vector<int> indeg(nc, 0), minrel(nc, INT32_MAX);
    for (uint32_t v = 0; v < n; v++) minrel[comp[v]] = std::min(minrel[comp[v]], (int)v);
    for (uint32_t v = 0; v < n; v++)
        for (uint32_t w : g[v])
            if (comp[v] != comp[w] && succ[comp[v]].insert(comp[w]).second) indeg[comp[w]]++;
    std::set<std::pair<int, int>> ready;  // (min relation id, component)
    for (int c = 0; c < nc; c++)
        if (!indeg[c]) ready.insert({minrel[c], c});
    std::vector<Stratum> out;
    while (!ready.empty()) {
        int c = ready.begin()->second;
        ready.erase(ready.begin());
        Stratum s;
        bool has_rule = false;
        for (uint32_t v = 0; v < n; v++)
            if (comp[v] == c) {
                s.rels.push_back(v);
                has_rule = has_rule || derived[v];
            }
        if (has_rule) out.push_back(s);
        for (int w : succ[c])
            if (--indeg[w] == 0) ready.insert({minrel[w], w});
    }
    return out;
}

// ------------------------------------------------------------------ rounds

struct Variant {
    const Rule* rule;
    int delta_atom;   // -1: all atoms read full
};

struct PendingOut {
    JoinOutput out;
    uint32_t producers = 0;   // variants that produced parts
};

void run_variant_on(Engine& E, const Variant& v, std::vector<const Index*>& src, std::map<uint32_t, PendingOut>& outs);

// Drop the rows of a raw (unsorted) table that are already in full, before any sorting: in
// late rounds most join output rediscovers known tuples, so the sort then only sees rows
// that may be new.  The join emits rows grouped by their leading columns, so consecutive
// probes of the full index touch the same ranges.  Returns the (possibly new) table.
// The result's columns lie t.n (the unfiltered count) values apart: see `stride`.
std::pair<DevPtr, TableView> prefilter(Engine& E, const Relation& R, DevPtr buf, TableView t, uint64_t& stride) {
    stride = t.n;
    // the relation is its body and, during recursive rounds, its head
    for (const Index* part : {&R.full[0], R.head.empty() ? nullptr : &R.head[0]}) {
        if (!part || part->n == 0 || t.n == 0) continue;
        DevPtr out = E.make(sizeof(uint32_t) * t.arity * stride);
        TableView o;
        memset(&o, 0, sizeof(o));
        o.arity = t.arity;
        for (uint32_t c = 0; c < t.arity; c++) o.col[c] = (uint32_t*)out->ptr + (size_t)c * stride;
        E.phase_begin(2);
        o.n = anti_filter(E, t, atom_of(*part), o, false);   // sorted next: order does not matter
        E.phase_end(2);
        buf = out;
        t = o;
    }
    return {buf, t};
}

// Rows of a sorted index absent from the relation's head (order kept).
Index minus_head(Engine& E, const Relation& R, const Index& d) {
    if (R.head.empty() || R.head[0].n == 0 || d.n == 0) return d;
    Perm p = identity_perm();
    for (int k = 0; k < kMaxArity; k++) p[k] = d.perm[k];
    Index o = make_index(E, d.arity, p, d.n);
    E.phase_begin(2);
    o.n = anti_filter(E, table_of(d), atom_of(R.head[0]), table_of(o));
    E.phase_end(2);
    return o;
}

// Head/body: merge every head into its body and rebuild the body's root offsets.
void flush_head(Engine& E, Relation& R) {
    if (R.head.empty()) return;
    if (R.head[0].n) {
        for (size_t k = 0; k < R.perms.size(); k++) {
            R.full[k] = merge_into(E, R.full[k], R.head[k]);
            build_roots(E, R.full[k], R.root_needed[k]);
        }
        check_sorted(E, R.full[0], R.name);
        E.head_flushes++;
    }
    for (size_t k = 0; k < R.head.size(); k++) R.head[k] = empty_index(R.arity, R.perms[k]);
}

// a ∪ b of two sorted, duplicate-free indexes (rows may occur in both).
Index union_sorted(Engine& E, const Index& a, const Index& b) {
    if (a.n == 0) return b;
    if (b.n == 0) return a;
    Perm p = identity_perm();
    for (int k = 0; k < kMaxArity; k++) p[k] = a.perm[k];
    Index m = make_index(E, a.arity, p, a.n + b.n);
    E.phase_begin(3);
    merge_rows(E, table_of(a), table_of(b), table_of(m));
    E.phase_end(3);
    Index u = make_index(E, a.arity, p, m.n);
    E.phase_begin(2);
    u.n = unique_anti(E, table_of(m), nullptr, table_of(u));
    E.phase_end(2);
    return u;
}

// Drop rows already in full from a raw output part, then sort it and drop duplicates.
Index sort_unique_index(Engine& E, DevPtr buf, TableView t, const Perm& perm, uint32_t arity, uint64_t stride) {
    if (t.n > 1) {
        Index out;
        E.phase_begin(1);
        const bool done = sort_unique_packed(E, t, [&](uint64_t m) {
            out = make_index(E, arity, perm, m);
            return table_of(out);
        });
        E.phase_end(1);
        if (done) return out;
    }
    Index sorted = sort_into_index(E, buf, t, perm, arity, stride);
    return compute_delta(E, sorted, empty_index(arity, perm), perm, arity, false);
}

// Rows of a raw table that are new to a relation in dense-bitmap form (each row's bit is
// tested and set, so the kept rows are distinct and absent from the relation), as a sorted
// index; `sorted` input stays sorted without a sort.
Index dense_reduce(Engine& E, Relation& R, const TableView& t, bool sorted) {
    Index o = make_index(E, R.arity, identity_perm(), t.n);
    E.phase_begin(2);
    o.n = dense_filter(E, t, R.dense_dom, (uint32_t*)R.dense->ptr, table_of(o));
    E.phase_end(2);
    if (sorted || o.n <= 1) return o;
    TableView ot = table_of(o);
    return sort_into_index(E, o.cols, ot, identity_perm(), R.arity, o.cap);
}

// Rows of a raw table set in a relation's dense bitmap (dense sink: the round's end extracts
// every row set since the last extraction, sorted and distinct).
void dense_mark(Engine& E, Relation& R, const TableView& t) {
    E.phase_begin(2);
    dense_set_rows(E, t, R.dense_dom, (uint32_t*)R.dense->ptr, (uint8_t*)R.dense_dirty->ptr);
    E.phase_end(2);
}

// The rows set in a relation's dense bitmap since the last extraction, as a sorted index.
Index dense_take(Engine& E, Relation& R) {
    Index o;
    E.phase_begin(2);
    o.n = dense_extract(E, R.arity, R.dense_dom, (const uint32_t*)R.dense->ptr, (uint32_t*)R.dense_old->ptr,
                        (uint8_t*)R.dense_dirty->ptr, R.dense_words, [&](uint64_t m) {
                            o = make_index(E, R.arity, identity_perm(), m);
                            return table_of(o);
                        });
    E.phase_end(2);
    return o;
}

Index reduce_part(Engine& E, Relation& R, DevPtr buf, TableView t) {
    if (R.dense && R.dense_dirty) {
        dense_mark(E, R, t);
        return empty_index(R.arity, identity_perm());
    }
    if (R.dense) return dense_reduce(E, R, t, false);
    uint64_t stride = 0;
    auto f = prefilter(E, R, buf, t, stride);
    return sort_unique_index(E, f.first, f.second, identity_perm(), R.arity, stride);
}

// Largest value + 1 of every column of every relation, over its rows and every row the rules
// can derive: a head column's values come from the body columns its variable is bound by, so
// they are below the smallest of those bounds (a fixpoint over the rules; constants count).
std::vector<std::array<uint32_t, kMaxArity>> column_domains(Engine& E) {
    std::vector<std::array<uint32_t, kMaxArity>> dom(E.rels.size());
    auto m = E.array<uint32_t>(kMaxArity);
    for (size_t r = 0; r < E.rels.size(); r++) {
        dom[r].fill(0);
        const Relation& R = E.rels[r];
        if (R.sink == DL_SINK_COUNT || R.full.empty() || R.full[0].n == 0) continue;
        DL_CUDA(cudaMemsetAsync(m.p, 0, sizeof(uint32_t) * kMaxArity, E.stream));
        for (uint32_t c = 0; c < R.arity; c++) column_max(E, R.full[0].col((int)c), R.full[0].n, m.p + c);
        uint32_t mx[kMaxArity];
        memcpy(mx, E.readback(m.p, kMaxArity / 2), sizeof(mx));
        for (uint32_t c = 0; c < R.arity; c++) dom[r][c] = mx[c] + 1;
    }
    for (bool changed = true; changed;) {
        changed = false;
        for (const Rule& q : E.rules) {
            for (uint32_t c = 0; c < q.head.arity; c++) {
                const dl_term& t = q.head.terms[c];
                uint32_t bound = 0;
                if (t.kind == DL_TERM_CONST) {
                    bound = t.id + 1;
                } else {
                    bound = UINT32_MAX;
                    for (const RuleAtom& a : q.body)
                        for (uint32_t k = 0; k < a.arity; k++)
                            if (a.terms[k].kind == DL_TERM_VAR && a.terms[k].id == t.id)
                                bound = std::min(bound, dom[a.rel][k]);
                    if (bound == UINT32_MAX) bound = E.V;
                }
                if (bound > dom[q.head.rel][c]) {
                    dom[q.head.rel][c] = bound;
                    changed = true;
                }
            }
        }
    }
    return dom;
}

void dense_end(Relation& R) {
    R.dense.reset();
    R.dense_old.reset();
    R.dense_dirty.reset();
    R.dense_words = 0;
}

// Gives a stratum's relations their dense bitmaps where the domain product is small enough.
void dense_begin(Engine& E, const Stratum& S) {
    if (E.dense_bytes <= 1) return;
    const auto dom = column_domains(E);
    const bool sink = !(E.flags & DL_FLAG_NO_DENSE_SINK);
    for (uint32_t r : S.rels) {
        Relation& R = E.rels[r];
        dense_end(R);
        if (R.sink == DL_SINK_COUNT) continue;
        long double bits = 1;
        for (uint32_t c = 0; c < R.arity; c++) bits *= (long double)std::max<uint32_t>(dom[r][c], 1);
        // the dense sink keeps a second copy (the bitmap as of the last extraction)
        const uint64_t room = E.budget > E.used ? (E.budget - E.used) / (sink ? 8 : 4) : 0;
        if (bits / 8 > (long double)std::min(E.dense_bytes, room)) continue;
        const uint64_t words = ((uint64_t)bits + 31) / 32;
        R.dense = E.make(sizeof(uint32_t) * words);
        R.dense_words = words;
        DL_CUDA(cudaMemsetAsync(R.dense->ptr, 0, sizeof(uint32_t) * words, E.stream));
        for (uint32_t c = 0; c < kMaxArity; c++) R.dense_dom[c] = c < R.arity ? std::max<uint32_t>(dom[r][c], 1) : 1;
        dense_set_rows(E, table_of(R.full[0]), R.dense_dom, (uint32_t*)R.dense->ptr);
        if (sink) {
            const uint64_t blocks = (words + kDenseBlockWords - 1) / kDenseBlockWords;
            R.dense_old = E.make(sizeof(uint32_t) * words);
            R.dense_dirty = E.make(blocks);
            DL_CUDA(cudaMemcpyAsync(R.dense_old->ptr, R.dense->ptr, sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice,
                                    E.stream));
            DL_CUDA(cudaMemsetAsync(R.dense_dirty->ptr, 0, blocks, E.stream));
        }
        E.dense_relations++;
    }
}

// Turn one round's join outputs for relation R into its new delta; merge into full.
// Returns |Δ|.
uint64_t absorb_round(Engine& E, Relation& R, PendingOut& P, bool keep_delta) {
    JoinOutput& jo = P.out;
    Index newrows = empty_index(R.arity, identity_perm());
    bool known_unique = false;
    bool filtered = false;   // rows already in full were dropped before sorting
    uint64_t raw = 0;
    for (auto& p : jo.parts) raw += p.n;
    Index d;
    if (R.dense && R.dense_dirty) {
        // dense sink: the joins set their rows' bits; raw parts of other variants are set too,
        // and the round's delta is every bit set since the last extraction (sorted, distinct,
        // absent from the relation)
        for (auto& p : jo.parts) dense_mark(E, R, p);
        jo.parts.clear();
        jo.owners.clear();
        jo.rparts.clear();
        d = dense_take(E, R);
        filtered = true;
    } else if (!jo.rparts.empty() || raw > E.chunk_rows) {
        // reduce every part on its own, then union (memory stays proportional to new tuples)
        Index acc = empty_index(R.arity, identity_perm());
        for (size_t i = 0; i < jo.parts.size(); i++) acc = union_sorted(E, acc, reduce_part(E, R, jo.owners[i], jo.parts[i]));
        jo.parts.clear();
        jo.owners.clear();
        for (Index& rp : jo.rparts) acc = union_sorted(E, acc, rp);
        jo.rparts.clear();
        d = acc;
    } else if (jo.parts.size() == 1 && jo.sorted_unique && R.dense) {
        d = dense_reduce(E, R, jo.parts[0], true);   // sorted and distinct already: no sort
        filtered = true;
    } else if (jo.parts.size() == 1 && jo.sorted_unique) {
        newrows.n = jo.parts[0].n;
        newrows.cap = newrows.n;
        newrows.cols = jo.owners[0];
        known_unique = true;
    } else if (!jo.parts.empty()) {
        uint64_t tot = 0;
        for (auto& p : jo.parts) tot += p.n;
        if (tot >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "round output of 2^32 rows or more");
        DevPtr buf = E.make(sizeof(uint32_t) * R.arity * tot);
        TableView t;
        memset(&t, 0, sizeof(t));
        t.arity = R.arity;
        t.n = tot;
        for (uint32_t c = 0; c < R.arity; c++) t.col[c] = (uint32_t*)buf->ptr + (size_t)c * tot;
        uint64_t off = 0;
        for (auto& p : jo.parts) {
            for (uint32_t c = 0; c < R.arity; c++)
                DL_CUDA(cudaMemcpyAsync(t.col[c] + off, p.col[c], sizeof(uint32_t) * p.n, cudaMemcpyDeviceToDevice,
                                        E.stream));
            off += p.n;
        }
        jo.parts.clear();
        jo.owners.clear();
        if (R.dense) {
            d = dense_reduce(E, R, t, false);
        } else {
            uint64_t stride = 0;
            auto f = prefilter(E, R, buf, t, stride);
            d = sort_unique_index(E, f.first, f.second, identity_perm(), R.arity, stride);
        }
        filtered = true;
    }
    if (!d.cols && d.n == 0) {
        d = compute_delta(E, newrows, filtered ? empty_index(R.arity, identity_perm()) : R.full[0], identity_perm(),
                          R.arity, known_unique);
        if (!filtered) d = minus_head(E, R, d);
    }
    jo.parts.clear();
    jo.owners.clear();
    E.delta_rows += d.n;
    if (keep_delta) {
        for (size_t k = 0; k < R.perms.size(); k++) R.delta[k] = empty_index(R.arity, R.perms[k]);
        R.delta[0] = d;
    }
    if (d.n == 0) return 0;
    // Recursive rounds (head/body form): Δ is merged into the small head; the body, and its
    // root offsets, stay as they are until the head outgrows E.head_percent of it (paper
    // Section 4, Merge: new tuples go to the head, which is flushed into the body by one
    // merge-path pass above a threshold).  Round 1 merges straight into full.
    const bool to_head = keep_delta && !R.head.empty();
    if (to_head) {
        R.head[0] = merge_into(E, R.head[0], d);
        check_sorted(E, R.head[0], R.name);
    } else {
        R.full[0] = merge_into(E, R.full[0], d);
        check_sorted(E, R.full[0], R.name);
        build_roots(E, R.full[0], R.root_needed[0]);
    }
    for (size_t k = 1; k < R.perms.size(); k++) {
        Index dk = permuted_sorted(E, d, R.perms[k]);
        if (to_head) {
            R.head[k] = merge_into(E, R.head[k], dk);
        } else {
            R.full[k] = merge_into(E, R.full[k], dk);
            build_roots(E, R.full[k], R.root_needed[k]);
        }
        if (keep_delta) {
            build_roots(E, dk, R.root_needed[k]);
            R.delta[k] = dk;
        }
    }
    if (to_head && E.head_percent != UINT32_MAX && R.head[0].n * 100 > (uint64_t)E.head_percent * R.full[0].n)
        flush_head(E, R);
    if (keep_delta) {
        Index d0 = d;
        build_roots(E, d0, R.root_needed[0]);
        R.delta[0] = d0;
    }
    R.full_perms_built = true;
    return d.n;
}

void run_variant(Engine& E, const Variant& v, std::map<uint32_t, PendingOut>& outs) {
    const Rule& r = *v.rule;
    std::vector<const Index*> src(r.body.size());
    std::vector<std::pair<size_t, const Index*>> heads;   // atoms reading a relation in head/body form
    for (size_t a = 0; a < r.body.size(); a++) {
        Relation& B = E.rels[r.body[a].rel];
        uint32_t slot = perm_slot(B, atom_perm(r, (uint32_t)a));
        src[a] = (int)a == v.delta_atom ? &B.delta[slot] : &B.full[slot];
        if ((int)a != v.delta_atom && slot < B.head.size() && B.head[slot].n) heads.push_back({a, &B.head[slot]});
    }
    if (heads.size() > 16) throw Error(DL_ERR_UNSUPPORTED, "more than 16 atoms read relations in head/body form");
    // full = body ∪ head (disjoint): the variant is the union of its evaluations with each such
    // atom reading either part
    const std::vector<const Index*> bodies = src;
    for (uint32_t m = 0; m < (1u << heads.size()); m++) {
        src = bodies;
        for (size_t h = 0; h < heads.size(); h++)
            if ((m >> h) & 1u) src[heads[h].first] = heads[h].second;
        run_variant_on(E, v, src, outs);
    }
}

void run_variant_on(Engine& E, const Variant& v, std::vector<const Index*>& src, std::map<uint32_t, PendingOut>& outs) {
    const Rule& r = *v.rule;
    std::vector<const Index*> nsrc(r.neg.size());   // negated relations: lower strata, read in full
    for (size_t a = 0; a < r.neg.size(); a++) {
        Relation& B = E.rels[r.neg[a].rel];
        nsrc[a] = &B.full[perm_slot(B, neg_perm(r, (uint32_t)a))];
    }
    Relation& H = E.rels[r.head.rel];
    PendingOut& po = outs[r.head.rel];
    JoinOutput jo;
    if (H.sink != DL_SINK_COUNT)
        // each chunk is reduced (rows already in the relation dropped, sorted, deduplicated) and
        // folded into one accumulated part at once, so memory follows the new rows, not the
        // raw bindings of all chunks
        jo.chunk_sink = [&E, &H, &jo](DevPtr buf, TableView t) {
            Index rp = reduce_part(E, H, buf, t);
            if (!rp.n) return;
            if (jo.rparts.empty()) jo.rparts.push_back(rp);
            else jo.rparts[0] = union_sorted(E, jo.rparts[0], rp);
        };
    run_join(E, r, src, nsrc, H, jo);
    if (!jo.parts.empty() || !jo.rparts.empty()) {
        po.producers++;
        po.out.sorted_unique = (po.producers == 1) && jo.sorted_unique && jo.rparts.empty();
        for (size_t i = 0; i < jo.parts.size(); i++) {
            po.out.parts.push_back(jo.parts[i]);
            po.out.owners.push_back(jo.owners[i]);
        }
        for (Index& rp : jo.rparts) po.out.rparts.push_back(rp);
        if (jo.parts.size() > 1) po.out.sorted_unique = false;
    }
}

void validate_program(Engine& E) {
    for (size_t ri = 0; ri < E.rules.size(); ri++) {
        const Rule& r = E.rules[ri];
        for (const RuleAtom& a : r.body)
            if (E.rels[a.rel].sink == DL_SINK_COUNT)
                throw Error(DL_ERR_UNSUPPORTED, "count sink '" + E.rels[a.rel].name + "' used in a rule body");
        if (E.rels[r.head.rel].sink == DL_SINK_COUNT) {
            int n = 0;
            for (const Rule& q : E.rules) n += q.head.rel == r.head.rel;
            std::set<uint32_t> hv;
            bool ok = n == 1 && r.head.arity == r.order.size();
            for (uint32_t c = 0; c < r.head.arity && ok; c++)
                ok = r.head.terms[c].kind == DL_TERM_VAR && hv.insert(r.head.terms[c].id).second;
            if (!ok)
                throw Error(DL_ERR_UNSUPPORTED, "count sink '" + E.rels[r.head.rel].name +
                                                    "' needs exactly one rule whose head lists each body variable once");
        }
    }
}

void fixpoint(Engine& E, dl_stats* st) {
    auto t0 = std::chrono::steady_clock::now();
    const uint64_t launches0 = E.launches;
    const uint64_t hub0 = E.hub_keys, slices0 = E.join_slices;
    const uint64_t tuned0 = E.tuned_levels, hits0 = E.tune_hits, flush0 = E.head_flushes, dense0 = E.dense_relations;
    E.join_rows = E.count_rows = E.delta_rows = 0;
    E.peak = E.used;
    E.event_next = 0;
    for (auto& v : E.phases.ev) v.clear();
    E.kev.clear();
    uint64_t klaunch0[DL_KERNEL_KINDS];
    memcpy(klaunch0, E.klaunch, sizeof(klaunch0));
    validate_program(E);
    for (Relation& R : E.rels) flush_pending(E, R);
    // plan: index permutations each atom reads; roots for every index a join probes
    for (const Rule& r : E.rules) {
        for (uint32_t a = 0; a < r.body.size(); a++) {
            Relation& B = E.rels[r.body[a].rel];
            uint32_t slot = perm_slot(B, atom_perm(r, a));
            B.root_needed[slot] = true;
        }
        for (uint32_t a = 0; a < r.neg.size(); a++) {
            Relation& B = E.rels[r.neg[a].rel];
            B.root_needed[perm_slot(B, neg_perm(r, a))] = true;
        }
    }
    for (Relation& R : E.rels) {
        if (R.sink == DL_SINK_COUNT) {
            R.sink_count = 0;
            R.sink_digest[0] = R.sink_digest[1] = 0;
            R.sink_inst.assign(3ull * E.instances, 0);
            continue;
        }
        ensure_full_perms(E, R);
    }
    E.strata = stratify(E);
    for (auto& R : E.rels) R.stratum = -1;
    for (size_t s = 0; s < E.strata.size(); s++)
        for (uint32_t r : E.strata[s].rels) E.rels[r].stratum = (int)s;
    E.inst_rounds.assign(E.strata.size(), std::vector<uint32_t>());

    for (size_t s = 0; s < E.strata.size(); s++) {
        Stratum& S = E.strata[s];
        std::vector<Variant> round1, rec;
        for (const Rule& r : E.rules) {
            if (E.rels[r.head.rel].stratum != (int)s) continue;
            for (uint32_t a = 0; a < r.body.size(); a++) {   // indexes fixed during this stratum
                Relation& B = E.rels[r.body[a].rel];
                if (B.stratum != (int)s) build_hubs(E, B.full[perm_slot(B, atom_perm(r, a))]);
            }
            bool is_rec = false;
            for (const RuleAtom& a : r.body) is_rec = is_rec || E.rels[a.rel].stratum == (int)s;
            if (!is_rec) {
                round1.push_back({&r, -1});
            } else {
                for (size_t j = 0; j < r.body.size(); j++)
                    if (E.rels[r.body[j].rel].stratum == (int)s) rec.push_back({&r, (int)j});
            }
        }
        // Batched form: last[i] = last round in which instance i had a non-empty delta.
        DArray<uint32_t> last;
        if (E.instances) {
            last = E.array<uint32_t>(E.instances);
            DL_CUDA(cudaMemsetAsync(last.p, 0, sizeof(uint32_t) * E.instances, E.stream));
        }
        // Round 1: non-recursive rules over full relations; Δ1 = everything now in the stratum.
        std::map<uint32_t, PendingOut> outs;
        for (const Variant& v : round1) run_variant(E, v, outs);
        bool any = false;
        for (uint32_t r : S.rels) {
            Relation& R = E.rels[r];
            if (R.sink == DL_SINK_COUNT) continue;
            absorb_round(E, R, outs[r], false);
            if (!rec.empty()) {
                for (size_t k = 0; k < R.perms.size(); k++) R.delta[k] = R.full[k];
                any = any || R.full[0].n > 0;
                if (E.instances) mark_runs(E, R.full[0].col(0), R.full[0].n, last.p, 1);
            }
        }
        uint32_t t = 1;
        if (!rec.empty() && any) {
            // the stratum's relations take the head/body form (and, where their column domains
            // are small, a dense bitmap) for the rounds
            dense_begin(E, S);
            for (uint32_t r : S.rels) {
                Relation& R = E.rels[r];
                if (R.sink == DL_SINK_COUNT) continue;
                R.head.clear();
                for (size_t k = 0; k < R.perms.size(); k++) R.head.push_back(empty_index(R.arity, R.perms[k]));
            }
            try {
                for (;;) {
                    t++;
                    outs.clear();
                    for (const Variant& v : rec) run_variant(E, v, outs);
                    uint64_t nd = 0;
                    for (uint32_t r : S.rels) {
                        Relation& R = E.rels[r];
                        if (R.sink == DL_SINK_COUNT) continue;
                        nd += absorb_round(E, R, outs[r], true);
                        if (E.instances) mark_runs(E, R.delta[0].col(0), R.delta[0].n, last.p, t);
                    }
                    if (nd == 0) break;
                }
            } catch (...) {
                // keep the completed rounds: merge what the heads hold back into the bodies
                outs.clear();
                for (uint32_t r : S.rels) {
                    try {
                        flush_head(E, E.rels[r]);
                    } catch (...) {
                    }
                    E.rels[r].head.clear();
                    dense_end(E.rels[r]);
                }
                throw;
            }
            for (uint32_t r : S.rels) {
                flush_head(E, E.rels[r]);
                E.rels[r].head.clear();
                dense_end(E.rels[r]);
            }
        }
        S.rounds = t;
        if (E.instances) {
            std::vector<uint32_t>& ir = E.inst_rounds[s];
            ir.assign(E.instances, 1);
            if (!rec.empty()) {
                DL_CUDA(cudaMemcpyAsync(ir.data(), last.p, sizeof(uint32_t) * E.instances, cudaMemcpyDeviceToHost,
                                        E.stream));
                E.sync();
                for (uint32_t& x : ir) x = x + 1;   // first empty round follows the last non-empty one
            }
        }
        for (uint32_t r : S.rels) {
            Relation& R = E.rels[r];
            for (size_t k = 0; k < R.delta.size(); k++) R.delta[k] = empty_index(R.arity, R.perms[k]);
        }
    }
    E.sync();
    if (st) {
        memset(st, 0, sizeof(*st));
        st->nstrata = (uint32_t)E.strata.size();
        for (size_t s = 0; s < E.strata.size(); s++) {
            st->total_rounds += E.strata[s].rounds;
            if (s < DL_MAX_STRATA) {
                st->rounds[s] = E.strata[s].rounds;
                st->stratum_first_rel[s] = E.strata[s].rels.front();
            }
        }
        st->join_rows = E.join_rows;
        st->count_rows = E.count_rows;
        st->delta_rows = E.delta_rows;
        st->peak_bytes = E.peak;
        st->kernel_launches = E.launches - launches0;
        st->hub_keys = (uint32_t)(E.hub_keys - hub0);
        st->join_slices = (uint32_t)(E.join_slices - slices0);
        st->tuned_levels = (uint32_t)(E.tuned_levels - tuned0);
        st->tune_hits = (uint32_t)(E.tune_hits - hits0);
        st->head_flushes = (uint32_t)(E.head_flushes - flush0);
        st->dense_relations = (uint32_t)(E.dense_relations - dense0);
        double* ms[4] = {&st->ms_join, &st->ms_sort, &st->ms_dedup, &st->ms_merge};
        for (int k = 0; k < 4; k++)
            for (auto& pr : E.phases.ev[k]) {
                float f = 0;
                if (pr.second && cudaEventElapsedTime(&f, pr.first, pr.second) == cudaSuccess) *ms[k] += f;
            }
        for (int k = 0; k < DL_KERNEL_KINDS; k++) st->kernels[k].launches = E.klaunch[k] - klaunch0[k];
        for (const KernelEvent& ke : E.kev) {
            float f = 0;
            if (cudaEventElapsedTime(&f, ke.a, ke.b) != cudaSuccess) continue;
            st->kernels[ke.kind].ms += f;
            st->kernels[ke.kind].alg_bytes += ke.bytes;
            st->kernels[ke.kind].units += ke.units;
            st->kernels[ke.kind].entries += ke.entries;
            if (f > st->top.ms) {
                st->top_kind = (uint32_t)ke.kind;
                st->top.launches = 1;
                st->top.ms = f;
                st->top.alg_bytes = ke.bytes;
                st->top.units = ke.units;
                st->top.entries = ke.entries;
            }
        }
        st->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
}

int guard(dl_engine* h, const std::function<void(Engine&)>& fn) {
    if (!h) return DL_ERR_ARG;
    Engine& E = *reinterpret_cast<Engine*>(h);
    E.err.clear();
    try {
        DL_CUDA(cudaSetDevice(E.device));
        fn(E);
        return DL_OK;
    } catch (const Error& x) {
        E.err = x.what();
        return x.code;
    } catch (const std::bad_alloc&) {
        E.err = "host out of memory";
        return DL_ERR_CAPACITY;
    } catch (const std::exception& x) {
        E.err = x.what();
        return DL_ERR_CUDA;
    }
}

Relation& rel_of(Engine& E, dl_rel_id r) {
    if (r >= E.rels.size()) throw Error(DL_ERR_ARG, "bad relation id " + std::to_string(r));
    return E.rels[r];
}

void load_table(Engine& E, Relation& R, DevPtr buf, TableView t) {
    if (R.sink == DL_SINK_COUNT) throw Error(DL_ERR_STATE, "cannot load facts into a count sink");
    update_max_value(E, t);
    R.pending.push_back({buf, t});
}

void plain_only(Engine& E, const char* what) {
    if (E.instances) throw Error(DL_ERR_STATE, std::string(what) + " is not available on a batched engine");
}

}  // namespace
}  // namespace dl

using namespace dl;

extern "C" {

const char* dl_version(void) { return kVersion; }

int dl_engine_create(const dl_config* cfg, dl_engine** out) {
    if (!out) return DL_ERR_ARG;
    *out = nullptr;
    dl_config c;
    memset(&c, 0, sizeof(c));
    c.device = -1;
    if (cfg) c = *cfg;
    if ((c.alloc == nullptr) != (c.free == nullptr)) return DL_ERR_ARG;
    Engine* E = new (std::nothrow) Engine();
    if (!E) return DL_ERR_CAPACITY;
    try {
        if (c.device < 0) DL_CUDA(cudaGetDevice(&E->device));
        else E->device = c.device;
        DL_CUDA(cudaSetDevice(E->device));
        if (c.stream) {
            E->stream = (cudaStream_t)c.stream;
        } else {
            DL_CUDA(cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking));
            E->own_stream = true;
        }
        size_t fr = 0, tot = 0;
        DL_CUDA(cudaMemGetInfo(&fr, &tot));
        E->budget = c.arena_bytes ? c.arena_bytes : (uint64_t)(fr * 0.9);
        E->ualloc = c.alloc;
        E->ufree = c.free;
        E->uuser = c.alloc_user;
        E->flags = c.flags;
        E->tile_units = c.tile_units;
        int sms = 0;
        DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device));
        E->sms = (uint32_t)std::max(sms, 1);
        E->instances = c.instances;
        if (c.chunk_rows) E->chunk_rows = c.chunk_rows;
        if (c.hub_rows) E->hub_rows = c.hub_rows;
        if (c.head_percent) E->head_percent = c.head_percent;
        if (c.dense_bytes) E->dense_bytes = c.dense_bytes;
        E->frontier_bytes = c.frontier_bytes;
        if (c.tune_cache) {
            E->tune_path = c.tune_cache;
            tune_load(*E, E->tune_path);
        }
        if (!E->ualloc) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = E->device;
            DL_CUDA(cudaMemPoolCreate(&E->pool, &props));
            uint64_t thr = UINT64_MAX;
            DL_CUDA(cudaMemPoolSetAttribute(E->pool, cudaMemPoolAttrReleaseThreshold, &thr));
        }
    } catch (const Error& x) {
        int code = x.code;
        delete E;
        return code;
    }
    *out = reinterpret_cast<dl_engine*>(E);
    return DL_OK;
}

int dl_engine_set_flags(dl_engine* e, uint32_t flags) {
    return guard(e, [&](Engine& E) { E.flags = flags; });
}

void dl_engine_destroy(dl_engine* e) {
    if (!e) return;
    Engine* E = reinterpret_cast<Engine*>(e);
    cudaSetDevice(E->device);
    delete E;
}

const char* dl_last_error(const dl_engine* e) {
    if (!e) return "null engine";
    return reinterpret_cast<const Engine*>(e)->err.c_str();
}

int dl_relation_create(dl_engine* e, const char* name, uint32_t arity, dl_rel_id* out) {
    return guard(e, [&](Engine& E) {
        if (!name || !*name) throw Error(DL_ERR_ARG, "empty relation name");
        const uint32_t stored = arity + (E.instances ? 1 : 0);
        if (arity < 1 || stored > DL_MAX_ARITY) throw Error(DL_ERR_ARG, "arity out of range");
        for (auto& r : E.rels)
            if (r.name == name) throw Error(DL_ERR_ARG, std::string("duplicate relation name ") + name);
        Relation R;
        R.name = name;
        R.arity = stored;
        R.user_arity = arity;
        R.perms.push_back(identity_perm());
        R.full.push_back(empty_index(stored, identity_perm()));
        R.delta.push_back(empty_index(stored, identity_perm()));
        R.root_needed.push_back(false);
        E.rels.push_back(std::move(R));
        if (out) *out = (dl_rel_id)(E.rels.size() - 1);
    });
}

int dl_relation_set_sink(dl_engine* e, dl_rel_id rel, uint32_t sink) {
    return guard(e, [&](Engine& E) {
        Relation& R = rel_of(E, rel);
        if (sink != DL_SINK_STORE && sink != DL_SINK_COUNT) throw Error(DL_ERR_ARG, "bad sink");
        if (sink == DL_SINK_COUNT && (R.full[0].n || !R.pending.empty()))
            throw Error(DL_ERR_STATE, "relation already holds tuples");
        R.sink = sink;
    });
}

int dl_load_facts(dl_engine* e, dl_rel_id rel, const uint32_t* const* cols, uint64_t nrows) {
    return guard(e, [&](Engine& E) {
        plain_only(E, "dl_load_facts");
        Relation& R = rel_of(E, rel);
        if (nrows == 0) return;
        if (!cols) throw Error(DL_ERR_ARG, "null column array");
        for (uint32_t c = 0; c < R.arity; c++)
            if (!cols[c]) throw Error(DL_ERR_ARG, "null column pointer");
        if (nrows >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "2^32 rows or more in one load");
        DevPtr buf = E.make(sizeof(uint32_t) * R.arity * nrows);
        TableView t;
        memset(&t, 0, sizeof(t));
        t.arity = R.arity;
        t.n = nrows;
        for (uint32_t c = 0; c < R.arity; c++) {
            t.col[c] = (uint32_t*)buf->ptr + (size_t)c * nrows;
            DL_CUDA(cudaMemcpyAsync(t.col[c], cols[c], sizeof(uint32_t) * nrows, cudaMemcpyHostToDevice, E.stream));
        }
        load_table(E, R, buf, t);
    });
}

int dl_load_facts_rows(dl_engine* e, dl_rel_id rel, const uint32_t* rows, uint64_t nrows) {
    if (!e) return DL_ERR_ARG;
    Engine& E = *reinterpret_cast<Engine*>(e);
    if (rel >= E.rels.size()) {
        E.err = "bad relation id";
        return DL_ERR_ARG;
    }
    if (nrows == 0) return DL_OK;
    if (!rows) {
        E.err = "null rows";
        return DL_ERR_ARG;
    }
    const uint32_t a = E.rels[rel].user_arity;
    std::vector<std::vector<uint32_t>> cols(a, std::vector<uint32_t>(nrows));
    for (uint64_t i = 0; i < nrows; i++)
        for (uint32_t c = 0; c < a; c++) cols[c][i] = rows[i * a + c];
    std::vector<const uint32_t*> ptrs(a);
    for (uint32_t c = 0; c < a; c++) ptrs[c] = cols[c].data();
    return dl_load_facts(e, rel, ptrs.data(), nrows);
}

int dl_load_facts_device(dl_engine* e, dl_rel_id rel, const uint32_t* const* dcols, uint64_t nrows) {
    return guard(e, [&](Engine& E) {
        plain_only(E, "dl_load_facts_device");
        Relation& R = rel_of(E, rel);
        if (nrows == 0) return;
        if (!dcols) throw Error(DL_ERR_ARG, "null column array");
        if (nrows >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "2^32 rows or more in one load");
        DevPtr buf = E.make(sizeof(uint32_t) * R.arity * nrows);
        TableView t;
        memset(&t, 0, sizeof(t));
        t.arity = R.arity;
        t.n = nrows;
        for (uint32_t c = 0; c < R.arity; c++) {
            if (!dcols[c]) throw Error(DL_ERR_ARG, "null column pointer");
            t.col[c] = (uint32_t*)buf->ptr + (size_t)c * nrows;
            DL_CUDA(cudaMemcpyAsync(t.col[c], dcols[c], sizeof(uint32_t) * nrows, cudaMemcpyDeviceToDevice, E.stream));
        }
        load_table(E, R, buf, t);
    });
}

int dl_relation_clear(dl_engine* e, dl_rel_id rel) {
    return guard(e, [&](Engine& E) {
        Relation& R = rel_of(E, rel);
        R.pending.clear();
        for (size_t k = 0; k < R.perms.size(); k++) {
            R.full[k] = empty_index(R.arity, R.perms[k]);
            R.delta[k] = empty_index(R.arity, R.perms[k]);
        }
        R.full_perms_built = true;
        R.sink_count = 0;
        R.sink_digest[0] = R.sink_digest[1] = 0;
        R.sink_inst.assign(3ull * E.instances, 0);
    });
}

// Validate a rule given through the ABI and convert it (throws Error; changes nothing).
Rule parse_rule(Engine& E, const dl_atom* head, const dl_atom* body, uint32_t nbody, const uint32_t* var_order,
                uint32_t nvars, const dl_atom* neg = nullptr, uint32_t nneg = 0, const dl_cmp* cmps = nullptr,
                uint32_t ncmp = 0) {
    if (!head || !body) throw Error(DL_ERR_ARG, "null head or body");
    if (nbody == 0 || nbody > DL_MAX_BODY) throw Error(DL_ERR_ARG, "body size out of range");
    if (nneg > DL_MAX_NEG || ncmp > DL_MAX_CMP) throw Error(DL_ERR_ARG, "too many negated atoms or comparisons");
    if ((nneg && !neg) || (ncmp && !cmps)) throw Error(DL_ERR_ARG, "null negated atoms or comparisons");
    Rule r;
    auto read = [&](const dl_atom& a, RuleAtom& ra) {
        Relation& R = rel_of(E, a.rel);
        if (a.arity != R.user_arity) throw Error(DL_ERR_ARG, "arity mismatch for relation " + R.name);
        if (!a.terms) throw Error(DL_ERR_ARG, "null terms");
        ra.rel = a.rel;
        ra.arity = a.arity;
        for (uint32_t c = 0; c < a.arity; c++) {
            if (a.terms[c].kind != DL_TERM_VAR && a.terms[c].kind != DL_TERM_CONST)
                throw Error(DL_ERR_ARG, "bad term kind");
            if (a.terms[c].kind == DL_TERM_VAR && a.terms[c].id >= 1024) throw Error(DL_ERR_ARG, "variable id >= 1024");
            ra.terms[c] = a.terms[c];
        }
    };
    std::set<uint32_t> bvars;
    bool unsupported_const = false, unsupported_repeat = false;
    for (uint32_t b = 0; b < nbody; b++) {
        RuleAtom ra;
        read(body[b], ra);
        std::set<uint32_t> here;
        for (uint32_t c = 0; c < ra.arity; c++) {
            if (ra.terms[c].kind == DL_TERM_CONST) {
                unsupported_const = true;
                continue;
            }
            if (!here.insert(ra.terms[c].id).second) unsupported_repeat = true;
            bvars.insert(ra.terms[c].id);
        }
        r.body.push_back(ra);
    }
    read(*head, r.head);
    for (uint32_t c = 0; c < r.head.arity; c++)
        if (r.head.terms[c].kind == DL_TERM_VAR && !bvars.count(r.head.terms[c].id))
            throw Error(DL_ERR_ARG, "head variable not bound by the body");
    bool neg_unsupported = false;
    for (uint32_t n = 0; n < nneg; n++) {
        RuleAtom ra;
        read(neg[n], ra);
        if (E.rels[ra.rel].sink == DL_SINK_COUNT) throw Error(DL_ERR_ARG, "a count sink cannot be negated");
        std::set<uint32_t> here;
        for (uint32_t c = 0; c < ra.arity; c++) {
            if (ra.terms[c].kind == DL_TERM_CONST) {
                neg_unsupported = true;
                continue;
            }
            if (!bvars.count(ra.terms[c].id)) throw Error(DL_ERR_ARG, "negated atom variable not bound by a positive atom");
            if (!here.insert(ra.terms[c].id).second) neg_unsupported = true;
        }
        r.neg.push_back(ra);
    }
    for (uint32_t k = 0; k < ncmp; k++) {
        const dl_cmp& q = cmps[k];
        if (q.op > DL_CMP_NE) throw Error(DL_ERR_ARG, "bad comparison operator");
        for (const dl_term* t : {&q.a, &q.b}) {
            if (t->kind != DL_TERM_VAR && t->kind != DL_TERM_CONST) throw Error(DL_ERR_ARG, "bad term kind");
            if (t->kind == DL_TERM_VAR && !bvars.count(t->id))
                throw Error(DL_ERR_ARG, "comparison variable not bound by a positive atom");
        }
        RuleCmp rc;
        rc.op = q.op;
        rc.a = q.a;
        rc.b = q.b;
        r.cmps.push_back(rc);
    }
    if (bvars.size() + (E.instances ? 1 : 0) > DL_MAX_VARS) throw Error(DL_ERR_ARG, "too many variables");
    if (!var_order || nvars != bvars.size()) throw Error(DL_ERR_ARG, "variable order must list every body variable once");
    std::set<uint32_t> ord(var_order, var_order + nvars);
    if (ord != bvars) throw Error(DL_ERR_ARG, "variable order is not a permutation of the body variables");
    if (neg_unsupported)
        throw Error(DL_ERR_UNSUPPORTED, "negated atoms take distinct variables only on the GPU path");
    r.order.assign(var_order, var_order + nvars);
    if (unsupported_const || unsupported_repeat) {
        // A constant or a repeated variable in a body atom becomes a fresh variable f with the
        // comparisons f <= t and t <= f (equality; t the constant or the first occurrence),
        // checked at f's level: a constant's f leads the variable order (its level keeps only
        // that value of the column), a repeat's f follows its variable.  Same bindings.
        uint32_t next = 1024;   // user variable ids are below 1024
        std::vector<uint32_t> lead;
        std::vector<std::pair<uint32_t, uint32_t>> after;   // (fresh, original)
        for (RuleAtom& ra : r.body) {
            std::set<uint32_t> here;
            for (uint32_t c = 0; c < ra.arity; c++) {
                dl_term& t = ra.terms[c];
                const bool is_const = t.kind == DL_TERM_CONST;
                if (!is_const && here.insert(t.id).second) continue;
                const uint32_t f = next++;
                RuleCmp le1, le2;
                le1.op = le2.op = DL_CMP_LE;
                le1.a.kind = DL_TERM_VAR;
                le1.a.id = f;
                le1.b = t;
                le2.a = t;
                le2.b = le1.a;
                r.cmps.push_back(le1);
                r.cmps.push_back(le2);
                if (is_const) lead.push_back(f);
                else after.push_back({f, t.id});
                t.kind = DL_TERM_VAR;
                t.id = f;
            }
        }
        std::vector<uint32_t> order(lead);
        for (uint32_t v : r.order) {
            order.push_back(v);
            for (auto& fa : after)
                if (fa.second == v) order.push_back(fa.first);
        }
        r.order = order;
        if (r.order.size() + (E.instances ? 1 : 0) > DL_MAX_VARS)
            throw Error(DL_ERR_UNSUPPORTED, "too many variables once body constants and repeats are rewritten");
        if (r.cmps.size() > DL_MAX_CMP)
            throw Error(DL_ERR_UNSUPPORTED, "too many comparisons once body constants and repeats are rewritten");
    }
    if (E.instances) {
        // batched form: the instance id is column 0 of every atom and the first join variable
        const uint32_t inst_var = 0x7fffffffu;
        auto shift = [&](RuleAtom& ra) {
            for (uint32_t c = ra.arity; c > 0; c--) ra.terms[c] = ra.terms[c - 1];
            ra.terms[0].kind = DL_TERM_VAR;
            ra.terms[0].id = inst_var;
            ra.arity++;
        };
        for (RuleAtom& b : r.body) shift(b);
        for (RuleAtom& b : r.neg) shift(b);
        shift(r.head);
        r.order.insert(r.order.begin(), inst_var);
    }
    for (uint32_t c = 0; c < r.head.arity; c++)
        if (r.head.terms[c].kind == DL_TERM_CONST && r.head.terms[c].id == 0xffffffffu)
            throw Error(DL_ERR_UNSUPPORTED, "value 0xFFFFFFFF is reserved");
    return r;
}

void add_rule(Engine& E, const Rule& r, dl_rule_id* out) {
    for (uint32_t c = 0; c < r.head.arity; c++)
        if (r.head.terms[c].kind == DL_TERM_CONST) E.V = std::max(E.V, r.head.terms[c].id + 1);
    E.rules.push_back(r);
    if (out) *out = (dl_rule_id)(E.rules.size() - 1);
}

int dl_rule_add(dl_engine* e, const dl_atom* head, const dl_atom* body, uint32_t nbody, const uint32_t* var_order,
                uint32_t nvars, dl_rule_id* out) {
    return guard(e, [&](Engine& E) { add_rule(E, parse_rule(E, head, body, nbody, var_order, nvars), out); });
}

// Helper-relation splitting (Section 5): the variables of the factored atoms that the rest of
// the rule (other atoms or the head) also uses, in the rule's variable order.
std::vector<uint32_t> split_columns(const dl_atom* head, const dl_atom* body, uint32_t nbody, const uint32_t* var_order,
                                    uint32_t nvars, uint64_t mask) {
    if (!head || !body || !var_order) throw Error(DL_ERR_ARG, "null head, body or variable order");
    if (nbody == 0 || nbody > DL_MAX_BODY) throw Error(DL_ERR_ARG, "body size out of range");
    const uint64_t all = (1ull << nbody) - 1;
    if (mask == 0 || (mask & ~all) || mask == all)
        throw Error(DL_ERR_ARG, "the split must factor out a non-empty proper subset of the body atoms");
    std::set<uint32_t> inside, outside;
    auto vars = [](const dl_atom& a, std::set<uint32_t>& to) {
        if (!a.terms) throw Error(DL_ERR_ARG, "null terms");
        for (uint32_t c = 0; c < a.arity; c++)
            if (a.terms[c].kind == DL_TERM_VAR) to.insert(a.terms[c].id);
    };
    for (uint32_t b = 0; b < nbody; b++) vars(body[b], ((mask >> b) & 1) ? inside : outside);
    vars(*head, outside);
    std::vector<uint32_t> cols;
    for (uint32_t k = 0; k < nvars; k++)
        if (inside.count(var_order[k]) && outside.count(var_order[k])) cols.push_back(var_order[k]);
    if (cols.empty())
        throw Error(DL_ERR_UNSUPPORTED, "the factored atoms share no variable with the rest of the rule");
    return cols;
}

int dl_rule_add_ex(dl_engine* e, const dl_atom* head, const dl_atom* body, uint32_t nbody, const dl_atom* neg,
                   uint32_t nneg, const dl_cmp* cmps, uint32_t ncmp, const uint32_t* var_order, uint32_t nvars,
                   dl_rule_id* out) {
    return guard(e, [&](Engine& E) {
        add_rule(E, parse_rule(E, head, body, nbody, var_order, nvars, neg, nneg, cmps, ncmp), out);
    });
}

int dl_split_columns(const dl_atom* head, const dl_atom* body, uint32_t nbody, const uint32_t* var_order,
                     uint32_t nvars, uint64_t mask, uint32_t* cols, uint32_t cap, uint32_t* ncols) {
    try {
        const std::vector<uint32_t> c = split_columns(head, body, nbody, var_order, nvars, mask);
        if (ncols) *ncols = (uint32_t)c.size();
        if (cols) {
            if (cap < c.size()) return DL_ERR_ARG;
            std::copy(c.begin(), c.end(), cols);
        }
        return DL_OK;
    } catch (const Error& ex) {
        return ex.code;
    } catch (...) {
        return DL_ERR_ARG;
    }
}

int dl_rule_add_split(dl_engine* e, const dl_atom* head, const dl_atom* body, uint32_t nbody, const uint32_t* var_order,
                      uint32_t nvars, uint64_t mask, const char* helper_name, dl_rel_id* helper_rel,
                      dl_rule_id* helper_rule, dl_rule_id* consumer_rule) {
    return guard(e, [&](Engine& E) {
        parse_rule(E, head, body, nbody, var_order, nvars);   // the unsplit rule must be valid
        const std::vector<uint32_t> cols = split_columns(head, body, nbody, var_order, nvars, mask);
        if (!helper_name || !*helper_name) throw Error(DL_ERR_ARG, "empty helper relation name");
        for (auto& r : E.rels)
            if (r.name == helper_name) throw Error(DL_ERR_ARG, std::string("duplicate relation name ") + helper_name);
        if (cols.size() + (E.instances ? 1 : 0) > DL_MAX_ARITY)
            throw Error(DL_ERR_UNSUPPORTED, "the helper relation would have more than DL_MAX_ARITY columns");
        const dl_rel_id hid = (dl_rel_id)E.rels.size();
        std::vector<dl_term> hterms;
        for (uint32_t v : cols) hterms.push_back({DL_TERM_VAR, v});
        const dl_atom hatom = {hid, (uint32_t)cols.size(), hterms.data()};
        std::vector<dl_atom> hbody, cbody;
        std::set<uint32_t> hvars, cvars(cols.begin(), cols.end());
        for (uint32_t b = 0; b < nbody; b++) {
            const bool in = (mask >> b) & 1;
            (in ? hbody : cbody).push_back(body[b]);
            for (uint32_t c = 0; c < body[b].arity; c++)
                if (body[b].terms[c].kind == DL_TERM_VAR) (in ? hvars : cvars).insert(body[b].terms[c].id);
        }
        cbody.push_back(hatom);
        std::vector<uint32_t> horder, corder;   // the rule's order restricted to each body
        for (uint32_t k = 0; k < nvars; k++) {
            if (hvars.count(var_order[k])) horder.push_back(var_order[k]);
            if (cvars.count(var_order[k])) corder.push_back(var_order[k]);
        }
        // the helper relation exists while the two rules are checked; removed again on failure
        Relation R;
        R.name = helper_name;
        R.arity = (uint32_t)cols.size() + (E.instances ? 1 : 0);
        R.user_arity = (uint32_t)cols.size();
        R.perms.push_back(identity_perm());
        R.full.push_back(empty_index(R.arity, identity_perm()));
        R.delta.push_back(empty_index(R.arity, identity_perm()));
        R.root_needed.push_back(false);
        E.rels.push_back(std::move(R));
        Rule hr, cr;
        try {
            hr = parse_rule(E, &hatom, hbody.data(), (uint32_t)hbody.size(), horder.data(), (uint32_t)horder.size());
            cr = parse_rule(E, head, cbody.data(), (uint32_t)cbody.size(), corder.data(), (uint32_t)corder.size());
        } catch (...) {
            E.rels.pop_back();
            throw;
        }
        add_rule(E, hr, helper_rule);
        add_rule(E, cr, consumer_rule);
        if (helper_rel) *helper_rel = hid;
    });
}

int dl_fixpoint(dl_engine* e, dl_stats* stats) {
    return guard(e, [&](Engine& E) {
        E.in_fixpoint = true;
        try {
            fixpoint(E, stats);
        } catch (...) {
            E.in_fixpoint = false;
            throw;
        }
        E.in_fixpoint = false;
    });
}

int dl_stratum_info(dl_engine* e, uint32_t s, dl_rel_id* rels, uint32_t cap, uint32_t* nrels, uint32_t* rounds) {
    return guard(e, [&](Engine& E) {
        if (s >= E.strata.size()) throw Error(DL_ERR_ARG, "bad stratum");
        const Stratum& S = E.strata[s];
        if (nrels) *nrels = (uint32_t)S.rels.size();
        if (rounds) *rounds = S.rounds;
        if (rels)
            for (uint32_t i = 0; i < S.rels.size() && i < cap; i++) rels[i] = S.rels[i];
    });
}

int dl_relation_size(dl_engine* e, dl_rel_id rel, uint64_t* nrows) {
    return guard(e, [&](Engine& E) {
        Relation& R = rel_of(E, rel);
        if (!nrows) throw Error(DL_ERR_ARG, "null output");
        flush_pending(E, R);
        *nrows = R.sink == DL_SINK_COUNT ? R.sink_count : R.full[0].n;
    });
}

static int fetch_impl(dl_engine* e, dl_rel_id rel, uint32_t* const* cols, uint64_t cap, uint64_t* nrows, bool device) {
    return guard(e, [&](Engine& E) {
        plain_only(E, "dl_fetch");
        Relation& R = rel_of(E, rel);
        if (R.sink == DL_SINK_COUNT) throw Error(DL_ERR_STATE, "count sinks hold no tuples; use dl_fetch_digest");
        flush_pending(E, R);
        const Index& ix = R.full[0];
        if (nrows) *nrows = ix.n;
        if (!cols) return;
        if (cap < ix.n) throw Error(DL_ERR_ARG, "cap_rows smaller than the relation");
        for (uint32_t c = 0; c < R.arity; c++) {
            if (!cols[c]) throw Error(DL_ERR_ARG, "null column pointer");
            if (ix.n)
                DL_CUDA(cudaMemcpyAsync(cols[c], ix.col((int)c), sizeof(uint32_t) * ix.n,
                                        device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, E.stream));
        }
        E.sync();
    });
}

int dl_fetch(dl_engine* e, dl_rel_id rel, uint32_t* const* cols_out, uint64_t cap_rows, uint64_t* nrows_out) {
    return fetch_impl(e, rel, cols_out, cap_rows, nrows_out, false);
}

int dl_fetch_device(dl_engine* e, dl_rel_id rel, uint32_t* const* dcols_out, uint64_t cap_rows, uint64_t* nrows_out) {
    return fetch_impl(e, rel, dcols_out, cap_rows, nrows_out, true);
}

int dl_fetch_digest(dl_engine* e, dl_rel_id rel, uint64_t* count, uint64_t digest[2]) {
    return guard(e, [&](Engine& E) {
        Relation& R = rel_of(E, rel);
        if (!count || !digest) throw Error(DL_ERR_ARG, "null output");
        flush_pending(E, R);
        if (R.sink == DL_SINK_COUNT) {
            *count = R.sink_count;
            digest[0] = R.sink_digest[0];
            digest[1] = R.sink_digest[1];
            return;
        }
        auto d = E.array<uint64_t>(3);
        DL_CUDA(cudaMemsetAsync(d.p, 0, 24, E.stream));
        table_digest(E, table_of(R.full[0]), (unsigned long long*)d.p);
        const uint64_t* h = E.readback(d.p, 3);
        *count = h[0];
        digest[0] = h[1];
        digest[1] = h[2];
    });
}

int dl_load_facts_instance(dl_engine* e, dl_rel_id rel, uint32_t inst, const uint32_t* const* cols, uint64_t nrows) {
    return guard(e, [&](Engine& E) {
        if (!E.instances) throw Error(DL_ERR_STATE, "dl_load_facts_instance needs a batched engine");
        Relation& R = rel_of(E, rel);
        if (inst >= E.instances) throw Error(DL_ERR_ARG, "instance out of range");
        if (nrows == 0) return;
        if (!cols) throw Error(DL_ERR_ARG, "null column array");
        for (uint32_t c = 0; c < R.user_arity; c++)
            if (!cols[c]) throw Error(DL_ERR_ARG, "null column pointer");
        if (nrows >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "2^32 rows or more in one load");
        DevPtr buf = E.make(sizeof(uint32_t) * R.arity * nrows);
        TableView t;
        memset(&t, 0, sizeof(t));
        t.arity = R.arity;
        t.n = nrows;
        for (uint32_t c = 0; c < R.arity; c++) t.col[c] = (uint32_t*)buf->ptr + (size_t)c * nrows;
        fill_u32(E, t.col[0], nrows, inst);
        for (uint32_t c = 0; c < R.user_arity; c++)
            DL_CUDA(cudaMemcpyAsync(t.col[c + 1], cols[c], sizeof(uint32_t) * nrows, cudaMemcpyHostToDevice, E.stream));
        load_table(E, R, buf, t);
    });
}

int dl_fetch_instance(dl_engine* e, dl_rel_id rel, uint32_t inst, uint32_t* const* cols_out, uint64_t cap_rows,
                      uint64_t* nrows_out) {
    return guard(e, [&](Engine& E) {
        if (!E.instances) throw Error(DL_ERR_STATE, "dl_fetch_instance needs a batched engine");
        Relation& R = rel_of(E, rel);
        if (inst >= E.instances) throw Error(DL_ERR_ARG, "instance out of range");
        flush_pending(E, R);
        const Index& ix = R.full[0];
        uint64_t lo = 0, hi = 0;
        find_range(E, ix.col(0), ix.n, inst, &lo, &hi);
        if (nrows_out) *nrows_out = hi - lo;
        if (!cols_out) return;
        if (cap_rows < hi - lo) throw Error(DL_ERR_ARG, "cap_rows smaller than the instance's relation");
        for (uint32_t c = 0; c < R.user_arity; c++) {
            if (!cols_out[c]) throw Error(DL_ERR_ARG, "null column pointer");
            if (hi > lo)
                DL_CUDA(cudaMemcpyAsync(cols_out[c], ix.col((int)c + 1) + lo, sizeof(uint32_t) * (hi - lo),
                                        cudaMemcpyDeviceToHost, E.stream));
        }
        E.sync();
    });
}

int dl_instance_digest(dl_engine* e, dl_rel_id rel, uint32_t inst, uint64_t* count, uint64_t digest[2]) {
    return guard(e, [&](Engine& E) {
        if (!E.instances) throw Error(DL_ERR_STATE, "dl_instance_digest needs a batched engine");
        Relation& R = rel_of(E, rel);
        if (inst >= E.instances) throw Error(DL_ERR_ARG, "instance out of range");
        if (!count || !digest) throw Error(DL_ERR_ARG, "null output");
        if (R.sink == DL_SINK_COUNT) {
            const bool have = R.sink_inst.size() == 3ull * E.instances;
            *count = have ? R.sink_inst[3ull * inst] : 0;
            digest[0] = have ? R.sink_inst[3ull * inst + 1] : 0;
            digest[1] = have ? R.sink_inst[3ull * inst + 2] : 0;
            return;
        }
        flush_pending(E, R);
        const Index& ix = R.full[0];
        uint64_t lo = 0, hi = 0;
        find_range(E, ix.col(0), ix.n, inst, &lo, &hi);
        // the instance's rows without the instance column: the digest of the instance alone
        TableView t;
        memset(&t, 0, sizeof(t));
        t.arity = R.user_arity;
        t.n = hi - lo;
        for (uint32_t c = 0; c < R.user_arity; c++) t.col[c] = ix.col((int)c + 1) + lo;
        auto d = E.array<uint64_t>(3);
        DL_CUDA(cudaMemsetAsync(d.p, 0, 24, E.stream));
        table_digest(E, t, (unsigned long long*)d.p);
        const uint64_t* h = E.readback(d.p, 3);
        *count = h[0];
        digest[0] = h[1];
        digest[1] = h[2];
    });
}

int dl_instance_rounds(dl_engine* e, uint32_t inst, uint32_t* rounds, uint32_t cap, uint32_t* nstrata) {
    return guard(e, [&](Engine& E) {
        if (!E.instances) throw Error(DL_ERR_STATE, "dl_instance_rounds needs a batched engine");
        if (inst >= E.instances) throw Error(DL_ERR_ARG, "instance out of range");
        if (nstrata) *nstrata = (uint32_t)E.inst_rounds.size();
        if (rounds)
            for (uint32_t s = 0; s < E.inst_rounds.size() && s < cap; s++)
                rounds[s] = E.inst_rounds[s].empty() ? 0 : E.inst_rounds[s][inst];
    });
}

int dl_tune_save(dl_engine* e, const char* path) {
    return guard(e, [&](Engine& E) {
        if (!path || !*path) throw Error(DL_ERR_ARG, "null path");
        if (!tune_write(E, path)) throw Error(DL_ERR_STATE, std::string("cannot write ") + path);
    });
}

int dl_partition_slices(const uint64_t* C, uint64_t K, uint32_t p, uint64_t* first_key, uint64_t* start_unit) {
    if (!C || !first_key || !start_unit || p == 0) return DL_ERR_ARG;
    const uint64_t T = K ? C[K - 1] : 0;
    const uint64_t step = (T + p - 1) / p;
    for (uint32_t b = 0; b < p; b++) {
        const uint64_t s = std::min<uint64_t>((uint64_t)b * step, T);
        start_unit[b] = s;
        first_key[b] = upper_bound_u64(C, 0, K, s);
    }
    return DL_OK;
}

int dl_decode_unit(const uint64_t* C, const uint64_t* d2, uint64_t K, uint64_t g, uint64_t* key, uint64_t* i1,
                   uint64_t* i2) {
    if (!C || !d2 || !key || !i1 || !i2 || K == 0 || g >= C[K - 1]) return DL_ERR_ARG;
    const uint64_t k = upper_bound_u64(C, 0, K, g);
    const uint64_t local = g - (k ? C[k - 1] : 0);
    if (d2[k] == 0) return DL_ERR_ARG;
    *key = k;
    *i1 = local / d2[k];
    *i2 = local % d2[k];
    return DL_OK;
}

}  // extern "C"
