// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dl.h"

namespace dl {

constexpr int kMaxArity = DL_MAX_ARITY;
constexpr int kMaxVars = DL_MAX_VARS;
constexpr int kMaxAtoms = DL_MAX_BODY;
constexpr int kMaxSrc = 8;   // atoms that mention one variable (sources of one join level)
constexpr uint32_t kDenseRootLimit = 1u << 27;  // dense root offsets only below this domain size
constexpr int kDenseBlockShift = 8;              // dense relation bitmaps: 2^8 words per dirty block
constexpr uint64_t kDenseBlockWords = 1ull << kDenseBlockShift;

// ---------------------------------------------------------------- errors

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define DL_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t err_ = (call);                                                         \
        if (err_ != cudaSuccess)                                                           \
            throw ::dl::Error(DL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(err_)); \
    } while (0)

#define DL_CHECK_LAUNCH() DL_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- memory

class Engine;

// Device allocation owned through a shared pointer so that an index can be aliased by
// several versions (e.g. the first-round delta is the full relation).
struct DevMem {
    Engine* eng = nullptr;
    void* ptr = nullptr;
    size_t bytes = 0;
    DevMem(Engine* e, size_t b);
    ~DevMem();
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
};
using DevPtr = std::shared_ptr<DevMem>;

template <class T>
struct DArray {                 // typed view on a DevPtr
    DevPtr mem;
    T* p = nullptr;
    uint64_t n = 0;
};

// One sorted SoA copy of a relation in a column permutation: col[k] holds relation column
// perm[k].  Rows are distinct and sorted lexicographically over col[0], col[1], ...
struct Index {
    uint32_t arity = 0;
    uint8_t perm[kMaxArity] = {0};
    uint64_t n = 0;
    DevPtr cols;                // arity * cap uint32 (column k at offset k * cap)
    uint64_t cap = 0;
    DevPtr root;                // dense offsets over col[0]: V + 1 uint32 (optional)
    uint32_t rootV = 0;
    DevPtr hub;                 // int32 per col[0] value: bitmap slot of a heavy key, else -1
    DevPtr bits;                // per heavy key: bitmap of its col[1] values over [0, V)
    uint32_t bmwords = 0;       // uint32 words per bitmap (0 = no bitmaps)
    uint32_t hubmin = 0;        // rows of the lightest key with a bitmap
    uint32_t* col(int k) const { return cols ? (uint32_t*)cols->ptr + (size_t)k * cap : nullptr; }
    const uint32_t* root_ptr() const { return root ? (const uint32_t*)root->ptr : nullptr; }
};

// ---------------------------------------------------------------- device views

struct AtomView {               // an index as the join kernels see it
    const uint32_t* col[kMaxArity];
    const uint32_t* root;       // dense root offsets or nullptr
    const int32_t* hub;         // heavy-key bitmap slots or nullptr
    const uint32_t* bits;
    uint32_t bmwords;
    uint32_t hubmin;            // rows of the lightest key with a bitmap
    uint32_t n;
    uint32_t V;
    uint32_t arity;
};
constexpr uint32_t kHubMinRows = 512;              // default: keys with this many rows get a bitmap
constexpr uint64_t kHubBitmapBytes = 1024ull << 20; // bitmap memory per index (at most)


struct TableView {              // a plain SoA table (not necessarily sorted)
    uint32_t* col[kMaxArity];
    uint64_t n;
    uint32_t arity;
};

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t lo, uint32_t hi,
                                                    uint32_t v) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* __restrict__ a, uint32_t lo, uint32_t hi,
                                                    uint32_t v) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first k in [lo, hi) with C[k] > g (C non-decreasing)
__host__ __device__ __forceinline__ uint64_t upper_bound_u64(const uint64_t* C, uint64_t lo, uint64_t hi, uint64_t g) {
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (C[mid] <= g) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Narrow [lo, hi) of an index to the rows whose column d equals v.  At depth 0 the range is
// always the whole index, so the dense root offsets answer in O(1) when present.
__device__ __forceinline__ bool narrow(const AtomView& a, int d, uint32_t v, uint32_t& lo, uint32_t& hi) {
    if (d == 0 && a.root) {
        if (v >= a.V) return false;
        lo = __ldg(a.root + v);
        hi = __ldg(a.root + v + 1);
        return lo < hi;
    }
    const uint32_t* c = a.col[d];
    uint32_t l = lower_bound_u32(c, lo, hi, v);
    if (l >= hi || __ldg(c + l) != v) return false;
    hi = upper_bound_u32(c, l + 1, hi, v);
    lo = l;
    return true;
}

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Tuple hash of the public digest definition (dl_fetch_digest).
__host__ __device__ __forceinline__ uint64_t tuple_hash_step(uint64_t h, uint32_t v, uint32_t j) {
    return mix64(h ^ ((uint64_t)v + 0x9E3779B97F4A7C15ULL * (uint64_t)(j + 1)));
}
constexpr uint64_t kTupleHashSeed = 0x243F6A8885A308D3ULL;

// ---------------------------------------------------------------- primitives (prims.cu)

struct Stream;  // fwd

// Exclusive (or inclusive) scan of n uint64 values in place; returns the total through
// *total_dev (device pointer, may be null).  tmp allocated from the engine.
void scan_u64(Engine& E, uint64_t* data, uint64_t n, bool inclusive, uint64_t* total_dev);
void scan_u32(Engine& E, uint32_t* data, uint64_t n, uint64_t* total_dev, bool inclusive = false);

// Sort the rows of t (arity columns, n rows) lexicographically, col[0] most significant.
// tmp must have the same shape; on return t holds the sorted rows (buffers may be swapped).
// Sorted distinct rows of t written to the table alloc_out(count) returns, through packed
// keys (sorted, deduplicated, unpacked once); false (nothing done) when the rows' varying
// bits do not fit in 64 bits or packing would not shrink them.
bool sort_unique_packed(Engine& E, const TableView& t, const std::function<TableView(uint64_t)>& alloc_out);

// allow_pack: rows whose varying bits fit in 64 bits are sorted as packed keys.
void radix_sort_rows(Engine& E, TableView& t, TableView& tmp, int* passes_out, bool allow_pack = true);

// Dense relation bitmaps (column c of the relation below dom[c]; bit index in mixed radix,
// column 0 most significant).  dense_set_rows sets the rows' bits; dense_filter keeps, in
// input order, the rows whose bit was clear and sets it (so the kept rows are distinct and
// new), returning their count (synchronises).  A row outside the domain is DL_ERR_STATE.
// With `dirty` (one byte per kDenseBlockWords words), every bit that goes from 0 to 1 marks
// its block, and dense_extract later lists the bits set since the last extraction.
void dense_set_rows(Engine& E, const TableView& t, const uint32_t* dom, uint32_t* bits, uint8_t* dirty = nullptr);
uint64_t dense_filter(Engine& E, const TableView& in, const uint32_t* dom, uint32_t* bits, const TableView& out);
// Rows whose bits are set in `bits` but not in `old`, looked for in the blocks marked dirty:
// written in bit order (sorted lexicographically, distinct) to the table alloc_out(count)
// returns; then old = bits and dirty = 0 in those blocks.  Returns the count (synchronises).
uint64_t dense_extract(Engine& E, uint32_t arity, const uint32_t* dom, const uint32_t* bits, uint32_t* old,
                       uint8_t* dirty, uint64_t nwords, const std::function<TableView(uint64_t)>& alloc_out);

// Keep rows that differ from their predecessor and (if full.n > 0) are absent from full.
// in is sorted; writes the kept rows, in order, to out; returns the count (synchronises).
uint64_t unique_anti(Engine& E, const TableView& in, const AtomView* full, const TableView& out);

// Keep the rows of in (any order) that are absent from full; order is kept; returns the
// count (synchronises).
// keep_order = false: one pass, rows come out in no particular order.
uint64_t anti_filter(Engine& E, const TableView& in, const AtomView& full, const TableView& out, bool keep_order = true);

// out = merge(a, b) of two sorted, disjoint tables (a.n + b.n rows).
void merge_rows(Engine& E, const TableView& a, const TableView& b, const TableView& out);

// Dense root offsets: root[v] = first row with col0 >= v, v in [0, V].
void build_root(Engine& E, const uint32_t* col0, uint64_t n, uint32_t* root, uint32_t V);

// Max over the columns (for the value domain) -> *out_dev (uint32, atomicMax).
void column_max(Engine& E, const uint32_t* col, uint64_t n, uint32_t* out_dev);

// Order-independent digest of a table: d[0] += count, d[1] += sum, d[2] ^= xor.
void table_digest(Engine& E, const TableView& t, unsigned long long* d);

// Gather columns: out.col[k] = in.col[perm[k]] (a device copy).
void permute_copy(Engine& E, const TableView& in, const uint8_t* perm, const TableView& out);

// out[i] = v for i < n.
void fill_u32(Engine& E, uint32_t* out, uint64_t n, uint32_t v);

// For a table sorted on col0: last[col0[i]] = t for the first row of every run.
void mark_runs(Engine& E, const uint32_t* col0, uint64_t n, uint32_t* last, uint32_t t);

// [lower_bound, upper_bound) of v in the sorted column col0[0..n) (synchronises).
void find_range(Engine& E, const uint32_t* col0, uint64_t n, uint32_t v, uint64_t* lo, uint64_t* hi);

// Bitmaps of the col[1] values of heavy keys: one block per
// key in hub_keys, bit v of bitmap slot b set iff (hub_keys[b], v) is a row.
void build_hub_bits(Engine& E, const uint32_t* col0_root, const uint32_t* col1, const uint32_t* hub_keys,
                    uint32_t nhubs, uint32_t* bits, uint32_t bmwords);

// Check that rows are strictly increasing; returns number of violations (synchronises).
uint64_t count_order_violations(Engine& E, const TableView& t);

}  // namespace dl
