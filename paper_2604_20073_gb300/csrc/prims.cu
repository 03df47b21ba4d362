// Data-parallel primitives of the semi-naive loop: device prefix scan, LSD radix sort of
// SoA rows, adjacent dedup + anti-join against the full relation (Compute Delta), merge-path
// merge (Merge), dense root offsets (Build Index), digests.
//
// Paper context: Section 4 names the phases Compute Delta (filter new tuples against the
// full relation), Build Index (sort new tuples into lexicographic SoA order) and Merge
// (single-pass GPU merge path, Green et al. 2012); Algorithm 1 uses prefix sums for the
// work histogram and for the count -> offset step.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <functional>

#include "engine.h"

namespace dl {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread; *total gets the block sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T& total) {
    __shared__ T warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    T x = warp_inclusive_scan(v);
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_sums[lane] : T(0);
        w = warp_inclusive_scan(w);
        warp_sums[lane] = w;
    }
    __syncthreads();
    T prefix = warp ? warp_sums[warp - 1] : T(0);
    total = warp_sums[nwarps - 1];
    __syncthreads();
    return prefix + x - v;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, uint64_t n, T* __restrict__ sums) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += in[base + k];
    T total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_down(T* __restrict__ data, uint64_t n, const T* __restrict__ offs, bool inclusive,
                            uint64_t* total_out) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = base + k < n ? data[base + k] : T(0);
        s += v[k];
    }
    T total;
    T run = block_exclusive_scan(s, total) + (offs ? offs[blockIdx.x] : T(0));
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        T x = v[k];
        if (base + k < n) data[base + k] = inclusive ? run + x : run;
        run += x;
    }
    if (total_out && threadIdx.x == 0) *total_out = (uint64_t)total;
}

template <typename T>
void scan_impl(Engine& E, T* data, uint64_t n, bool inclusive, uint64_t* total_dev) {
    if (n == 0) {
        if (total_dev) DL_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), E.stream));
        return;
    }
    uint64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        KernelScope ks(E, DL_K_SCAN, 2 * sizeof(T) * n);
        k_scan_down<T><<<1, kScanThreads, 0, E.stream>>>(data, n, nullptr, inclusive, total_dev);
        DL_CHECK_LAUNCH();
        return;
    }
    auto sums = E.array<T>(nb);
    {
        KernelScope ks(E, DL_K_SCAN, sizeof(T) * n);
        k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, E.stream>>>(data, n, sums.p);
        DL_CHECK_LAUNCH();
    }
    scan_impl<T>(E, sums.p, nb, false, total_dev);
    KernelScope ks(E, DL_K_SCAN, 2 * sizeof(T) * n);
    k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, E.stream>>>(data, n, sums.p, inclusive, nullptr);
    DL_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ radix sort

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void k_varying_bits(const uint32_t* __restrict__ col, uint64_t n, uint32_t* out) {
    uint32_t first = col[0];
    uint32_t acc = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        acc |= col[i] ^ first;
#pragma unroll
    for (int o = 16; o; o >>= 1) acc |= __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(out, acc);
}

__global__ void k_radix_hist(const uint32_t* __restrict__ key, uint64_t n, uint32_t shift,
                             uint32_t* __restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
    for (int j = threadIdx.x; j < kSortTile; j += blockDim.x) {
        uint64_t i = base + j;
        uint32_t d = i < n ? (key[i] >> shift) & (kRadix - 1) : 0xffffffffu;
        unsigned peers = __match_any_sync(kFull, d);
        if (i < n && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(uint64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: warp w of the block owns the contiguous rows [base + w*32*I, base + (w+1)*32*I);
// iteration j handles row base + w*32*I + j*32 + lane, so (j, lane) order is row order.  Each
// row's rank within its digit is found with a warp match; the tile's rows are then staged in
// shared memory in digit order and written out so that consecutive threads store consecutive
// rows of one digit's run (coalesced), instead of every lane storing to a different run.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const __grid_constant__ TableView src,
                                                                const __grid_constant__ TableView dst, int keycol,
                                                                uint32_t shift, const uint32_t* __restrict__ offs,
                                                                uint32_t ntiles) {
    extern __shared__ uint32_t stage[];                  // arity x kSortTile rows, digit order
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    __shared__ uint32_t lstart[kRadix], gstart[kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t n = src.n;
    const uint64_t tbase = (uint64_t)blockIdx.x * kSortTile;
    const uint32_t tn = (uint32_t)min((uint64_t)kSortTile, n - tbase);
    const uint64_t wbase = tbase + (uint64_t)warp * 32 * kSortItems;
    const unsigned lt = (1u << lane) - 1;
    uint32_t rank[kSortItems], dig[kSortItems];
    const uint32_t* key = src.col[keycol];
#pragma unroll
    for (int j = 0; j < kSortItems; j++) {
        uint64_t i = wbase + (uint64_t)j * 32 + lane;
        bool valid = i < n;
        uint32_t d = valid ? (key[i] >> shift) & (kRadix - 1) : 0xffffffffu;
        unsigned peers = __match_any_sync(kFull, d);
        uint32_t before = valid ? wcnt[warp][d] : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt);
        dig[j] = d;
    }
    __syncthreads();
    // per digit (one per thread): the warps' prefix within the digit, the tile's digit total
    uint32_t tot = 0;
    {
        const int d = threadIdx.x;
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = tot;
            tot += c;
        }
        gstart[d] = offs[(uint64_t)d * ntiles + blockIdx.x];
    }
    uint32_t all;
    const uint32_t ls = block_exclusive_scan(tot, all);   // the digit's first row in the tile
    lstart[threadIdx.x] = ls;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; j++) {
        uint64_t i = wbase + (uint64_t)j * 32 + lane;
        if (i < n) {
            const uint32_t lp = lstart[dig[j]] + wcnt[warp][dig[j]] + rank[j];
            for (uint32_t c = 0; c < src.arity; c++) stage[c * kSortTile + lp] = src.col[c][i];
        }
    }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < tn; p += kSortThreads) {
        const uint32_t d = (stage[keycol * kSortTile + p] >> shift) & (kRadix - 1);
        const uint64_t to = (uint64_t)gstart[d] + (p - lstart[d]);
        for (uint32_t c = 0; c < src.arity; c++) dst.col[c][to] = stage[c * kSortTile + p];
    }
}

// Packed sort keys: the varying low bits of every column (column 0 most significant)
// concatenated into one 64-bit key, held as one (width <= 32) or two uint32 columns.
struct PackSpec {
    uint32_t arity, kcols;
    uint32_t width[kMaxArity];      // varying low bits of each column
    uint32_t high[kMaxArity];       // the constant bits above them (from the first row)
};

__global__ void k_pack_keys(const __grid_constant__ TableView t, const __grid_constant__ PackSpec S,
                            uint32_t* __restrict__ khi, uint32_t* __restrict__ klo) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < t.n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
        for (uint32_t c = 0; c < S.arity; c++) {
            const uint32_t w = S.width[c];
            if (!w) continue;
            k = (k << w) | (uint64_t)(t.col[c][i] & (w == 32 ? 0xFFFFFFFFu : (1u << w) - 1u));
        }
        if (S.kcols == 2) {
            khi[i] = (uint32_t)(k >> 32);
            klo[i] = (uint32_t)k;
        } else {
            klo[i] = (uint32_t)k;
        }
    }
}

__global__ void k_unpack_keys(const uint32_t* __restrict__ khi, const uint32_t* __restrict__ klo, uint64_t n,
                              const __grid_constant__ PackSpec S, const __grid_constant__ TableView t) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = S.kcols == 2 ? ((uint64_t)khi[i] << 32) | klo[i] : klo[i];
        for (int c = (int)S.arity - 1; c >= 0; c--) {
            const uint32_t w = S.width[c];
            const uint32_t low = w ? (uint32_t)(k & (w == 32 ? 0xFFFFFFFFull : ((1ull << w) - 1))) : 0u;
            t.col[c][i] = S.high[c] | low;
            k = w == 64 ? 0 : (k >> w);
        }
    }
}

// ------------------------------------------------------------- compaction

constexpr int kCompThreads = 256;
constexpr int kCompItems = 16;
constexpr int kCompTile = kCompThreads * kCompItems;

__device__ __forceinline__ bool row_equal(const TableView& t, uint64_t i, uint64_t j) {
    for (uint32_t c = 0; c < t.arity; c++)
        if (t.col[c][i] != t.col[c][j]) return false;
    return true;
}

__device__ bool contains_row(const AtomView& a, const TableView& t, uint64_t i) {
    uint32_t lo = 0, hi = a.n;
    for (uint32_t c = 0; c < a.arity; c++)
        if (!narrow(a, (int)c, t.col[c][i], lo, hi)) return false;
    return true;
}

struct UniqueAnti {
    TableView in;
    AtomView full;
    bool use_full;
    __device__ bool operator()(uint64_t i) const {
        if (i > 0 && row_equal(in, i, i - 1)) return false;
        return !use_full || !contains_row(full, in, i);
    }
};

// Is row i absent from full?  Called by all 32 lanes of a warp on 32 consecutive rows.  Rows
// usually arrive grouped by their leading columns (joins emit them in prefix order), so only
// the first lane of each run of equal leading columns narrows the full index down to that
// prefix; the rest of the run takes the range by shuffle and searches the last column only.
__device__ __forceinline__ bool absent_row_warp(const AtomView& full, const TableView& in, uint64_t i, bool valid) {
    const int lane = threadIdx.x & 31;
    const uint32_t a = in.arity;
    bool head = true;
    if (valid && a > 1 && lane > 0 && i > 0) {
        head = false;
        for (uint32_t c = 0; c + 1 < a; c++)
            if (in.col[c][i] != in.col[c][i - 1]) {
                head = true;
                break;
            }
    }
    uint32_t lo = 0, hi = full.n, pok = 1;
    if (head && valid)
        for (uint32_t c = 0; c + 1 < a && pok; c++) pok = narrow(full, (int)c, in.col[c][i], lo, hi) ? 1u : 0u;
    const unsigned heads = __ballot_sync(kFull, head);
    const int src = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    lo = __shfl_sync(kFull, lo, src);
    hi = __shfl_sync(kFull, hi, src);
    pok = __shfl_sync(kFull, pok, src);
    if (!valid) return false;
    if (!pok) return true;
    uint32_t l = lo, h = hi;
    return !narrow(full, (int)a - 1, in.col[a - 1][i], l, h);
}

__global__ void k_absent_count(const __grid_constant__ TableView in, const __grid_constant__ AtomView full,
                               uint64_t* __restrict__ block_count) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t c = 0;
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        if (absent_row_warp(full, in, i, i < in.n)) c++;
    }
    uint64_t total;
    block_exclusive_scan(c, total);
    if (threadIdx.x == 0) block_count[blockIdx.x] = total;
}

__global__ void k_absent_write(const __grid_constant__ TableView in, const __grid_constant__ AtomView full,
                               const __grid_constant__ TableView out, const uint64_t* __restrict__ block_off) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t run = block_off[blockIdx.x];
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        const uint32_t f = absent_row_warp(full, in, i, i < in.n) ? 1u : 0u;
        uint32_t total;
        const uint32_t pos = block_exclusive_scan(f, total);
        if (f)
            for (uint32_t c = 0; c < in.arity; c++) out.col[c][run + pos] = in.col[c][i];
        run += total;
    }
}

// Unordered variant (one pass): each warp appends its absent rows at an offset taken from
// one global counter with a single atomic; rows keep no particular order.
__global__ void k_absent_append(const __grid_constant__ TableView in, const __grid_constant__ AtomView full,
                                const __grid_constant__ TableView out, unsigned long long* __restrict__ counter) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        const bool f = absent_row_warp(full, in, i, i < in.n);
        const unsigned ball = __ballot_sync(kFull, f);
        if (!ball) continue;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(counter, (unsigned long long)__popc(ball));
        at = __shfl_sync(kFull, at, 0);
        if (f) {
            const uint64_t o = at + __popc(ball & ((1u << lane) - 1));
            for (uint32_t c = 0; c < in.arity; c++) out.col[c][o] = in.col[c][i];
        }
    }
}

template <class Pred>
__global__ void k_flag_count(const __grid_constant__ Pred pred, uint64_t n, uint64_t* __restrict__ block_count) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t c = 0;
    for (int j = threadIdx.x; j < kCompTile; j += blockDim.x) {
        uint64_t i = base + j;
        if (i < n && pred(i)) c++;
    }
    uint64_t total;
    block_exclusive_scan(c, total);
    if (threadIdx.x == 0) block_count[blockIdx.x] = total;
}

template <class Pred>
__global__ void k_flag_write(const __grid_constant__ Pred pred, const __grid_constant__ TableView in,
                             const __grid_constant__ TableView out, const uint64_t* __restrict__ block_off) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t run = block_off[blockIdx.x];
    for (int j = 0; j < kCompItems; j++) {
        uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        uint32_t f = (i < in.n && pred(i)) ? 1u : 0u;
        uint32_t total;
        uint32_t pos = block_exclusive_scan(f, total);
        if (f)
            for (uint32_t c = 0; c < in.arity; c++) out.col[c][run + pos] = in.col[c][i];
        run += total;
    }
}

// Distinct packed keys (sorted): a row is kept when its key differs from the previous one.
__device__ __forceinline__ bool key_starts(const uint32_t* khi, const uint32_t* klo, uint64_t i) {
    return i == 0 || klo[i] != klo[i - 1] || (khi && khi[i] != khi[i - 1]);
}

__global__ void k_key_distinct_count(const uint32_t* __restrict__ khi, const uint32_t* __restrict__ klo, uint64_t n,
                                     uint64_t* __restrict__ block_count) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t c = 0;
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        if (i < n && key_starts(khi, klo, i)) c++;
    }
    uint64_t total;
    block_exclusive_scan(c, total);
    if (threadIdx.x == 0) block_count[blockIdx.x] = total;
}

__global__ void k_key_distinct_write(const uint32_t* __restrict__ khi, const uint32_t* __restrict__ klo, uint64_t n,
                                     const __grid_constant__ PackSpec S, const __grid_constant__ TableView out,
                                     const uint64_t* __restrict__ block_off) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t run = block_off[blockIdx.x];
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        const uint32_t f = (i < n && key_starts(khi, klo, i)) ? 1u : 0u;
        uint32_t total;
        const uint32_t pos = block_exclusive_scan(f, total);
        if (f) {
            uint64_t k = S.kcols == 2 ? ((uint64_t)khi[i] << 32) | klo[i] : klo[i];
            for (int c = (int)S.arity - 1; c >= 0; c--) {
                const uint32_t w = S.width[c];
                const uint32_t low = w ? (uint32_t)(k & (w == 32 ? 0xFFFFFFFFull : ((1ull << w) - 1))) : 0u;
                out.col[c][run + pos] = S.high[c] | low;
                k >>= w;
            }
        }
        run += total;
    }
}

// Dense relation bitmaps: bit v0 * d1 * d2 ... + v1 * d2 ... + v(a-1) of a relation whose column c
// holds values below dom.d[c].
struct DenseDom {
    uint32_t arity;
    uint32_t d[kMaxArity];
};

__device__ __forceinline__ uint64_t dense_index(const TableView& t, uint64_t i, const DenseDom& D, bool& ok) {
    uint64_t idx = 0;
    for (uint32_t c = 0; c < D.arity; c++) {
        const uint32_t v = t.col[c][i];
        ok = ok && v < D.d[c];
        idx = idx * D.d[c] + v;
    }
    return idx;
}

__global__ void k_dense_set(const __grid_constant__ TableView t, const __grid_constant__ DenseDom D,
                            uint32_t* __restrict__ bits, uint8_t* __restrict__ dirty,
                            unsigned long long* __restrict__ bad) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < t.n; i += (uint64_t)gridDim.x * blockDim.x) {
        bool ok = true;
        const uint64_t idx = dense_index(t, i, D, ok);
        if (!ok) {
            atomicAdd(bad, 1ull);
            continue;
        }
        uint32_t* w = bits + (idx >> 5);
        const uint32_t m = 1u << (idx & 31);
        if (__ldcg(w) & m) continue;   // set already (bits only go from 0 to 1 here)
        if (!(atomicOr(w, m) & m) && dirty) dirty[idx >> (5 + kDenseBlockShift)] = 1;
    }
}

// Dense extraction: the bits set in `bits` but not in `old`.  A warp takes a group of 32
// consecutive blocks of kDenseBlockWords words: lane l reads block l's dirty byte, and the warp
// walks the dirty blocks of the group in order, 8 words per lane.  Count pass: per group.
constexpr int kExtractWarps = 8;
constexpr int kWordsPerLane = (int)(kDenseBlockWords / 32);

__device__ __forceinline__ uint32_t block_new_words(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ old,
                                                    uint64_t w0, uint64_t nwords, uint32_t (&nw)[kWordsPerLane]) {
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kWordsPerLane; k++) {
        nw[k] = w0 + k < nwords ? bits[w0 + k] & ~old[w0 + k] : 0u;
        c += __popc(nw[k]);
    }
    return c;
}

__global__ void k_dense_group_count(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ old,
                                    const uint8_t* __restrict__ dirty, uint64_t nwords, uint64_t nblocks,
                                    uint64_t ngroups, uint64_t* __restrict__ gcnt) {
    const uint64_t g = blockIdx.x * (uint64_t)kExtractWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ngroups) return;
    const uint64_t b0 = g * 32;
    uint32_t m = __ballot_sync(0xffffffffu, b0 + lane < nblocks && dirty[b0 + lane]);
    uint32_t c = 0;
    while (m) {
        const uint64_t b = b0 + (uint64_t)(__ffs(m) - 1);
        m &= m - 1;
        uint32_t nw[kWordsPerLane];
        c += block_new_words(bits, old, b * kDenseBlockWords + (uint64_t)lane * kWordsPerLane, nwords, nw);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) gcnt[g] = c;
}

// Write pass: per dirty block, 32 words at a time (word k of the step on lane k): the step's
// new rows are dealt out in bit order, row p to lane p mod 32, so consecutive lanes store
// consecutive rows (coalesced).  The lane of row p is found by a search over the lanes'
// exclusive counts, the bit by its rank in that lane's word; the word's first index is
// decoded into columns once (mixed radix) and the bit's offset added with carries.  Then the
// block's old words take the current bits and the block is clean again.
__global__ void k_dense_group_write(const uint32_t* __restrict__ bits, uint32_t* __restrict__ old,
                                    uint8_t* __restrict__ dirty, uint64_t nwords, uint64_t nblocks, uint64_t ngroups,
                                    const uint64_t* __restrict__ goff, const __grid_constant__ DenseDom D,
                                    const __grid_constant__ TableView out) {
    const uint64_t g = blockIdx.x * (uint64_t)kExtractWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ngroups) return;
    const uint64_t b0 = g * 32;
    const bool mine = b0 + lane < nblocks && dirty[b0 + lane];
    uint32_t m = __ballot_sync(0xffffffffu, mine);
    uint64_t run = goff[g];
    while (m) {
        const uint64_t b = b0 + (uint64_t)(__ffs(m) - 1);
        m &= m - 1;
        for (int step = 0; step < kWordsPerLane; step++) {
            const uint64_t w = b * kDenseBlockWords + (uint64_t)step * 32 + lane;
            const uint32_t x = w < nwords ? bits[w] & ~old[w] : 0u;
            const uint32_t c = __popc(x);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - c, n = __shfl_sync(0xffffffffu, incl, 31);
            if (n == 0) continue;
            if (x) old[w] |= x;
            // the lane's word's first bit index, as columns (columns at and above D.arity: 0)
            uint32_t dig[kMaxArity];
            {
                uint64_t q = w * 32;
#pragma unroll
                for (int col = kMaxArity - 1; col >= 0; col--) {
                    dig[col] = 0;
                    if (col < (int)D.arity) {
                        dig[col] = (uint32_t)(q % D.d[col]);
                        q /= D.d[col];
                    }
                }
            }
            for (uint32_t j = 0; j < n; j += 32) {
                const uint32_t p = j + lane;
                // source lane: the last lane whose exclusive count is <= p
                int src = 0;
#pragma unroll
                for (int h = 16; h; h >>= 1) {
                    const uint32_t e = __shfl_sync(0xffffffffu, excl, src + h);
                    if (e <= p) src += h;
                }
                const uint32_t xs = __shfl_sync(0xffffffffu, x, src);
                const uint32_t k = p - __shfl_sync(0xffffffffu, excl, src);
                uint32_t add = p < n ? (uint32_t)__fns(xs, 0, (int)k + 1) : 0u;
                uint32_t v[kMaxArity];
#pragma unroll
                for (int col = 0; col < kMaxArity; col++) v[col] = __shfl_sync(0xffffffffu, dig[col], src);
#pragma unroll
                for (int col = kMaxArity - 1; col >= 0; col--) {
                    if (col >= (int)D.arity || !add) continue;
                    uint64_t t = (uint64_t)v[col] + add;
                    add = 0;
                    while (t >= D.d[col]) {
                        t -= D.d[col];
                        add++;
                    }
                    v[col] = (uint32_t)t;
                }
                if (p < n) {
#pragma unroll
                    for (int col = 0; col < kMaxArity; col++)
                        if (col < (int)D.arity) out.col[col][run + p] = v[col];
                }
            }
            run += n;
        }
    }
    if (mine) dirty[b0 + lane] = 0;
}

// Test-and-set every row's bit: a row is new iff its bit was clear (it is neither in the
// relation nor earlier in this input).  flags[i] = 1 for new rows; per-tile counts.  Bits only
// go from 0 to 1 here, so a set bit read from L2 settles the row without the atomic; most
// rows of a projecting rule are duplicates, and a plain load costs far less than an atomic.
__global__ void k_dense_flags(const __grid_constant__ TableView t, const __grid_constant__ DenseDom D,
                              uint32_t* __restrict__ bits, uint8_t* __restrict__ flags,
                              uint64_t* __restrict__ block_count, unsigned long long* __restrict__ bad) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t c = 0;
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        if (i >= t.n) continue;
        bool ok = true;
        const uint64_t idx = dense_index(t, i, D, ok);
        uint8_t f = 0;
        if (!ok) {
            atomicAdd(bad, 1ull);
        } else {
            const uint32_t m = 1u << (idx & 31);
            uint32_t* w = bits + (idx >> 5);
            f = (__ldcg(w) & m) ? 0 : (atomicOr(w, m) & m) ? 0 : 1;
        }
        flags[i] = f;
        c += f;
    }
    uint64_t total;
    block_exclusive_scan(c, total);
    if (threadIdx.x == 0) block_count[blockIdx.x] = total;
}

__global__ void k_dense_write(const __grid_constant__ TableView in, const uint8_t* __restrict__ flags,
                              const __grid_constant__ TableView out, const uint64_t* __restrict__ block_off) {
    const uint64_t base = (uint64_t)blockIdx.x * kCompTile;
    uint64_t run = block_off[blockIdx.x];
    for (int j = 0; j < kCompItems; j++) {
        const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
        const uint32_t f = i < in.n ? flags[i] : 0u;
        uint32_t total;
        const uint32_t pos = block_exclusive_scan(f, total);
        if (f)
            for (uint32_t c = 0; c < in.arity; c++) out.col[c][run + pos] = in.col[c][i];
        run += total;
    }
}

// ------------------------------------------------------------------ merge

constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 8;                            // output rows per thread
constexpr int kMergeTile = kMergeThreads * kMergeItems;   // output rows per CTA

// lexicographic a[i] < b[j]
__device__ __forceinline__ bool row_less(const TableView& a, uint64_t i, const TableView& b, uint64_t j) {
    for (uint32_t c = 0; c < a.arity; c++) {
        uint32_t x = a.col[c][i], y = b.col[c][j];
        if (x != y) return x < y;
    }
    return false;
}

// Merge path (Green et al., the paper's Section 4 Merge): the number of a-rows among the first
// `diag` rows of merge(a, b), a first on ties.
__device__ __forceinline__ uint64_t merge_split(const TableView& a, const TableView& b, uint64_t diag) {
    uint64_t lo = diag > b.n ? diag - b.n : 0, hi = diag < a.n ? diag : a.n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (!row_less(b, diag - 1 - mid, a, mid)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Rows x < y of the staged window (column c of row r at s[c * kMergeTile + r]).
__device__ __forceinline__ bool staged_less(const uint32_t* s, uint32_t arity, uint32_t x, uint32_t y) {
    for (uint32_t c = 0; c < arity; c++) {
        const uint32_t u = s[c * kMergeTile + x], v = s[c * kMergeTile + y];
        if (u != v) return u < v;
    }
    return false;
}

// Merge-path splits of every tile boundary (one thread each, all searches in parallel).
__global__ void k_merge_splits(const __grid_constant__ TableView a, const __grid_constant__ TableView b,
                               uint64_t ntiles, uint64_t* __restrict__ split) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    split[t] = merge_split(a, b, min(t * (uint64_t)kMergeTile, a.n + b.n));
}

// One CTA per kMergeTile output rows: the CTA stages the a- and b-windows between its two
// splits in shared memory with coalesced loads (each thread's loads of a column issued
// before its stores), each thread merges its kMergeItems outputs from shared memory and
// records the staged row each output takes (2 bytes, not the row: a smaller footprint keeps
// more CTAs resident), and the tile is written back with coalesced stores through those
// indexes (every input and output row crosses HBM once).
__global__ void __launch_bounds__(kMergeThreads) k_merge(const __grid_constant__ TableView a,
                                                         const __grid_constant__ TableView b,
                                                         const __grid_constant__ TableView out,
                                                         const uint64_t* __restrict__ split) {
    extern __shared__ uint32_t smem[];
    const uint32_t arity = a.arity;
    uint32_t* sin = smem;                                  // arity x kMergeTile: a-window, then b-window
    uint16_t* sidx = (uint16_t*)(smem + (size_t)arity * kMergeTile);   // kMergeTile: staged row of each output
    const uint64_t total = a.n + b.n;
    const uint64_t d0 = (uint64_t)blockIdx.x * kMergeTile, d1 = min(d0 + kMergeTile, total);
    const uint64_t i0 = split[blockIdx.x], i1 = split[blockIdx.x + 1];
    const uint64_t j0 = d0 - i0;
    const uint32_t na = (uint32_t)(i1 - i0), n = (uint32_t)(d1 - d0), nb = n - na;
    if (na == 0 || nb == 0) {
        // the tile comes from one side only (the common case when a small delta is merged into
        // a large relation): a straight coalesced copy
        for (uint32_t c = 0; c < arity; c++) {
            const uint32_t* src = na ? a.col[c] + i0 : b.col[c] + j0;
            uint32_t* oc = out.col[c] + d0;
            for (uint32_t t = threadIdx.x; t < n; t += kMergeThreads) oc[t] = src[t];
        }
        return;
    }
    for (uint32_t c = 0; c < arity; c++) {
        const uint32_t* ac = a.col[c] + i0;
        const uint32_t* bc = b.col[c] + j0;
        uint32_t r[kMergeItems];
#pragma unroll
        for (int k = 0; k < kMergeItems; k++) {
            const uint32_t t = threadIdx.x + (uint32_t)k * kMergeThreads;
            r[k] = t < na ? ac[t] : t < n ? bc[t - na] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kMergeItems; k++) {
            const uint32_t t = threadIdx.x + (uint32_t)k * kMergeThreads;
            if (t < n) sin[c * kMergeTile + t] = r[k];
        }
    }
    __syncthreads();
    const uint32_t dd = min((uint32_t)threadIdx.x * kMergeItems, n);
    uint32_t lo = dd > nb ? dd - nb : 0, hi = min(dd, na);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (!staged_less(sin, arity, na + (dd - 1 - mid), mid)) lo = mid + 1; else hi = mid;
    }
    uint32_t ia = lo, ib = dd - lo;
    const uint32_t end = min(dd + kMergeItems, n);
    for (uint32_t k = dd; k < end; k++) {
        const bool take_a = ib >= nb || (ia < na && !staged_less(sin, arity, na + ib, ia));
        sidx[k] = (uint16_t)(take_a ? ia++ : na + ib++);
    }
    __syncthreads();
    for (uint32_t c = 0; c < arity; c++) {
        uint32_t* oc = out.col[c] + d0;
        for (uint32_t t = threadIdx.x; t < n; t += kMergeThreads) oc[t] = sin[c * kMergeTile + sidx[t]];
    }
}

// ------------------------------------------------------------------ misc

__global__ void k_build_root(const uint32_t* __restrict__ col0, uint32_t n, uint32_t* __restrict__ root, uint32_t V) {
    uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v > V) return;
    root[v] = v == V ? n : lower_bound_u32(col0, 0, n, (uint32_t)v);
}

__global__ void k_column_max(const uint32_t* __restrict__ col, uint64_t n, uint32_t* out) {
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, col[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_digest(const __grid_constant__ TableView t, unsigned long long* d) {
    unsigned long long s = 0, x = 0, c = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < t.n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t h = kTupleHashSeed;
        for (uint32_t j = 0; j < t.arity; j++) h = tuple_hash_step(h, t.col[j][i], j);
        s += h;
        x ^= h;
        c++;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(kFull, s, o);
        x ^= __shfl_xor_sync(kFull, x, o);
        c += __shfl_xor_sync(kFull, c, o);
    }
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(&d[0], c);
        atomicAdd(&d[1], s);
        atomicXor(&d[2], x);
    }
}

__global__ void k_order_violations(const __grid_constant__ TableView t, unsigned long long* out) {
    unsigned long long c = 0;
    for (uint64_t i = 1 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < t.n; i += (uint64_t)gridDim.x * blockDim.x)
        if (!row_less(t, i - 1, t, i)) c++;
    if (c) atomicAdd(out, c);
}

__global__ void k_fill_u32(uint32_t* __restrict__ out, uint64_t n, uint32_t v) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

__global__ void k_mark_runs(const uint32_t* __restrict__ col0, uint64_t n, uint32_t* __restrict__ last, uint32_t t) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (i == 0 || col0[i] != col0[i - 1]) last[col0[i]] = t;
}

__global__ void k_find_range(const uint32_t* __restrict__ col0, uint64_t n, uint32_t v, unsigned long long* out) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (col0[mid] < v) lo = mid + 1; else hi = mid;
    }
    uint64_t lo2 = lo, hi2 = n;
    while (lo2 < hi2) {
        uint64_t mid = (lo2 + hi2) >> 1;
        if (col0[mid] <= v) lo2 = mid + 1; else hi2 = mid;
    }
    out[0] = lo;
    out[1] = lo2;
}

__global__ void k_hub_bits(const uint32_t* __restrict__ root, const uint32_t* __restrict__ col1,
                           const uint32_t* __restrict__ hub_keys, uint32_t* __restrict__ bits, uint32_t bmwords) {
    const uint32_t key = hub_keys[blockIdx.x];
    uint32_t* bm = bits + (uint64_t)blockIdx.x * bmwords;
    for (uint32_t r = root[key] + threadIdx.x; r < root[key + 1]; r += blockDim.x) {
        const uint32_t v = col1[r];
        atomicOr(bm + (v >> 5), 1u << (v & 31));
    }
}

unsigned grid_for(uint64_t n, int threads, unsigned cap = 152u * 16u) {
    uint64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, cap));
}

}  // namespace

void scan_u64(Engine& E, uint64_t* data, uint64_t n, bool inclusive, uint64_t* total_dev) {
    scan_impl<unsigned long long>(E, (unsigned long long*)data, n, inclusive, total_dev);
}

void scan_u32(Engine& E, uint32_t* data, uint64_t n, uint64_t* total_dev, bool inclusive) {
    scan_impl<uint32_t>(E, data, n, inclusive, total_dev);
}

void radix_sort_rows(Engine& E, TableView& t, TableView& tmp, int* passes_out, bool allow_pack) {
    int passes = 0;
    const uint64_t n = t.n;
    // the scatter's staging buffer: up to kMaxArity x kSortTile rows (raised once per device)
    static std::atomic<uint64_t> attr_set{0};
    const uint64_t bit = 1ull << (E.device & 63);
    if (!(attr_set.load() & bit)) {
        DL_CUDA(cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(uint32_t) * kMaxArity * kSortTile)));
        attr_set.fetch_or(bit);
    }
    if (n > 1) {
        if (n >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "sort of 2^32 rows or more");
        auto bits = E.array<uint32_t>(kMaxArity);
        DL_CUDA(cudaMemsetAsync(bits.p, 0, sizeof(uint32_t) * kMaxArity, E.stream));
        for (uint32_t c = 0; c < t.arity; c++) {
            KernelScope ks(E, DL_K_SORT, 4 * n);
            k_varying_bits<<<grid_for(n, 256), 256, 0, E.stream>>>(t.col[c], n, bits.p + c);
            DL_CHECK_LAUNCH();
        }
        uint32_t hbits[kMaxArity];
        const uint64_t* hb = E.readback(bits.p, kMaxArity / 2);
        memcpy(hbits, hb, sizeof(uint32_t) * t.arity);
        // Rows whose varying bits fit in 64 bits are sorted as one packed key (one or two
        // columns instead of all of them, and no pass over constant bits), then unpacked
        // in place: the same order, fewer bytes per pass.
        uint32_t wsum = 0;
        PackSpec S;
        memset(&S, 0, sizeof(S));
        S.arity = t.arity;
        for (uint32_t c = 0; c < t.arity; c++) {
            S.width[c] = hbits[c] ? 32u - (uint32_t)__builtin_clz(hbits[c]) : 0u;
            wsum += S.width[c];
        }
        S.kcols = wsum > 32 ? 2 : 1;
        if (allow_pack && t.arity >= 2 && wsum <= 64 && S.kcols < t.arity) {
            uint32_t first[kMaxArity];
            for (uint32_t c = 0; c < t.arity; c++)
                DL_CUDA(cudaMemcpyAsync(first + c, t.col[c], sizeof(uint32_t), cudaMemcpyDeviceToHost, E.stream));
            E.sync();
            for (uint32_t c = 0; c < t.arity; c++)
                S.high[c] = S.width[c] == 32 ? 0u : (first[c] & ~((1u << S.width[c]) - 1u));
            auto keys = E.array<uint32_t>(4 * n);   // key columns and their sort buffers
            TableView kt, kt2;
            memset(&kt, 0, sizeof(kt));
            memset(&kt2, 0, sizeof(kt2));
            kt.arity = kt2.arity = S.kcols;
            kt.n = kt2.n = n;
            for (uint32_t c = 0; c < S.kcols; c++) {
                kt.col[c] = keys.p + (uint64_t)c * n;
                kt2.col[c] = keys.p + (uint64_t)(2 + c) * n;
            }
            uint32_t* khi = S.kcols == 2 ? kt.col[0] : nullptr;
            uint32_t* klo = kt.col[S.kcols - 1];
            {
                KernelScope ks(E, DL_K_SORT, (4ull * t.arity + 4ull * S.kcols) * n);
                k_pack_keys<<<grid_for(n, 256), 256, 0, E.stream>>>(t, S, khi, klo);
                DL_CHECK_LAUNCH();
            }
            radix_sort_rows(E, kt, kt2, &passes, false);
            khi = S.kcols == 2 ? kt.col[0] : nullptr;
            klo = kt.col[S.kcols - 1];
            {
                KernelScope ks(E, DL_K_SORT, (4ull * t.arity + 4ull * S.kcols) * n);
                k_unpack_keys<<<grid_for(n, 256), 256, 0, E.stream>>>(khi, klo, n, S, t);
                DL_CHECK_LAUNCH();
            }
            if (passes_out) *passes_out = passes;
            return;
        }
        const uint32_t ntiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
        auto hist = E.array<uint32_t>((uint64_t)kRadix * ntiles);
        for (int c = (int)t.arity - 1; c >= 0; c--) {
            uint32_t vb = hbits[c];
            if (!vb) continue;
            int lo = __builtin_ctz(vb), hi = 31 - __builtin_clz(vb);
            for (int shift = lo; shift <= hi; shift += kRadixBits) {
                {
                    KernelScope ks(E, DL_K_SORT, 4 * n);
                    k_radix_hist<<<ntiles, kSortThreads, 0, E.stream>>>(t.col[c], n, shift, hist.p, ntiles);
                    DL_CHECK_LAUNCH();
                }
                scan_u32(E, hist.p, (uint64_t)kRadix * ntiles, nullptr);
                TableView dst = tmp;
                dst.n = n;
                KernelScope ks(E, DL_K_SORT, (4 + 8ull * t.arity) * n);
                k_radix_scatter<<<ntiles, kSortThreads, sizeof(uint32_t) * t.arity * kSortTile, E.stream>>>(
                    t, dst, c, shift, hist.p, ntiles);
                DL_CHECK_LAUNCH();
                std::swap(t, tmp);
                t.n = n;
                passes++;
            }
        }
    }
    if (passes_out) *passes_out = passes;
}

bool sort_unique_packed(Engine& E, const TableView& t, const std::function<TableView(uint64_t)>& alloc_out) {
    const uint64_t n = t.n;
    if (n < 2 || t.arity < 2) return false;
    if (n >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "sort of 2^32 rows or more");
    auto bits = E.array<uint32_t>(kMaxArity);
    DL_CUDA(cudaMemsetAsync(bits.p, 0, sizeof(uint32_t) * kMaxArity, E.stream));
    for (uint32_t c = 0; c < t.arity; c++) {
        KernelScope ks(E, DL_K_SORT, 4 * n);
        k_varying_bits<<<grid_for(n, 256), 256, 0, E.stream>>>(t.col[c], n, bits.p + c);
        DL_CHECK_LAUNCH();
    }
    uint32_t hbits[kMaxArity];
    memcpy(hbits, E.readback(bits.p, kMaxArity / 2), sizeof(uint32_t) * t.arity);
    PackSpec S;
    memset(&S, 0, sizeof(S));
    S.arity = t.arity;
    uint32_t wsum = 0;
    for (uint32_t c = 0; c < t.arity; c++) {
        S.width[c] = hbits[c] ? 32u - (uint32_t)__builtin_clz(hbits[c]) : 0u;
        wsum += S.width[c];
    }
    S.kcols = wsum > 32 ? 2 : 1;
    if (wsum > 64 || S.kcols >= t.arity) return false;
    uint32_t first[kMaxArity];
    for (uint32_t c = 0; c < t.arity; c++)
        DL_CUDA(cudaMemcpyAsync(first + c, t.col[c], sizeof(uint32_t), cudaMemcpyDeviceToHost, E.stream));
    E.sync();
    for (uint32_t c = 0; c < t.arity; c++) S.high[c] = S.width[c] == 32 ? 0u : (first[c] & ~((1u << S.width[c]) - 1u));
    auto keys = E.array<uint32_t>(4 * n);
    TableView kt, kt2;
    memset(&kt, 0, sizeof(kt));
    memset(&kt2, 0, sizeof(kt2));
    kt.arity = kt2.arity = S.kcols;
    kt.n = kt2.n = n;
    for (uint32_t c = 0; c < S.kcols; c++) {
        kt.col[c] = keys.p + (uint64_t)c * n;
        kt2.col[c] = keys.p + (uint64_t)(2 + c) * n;
    }
    {
        KernelScope ks(E, DL_K_SORT, (4ull * t.arity + 4ull * S.kcols) * n);
        k_pack_keys<<<grid_for(n, 256), 256, 0, E.stream>>>(t, S, S.kcols == 2 ? kt.col[0] : nullptr, kt.col[S.kcols - 1]);
        DL_CHECK_LAUNCH();
    }
    radix_sort_rows(E, kt, kt2, nullptr, false);
    const uint32_t* khi = S.kcols == 2 ? kt.col[0] : nullptr;
    const uint32_t* klo = kt.col[S.kcols - 1];
    const uint64_t nb = (n + kCompTile - 1) / kCompTile;
    auto cnt = E.array<uint64_t>(nb + 1);
    {
        KernelScope ks(E, DL_K_DELTA, 8ull * S.kcols * n);
        k_key_distinct_count<<<(unsigned)nb, kCompThreads, 0, E.stream>>>(khi, klo, n, cnt.p);
        DL_CHECK_LAUNCH();
    }
    scan_u64(E, cnt.p, nb, false, cnt.p + nb);
    const uint64_t total = E.readback(cnt.p + nb, 1)[0];
    const TableView out = alloc_out(total);
    if (total) {
        KernelScope ks(E, DL_K_DELTA, 8ull * S.kcols * n + 4ull * t.arity * total);
        k_key_distinct_write<<<(unsigned)nb, kCompThreads, 0, E.stream>>>(khi, klo, n, S, out, cnt.p);
        DL_CHECK_LAUNCH();
    }
    return true;
}

void dense_set_rows(Engine& E, const TableView& t, const uint32_t* dom, uint32_t* bits, uint8_t* dirty) {
    if (!t.n) return;
    DenseDom D;
    memset(&D, 0, sizeof(D));
    D.arity = t.arity;
    for (uint32_t c = 0; c < t.arity; c++) D.d[c] = dom[c];
    auto bad = E.array<uint64_t>(1);
    DL_CUDA(cudaMemsetAsync(bad.p, 0, 8, E.stream));
    {
        KernelScope ks(E, DL_K_DELTA, 4ull * t.arity * t.n);
        k_dense_set<<<grid_for(t.n, 256), 256, 0, E.stream>>>(t, D, bits, dirty, (unsigned long long*)bad.p);
        DL_CHECK_LAUNCH();
    }
    if (E.readback(bad.p, 1)[0]) throw Error(DL_ERR_STATE, "a row lies outside its relation's dense domain");
}

uint64_t dense_filter(Engine& E, const TableView& in, const uint32_t* dom, uint32_t* bits, const TableView& out) {
    const uint64_t n = in.n;
    if (n == 0) return 0;
    DenseDom D;
    memset(&D, 0, sizeof(D));
    D.arity = in.arity;
    for (uint32_t c = 0; c < in.arity; c++) D.d[c] = dom[c];
    const uint64_t nb = (n + kCompTile - 1) / kCompTile;
    auto cnt = E.array<uint64_t>(nb + 2);
    auto flags = E.array<uint8_t>(n);
    DL_CUDA(cudaMemsetAsync(cnt.p + nb + 1, 0, 8, E.stream));
    {
        KernelScope ks(E, DL_K_DELTA, 4ull * in.arity * n);
        k_dense_flags<<<(unsigned)nb, kCompThreads, 0, E.stream>>>(in, D, bits, flags.p, cnt.p,
                                                                  (unsigned long long*)(cnt.p + nb + 1));
        DL_CHECK_LAUNCH();
    }
    scan_u64(E, cnt.p, nb, false, cnt.p + nb);
    const uint64_t* h = E.readback(cnt.p + nb, 2);
    const uint64_t total = h[0];
    if (h[1]) throw Error(DL_ERR_STATE, "a row lies outside its relation's dense domain");
    if (total) {
        KernelScope ks(E, DL_K_DELTA, (4ull * in.arity + 1) * n + 4ull * in.arity * total);
        k_dense_write<<<(unsigned)nb, kCompThreads, 0, E.stream>>>(in, flags.p, out, cnt.p);
        DL_CHECK_LAUNCH();
    }
    return total;
}

uint64_t dense_extract(Engine& E, uint32_t arity, const uint32_t* dom, const uint32_t* bits, uint32_t* old,
                       uint8_t* dirty, uint64_t nwords, const std::function<TableView(uint64_t)>& alloc_out) {
    DenseDom D;
    memset(&D, 0, sizeof(D));
    D.arity = arity;
    for (uint32_t c = 0; c < arity; c++) D.d[c] = dom[c];
    const uint64_t nblocks = (nwords + kDenseBlockWords - 1) / kDenseBlockWords;
    const uint64_t ngroups = (nblocks + 31) / 32;
    const uint64_t grid = (ngroups + kExtractWarps - 1) / kExtractWarps;
    if (grid >= (1ull << 31)) throw Error(DL_ERR_CAPACITY, "dense bitmap too large to extract");
    auto gcnt = E.array<uint64_t>(ngroups + 1);
    {
        KernelScope ks(E, DL_K_DELTA, nblocks);
        k_dense_group_count<<<(unsigned)grid, 32 * kExtractWarps, 0, E.stream>>>(bits, old, dirty, nwords, nblocks,
                                                                                 ngroups, gcnt.p);
        DL_CHECK_LAUNCH();
    }
    scan_u64(E, gcnt.p, ngroups, false, gcnt.p + ngroups);
    const uint64_t total = E.readback(gcnt.p + ngroups, 1)[0];
    const TableView out = alloc_out(total);
    if (total) {
        KernelScope ks(E, DL_K_DELTA, nblocks + 4ull * arity * total);
        k_dense_group_write<<<(unsigned)grid, 32 * kExtractWarps, 0, E.stream>>>(bits, old, dirty, nwords, nblocks,
                                                                                 ngroups, gcnt.p, D, out);
        DL_CHECK_LAUNCH();
    }
    return total;
}

uint64_t unique_anti(Engine& E, const TableView& in, const AtomView* full, const TableView& out) {
    const uint64_t n = in.n;
    if (n == 0) return 0;
    UniqueAnti pred;
    pred.in = in;
    pred.use_full = full && full->n > 0;
    if (full) pred.full = *full; else memset(&pred.full, 0, sizeof(pred.full));
    const uint64_t nb = (n + kCompTile - 1) / kCompTile;
    auto cnt = E.array<uint64_t>(nb + 1);
    const uint64_t rowb = 4ull * in.arity;
    {
        KernelScope ks(E, DL_K_DELTA, 2 * rowb * n);
        k_flag_count<UniqueAnti><<<(unsigned)nb, kCompThreads, 0, E.stream>>>(pred, n, cnt.p);
        DL_CHECK_LAUNCH();
    }
    scan_u64(E, cnt.p, nb, false, cnt.p + nb);
    const uint64_t total = E.readback(cnt.p + nb, 1)[0];
    if (total) {
        KernelScope ks(E, DL_K_DELTA, 2 * rowb * n + rowb * total);
        k_flag_write<UniqueAnti><<<(unsigned)nb, kCompThreads, 0, E.stream>>>(pred, in, out, cnt.p);
        DL_CHECK_LAUNCH();
    }
    return total;
}

uint64_t anti_filter(Engine& E, const TableView& in, const AtomView& full, const TableView& out, bool keep_order) {
    const uint64_t n = in.n;
    if (n == 0) return 0;
    if (!keep_order) {
        auto cnt = E.array<uint64_t>(1);
        DL_CUDA(cudaMemsetAsync(cnt.p, 0, 8, E.stream));
        {
            KernelScope ks(E, DL_K_DELTA, 4ull * in.arity * n);
            k_absent_append<<<(unsigned)((n + kCompTile - 1) / kCompTile), kCompThreads, 0, E.stream>>>(
                in, full, out, (unsigned long long*)cnt.p);
            DL_CHECK_LAUNCH();
        }
        return E.readback(cnt.p, 1)[0];
    }
    const uint64_t nb = (n + kCompTile - 1) / kCompTile;
    auto cnt = E.array<uint64_t>(nb + 1);
    const uint64_t rowb = 4ull * in.arity;
    {
        KernelScope ks(E, DL_K_DELTA, rowb * n);
        k_absent_count<<<(unsigned)nb, kCompThreads, 0, E.stream>>>(in, full, cnt.p);
        DL_CHECK_LAUNCH();
    }
    scan_u64(E, cnt.p, nb, false, cnt.p + nb);
    const uint64_t total = E.readback(cnt.p + nb, 1)[0];
    if (total) {
        KernelScope ks(E, DL_K_DELTA, rowb * n + rowb * total);
        k_absent_write<<<(unsigned)nb, kCompThreads, 0, E.stream>>>(in, full, out, cnt.p);
        DL_CHECK_LAUNCH();
    }
    return total;
}

void merge_rows(Engine& E, const TableView& a, const TableView& b, const TableView& out) {
    const uint64_t total = a.n + b.n;
    if (!total) return;
    const size_t smem = sizeof(uint32_t) * a.arity * kMergeTile + sizeof(uint16_t) * kMergeTile;
    // the kernel's dynamic shared memory limit, raised once per device (setting it twice is harmless)
    static std::atomic<uint64_t> attr_set{0};
    const uint64_t bit = 1ull << (E.device & 63);
    if (!(attr_set.load() & bit)) {
        DL_CUDA(cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(uint32_t) * 2ull * kMaxArity * kMergeTile)));
        attr_set.fetch_or(bit);
    }
    const uint64_t tiles = (total + kMergeTile - 1) / kMergeTile;
    if (tiles >= (1ull << 31)) throw Error(DL_ERR_CAPACITY, "merge of 2^31 tiles or more");
    auto split = E.array<uint64_t>(tiles + 1);
    {
        KernelScope ks(E, DL_K_MERGE, 16ull * (tiles + 1));
        k_merge_splits<<<(unsigned)((tiles + 1 + 255) / 256), 256, 0, E.stream>>>(a, b, tiles, split.p);
        DL_CHECK_LAUNCH();
    }
    KernelScope ks(E, DL_K_MERGE, 8ull * a.arity * total);
    k_merge<<<(unsigned)tiles, kMergeThreads, smem, E.stream>>>(a, b, out, split.p);
    DL_CHECK_LAUNCH();
}

void build_root(Engine& E, const uint32_t* col0, uint64_t n, uint32_t* root, uint32_t V) {
    const uint64_t cnt = (uint64_t)V + 1;
    KernelScope ks(E, DL_K_OTHER, 4 * cnt);
    k_build_root<<<(unsigned)((cnt + 255) / 256), 256, 0, E.stream>>>(col0, (uint32_t)n, root, V);
    DL_CHECK_LAUNCH();
}

void column_max(Engine& E, const uint32_t* col, uint64_t n, uint32_t* out_dev) {
    if (!n) return;
    KernelScope ks(E, DL_K_OTHER, 4 * n);
    k_column_max<<<grid_for(n, 256), 256, 0, E.stream>>>(col, n, out_dev);
    DL_CHECK_LAUNCH();
}

void table_digest(Engine& E, const TableView& t, unsigned long long* d) {
    if (!t.n) return;
    KernelScope ks(E, DL_K_OTHER, 4ull * t.arity * t.n);
    k_digest<<<grid_for(t.n, 256), 256, 0, E.stream>>>(t, d);
    DL_CHECK_LAUNCH();
}

void permute_copy(Engine& E, const TableView& in, const uint8_t* perm, const TableView& out) {
    for (uint32_t k = 0; k < in.arity; k++)
        if (in.n)
            DL_CUDA(cudaMemcpyAsync(out.col[k], in.col[perm[k]], sizeof(uint32_t) * in.n, cudaMemcpyDeviceToDevice,
                                    E.stream));
}

void fill_u32(Engine& E, uint32_t* out, uint64_t n, uint32_t v) {
    if (!n) return;
    KernelScope ks(E, DL_K_OTHER, 4 * n);
    k_fill_u32<<<grid_for(n, 256), 256, 0, E.stream>>>(out, n, v);
    DL_CHECK_LAUNCH();
}

void mark_runs(Engine& E, const uint32_t* col0, uint64_t n, uint32_t* last, uint32_t t) {
    if (!n) return;
    KernelScope ks(E, DL_K_OTHER, 8 * n);
    k_mark_runs<<<grid_for(n, 256), 256, 0, E.stream>>>(col0, n, last, t);
    DL_CHECK_LAUNCH();
}

void find_range(Engine& E, const uint32_t* col0, uint64_t n, uint32_t v, uint64_t* lo, uint64_t* hi) {
    if (!n) {
        *lo = *hi = 0;
        return;
    }
    auto r = E.array<uint64_t>(2);
    {
        KernelScope ks(E, DL_K_OTHER, 256);
        k_find_range<<<1, 1, 0, E.stream>>>(col0, n, v, (unsigned long long*)r.p);
        DL_CHECK_LAUNCH();
    }
    const uint64_t* h = E.readback(r.p, 2);
    *lo = h[0];
    *hi = h[1];
}

void build_hub_bits(Engine& E, const uint32_t* root, const uint32_t* col1, const uint32_t* hub_keys,
                    uint32_t nhubs, uint32_t* bits, uint32_t bmwords) {
    if (!nhubs) return;
    DL_CUDA(cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (uint64_t)nhubs * bmwords, E.stream));
    KernelScope ks(E, DL_K_OTHER, 4ull * nhubs * bmwords);
    k_hub_bits<<<nhubs, 256, 0, E.stream>>>(root, col1, hub_keys, bits, bmwords);
    DL_CHECK_LAUNCH();
}

uint64_t count_order_violations(Engine& E, const TableView& t) {
    if (t.n < 2) return 0;
    auto c = E.array<uint64_t>(1);
    DL_CUDA(cudaMemsetAsync(c.p, 0, 8, E.stream));
    {
        KernelScope ks(E, DL_K_OTHER, 4ull * t.arity * t.n);
        k_order_violations<<<grid_for(t.n, 256), 256, 0, E.stream>>>(t, (unsigned long long*)c.p);
        DL_CHECK_LAUNCH();
    }
    return E.readback(c.p, 1)[0];
}

}  // namespace dl
