// Worst-case-optimal join of one rule body, attribute at a time.
//
// Method (paper Section 2, "Join Processing and Worst-Case Optimal Join"): fix a variable
// order x1..xm; at level i the candidates for x_i are the intersection of the sorted
// projections of every atom that mentions x_i, each restricted to the rows that match the
// values already bound; only surviving prefixes continue.  Atoms are stored as flat
// lexicographically sorted SoA indexes whose column order follows the variable order
// (Section 4), so "restrict to the prefix" is range narrowing by binary search and the
// projection onto x_i is the next column of the narrowed range.
//
// GPU organisation (this library's design; the paper's is prior art):
//  * Levels run breadth-first.  The surviving prefixes of level i form a frontier (SoA:
//    the bound values plus, for each atom still needed later, its narrowed row range).
//  * Per level, a histogram pass gives every frontier entry a work count W = the size of
//    its smallest candidate source (Algorithm 1, Phase 1, generalised from the root to every
//    level); a device prefix scan flattens all entries into one space of T work units
//    (Figure 2).  CTAs take equal contiguous tiles of that space (Algorithm 2's slice),
//    so a heavy key is split across warps and CTAs; a unit is decoded to its entry by a
//    binary search on the prefix (Section 5's decode).
//  * A unit is one candidate row of the entry's driving source.  It survives if it starts
//    a run of its value (distinct candidates) and the value is present in every other
//    source's range (binary search).  Count pass -> prefix scan -> write pass (Algorithm 1,
//    Phases 2 and 3): survivors are ranked inside each CTA with a block scan and written in
//    unit order at the scanned offsets, without atomics.  Unit order is lexicographic
//    prefix order, so outputs come out sorted by the variable order.
//  * Candidate reuse: when the sources of level i+1 include an exact copy of level i's
//    sources (same index, same depth, same bound prefix; e.g. E(w,.) and E(x,.) of the
//    4-clique), their intersection for a prefix equals level i's surviving candidates for
//    that prefix, i.e. the values of the entry's siblings in the frontier.  Level i+1 then
//    reads that sibling run as one already-intersected source instead of re-intersecting.
#include <algorithm>
#include <cstdio>
#include <string>

#include "engine.h"

namespace dl {

namespace {

constexpr int kJoinThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint8_t kVirtual = 0xff;   // source = the entry's sibling run in the frontier

enum { MODE_FRONTIER = 0, MODE_HEAD = 1, MODE_COUNT = 2 };
// A comparison applied at a level: relation of the level's value v to the other operand.
enum { F_LT = 0, F_LE = 1, F_GT = 2, F_GE = 3, F_NE = 4 };
constexpr int kMaxNeg = DL_MAX_NEG;
constexpr int kMaxCmp = DL_MAX_CMP;

struct LevelParams {
    AtomView atom[kMaxAtoms];
    uint32_t level;                       // values fval[0..level) are bound by the frontier
    uint32_t nsrc;
    uint8_t src_atom[kMaxSrc + 1];        // atom of each source, kVirtual for the sibling run
    uint8_t src_depth[kMaxSrc + 1];
    uint8_t src_need_range[kMaxSrc + 1];  // 1: the narrowed range is carried to the next level
    int8_t src_keypos[kMaxSrc + 1];       // depth-1 source: order position of its depth-0 value
    int8_t slot_in[kMaxAtoms];            // frontier slot of each atom's range, -1 = whole index
    int8_t lazy_pos[kMaxAtoms];           // atom whose depth-0 check was deferred: position of that value
    uint64_t nF;
    const uint32_t* fval[kMaxVars];
    const uint32_t* flo[kMaxAtoms];
    const uint32_t* fhi[kMaxAtoms];
    const uint32_t* sibcol;               // the previous level's values, indexed as the sibling runs are
    const uint32_t* seg;                  // sibling run of each entry: inclusive segment number
    const uint32_t* segstart;             // first entry of each segment (+ end sentinel)
    unsigned long long* C;                // per entry: W, then inclusive prefix
    uint8_t* drv;                         // per entry: driving source
    uint64_t T;
    uint64_t tile;
    uint64_t tile_base;                   // first tile of this launch (chunked writes)
    uint64_t out_base;                    // output offset of tile_base (chunked writes)
    uint32_t naive;                       // one frontier entry per CTA (ablation baseline)
    unsigned long long* block_count;      // count pass: per-tile counts; write pass: exclusive offsets
    int mode;
    uint32_t* oval[kMaxVars];
    uint32_t* oparent;                    // frontier out: parent entry (when the next level reuses)
    uint32_t ncarry;
    int8_t carry_src[kMaxAtoms];          // source index providing the range, or -1
    int8_t carry_slot[kMaxAtoms];         // otherwise: input slot (-1 = whole index)
    uint8_t carry_atom[kMaxAtoms];
    uint32_t* olo[kMaxAtoms];
    uint32_t* ohi[kMaxAtoms];
    uint32_t head_arity;
    int8_t head_pos[kMaxArity];           // order position of head column, -1 = constant
    int8_t head_lvl;                      // MODE_COUNT: the head column holding the level's variable
    int8_t head_shared;                   // MODE_COUNT: leading head columns shared by an entry's siblings
    uint32_t head_const[kMaxArity];
    uint32_t* ocol[kMaxArity];
    unsigned long long* digest;           // MODE_COUNT: [count, sum, xor]
    // filters whose last variable is this level's (comparisons, negated atoms)
    uint32_t ncmp, nneg;
    uint8_t cmp_op[kMaxCmp];              // F_*: v op w
    int8_t cmp_pos[kMaxCmp];              // order position of w, -1 = the constant cmp_const
    uint32_t cmp_const[kMaxCmp];
    AtomView neg[kMaxNeg];                // a negated atom's index, columns in order-position order
    int8_t neg_pos[kMaxNeg][kMaxArity];   // order position of each of its columns (the last: level)
};

// The level's filters for candidate v of entry e: every comparison holds and no negated
// atom holds the bound tuple.
__device__ __noinline__ bool filters_pass(const LevelParams& P, uint64_t e, uint32_t v) {
    for (uint32_t f = 0; f < P.ncmp; f++) {
        const uint32_t w = P.cmp_pos[f] < 0 ? P.cmp_const[f] : __ldg(P.fval[P.cmp_pos[f]] + e);
        const uint8_t op = P.cmp_op[f];
        const bool ok = op == F_LT ? v < w : op == F_LE ? v <= w : op == F_GT ? v > w : op == F_GE ? v >= w : v != w;
        if (!ok) return false;
    }
    for (uint32_t n = 0; n < P.nneg; n++) {
        const AtomView& A = P.neg[n];
        uint32_t lo = 0, hi = A.n;
        bool in = A.n > 0;
        for (uint32_t c = 0; c < A.arity && in; c++) {
            const int pos = P.neg_pos[n][c];
            in = narrow(A, (int)c, pos == (int)P.level ? v : __ldg(P.fval[pos] + e), lo, hi);
        }
        if (in) return false;
    }
    return true;
}

// Row range of source s for frontier entry e, and the column its candidates live in.
__device__ __forceinline__ const uint32_t* src_range(const LevelParams& P, int s, uint64_t e, uint32_t& lo,
                                                     uint32_t& hi) {
    const int a = P.src_atom[s];
    if (a == kVirtual) {
        const uint32_t g = __ldg(P.seg + e) - 1;
        lo = __ldg(P.segstart + g);
        hi = __ldg(P.segstart + g + 1);
        return P.sibcol;
    }
    const int d = P.src_depth[s];
    if (d == 0) {
        lo = 0;
        hi = P.atom[a].n;
    } else if (P.slot_in[a] >= 0) {
        const int slot = P.slot_in[a];
        lo = __ldg(P.flo[slot] + e);
        hi = __ldg(P.fhi[slot] + e);
    } else {
        // the atom's depth-0 value was bound earlier with its check deferred: narrow now
        const uint32_t v0 = __ldg(P.fval[P.lazy_pos[a]] + e);
        lo = 0;
        hi = P.atom[a].n;
        if (!narrow(P.atom[a], 0, v0, lo, hi)) lo = hi = 0;
    }
    return P.atom[a].col[d];
}

// Histogram (Algorithm 1, Phase 1, at every level): each entry's work W = the size of its
// smallest candidate source, which drives the entry.  The sum of W over the entries (the
// scan's total T) is the level's algorithmic work: every candidate of the smallest source is
// examined once.
__global__ void k_wcoj_hist(const __grid_constant__ LevelParams P) {
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (e >= P.nF) return;
    unsigned long long best = ~0ull;
    uint32_t bs = 0;
    for (uint32_t s = 0; s < P.nsrc; s++) {
        const int a = P.src_atom[s], d = P.src_depth[s];
        unsigned long long len;
        if (a != kVirtual && d == 0) {
            const AtomView& A = P.atom[a];
            len = A.n == 0 ? 0 : (A.root ? A.V : A.n);
        } else {
            uint32_t lo, hi;
            src_range(P, (int)s, e, lo, hi);
            len = hi - lo;
        }
        if (len < best) { best = len; bs = s; }
    }
    P.C[e] = best == ~0ull ? 0 : best;
    P.drv[e] = (uint8_t)bs;
}

struct Unit {
    uint64_t e;
    uint32_t v;
    uint32_t lo[kMaxSrc + 1], hi[kMaxSrc + 1];
};

// Decode unit u of the flat space into (entry, local) and evaluate it (F: the level has
// filters).
template <bool F>
__device__ __forceinline__ bool eval_unit(const LevelParams& P, uint64_t u, uint64_t e0, uint64_t e1, Unit& U) {
    uint64_t e;
    if (P.naive) e = e0;
    else e = upper_bound_u64((const uint64_t*)P.C, e0, e1, u);
    const uint64_t local = u - (e ? P.C[e - 1] : 0);
    U.e = e;
    const int s0 = P.drv[e];
    uint32_t v, d_lo, d_hi;   // the driving source's narrowed range for v
    {
        const int a = P.src_atom[s0], d = P.src_depth[s0];
        if (a != kVirtual && d == 0 && P.atom[a].root) {
            const AtomView& A = P.atom[a];
            v = (uint32_t)local;                       // iterate the dense value domain
            d_lo = __ldg(A.root + v);
            d_hi = __ldg(A.root + v + 1);
            if (d_lo >= d_hi) return false;
        } else {
            uint32_t lo, hi;
            const uint32_t* col = src_range(P, s0, e, lo, hi);
            const uint32_t r = lo + (uint32_t)local;
            v = __ldg(col + r);
            if (r > lo && __ldg(col + r - 1) == v) return false;   // not the first row of its value
            d_lo = r;
            d_hi = P.src_need_range[s0] ? upper_bound_u32(col, r + 1, hi, v) : r + 1;
        }
    }
    U.v = v;
#pragma unroll
    for (int s = 0; s < kMaxSrc + 1; s++) {
        if (s >= (int)P.nsrc) break;
        if (s == s0) {               // the driver holds v by construction
            U.lo[s] = d_lo;
            U.hi[s] = d_hi;
            continue;
        }
        const int a = P.src_atom[s], d = P.src_depth[s];
        uint32_t lo, hi;
        const uint32_t* col = src_range(P, s, e, lo, hi);
        if (P.src_need_range[s]) {
            if (!narrow(P.atom[a], d, v, lo, hi)) return false;
        } else if (a != kVirtual && d == 0 && P.atom[a].root) {
            const AtomView& A = P.atom[a];
            if (v >= A.V || __ldg(A.root + v) >= __ldg(A.root + v + 1)) return false;
        } else {
            const uint32_t l = lower_bound_u32(col, lo, hi, v);
            if (l >= hi || __ldg(col + l) != v) return false;
        }
        U.lo[s] = lo;
        U.hi[s] = hi;
    }
    if (F && !filters_pass(P, e, v)) return false;
    return true;
}

__device__ __forceinline__ uint32_t value_at(const LevelParams& P, const Unit& U, int pos) {
    return pos == (int)P.level ? U.v : __ldg(P.fval[pos] + U.e);
}

__device__ __forceinline__ void tile_bounds(const LevelParams& P, uint64_t& lo, uint64_t& hi) {
    if (P.naive) {
        const uint64_t e = blockIdx.x;
        lo = e ? P.C[e - 1] : 0;
        hi = P.C[e];
    } else {
        lo = (P.tile_base + blockIdx.x) * P.tile;
        hi = min(lo + P.tile, P.T);
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T ws[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : T(0);
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

__device__ __forceinline__ void tile_entries(const LevelParams& P, uint64_t tlo, uint64_t thi, uint64_t& e0,
                                             uint64_t& e1) {
    __shared__ uint64_t s_e0, s_e1;
    if (threadIdx.x == 0) {
        if (P.naive) {
            s_e0 = blockIdx.x;
            s_e1 = blockIdx.x + 1;
        } else if (tlo < thi) {
            s_e0 = upper_bound_u64((const uint64_t*)P.C, 0, P.nF, tlo);
            s_e1 = upper_bound_u64((const uint64_t*)P.C, s_e0, P.nF, thi - 1) + 1;
        } else {
            s_e0 = s_e1 = 0;
        }
    }
    __syncthreads();
    e0 = s_e0;
    e1 = s_e1;
}

template <bool F>
__global__ void __launch_bounds__(kJoinThreads, 8) k_wcoj_count(const __grid_constant__ LevelParams P) {
    uint64_t tlo, thi, e0, e1;
    tile_bounds(P, tlo, thi);
    tile_entries(P, tlo, thi, e0, e1);
    unsigned long long cnt = 0, hs = 0, hx = 0;
    Unit U;
    for (uint64_t u = tlo + threadIdx.x; u < thi; u += blockDim.x) {
        if (!eval_unit<F>(P, u, e0, e1, U)) continue;
        cnt++;
        if (P.mode == MODE_COUNT) {
            uint64_t h = kTupleHashSeed;
            for (uint32_t c = 0; c < P.head_arity; c++) {
                const int pos = P.head_pos[c];
                h = tuple_hash_step(h, pos < 0 ? P.head_const[c] : value_at(P, U, pos), c);
            }
            hs += h;
            hx ^= h;
        }
    }
    const unsigned long long total = block_sum(cnt);
    if (P.mode == MODE_COUNT) {
        const unsigned long long s = block_sum(hs);
#pragma unroll
        for (int o = 16; o; o >>= 1) hx ^= __shfl_xor_sync(kFull, hx, o);
        if ((threadIdx.x & 31) == 0 && hx) atomicXor(&P.digest[2], hx);
        if (threadIdx.x == 0 && total) {
            atomicAdd(&P.digest[0], total);
            atomicAdd(&P.digest[1], s);
        }
    }
    if (threadIdx.x == 0) P.block_count[blockIdx.x] = total;
}

// Count pass of a count sink's rule in the batched form: every survivor's row hash (over the
// head's columns after the instance id, numbered from 0, so that it equals the digest of the
// instance evaluated alone) goes to its instance's accumulators [count, sum, xor].
template <bool F>
__global__ void __launch_bounds__(kJoinThreads, 8) k_wcoj_count_inst(const __grid_constant__ LevelParams P) {
    uint64_t tlo, thi, e0, e1;
    tile_bounds(P, tlo, thi);
    tile_entries(P, tlo, thi, e0, e1);
    unsigned long long cnt = 0;
    Unit U;
    for (uint64_t u = tlo + threadIdx.x; u < thi; u += blockDim.x) {
        if (!eval_unit<F>(P, u, e0, e1, U)) continue;
        cnt++;
        uint64_t h = kTupleHashSeed;
        for (uint32_t c = 1; c < P.head_arity; c++) {
            const int pos = P.head_pos[c];
            h = tuple_hash_step(h, pos < 0 ? P.head_const[c] : value_at(P, U, pos), c - 1);
        }
        unsigned long long* d = P.digest + 3ull * __ldg(P.fval[0] + U.e);
        atomicAdd(d, 1ull);
        atomicAdd(d + 1, (unsigned long long)h);
        atomicXor(d + 2, (unsigned long long)h);
    }
    const unsigned long long total = block_sum(cnt);
    if (threadIdx.x == 0) P.block_count[blockIdx.x] = total;
}

__device__ __forceinline__ uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t& total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const uint32_t pre = warp ? ws[warp - 1] : 0;
    total = ws[nw - 1];
    __syncthreads();
    return pre + x - v;
}

template <bool F>
__global__ void __launch_bounds__(kJoinThreads, 4) k_wcoj_write(const __grid_constant__ LevelParams P) {
    uint64_t tlo, thi, e0, e1;
    tile_bounds(P, tlo, thi);
    tile_entries(P, tlo, thi, e0, e1);
    uint64_t run = P.block_count[P.tile_base + blockIdx.x] - P.out_base;
    Unit U;
    for (uint64_t base = tlo; base < thi; base += blockDim.x) {
        const uint64_t u = base + threadIdx.x;
        const uint32_t f = (u < thi && eval_unit<F>(P, u, e0, e1, U)) ? 1u : 0u;
        uint32_t total;
        const uint32_t pos = block_exclusive_scan_u32(f, total);
        if (f) {
            const uint64_t o = run + pos;
            if (P.mode == MODE_HEAD) {
                for (uint32_t c = 0; c < P.head_arity; c++) {
                    const int hp = P.head_pos[c];
                    P.ocol[c][o] = hp < 0 ? P.head_const[c] : value_at(P, U, hp);
                }
            } else {
                for (uint32_t k = 0; k <= P.level; k++) P.oval[k][o] = value_at(P, U, (int)k);
                if (P.oparent) P.oparent[o] = (uint32_t)U.e;
#pragma unroll
                for (int c = 0; c < kMaxAtoms; c++) {
                    if (c >= (int)P.ncarry) break;
                    const int s = P.carry_src[c];
                    uint32_t lo, hi;
                    if (s >= 0) {
                        // registers hold the ranges by source index; select without local arrays
                        lo = 0;
                        hi = 0;
#pragma unroll
                        for (int q = 0; q < kMaxSrc + 1; q++)
                            if (q == s) { lo = U.lo[q]; hi = U.hi[q]; }
                    } else if (P.carry_slot[c] >= 0) {
                        lo = __ldg(P.flo[P.carry_slot[c]] + U.e);
                        hi = __ldg(P.fhi[P.carry_slot[c]] + U.e);
                    } else {
                        lo = 0;
                        hi = P.atom[P.carry_atom[c]].n;
                    }
                    P.olo[c][o] = lo;
                    P.ohi[c][o] = hi;
                }
            }
        }
        run += total;
    }
}

// ------------------------------------------------------------ warp-major kernels
//
// Used when a level averages at least 32 units per frontier entry.  A warp owns a
// contiguous range of the unit space and walks the entries overlapping it; the entry's
// state (driver, source ranges) is loaded once and shared by the 32 lanes, which take the
// entry's units 32 at a time.  No per-unit decode, and the lanes of a step probe the same
// ranges.  The count pass leaves one count per warp; after the scan the write pass ranks a
// step's survivors with a ballot, so output stays in unit order.

constexpr int kWarps = kJoinThreads / 32;

// How a probe source is searched, packed into its (lo, hi) pair: an ordinary range has
// lo <= hi < kRootMark (indexes hold fewer than 2^32 - 2 rows).
constexpr uint32_t kRootMark = 0xFFFFFFFEu;   // col = dense root offsets, hi = their domain size
constexpr uint32_t kBitsMark = 0xFFFFFFFFu;   // col = a heavy key's bitmap, hi = its width in bits

// An entry's sources with the driver held apart: probe slot k holds source k + (k >= s0).
// Slots are written and read with compile-time indexes only, so they stay in registers.
template <int NS>
struct EntryState {
    static constexpr int NP = NS > 1 ? NS - 1 : 1;
    uint64_t e;
    uint32_t eoff;                // (warp range start - the entry's first unit) mod 2^32
    const uint32_t* col[NP];
    uint32_t lo[NP], hi[NP];
    const uint32_t* dcol;         // the driver (dlo == kRootMark: iterate the dense domain)
    uint32_t dlo, dhi;
    int s0;
};

// Source s's search state for entry e.
__device__ __forceinline__ const uint32_t* probe_state(const LevelParams& P, int s, uint64_t e, uint32_t& lo,
                                                       uint32_t& hi) {
    const int a = P.src_atom[s];
    if (a != kVirtual && P.src_depth[s] == 0 && P.atom[a].root) {
        lo = kRootMark;
        hi = P.atom[a].V;
        return P.atom[a].root;
    }
    const uint32_t* col = src_range(P, s, e, lo, hi);
    // a membership-only probe into a heavy key's rows: test its bitmap instead
    if (a != kVirtual && P.src_depth[s] == 1 && !P.src_need_range[s] && P.atom[a].hub &&
        hi - lo >= P.atom[a].hubmin) {
        const uint32_t key = __ldg(P.fval[P.src_keypos[s]] + e);
        const int32_t slot = key < P.atom[a].V ? __ldg(P.atom[a].hub + key) : -1;
        if (slot >= 0) {
            lo = kBitsMark;
            hi = P.atom[a].bmwords * 32u;
            return P.atom[a].bits + (uint64_t)slot * P.atom[a].bmwords;
        }
    }
    return col;
}

// Loads entry e for a warp whose range starts at unit wlo; returns the entry's end unit.
template <int NS>
__device__ __forceinline__ uint64_t entry_load(const LevelParams& P, EntryState<NS>& S, uint64_t e, uint64_t wlo) {
    S.e = e;
    S.eoff = (uint32_t)(wlo - (e ? P.C[e - 1] : 0));
    S.s0 = P.drv[e];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s < (int)P.nsrc && s != S.s0) {
            uint32_t lo, hi;
            const uint32_t* col = probe_state(P, s, e, lo, hi);
            constexpr int NP = EntryState<NS>::NP;
            const int below = s < NP ? s : NP - 1, above = s > 0 ? s - 1 : 0;   // compile-time
            if (s < S.s0) {
                S.col[below] = col;
                S.lo[below] = lo;
                S.hi[below] = hi;
            } else {
                S.col[above] = col;
                S.lo[above] = lo;
                S.hi[above] = hi;
            }
        }
    }
    const int a = P.src_atom[S.s0];
    if (a != kVirtual && P.src_depth[S.s0] == 0 && P.atom[a].root) {
        S.dcol = P.atom[a].root;
        S.dlo = kRootMark;
        S.dhi = P.atom[a].V;
    } else {
        S.dcol = src_range(P, S.s0, e, S.dlo, S.dhi);
    }
    return P.C[e];
}

// The entry's unit `local` (counted from its first unit): the candidate value v and whether
// every probe source holds it.  nlo/nhi (probe slots) and dnlo/dnhi (driver) receive the
// narrowed ranges.
template <int NS>
__device__ __forceinline__ bool entry_eval(const LevelParams& P, const EntryState<NS>& S, uint32_t local,
                                           uint32_t& v, uint32_t (&nlo)[EntryState<NS>::NP],
                                           uint32_t (&nhi)[EntryState<NS>::NP], uint32_t& dnlo, uint32_t& dnhi) {
    bool ok;
    if (S.dlo == kRootMark) {
        v = local;                                 // iterate the dense value domain
        dnlo = __ldg(S.dcol + v);
        dnhi = __ldg(S.dcol + v + 1);
        ok = dnlo < dnhi;
    } else {
        const uint32_t r = S.dlo + local;
        v = __ldg(S.dcol + r);
        // A driver whose atom has later columns repeats a value over that value's rows: only
        // the first row of a value is a candidate.  Otherwise (the atom's last column under a
        // bound prefix, or a sibling run) the values are distinct.
        const bool need = P.src_need_range[S.s0];
        ok = !(need && r > S.dlo && __ldg(S.dcol + r - 1) == v);
        dnlo = r;
        dnhi = (ok && need) ? upper_bound_u32(S.dcol, r + 1, S.dhi, v) : r + 1;
    }
#pragma unroll
    for (int k = 0; k < NS - 1; k++) {
        if (ok && k + 1 < (int)P.nsrc) {
            if (S.lo[k] == kRootMark) {
                const uint32_t l = v < S.hi[k] ? __ldg(S.col[k] + v) : 0;
                const uint32_t h = v < S.hi[k] ? __ldg(S.col[k] + v + 1) : 0;
                ok = l < h;
                nlo[k] = l;
                nhi[k] = h;
            } else if (S.lo[k] == kBitsMark) {
                ok = v < S.hi[k] && ((__ldg(S.col[k] + (v >> 5)) >> (v & 31)) & 1u);   // one bit test
                nlo[k] = 0;
                nhi[k] = 0;
            } else {
                const uint32_t l = lower_bound_u32(S.col[k], S.lo[k], S.hi[k], v);
                ok = l < S.hi[k] && __ldg(S.col[k] + l) == v;
                nlo[k] = l;
                const int q = k + (k >= S.s0 ? 1 : 0);
                nhi[k] = (ok && P.src_need_range[q]) ? upper_bound_u32(S.col[k], l + 1, S.hi[k], v) : l + 1;
            }
        }
    }
    return ok;
}

__device__ __forceinline__ void warp_range(const LevelParams& P, uint64_t& wlo, uint64_t& whi) {
    const uint64_t tlo = (P.tile_base + blockIdx.x) * P.tile;
    const uint64_t thi = min(tlo + P.tile, P.T);
    const uint64_t per = (P.tile + kWarps - 1) / kWarps;
    wlo = min(tlo + (threadIdx.x >> 5) * per, thi);
    whi = min(wlo + per, thi);
}

// Value of head column c (not the level's variable) for frontier entry e.
__device__ __forceinline__ uint32_t head_value(const LevelParams& P, int c, uint64_t e) {
    const int pos = P.head_pos[c];
    return pos < 0 ? P.head_const[c] : __ldg(P.fval[pos] + e);
}

template <int NS, bool F>
__global__ void __launch_bounds__(kJoinThreads, NS <= 2 ? 8 : 4) k_wcoj_count_wm(const __grid_constant__ LevelParams P) {
    const int lane = threadIdx.x & 31;
    // the warp's range lives in shared memory between entries (registers are the limit here)
    __shared__ unsigned long long s_wlo[kWarps], s_whi[kWarps];
    {
        uint64_t wlo, whi;
        warp_range(P, wlo, whi);
        if (lane == 0) {
            s_wlo[threadIdx.x >> 5] = wlo;
            s_whi[threadIdx.x >> 5] = whi;
        }
        __syncwarp();
    }
    uint32_t cnt = 0;
    unsigned long long hs = 0, hx = 0;
    if (s_wlo[threadIdx.x >> 5] < s_whi[threadIdx.x >> 5]) {
        // unit positions below are relative to wlo (a warp range spans fewer than 2^32 units)
        uint64_t e = upper_bound_u64((const uint64_t*)P.C, 0, P.nF, s_wlo[threadIdx.x >> 5]);
        EntryState<NS> S;
        uint32_t r = 0;
        uint64_t hpre = 0;        // MODE_COUNT: row hash over the head columns before head_lvl
        uint64_t hsh = 0;         // hash of the columns shared by the current sibling run
        uint32_t run = 0xFFFFFFFFu;
        for (;;) {
            const uint64_t wlo = s_wlo[threadIdx.x >> 5], whi = s_whi[threadIdx.x >> 5];
            const uint32_t stop = (uint32_t)(min(entry_load(P, S, e, wlo), whi) - wlo);
            if (P.mode == MODE_COUNT) {
                int c0 = 0;
                if (P.head_shared > 0) {
                    const uint32_t g = __ldg(P.seg + e);
                    if (g != run) {
                        run = g;
                        hsh = kTupleHashSeed;
                        for (int c = 0; c < P.head_shared; c++) hsh = tuple_hash_step(hsh, head_value(P, c, e), c);
                    }
                    c0 = P.head_shared;
                    hpre = hsh;
                } else {
                    hpre = kTupleHashSeed;
                }
                for (int c = c0; c < P.head_lvl; c++) hpre = tuple_hash_step(hpre, head_value(P, c, e), c);
            }
            for (uint32_t b = r; b < stop; b += 32) {
                const uint32_t rr = b + lane;
                uint32_t v, nlo[EntryState<NS>::NP], nhi[EntryState<NS>::NP], dnlo, dnhi;
                if (rr >= stop || !entry_eval(P, S, rr + S.eoff, v, nlo, nhi, dnlo, dnhi)) continue;
                if (F && !filters_pass(P, e, v)) continue;
                cnt++;
                if (P.mode == MODE_COUNT) {
                    uint64_t h = tuple_hash_step(hpre, v, P.head_lvl);
                    for (uint32_t c = P.head_lvl + 1; c < P.head_arity; c++) h = tuple_hash_step(h, head_value(P, c, e), c);
                    hs += h;
                    hx ^= h;
                }
            }
            r = stop;
            const uint64_t at = s_wlo[threadIdx.x >> 5] + r;
            if (at >= s_whi[threadIdx.x >> 5]) break;
            e++;
            while (P.C[e] <= at) e++;   // entries without units
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(kFull, cnt, o);
        hs += __shfl_xor_sync(kFull, hs, o);
        hx ^= __shfl_xor_sync(kFull, hx, o);
    }
    if (lane == 0) {
        P.block_count[(uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)] = cnt;
        if (P.mode == MODE_COUNT && cnt) {
            atomicAdd(&P.digest[0], (unsigned long long)cnt);
            atomicAdd(&P.digest[1], hs);
            atomicXor(&P.digest[2], hx);
        }
    }
}

template <int NS, bool F>
__global__ void __launch_bounds__(kJoinThreads, NS <= 2 ? 6 : 4) k_wcoj_write_wm(const __grid_constant__ LevelParams P) {
    const int lane = threadIdx.x & 31;
    uint64_t wlo, whi;
    warp_range(P, wlo, whi);
    if (wlo >= whi) return;
    uint64_t o = P.block_count[(P.tile_base + blockIdx.x) * kWarps + (threadIdx.x >> 5)] - P.out_base;
    uint64_t e = upper_bound_u64((const uint64_t*)P.C, 0, P.nF, wlo);
    EntryState<NS> S;
    const uint32_t span = (uint32_t)(whi - wlo);   // unit positions relative to wlo
    uint32_t r = 0;
    const unsigned lt = (1u << lane) - 1;
    for (;;) {
        const uint32_t stop = (uint32_t)(min(entry_load(P, S, e, wlo), whi) - wlo);
        for (uint32_t b = r; b < stop; b += 32) {
            const uint32_t rr = b + lane;
            uint32_t v = 0, nlo[EntryState<NS>::NP], nhi[EntryState<NS>::NP], dnlo = 0, dnhi = 0;
            const bool f = rr < stop && entry_eval(P, S, rr + S.eoff, v, nlo, nhi, dnlo, dnhi) &&
                           (!F || filters_pass(P, e, v));
            const unsigned ball = __ballot_sync(kFull, f);
            if (f) {
                const uint64_t w = o + __popc(ball & lt);
                if (P.mode == MODE_HEAD) {
                    for (uint32_t c = 0; c < P.head_arity; c++) {
                        const int hp = P.head_pos[c];
                        P.ocol[c][w] = hp < 0 ? P.head_const[c] : (hp == (int)P.level ? v : __ldg(P.fval[hp] + e));
                    }
                } else {
                    for (uint32_t k = 0; k < P.level; k++) P.oval[k][w] = __ldg(P.fval[k] + e);
                    P.oval[P.level][w] = v;
                    if (P.oparent) P.oparent[w] = (uint32_t)e;
                    for (uint32_t c = 0; c < P.ncarry; c++) {
                        const int s = P.carry_src[c];
                        if (s == S.s0) {
                            P.olo[c][w] = dnlo;
                            P.ohi[c][w] = dnhi;
                        } else if (s < 0) {
                            const int slot = P.carry_slot[c];
                            P.olo[c][w] = slot >= 0 ? __ldg(P.flo[slot] + e) : 0;
                            P.ohi[c][w] = slot >= 0 ? __ldg(P.fhi[slot] + e) : P.atom[P.carry_atom[c]].n;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < NS - 1; k++) {
                        if (k + 1 >= (int)P.nsrc) continue;
                        const int q = k + (k >= S.s0 ? 1 : 0);   // the probe slot's source
                        for (uint32_t c = 0; c < P.ncarry; c++)
                            if (P.carry_src[c] == q) {
                                P.olo[c][w] = nlo[k];
                                P.ohi[c][w] = nhi[k];
                            }
                    }
                }
            }
            o += __popc(ball);
        }
        r = stop;
        if (r >= span) break;
        e++;
        while (P.C[e] <= wlo + r) e++;
    }
}

#define DL_NS_DISPATCH_F(KERNEL, NSRC, F, GRID, STREAM, PARAMS)                                     \
    do {                                                                                            \
        if ((NSRC) <= 1) KERNEL<1, F><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);               \
        else if ((NSRC) <= 2) KERNEL<2, F><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);          \
        else if ((NSRC) <= 3) KERNEL<3, F><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);          \
        else if ((NSRC) <= 4) KERNEL<4, F><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);          \
        else KERNEL<kMaxSrc + 1, F><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);                \
    } while (0)
// by source count and by whether the level has filters
#define DL_NS_DISPATCH(KERNEL, NSRC, FILT, GRID, STREAM, PARAMS)                                    \
    do {                                                                                            \
        if (FILT) DL_NS_DISPATCH_F(KERNEL, NSRC, true, GRID, STREAM, PARAMS);                       \
        else DL_NS_DISPATCH_F(KERNEL, NSRC, false, GRID, STREAM, PARAMS);                           \
    } while (0)

// Sibling runs of a frontier: seg[k] = 1 if entry k starts a new parent's run.
__global__ void k_seg_flags(const uint32_t* __restrict__ parent, uint64_t n, uint32_t* __restrict__ seg) {
    const uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (k < n) seg[k] = (k == 0 || parent[k] != parent[k - 1]) ? 1u : 0u;
}

// After an inclusive scan seg[k] is the 1-based run number; record each run's first entry.
__global__ void k_seg_starts(const uint32_t* __restrict__ parent, const uint32_t* __restrict__ seg, uint64_t n,
                             uint32_t* __restrict__ segstart) {
    const uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (k == 0 || parent[k] != parent[k - 1]) segstart[seg[k] - 1] = (uint32_t)k;
    if (k == n - 1) segstart[seg[k]] = (uint32_t)n;
}

// ---------------------------------------------------------------- host plan

struct Src {
    int atom;
    int depth;
};

struct Plan {
    uint32_t m = 0, natoms = 0;
    uint8_t colpos[kMaxAtoms][kMaxArity];   // order position held by index column k of atom a
    uint8_t arity[kMaxAtoms];
    int first_level[kMaxAtoms], last_level[kMaxAtoms];
    int touch_level[kMaxAtoms];             // level whose pass first narrows the atom's range
    int lazy_pos[kMaxAtoms];                // deferred depth-0 check: the value's position, else -1
    std::vector<std::vector<Src>> src;      // per level: the atoms binding the level's variable
    std::vector<uint32_t> reuse_mask;       // per level: atoms replaced by the previous level's siblings
    std::vector<uint32_t> defer_mask;       // per level: atoms whose depth-0 check moves to their next level
};

// filter_levels: bit l set when level l applies a comparison or a negated atom; the level
// after it then cannot reuse its siblings (they passed filters on the previous variable
// that need not hold for the next one).
Plan make_plan(const Rule& R, const std::vector<const Index*>& idx, uint64_t filter_levels) {
    Plan p;
    p.m = (uint32_t)R.order.size();
    p.natoms = (uint32_t)R.body.size();
    for (uint32_t a = 0; a < p.natoms; a++) {
        const RuleAtom& A = R.body[a];
        std::vector<int> pos;
        for (uint32_t c = 0; c < A.arity; c++)
            pos.push_back((int)(std::find(R.order.begin(), R.order.end(), A.terms[c].id) - R.order.begin()));
        std::sort(pos.begin(), pos.end());
        p.arity[a] = (uint8_t)A.arity;
        for (uint32_t k = 0; k < A.arity; k++) p.colpos[a][k] = (uint8_t)pos[k];
        p.first_level[a] = pos.front();
        p.last_level[a] = pos.back();
    }
    p.src.resize(p.m);
    p.reuse_mask.assign(p.m, 0);
    p.defer_mask.assign(p.m, 0);
    for (uint32_t l = 0; l < p.m; l++)
        for (uint32_t a = 0; a < p.natoms; a++)
            for (uint32_t k = 0; k < p.arity[a]; k++)
                if (p.colpos[a][k] == l) p.src[l].push_back({(int)a, (int)k});
    // Candidate reuse at level l: every source applied at level l-1 has a twin among level
    // l's sources (same index, same depth, same bound prefix) whose atom has no variable after
    // level l; then the intersection of those twins, for an entry's prefix, is exactly the set
    // of the entry's siblings.  A depth-0 source at level l-1 whose atom has a later variable
    // may be left out of level l-1 (its check "the value occurs in column 0" is made at the
    // atom's next level instead, where its range is narrowed anyway) when that is what makes
    // the match possible.  Reuse is only taken when it replaces an intersection of >= 2
    // sources.
    for (uint32_t l = 1; l < p.m; l++) {
        if ((filter_levels >> (l - 1)) & 1u) continue;
        uint32_t defer = 0;
        std::vector<Src> applied;
        for (const Src& b : p.src[l - 1]) {
            if (b.depth == 0 && p.last_level[b.atom] > (int)l - 1) defer |= 1u << b.atom;
            else applied.push_back(b);
        }
        if (applied.size() < 2) continue;
        uint32_t used = 0;
        bool ok = true;
        for (const Src& b : applied) {
            bool found = false;
            for (const Src& a : p.src[l]) {
                if ((used >> a.atom) & 1u) continue;
                if (idx[a.atom] != idx[b.atom] || a.depth != b.depth || p.last_level[a.atom] != (int)l) continue;
                bool same = true;
                for (int k = 0; k < a.depth && same; k++) same = p.colpos[a.atom][k] == p.colpos[b.atom][k];
                if (!same) continue;
                used |= 1u << a.atom;
                found = true;
                break;
            }
            if (!found) { ok = false; break; }
        }
        if (ok) {
            p.reuse_mask[l] = used;
            p.defer_mask[l - 1] = defer;
        }
    }
    for (uint32_t a = 0; a < p.natoms; a++) {
        p.touch_level[a] = p.first_level[a];
        p.lazy_pos[a] = -1;
        if ((p.defer_mask[p.first_level[a]] >> a) & 1u) {
            p.lazy_pos[a] = p.first_level[a];
            p.touch_level[a] = p.colpos[a][1];
        }
    }
    return p;
}

// Units per CTA tile for a level of T units.  Each warp starts with a search for its first
// entry, which larger tiles amortise; at least eight waves of resident CTAs (8 per SM) keep
// the tail of the launch short.
uint32_t auto_tile(const Engine& E, uint64_t T) {
    const uint64_t waves = 8ull * 8ull * E.sms;
    uint32_t t = 4096;
    while (t < (1u << 16) && T / (2ull * t) >= waves) t *= 2;
    return t;
}

void launch_seg(Engine& E, const uint32_t* parent, uint64_t n, uint32_t* seg, uint32_t* segstart) {
    const unsigned g = (unsigned)((n + 255) / 256);
    {
        KernelScope ks(E, DL_K_OTHER, 12 * n);
        k_seg_flags<<<g, 256, 0, E.stream>>>(parent, n, seg);
        DL_CHECK_LAUNCH();
    }
    scan_u32(E, seg, n, nullptr, true);
    KernelScope ks(E, DL_K_OTHER, 16 * n);
    k_seg_starts<<<g, 256, 0, E.stream>>>(parent, seg, n, segstart);
    DL_CHECK_LAUNCH();
}

}  // namespace

// Index permutation an atom needs: its columns sorted by the order position of their variable.
Perm atom_perm(const Rule& R, uint32_t a) {
    const RuleAtom& A = R.body[a];
    std::vector<std::pair<int, int>> pc;
    for (uint32_t c = 0; c < A.arity; c++)
        pc.push_back({(int)(std::find(R.order.begin(), R.order.end(), A.terms[c].id) - R.order.begin()), (int)c});
    std::sort(pc.begin(), pc.end());
    Perm p = identity_perm();
    for (uint32_t k = 0; k < A.arity; k++) p[k] = (uint8_t)pc[k].second;
    return p;
}

// Index permutation a negated atom needs: the same rule as for positive atoms.
Perm neg_perm(const Rule& R, uint32_t n) {
    const RuleAtom& A = R.neg[n];
    std::vector<std::pair<int, int>> pc;
    for (uint32_t c = 0; c < A.arity; c++)
        pc.push_back({(int)(std::find(R.order.begin(), R.order.end(), A.terms[c].id) - R.order.begin()), (int)c});
    std::sort(pc.begin(), pc.end());
    Perm p = identity_perm();
    for (uint32_t k = 0; k < A.arity; k++) p[k] = (uint8_t)pc[k].second;
    return p;
}

// Filters of a rule placed at the level of their last variable.
struct LevelFilters {
    std::vector<uint8_t> op;
    std::vector<int8_t> pos;
    std::vector<uint32_t> cst;
    std::vector<int> neg;                     // negated atom ids
};

// Returns false when a comparison can never hold (the rule derives nothing).
bool place_filters(const Rule& R, const std::vector<const Index*>& nsrc, std::vector<LevelFilters>& lf,
                   uint64_t& levels) {
    auto pos_of = [&](uint32_t id) {
        return (int)(std::find(R.order.begin(), R.order.end(), id) - R.order.begin());
    };
    lf.assign(R.order.size(), LevelFilters());
    levels = 0;
    for (const RuleCmp& q : R.cmps) {
        const bool av = q.a.kind == DL_TERM_VAR, bv = q.b.kind == DL_TERM_VAR;
        if (!av && !bv) {
            const uint32_t a = q.a.id, b = q.b.id;
            if (!(q.op == DL_CMP_LT ? a < b : q.op == DL_CMP_LE ? a <= b : a != b)) return false;
            continue;
        }
        if (av && bv && q.a.id == q.b.id) {
            if (q.op != DL_CMP_LE) return false;   // x < x and x != x never hold
            continue;
        }
        const int pa = av ? pos_of(q.a.id) : -1, pb = bv ? pos_of(q.b.id) : -1;
        // v is the operand bound last; op is rewritten as "v op' w"
        const bool v_is_a = pa > pb;
        uint8_t op;
        if (q.op == DL_CMP_NE) op = F_NE;
        else if (q.op == DL_CMP_LT) op = v_is_a ? F_LT : F_GT;
        else op = v_is_a ? F_LE : F_GE;
        const int lvl = v_is_a ? pa : pb;
        const dl_term& w = v_is_a ? q.b : q.a;
        LevelFilters& L = lf[lvl];
        L.op.push_back(op);
        L.pos.push_back(w.kind == DL_TERM_VAR ? (int8_t)pos_of(w.id) : (int8_t)-1);
        L.cst.push_back(w.kind == DL_TERM_VAR ? 0u : w.id);
        levels |= 1ull << lvl;
    }
    for (uint32_t n = 0; n < R.neg.size(); n++) {
        if (nsrc[n]->n == 0) continue;        // nothing to exclude
        int lvl = 0;
        for (uint32_t c = 0; c < R.neg[n].arity; c++) lvl = std::max(lvl, pos_of(R.neg[n].terms[c].id));
        lf[lvl].neg.push_back((int)n);
        levels |= 1ull << lvl;
    }
    return true;
}

// True when a rule's head lists exactly the variable order: the join then emits rows that are
// already sorted in the head's canonical order and distinct.
bool head_is_order(const Rule& R) {
    if (R.head.arity != R.order.size()) return false;
    for (uint32_t c = 0; c < R.head.arity; c++)
        if (R.head.terms[c].kind != DL_TERM_VAR || R.head.terms[c].id != R.order[c]) return false;
    return true;
}

namespace {

// Entry cut points for slicing a level's input entries [0, nF) into s parts of about equal
// output: the count pass left the exclusive output offset of every count slot (a tile, or a
// warp's range in a tile) in bc; cut k is the entry holding the unit where output k * total / s
// begins (that entry starts the next part, so parts hold whole entries).
__global__ void k_slice_cuts(const unsigned long long* __restrict__ bc, uint64_t ncounts,
                             const unsigned long long* __restrict__ C, uint64_t nF, uint64_t T, uint64_t tile, int wm,
                             uint64_t total, uint32_t s, unsigned long long* __restrict__ cuts) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s) return;
    if (k == 0) {
        cuts[0] = 0;
        return;
    }
    const uint64_t target = total / s * k + (total % s) * k / s;
    // last count slot whose first output is <= target
    uint64_t i = upper_bound_u64((const uint64_t*)bc, 0, ncounts, target);
    i = i ? i - 1 : 0;
    uint64_t unit;
    if (wm) {
        const uint64_t per = (tile + kWarps - 1) / kWarps;
        unit = (i / kWarps) * tile + (i % kWarps) * per;
    } else {
        unit = i * tile;
    }
    if (unit > T) unit = T;
    cuts[k] = unit >= T ? nF : upper_bound_u64((const uint64_t*)C, 0, nF, unit);
}

// Autotuner key: the rule's shape (relation names, terms, variable order), the level, and the
// size bucket of its work (log2 of the units and of the frontier entries), its source count
// and whether it filters.
std::string tune_key(const Rule& R, uint32_t lvl, uint64_t T, uint64_t nF, uint32_t nsrc, bool filt) {
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the rule's structure
    auto mixin = [&](uint64_t v) {
        for (int k = 0; k < 8; k++) {
            h ^= (v >> (8 * k)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    auto atom = [&](const RuleAtom& a) {
        mixin(a.rel);
        mixin(a.arity);
        for (uint32_t c = 0; c < a.arity; c++) {
            mixin(a.terms[c].kind);
            mixin(a.terms[c].id);
        }
    };
    atom(R.head);
    for (const RuleAtom& a : R.body) atom(a);
    for (const RuleAtom& a : R.neg) atom(a);
    for (uint32_t v : R.order) mixin(v);
    for (const RuleCmp& q : R.cmps) {
        mixin(q.op);
        mixin(q.a.id);
        mixin(q.b.id);
    }
    auto lg = [](uint64_t x) { return x ? 63 - __builtin_clzll(x) : 0; };
    char buf[128];
    snprintf(buf, sizeof(buf), "%016llx:L%u:T%d:F%d:S%u:f%d", (unsigned long long)h, lvl, lg(T), lg(nF), nsrc,
             filt ? 1 : 0);
    return buf;
}

// A join frontier: the surviving prefixes of the levels so far (SoA), the narrowed ranges of
// the atoms still needed later, and the sibling runs when the next level reuses them.
struct Frontier {
    uint64_t n = 1;
    const uint32_t* vals[kMaxVars] = {nullptr};
    const uint32_t* lo[kMaxAtoms] = {nullptr};
    const uint32_t* hi[kMaxAtoms] = {nullptr};
    const uint32_t* seg = nullptr;
    const uint32_t* segstart = nullptr;
    int8_t slot_of[kMaxAtoms];
    DevPtr own_vals, own_rng, own_seg, own_parent;
    Frontier() {
        for (int a = 0; a < kMaxAtoms; a++) slot_of[a] = -1;
    }
};

struct JoinRun {
    Engine& E;
    const Rule& R;
    const std::vector<const Index*>& nsrc;
    Relation& head;
    JoinOutput& out;
    Plan plan;
    std::vector<LevelFilters> lf;
    bool count_sink = false;
    LevelParams base;

    JoinRun(Engine& e, const Rule& r, const std::vector<const Index*>& ns, Relation& h, JoinOutput& o)
        : E(e), R(r), nsrc(ns), head(h), out(o) {}

    // Bytes of frontier a level may hold at once before its input entries are processed in
    // slices (each slice carried through the remaining levels before the next).
    uint64_t frontier_cap() const {
        if (E.frontier_bytes) return E.frontier_bytes;
        const uint64_t left = E.budget > E.used ? E.budget - E.used : 0;
        return std::max<uint64_t>(64ull << 20, left / 3);
    }

    // Level lvl over the input entries [ea, eb) of frontier F.
    void level(uint32_t lvl, const Frontier& F, uint64_t ea, uint64_t eb);
};

void JoinRun::level(uint32_t lvl, const Frontier& F, uint64_t ea, uint64_t eb) {
    const uint64_t nF = eb - ea;
    if (nF == 0) return;
    const bool last = lvl + 1 == plan.m;
    const uint32_t reuse = plan.reuse_mask[lvl];
    const uint32_t defer = plan.defer_mask[lvl];
    const uint32_t next_reuse = last ? 0 : plan.reuse_mask[lvl + 1];
    LevelParams P = base;
    P.level = lvl;
    P.nF = nF;
    // per-entry inputs are read at entry - ea; a sibling run's values keep the frontier's own
    // indexing (runs may extend past the slice)
    for (uint32_t k = 0; k < lvl; k++) P.fval[k] = F.vals[k] + ea;
    P.sibcol = lvl ? F.vals[lvl - 1] : nullptr;
    for (uint32_t a = 0; a < plan.natoms; a++) {
        P.slot_in[a] = F.slot_of[a];
        if (F.slot_of[a] >= 0) {
            P.flo[F.slot_of[a]] = F.lo[F.slot_of[a]] + ea;
            P.fhi[F.slot_of[a]] = F.hi[F.slot_of[a]] + ea;
        }
    }
    P.seg = F.seg ? F.seg + ea : nullptr;
    P.segstart = F.segstart;
    {   // this level's filters
        const LevelFilters& L = lf[lvl];
        P.ncmp = (uint32_t)L.op.size();
        P.nneg = (uint32_t)L.neg.size();
        for (uint32_t f = 0; f < P.ncmp; f++) {
            P.cmp_op[f] = L.op[f];
            P.cmp_pos[f] = L.pos[f];
            P.cmp_const[f] = L.cst[f];
        }
        for (uint32_t k = 0; k < P.nneg; k++) {
            const int n = L.neg[k];
            const Perm np = neg_perm(R, (uint32_t)n);
            P.neg[k] = atom_of(*nsrc[n]);
            for (uint32_t c = 0; c < R.neg[n].arity; c++)
                P.neg_pos[k][c] = (int8_t)(std::find(R.order.begin(), R.order.end(), R.neg[n].terms[np[c]].id) -
                                           R.order.begin());
        }
    }
    // sources of this level (atoms covered by candidate reuse become one sibling source)
    P.nsrc = 0;
    for (const Src& s : plan.src[lvl]) {
        if (((reuse | defer) >> s.atom) & 1u) continue;
        P.src_atom[P.nsrc] = (uint8_t)s.atom;
        P.src_depth[P.nsrc] = (uint8_t)s.depth;
        P.src_need_range[P.nsrc] = plan.last_level[s.atom] > (int)lvl ? 1 : 0;
        P.src_keypos[P.nsrc] = s.depth == 1 ? (int8_t)plan.colpos[s.atom][0] : (int8_t)-1;
        P.nsrc++;
    }
    if (P.nsrc > (uint32_t)kMaxSrc) throw Error(DL_ERR_UNSUPPORTED, "more than 8 body atoms mention one variable");
    if (reuse) {
        P.src_atom[P.nsrc] = kVirtual;
        P.src_depth[P.nsrc] = 0;
        P.src_need_range[P.nsrc] = 0;
        P.nsrc++;
    }
    // carried atoms: touched at or before this level and still needed later (atoms the next
    // level replaces by its sibling source are not needed)
    P.ncarry = 0;
    if (!last)
        for (uint32_t a = 0; a < plan.natoms; a++)
            if (plan.touch_level[a] <= (int)lvl && plan.last_level[a] > (int)lvl && !((next_reuse >> a) & 1u)) {
                const int c = (int)P.ncarry++;
                P.carry_atom[c] = (uint8_t)a;
                P.carry_src[c] = -1;
                for (uint32_t s = 0; s < P.nsrc; s++)
                    if (P.src_atom[s] == a) P.carry_src[c] = (int8_t)s;
                P.carry_slot[c] = F.slot_of[a];
            }

    // algorithmic bytes of one frontier entry read (values + carried ranges + sibling run)
    uint32_t nslots_in = 0;
    for (uint32_t a = 0; a < plan.natoms; a++) nslots_in += F.slot_of[a] >= 0;
    const uint64_t entry_bytes = 4ull * (lvl + 2 * nslots_in) + (reuse ? 8 : 0);

    // Phase 1: histogram + prefix (C[nF] receives the total)
    auto C = E.array<uint64_t>(nF + 1);
    auto drv = E.array<uint8_t>(nF);
    P.C = (unsigned long long*)C.p;
    P.drv = drv.p;
    E.phase_begin(0);
    {
        KernelScope ks(E, DL_K_JOIN_HIST, (entry_bytes + 9) * nF, 1, 0, nF);
        k_wcoj_hist<<<(unsigned)((nF + 255) / 256), 256, 0, E.stream>>>(P);
        DL_CHECK_LAUNCH();
    }
    scan_u64(E, C.p, nF, true, C.p + nF);
    const uint64_t T = E.readback(C.p + nF, 1)[0];
    // algorithmic work of the level: every candidate of each entry's smallest source
    const uint64_t Tmin = T;
    if (T == 0) {
        E.phase_end(0);
        return;
    }
    P.T = T;
    const bool filt = P.ncmp || P.nneg;
    // Count pass with a given tile size and kernel shape: per-tile (striped) or per-warp
    // (warp-major) output counts, plus the count sink's digest at the last level.
    struct CountRun {
        uint32_t tile = 0;
        bool wm = false;
        uint64_t ntiles = 0, ncounts = 0;
        DArray<uint64_t> bc, dg;
        float ms = 0;
    };
    if (last && count_sink) {
        P.mode = MODE_COUNT;
        P.head_lvl = -1;
        for (uint32_t c = 0; c < P.head_arity; c++)
            if (P.head_pos[c] == (int)lvl) P.head_lvl = (int8_t)c;
        if (P.head_lvl < 0) throw Error(DL_ERR_STATE, "count sink head lacks the last variable");
        // leading head columns bound above the previous level are equal across a sibling run
        P.head_shared = 0;
        if (P.seg && lvl >= 2)
            while (P.head_shared < P.head_lvl && P.head_pos[P.head_shared] >= 0 &&
                   P.head_pos[P.head_shared] < (int)lvl - 1)
                P.head_shared++;
    } else {
        P.mode = last ? MODE_HEAD : MODE_FRONTIER;
    }
    auto count_with = [&](uint32_t tile, bool wmk, bool timed) {
        CountRun r;
        r.tile = tile;
        r.wm = wmk;
        r.ntiles = P.naive ? nF : (T + tile - 1) / tile;
        if (r.ntiles >= (1ull << 31)) throw Error(DL_ERR_CAPACITY, "join level exceeds 2^31 tiles");
        r.ncounts = wmk ? r.ntiles * kWarps : r.ntiles;
        r.bc = E.array<uint64_t>(r.ncounts + 1);
        P.tile = tile;
        P.block_count = (unsigned long long*)r.bc.p;
        const bool per_inst = P.mode == MODE_COUNT && E.instances;   // batched count sink
        if (per_inst) wmk = r.wm = false;
        if (P.mode == MODE_COUNT) {
            const uint64_t words = per_inst ? 3ull * E.instances : 3;
            r.dg = E.array<uint64_t>(words);
            DL_CUDA(cudaMemsetAsync(r.dg.p, 0, 8 * words, E.stream));
            P.digest = (unsigned long long*)r.dg.p;
        }
        cudaEvent_t a = nullptr, b = nullptr;
        if (timed) {
            a = E.next_event();
            b = E.next_event();
            DL_CUDA(cudaEventRecord(a, E.stream));
        }
        {
            KernelScope ks(E, DL_K_JOIN_COUNT, 4 * Tmin + (entry_bytes + 9) * nF, 1, Tmin, nF);
            if (per_inst && filt) k_wcoj_count_inst<true><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            else if (per_inst) k_wcoj_count_inst<false><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            else if (wmk) DL_NS_DISPATCH(k_wcoj_count_wm, P.nsrc, filt, (unsigned)r.ntiles, E.stream, P);
            else if (filt) k_wcoj_count<true><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            else k_wcoj_count<false><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            DL_CHECK_LAUNCH();
        }
        if (timed) {
            DL_CUDA(cudaEventRecord(b, E.stream));
            DL_CUDA(cudaEventSynchronize(b));
            DL_CUDA(cudaEventElapsedTime(&r.ms, a, b));
        }
        return r;
    };
    // Tile size (units per CTA) and kernel shape: the autotuner's cached choice for this
    // rule, level and size bucket; on a miss every candidate is timed once and the fastest is
    // kept (its counts are the ones used); without the autotuner, the fixed heuristic.
    CountRun cr;
    bool tuned = false;
    if ((E.flags & DL_FLAG_AUTOTUNE) && !P.naive && !E.tile_units) {
        const std::string key = tune_key(R, lvl, T, nF, P.nsrc, filt);
        auto it = E.tune.find(key);
        if (it != E.tune.end()) {
            cr = count_with(it->second.tile, it->second.wm, false);
            E.tune_hits++;
        } else {
            CountRun best;
            // shapes worth timing: a thread per unit decodes every unit's entry (hopeless when
            // entries average hundreds of units); a warp per entry range idles lanes on entries
            // of a few units
            const bool try_striped = T < 256 * nF, try_warp = T >= 4 * nF;
            for (uint32_t tile : {4096u, 16384u, 65536u})
                for (bool wmk : {false, true}) {
                    if ((wmk && !try_warp) || (!wmk && !try_striped)) continue;
                    CountRun r = count_with(tile, wmk, true);
                    if (!best.bc.mem || r.ms < best.ms) best = std::move(r);
                }
            E.tune[key] = {best.tile, best.wm, best.ms};
            E.tuned_levels++;
            cr = std::move(best);
        }
        tuned = true;
    }
    if (!tuned) {
        const uint32_t tile = E.tile_units ? E.tile_units : auto_tile(E, T);
        // warp-major kernels when entries average >= 32 units (one count per warp)
        cr = count_with(tile, !P.naive && T >= 32 * nF, false);
    }
    P.tile = cr.tile;
    P.block_count = (unsigned long long*)cr.bc.p;
    const bool wm = cr.wm;
    const uint64_t ntiles = cr.ntiles, ncounts = cr.ncounts;
    auto bc = cr.bc;
    auto launch_write = [&](uint64_t grid) {
        if (wm) DL_NS_DISPATCH(k_wcoj_write_wm, P.nsrc, filt, (unsigned)grid, E.stream, P);
        else if (filt) k_wcoj_write<true><<<(unsigned)grid, kJoinThreads, 0, E.stream>>>(P);
        else k_wcoj_write<false><<<(unsigned)grid, kJoinThreads, 0, E.stream>>>(P);
    };

    if (last && count_sink) {
        if (E.instances) {
            std::vector<uint64_t> d(3ull * E.instances);
            DL_CUDA(cudaMemcpyAsync(d.data(), cr.dg.p, 8 * d.size(), cudaMemcpyDeviceToHost, E.stream));
            E.sync();
            head.sink_inst.resize(d.size(), 0);
            for (uint64_t i = 0; i < E.instances; i++) {
                head.sink_inst[3 * i] += d[3 * i];
                head.sink_inst[3 * i + 1] += d[3 * i + 1];
                head.sink_inst[3 * i + 2] ^= d[3 * i + 2];
                head.sink_count += d[3 * i];
                head.sink_digest[0] += d[3 * i + 1];
                head.sink_digest[1] ^= d[3 * i + 2];
                E.count_rows += d[3 * i];
            }
        } else {
            const uint64_t* d = E.readback(cr.dg.p, 3);
            head.sink_count += d[0];
            head.sink_digest[0] += d[1];
            head.sink_digest[1] ^= d[2];
            E.count_rows += d[0];
        }
        E.phase_end(0);
        return;
    }

    // Phase 2: count -> exclusive offsets
    scan_u64(E, bc.p, ncounts, false, bc.p + ncounts);
    const uint64_t total = E.readback(bc.p + ncounts, 1)[0];
    if (total == 0) {
        E.phase_end(0);
        return;
    }

    // Phase 3: allocate exactly and write
    if (last) {
        E.join_rows += total;
        // Outputs above chunk_rows are written one tile range at a time; each chunk goes to the
        // caller's chunk sink (sorted, deduplicated, anti-joined) before the next.
        std::vector<uint64_t> off;
        const bool chunked = total > E.chunk_rows && out.chunk_sink;
        if (total >= (1ull << 32) && !chunked) throw Error(DL_ERR_CAPACITY, "rule output of 2^32 rows or more in one round");
        if (chunked) {
            std::vector<uint64_t> all(ncounts + 1);
            DL_CUDA(cudaMemcpyAsync(all.data(), bc.p, sizeof(uint64_t) * (ncounts + 1), cudaMemcpyDeviceToHost,
                                    E.stream));
            E.sync();
            off.resize(ntiles + 1);   // output offset of each tile's first unit
            for (uint64_t t = 0; t <= ntiles; t++) off[t] = all[wm ? t * kWarps : t];
        } else {
            off = {0, total};
        }
        const uint64_t nt = chunked ? ntiles : 1;
        uint64_t a = 0;
        while (a < nt) {
            uint64_t b = chunked ? (uint64_t)(std::upper_bound(off.begin() + a + 1, off.end(), off[a] + E.chunk_rows) -
                                              off.begin()) - 1
                                 : 1;
            if (b <= a) b = a + 1;
            const uint64_t rows = off[b] - off[a];
            if (rows) {
                auto buf = E.make(sizeof(uint32_t) * R.head.arity * rows);
                TableView tv;
                memset(&tv, 0, sizeof(tv));
                tv.arity = R.head.arity;
                tv.n = rows;
                for (uint32_t c = 0; c < R.head.arity; c++) {
                    tv.col[c] = (uint32_t*)buf->ptr + (size_t)c * rows;
                    P.ocol[c] = tv.col[c];
                }
                P.tile_base = chunked ? a : 0;
                P.out_base = off[a];
                const uint64_t grid = chunked ? b - a : ntiles;
                {
                    KernelScope ks(E, DL_K_JOIN_WRITE,
                                   (4 * Tmin + (entry_bytes + 9) * nF) * grid / ntiles + 4ull * R.head.arity * rows, 1,
                                   Tmin * grid / ntiles, nF * grid / ntiles);
                    launch_write(grid);
                    DL_CHECK_LAUNCH();
                }
                if (chunked) {
                    out.chunk_sink(buf, tv);
                } else {
                    out.parts.push_back(tv);
                    out.owners.push_back(buf);
                }
            }
            a = b;
        }
        E.phase_end(0);
        return;
    }

    // The next frontier's bytes per entry (values, carried ranges, parent and sibling runs).
    const uint64_t bpe = 4ull * (lvl + 1 + 2 * P.ncarry) + (next_reuse ? 12 : 0);
    if (total * bpe > frontier_cap() && nF > 1) {
        // Bounded memory: cut the input entries into slices of about equal output and carry
        // each slice through the remaining levels before the next (the paper's two-phase
        // allocation applied per slice).
        const uint64_t want = (total * bpe + frontier_cap() - 1) / frontier_cap();
        const uint32_t s = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(want, 2), 63);
        auto cuts = E.array<uint64_t>(64);
        {
            KernelScope ks(E, DL_K_OTHER, 8ull * s * 64);
            k_slice_cuts<<<1, 64, 0, E.stream>>>((const unsigned long long*)bc.p, ncounts, P.C, nF, T, P.tile, wm ? 1 : 0,
                                                 total, s, (unsigned long long*)cuts.p);
            DL_CHECK_LAUNCH();
        }
        const uint64_t* cutp = E.readback(cuts.p, s);
        std::vector<uint64_t> cut(cutp, cutp + s);
        cut.push_back(nF);
        E.phase_end(0);
        uint64_t prev = 0;
        bool split = false;
        for (uint32_t k = 1; k <= s; k++) {
            const uint64_t c = std::min<uint64_t>(std::max<uint64_t>(cut[k], prev), nF);
            if (c > prev && (prev > 0 || c < nF)) split = true;
            cut[k] = c;
            prev = c;
        }
        if (split) {
            E.join_slices += 1;
            C = DArray<uint64_t>();
            drv = DArray<uint8_t>();
            bc = DArray<uint64_t>();
            cr = CountRun();
            for (uint32_t k = 0; k < s; k++)
                if (cut[k + 1] > cut[k]) level(lvl, F, ea + cut[k], ea + cut[k + 1]);
            return;
        }
        E.phase_begin(0);   // a single entry holds (nearly) all of the output: no cut possible
    }
    if (next_reuse && (nF >= 0xFFFFFFFEull || total >= 0xFFFFFFFEull))
        throw Error(DL_ERR_CAPACITY, "join frontier of 2^32 - 2 entries or more");
    Frontier N;
    N.n = total;
    N.own_vals = E.make(sizeof(uint32_t) * (lvl + 1) * total);
    N.own_rng = E.make(sizeof(uint32_t) * 2 * std::max<uint32_t>(1, P.ncarry) * total);
    for (uint32_t k = 0; k <= lvl; k++) P.oval[k] = (uint32_t*)N.own_vals->ptr + (size_t)k * total;
    for (uint32_t c = 0; c < P.ncarry; c++) {
        P.olo[c] = (uint32_t*)N.own_rng->ptr + (size_t)(2 * c) * total;
        P.ohi[c] = (uint32_t*)N.own_rng->ptr + (size_t)(2 * c + 1) * total;
    }
    P.oparent = nullptr;
    if (next_reuse) {
        N.own_parent = E.make(sizeof(uint32_t) * total);
        P.oparent = (uint32_t*)N.own_parent->ptr;
    }
    {
        KernelScope ks(E, DL_K_JOIN_WRITE,
                       4 * Tmin + (entry_bytes + 9) * nF + 4ull * (lvl + 1 + 2 * P.ncarry + (next_reuse ? 1 : 0)) * total,
                       1, Tmin, nF);
        launch_write(ntiles);
        DL_CHECK_LAUNCH();
    }
    if (next_reuse) {
        N.own_seg = E.make(sizeof(uint32_t) * (2 * total + 1));
        uint32_t* seg = (uint32_t*)N.own_seg->ptr;
        uint32_t* segstart = seg + total;
        launch_seg(E, P.oparent, total, seg, segstart);
        N.seg = seg;
        N.segstart = segstart;
    }
    E.phase_end(0);
    for (uint32_t k = 0; k <= lvl; k++) N.vals[k] = P.oval[k];
    for (uint32_t c = 0; c < P.ncarry; c++) {
        N.slot_of[P.carry_atom[c]] = (int8_t)c;
        N.lo[c] = P.olo[c];
        N.hi[c] = P.ohi[c];
    }
    // this level's own buffers are no longer needed below
    C = DArray<uint64_t>();
    drv = DArray<uint8_t>();
    bc = DArray<uint64_t>();
    cr = CountRun();
    N.own_parent.reset();
    level(lvl + 1, N, 0, total);
}

}  // namespace

void run_join(Engine& E, const Rule& R, const std::vector<const Index*>& src, const std::vector<const Index*>& nsrc,
              Relation& head, JoinOutput& out) {
    JoinRun J(E, R, nsrc, head, out);
    uint64_t filter_levels = 0;
    if (!place_filters(R, nsrc, J.lf, filter_levels)) return;   // a comparison that never holds
    J.plan = make_plan(R, src, filter_levels);
    J.count_sink = head.sink == DL_SINK_COUNT;
    out.sorted_unique = head_is_order(R);

    LevelParams& P = J.base;
    memset(&P, 0, sizeof(P));
    for (uint32_t a = 0; a < J.plan.natoms; a++) {
        P.atom[a] = atom_of(*src[a]);
        if (src[a]->n == 0) return;      // an empty atom: the body has no binding
    }
    P.naive = (E.flags & DL_FLAG_NAIVE_ROOTS) ? 1 : 0;
    P.tile = E.tile_units;
    P.head_arity = R.head.arity;
    for (uint32_t c = 0; c < R.head.arity; c++) {
        if (R.head.terms[c].kind == DL_TERM_CONST) {
            P.head_pos[c] = -1;
            P.head_const[c] = R.head.terms[c].id;
        } else {
            P.head_pos[c] = (int8_t)(std::find(R.order.begin(), R.order.end(), R.head.terms[c].id) - R.order.begin());
        }
    }
    for (uint32_t a = 0; a < J.plan.natoms; a++) P.lazy_pos[a] = (int8_t)J.plan.lazy_pos[a];
    Frontier root;   // the empty prefix
    J.level(0, root, 0, 1);
}

}  // namespace dl
