// Device side of the worst-case-optimal join (kernels and their device helpers), included
// by wcoj.cu inside its anonymous namespace.  The method and the GPU organisation are
// described at the top of wcoj.cu.
#pragma once


constexpr int kJoinThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint8_t kVirtual = 0xff;   // source = the entry's sibling run in the frontier

enum { MODE_FRONTIER = 0, MODE_HEAD = 1, MODE_COUNT = 2, MODE_DENSE = 3 };
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
    unsigned long long* digest;           // MODE_COUNT: [count, sum, xor]; MODE_DENSE: [rows, new, bad]
    // MODE_DENSE: the head relation's dense bitmap; a row's bit is sum over head columns c of
    // value * dense_mul[c] (value < dense_dom[c]); the level's variable contributes
    // v * dense_lvl_mul (v < dense_lvl_dom), the other columns come from the entry
    uint32_t* dense_bits;
    uint8_t* dense_dirty;
    unsigned long long dense_mul[kMaxArity];
    uint32_t dense_dom[kMaxArity];
    unsigned long long dense_lvl_mul;
    uint32_t dense_lvl_dom;
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
// filters).  sC: the tile's entry ends staged in shared memory (sC[0] = the unit before entry
// e0, sC[1 + i] = C[e0 + i]), or null to search C in global memory.
template <bool F>
__device__ __forceinline__ bool eval_unit(const LevelParams& P, uint64_t u, uint64_t e0, uint64_t e1,
                                          const unsigned long long* sC, Unit& U) {
    uint64_t e, prev;
    if (P.naive) {
        e = e0;
        prev = e ? P.C[e - 1] : 0;
    } else if (sC) {
        uint32_t lo = 0, hi = (uint32_t)(e1 - e0);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (sC[1 + mid] <= u) lo = mid + 1; else hi = mid;
        }
        e = e0 + lo;
        prev = sC[lo];
    } else {
        e = upper_bound_u64((const uint64_t*)P.C, e0, e1, u);
        prev = e ? P.C[e - 1] : 0;
    }
    const uint64_t local = u - prev;
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

// MODE_DENSE: test-and-set bit idx of the head relation's bitmap; 1 if this call set it.  Bits
// only go from 0 to 1 during the stratum, so a set bit read through the non-coherent cached
// path settles the row without the atomic (most derived rows of a projecting rule are
// duplicates, and neighbouring entries hit the same words in L1); a stale clear bit only
// sends the row on to the atomic, which decides.  A newly set bit marks its block dirty for
// the round's extraction.
__device__ __forceinline__ uint32_t dense_claim(const LevelParams& P, uint64_t idx) {
    uint32_t* w = P.dense_bits + (idx >> 5);
    const uint32_t m = 1u << (idx & 31);
    if (__ldg(w) & m) return 0u;
    if (atomicOr(w, m) & m) return 0u;
    P.dense_dirty[idx >> (5 + kDenseBlockShift)] = 1;
    return 1u;
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

// A tile's entry ends staged in shared memory when the tile spans at most kStageC entries
// (the per-unit decode then searches shared memory instead of chasing C through L1/L2);
// returns null otherwise.  Every thread of the CTA calls it (it synchronises).
constexpr uint32_t kStageC = 3072;
__device__ __forceinline__ const unsigned long long* stage_entry_ends(const LevelParams& P, uint64_t e0, uint64_t e1,
                                                                      unsigned long long* buf) {
    if (P.naive || e1 - e0 > kStageC) return nullptr;
    const uint32_t ne = (uint32_t)(e1 - e0);
    for (uint32_t i = threadIdx.x; i <= ne; i += blockDim.x)
        buf[i] = i ? P.C[e0 + i - 1] : (e0 ? P.C[e0 - 1] : 0ull);
    __syncthreads();
    return buf;
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

// D: MODE_DENSE (every survivor's row is test-and-set in the head relation's bitmap).
template <bool F, bool D>
__global__ void __launch_bounds__(kJoinThreads, 8) k_wcoj_count(const __grid_constant__ LevelParams P) {
    uint64_t tlo, thi, e0, e1;
    tile_bounds(P, tlo, thi);
    tile_entries(P, tlo, thi, e0, e1);
    __shared__ unsigned long long s_ends[kStageC + 1];
    const unsigned long long* sC = stage_entry_ends(P, e0, e1, s_ends);
    unsigned long long cnt = 0, hs = 0, hx = 0;
    Unit U;
    for (uint64_t u = tlo + threadIdx.x; u < thi; u += blockDim.x) {
        if (!eval_unit<F>(P, u, e0, e1, sC, U)) continue;
        cnt++;
        if (D) {
            uint64_t idx = 0;
            bool in = true;
            for (uint32_t c = 0; c < P.head_arity; c++) {
                const int pos = P.head_pos[c];
                const uint32_t x = pos < 0 ? P.head_const[c] : value_at(P, U, pos);
                in = in && x < P.dense_dom[c];
                idx += (unsigned long long)x * P.dense_mul[c];
            }
            if (in) hs += dense_claim(P, idx);
            else hx = 1;   // a row outside the dense domain
        } else if (P.mode == MODE_COUNT) {
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
    if (D) {
        const unsigned long long s = block_sum(hs);
        const int bad = __syncthreads_or(hx != 0);
        if (threadIdx.x == 0 && total) {
            atomicAdd(&P.digest[0], total);
            atomicAdd(&P.digest[1], s);
            if (bad) atomicOr(&P.digest[2], 1ull);
        }
    } else if (P.mode == MODE_COUNT) {
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
    __shared__ unsigned long long s_ends[kStageC + 1];
    const unsigned long long* sC = stage_entry_ends(P, e0, e1, s_ends);
    unsigned long long cnt = 0;
    Unit U;
    for (uint64_t u = tlo + threadIdx.x; u < thi; u += blockDim.x) {
        if (!eval_unit<F>(P, u, e0, e1, sC, U)) continue;
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
    __shared__ unsigned long long s_ends[kStageC + 1];
    const unsigned long long* sC = stage_entry_ends(P, e0, e1, s_ends);
    uint64_t run = P.block_count[P.tile_base + blockIdx.x] - P.out_base;
    Unit U;
    for (uint64_t base = tlo; base < thi; base += blockDim.x) {
        const uint64_t u = base + threadIdx.x;
        const uint32_t f = (u < thi && eval_unit<F>(P, u, e0, e1, sC, U)) ? 1u : 0u;
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

// D: MODE_DENSE (every survivor's row is test-and-set in the head relation's bitmap).
template <int NS, bool F, bool D>
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
        uint64_t hpre = 0;        // MODE_COUNT: row hash over the head columns before head_lvl;
                                  // MODE_DENSE: the entry's part of the bit index (~0: outside)
        // hash of the columns shared by the current sibling run, and that run (warp-uniform,
        // kept in shared memory: registers are the limit here)
        __shared__ unsigned long long s_hsh[kWarps];
        __shared__ uint32_t s_run[kWarps];
        if (lane == 0) s_run[threadIdx.x >> 5] = 0xFFFFFFFFu;
        __syncwarp();
        for (;;) {
            const uint64_t wlo = s_wlo[threadIdx.x >> 5], whi = s_whi[threadIdx.x >> 5];
            const uint32_t stop = (uint32_t)(min(entry_load(P, S, e, wlo), whi) - wlo);
            if (D) {
                uint64_t ip = 0;
                bool in = true;
                for (uint32_t c = 0; c < P.head_arity; c++) {
                    if (P.head_pos[c] == (int)P.level) continue;
                    const uint32_t x = head_value(P, c, e);
                    in = in && x < P.dense_dom[c];
                    ip += (unsigned long long)x * P.dense_mul[c];
                }
                hpre = in ? ip : ~0ull;
            } else if (P.mode == MODE_COUNT) {
                int c0 = 0;
                if (P.head_shared > 0) {
                    const uint32_t g = __ldg(P.seg + e);
                    if (g != s_run[threadIdx.x >> 5]) {
                        uint64_t hsh = kTupleHashSeed;
                        for (int c = 0; c < P.head_shared; c++) hsh = tuple_hash_step(hsh, head_value(P, c, e), c);
                        __syncwarp();
                        if (lane == 0) {
                            s_run[threadIdx.x >> 5] = g;
                            s_hsh[threadIdx.x >> 5] = hsh;
                        }
                        __syncwarp();
                    }
                    c0 = P.head_shared;
                    hpre = s_hsh[threadIdx.x >> 5];
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
                if (D) {
                    if (hpre == ~0ull || v >= P.dense_lvl_dom) hx = 1;   // a row outside the dense domain
                    else hs += dense_claim(P, hpre + (unsigned long long)v * P.dense_lvl_mul);
                } else if (P.mode == MODE_COUNT) {
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
        if (D) hx |= __shfl_xor_sync(kFull, hx, o);
        else hx ^= __shfl_xor_sync(kFull, hx, o);
    }
    if (lane == 0) {
        P.block_count[(uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)] = cnt;
        if (D && cnt) {
            atomicAdd(&P.digest[0], (unsigned long long)cnt);
            atomicAdd(&P.digest[1], hs);
            if (hx) atomicOr(&P.digest[2], 1ull);
        } else if (P.mode == MODE_COUNT && cnt) {
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

#define DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, ...)                                   \
    do {                                                                                            \
        if ((NSRC) <= 1) KERNEL<1, __VA_ARGS__><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);     \
        else if ((NSRC) <= 2) KERNEL<2, __VA_ARGS__><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS); \
        else if ((NSRC) <= 3) KERNEL<3, __VA_ARGS__><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS); \
        else if ((NSRC) <= 4) KERNEL<4, __VA_ARGS__><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS); \
        else KERNEL<kMaxSrc + 1, __VA_ARGS__><<<(GRID), kJoinThreads, 0, (STREAM)>>>(PARAMS);      \
    } while (0)
// by source count and by whether the level has filters
#define DL_NS_DISPATCH(KERNEL, NSRC, FILT, GRID, STREAM, PARAMS)                                    \
    do {                                                                                            \
        if (FILT) DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, true);                       \
        else DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, false);                           \
    } while (0)
// the count kernels: also by MODE_DENSE
#define DL_NS_DISPATCH_D(KERNEL, NSRC, FILT, D, GRID, STREAM, PARAMS)                               \
    do {                                                                                            \
        if (D) {                                                                                    \
            if (FILT) DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, true, true);             \
            else DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, false, true);                 \
        } else {                                                                                    \
            if (FILT) DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, true, false);            \
            else DL_NS_DISPATCH_F(KERNEL, NSRC, GRID, STREAM, PARAMS, false, false);                \
        }                                                                                           \
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
