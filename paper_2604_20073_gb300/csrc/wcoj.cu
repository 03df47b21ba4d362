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
#include <algorithm>

#include "engine.h"

namespace dl {

namespace {

constexpr int kJoinThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

enum { MODE_FRONTIER = 0, MODE_HEAD = 1, MODE_COUNT = 2 };

struct LevelParams {
    AtomView atom[kMaxAtoms];
    uint32_t level;                       // values fval[0..level) are bound by the frontier
    uint32_t nsrc;
    uint8_t src_atom[kMaxAtoms];
    uint8_t src_depth[kMaxAtoms];
    uint8_t src_need_range[kMaxAtoms];    // 1: the narrowed range is carried to the next level
    int8_t slot_in[kMaxAtoms];            // frontier slot of each atom's range, -1 = whole index
    uint64_t nF;
    const uint32_t* fval[kMaxVars];
    const uint32_t* flo[kMaxAtoms];
    const uint32_t* fhi[kMaxAtoms];
    unsigned long long* C;                // per entry: W, then inclusive prefix
    uint8_t* drv;                         // per entry: driving source
    uint64_t T;
    uint64_t tile;
    uint32_t naive;                       // one frontier entry per CTA (ablation baseline)
    unsigned long long* block_count;      // count pass: per-tile counts; write pass: exclusive offsets
    int mode;
    uint32_t* oval[kMaxVars];
    uint32_t ncarry;
    int8_t carry_src[kMaxAtoms];          // source index providing the range, or -1
    int8_t carry_slot[kMaxAtoms];         // otherwise: input slot (-1 = whole index)
    uint8_t carry_atom[kMaxAtoms];
    uint32_t* olo[kMaxAtoms];
    uint32_t* ohi[kMaxAtoms];
    uint32_t head_arity;
    int8_t head_pos[kMaxArity];           // order position of head column, -1 = constant
    uint32_t head_const[kMaxArity];
    uint32_t* ocol[kMaxArity];
    unsigned long long* digest;           // MODE_COUNT: [count, sum, xor]
};

__global__ void k_wcoj_hist(const __grid_constant__ LevelParams P) {
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (e >= P.nF) return;
    unsigned long long best = ~0ull;
    uint32_t bs = 0;
    for (uint32_t s = 0; s < P.nsrc; s++) {
        const int a = P.src_atom[s], d = P.src_depth[s];
        const AtomView& A = P.atom[a];
        unsigned long long len;
        if (d == 0) {
            len = A.n == 0 ? 0 : (A.root ? A.V : A.n);
        } else {
            const int slot = P.slot_in[a];
            len = P.fhi[slot][e] - P.flo[slot][e];
        }
        if (len < best) { best = len; bs = s; }
    }
    P.C[e] = best == ~0ull ? 0 : best;
    P.drv[e] = (uint8_t)bs;
}

struct Unit {
    uint64_t e;
    uint32_t v;
    uint32_t lo[kMaxAtoms], hi[kMaxAtoms];
};

// Decode unit u of the flat space into (entry, local) and evaluate it.
__device__ __forceinline__ bool eval_unit(const LevelParams& P, uint64_t u, uint64_t e0, uint64_t e1, Unit& U) {
    uint64_t e, local;
    if (P.naive) {
        e = e0;
        local = u - (e ? P.C[e - 1] : 0);
    } else {
        e = upper_bound_u64((const uint64_t*)P.C, e0, e1, u);
        local = u - (e ? P.C[e - 1] : 0);
    }
    U.e = e;
    const int s0 = P.drv[e];
    uint32_t v;
    {
        const int a = P.src_atom[s0], d = P.src_depth[s0];
        const AtomView& A = P.atom[a];
        if (d == 0 && A.root) {
            v = (uint32_t)local;                       // iterate the dense value domain
            if (__ldg(A.root + v) >= __ldg(A.root + v + 1)) return false;
        } else {
            uint32_t lo = 0;
            if (d != 0) lo = P.flo[P.slot_in[a]][e];
            const uint32_t r = lo + (uint32_t)local;
            const uint32_t* col = A.col[d];
            v = __ldg(col + r);
            if (r > lo && __ldg(col + r - 1) == v) return false;   // not the first row of its value
        }
    }
    U.v = v;
#pragma unroll
    for (int s = 0; s < kMaxAtoms; s++) {
        if (s >= (int)P.nsrc) break;
        const int a = P.src_atom[s], d = P.src_depth[s];
        const AtomView& A = P.atom[a];
        uint32_t lo, hi;
        if (d == 0) {
            lo = 0;
            hi = A.n;
        } else {
            const int slot = P.slot_in[a];
            lo = P.flo[slot][e];
            hi = P.fhi[slot][e];
        }
        if (P.src_need_range[s]) {
            if (!narrow(A, d, v, lo, hi)) return false;
        } else if (d == 0 && A.root) {
            if (v >= A.V || __ldg(A.root + v) >= __ldg(A.root + v + 1)) return false;
        } else {
            const uint32_t* col = A.col[d];
            const uint32_t l = lower_bound_u32(col, lo, hi, v);
            if (l >= hi || __ldg(col + l) != v) return false;
        }
        U.lo[s] = lo;
        U.hi[s] = hi;
    }
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
        lo = (uint64_t)blockIdx.x * P.tile;
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

__global__ void __launch_bounds__(kJoinThreads) k_wcoj_count(const __grid_constant__ LevelParams P) {
    __shared__ uint64_t s_e0, s_e1;
    uint64_t tlo, thi;
    tile_bounds(P, tlo, thi);
    if (threadIdx.x == 0) {
        if (P.naive) {
            s_e0 = blockIdx.x;
            s_e1 = blockIdx.x + 1;
        } else if (tlo < thi) {
            s_e0 = upper_bound_u64((const uint64_t*)P.C, 0, P.nF, tlo);
            s_e1 = upper_bound_u64((const uint64_t*)P.C, s_e0, P.nF, thi - 1) + 1;
        }
    }
    __syncthreads();
    const uint64_t e0 = s_e0, e1 = s_e1;
    unsigned long long cnt = 0, hs = 0, hx = 0;
    Unit U;
    for (uint64_t u = tlo + threadIdx.x; u < thi; u += blockDim.x) {
        if (!eval_unit(P, u, e0, e1, U)) continue;
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

__global__ void __launch_bounds__(kJoinThreads) k_wcoj_write(const __grid_constant__ LevelParams P) {
    __shared__ uint64_t s_e0, s_e1;
    uint64_t tlo, thi;
    tile_bounds(P, tlo, thi);
    if (threadIdx.x == 0) {
        if (P.naive) {
            s_e0 = blockIdx.x;
            s_e1 = blockIdx.x + 1;
        } else if (tlo < thi) {
            s_e0 = upper_bound_u64((const uint64_t*)P.C, 0, P.nF, tlo);
            s_e1 = upper_bound_u64((const uint64_t*)P.C, s_e0, P.nF, thi - 1) + 1;
        }
    }
    __syncthreads();
    const uint64_t e0 = s_e0, e1 = s_e1;
    uint64_t run = P.block_count[blockIdx.x];
    Unit U;
    for (uint64_t base = tlo; base < thi; base += blockDim.x) {
        const uint64_t u = base + threadIdx.x;
        const uint32_t f = (u < thi && eval_unit(P, u, e0, e1, U)) ? 1u : 0u;
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
#pragma unroll
                for (int c = 0; c < kMaxAtoms; c++) {
                    if (c >= (int)P.ncarry) break;
                    const int s = P.carry_src[c];
                    uint32_t lo, hi;
                    if (s >= 0) {
                        // registers hold the ranges by source index; select without local arrays
                        lo = 0; hi = 0;
#pragma unroll
                        for (int q = 0; q < kMaxAtoms; q++)
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

// ---------------------------------------------------------------- host plan

struct Plan {
    uint32_t m = 0, natoms = 0;
    uint8_t colpos[kMaxAtoms][kMaxArity];   // order position held by index column k of atom a
    uint8_t arity[kMaxAtoms];
    int first_level[kMaxAtoms], last_level[kMaxAtoms];
};

Plan make_plan(const Rule& R) {
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
    return p;
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

// True when a rule's head lists exactly the variable order: the join then emits rows that are
// already sorted in the head's canonical order and distinct.
bool head_is_order(const Rule& R) {
    if (R.head.arity != R.order.size()) return false;
    for (uint32_t c = 0; c < R.head.arity; c++)
        if (R.head.terms[c].kind != DL_TERM_VAR || R.head.terms[c].id != R.order[c]) return false;
    return true;
}

void run_join(Engine& E, const Rule& R, const std::vector<const Index*>& src, Relation& head, JoinOutput& out) {
    const Plan plan = make_plan(R);
    const bool count_sink = head.sink == DL_SINK_COUNT;
    out.sorted_unique = head_is_order(R);

    LevelParams P;
    memset(&P, 0, sizeof(P));
    for (uint32_t a = 0; a < plan.natoms; a++) {
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

    // frontier state (host handles)
    uint64_t nF = 1;
    std::vector<DevPtr> f_vals_owner, f_rng_owner;
    const uint32_t* f_vals[kMaxVars] = {nullptr};
    const uint32_t* f_lo[kMaxAtoms] = {nullptr};
    const uint32_t* f_hi[kMaxAtoms] = {nullptr};
    int8_t slot_of[kMaxAtoms];
    for (int a = 0; a < kMaxAtoms; a++) slot_of[a] = -1;

    auto C = E.array<uint64_t>(1);
    for (uint32_t lvl = 0; lvl < plan.m; lvl++) {
        const bool last = lvl + 1 == plan.m;
        P.level = lvl;
        P.nF = nF;
        for (uint32_t k = 0; k < lvl; k++) P.fval[k] = f_vals[k];
        for (uint32_t a = 0; a < plan.natoms; a++) {
            P.slot_in[a] = slot_of[a];
            if (slot_of[a] >= 0) {
                P.flo[slot_of[a]] = f_lo[slot_of[a]];
                P.fhi[slot_of[a]] = f_hi[slot_of[a]];
            }
        }
        // sources of this level
        P.nsrc = 0;
        for (uint32_t a = 0; a < plan.natoms; a++)
            for (uint32_t k = 0; k < plan.arity[a]; k++)
                if (plan.colpos[a][k] == lvl) {
                    P.src_atom[P.nsrc] = (uint8_t)a;
                    P.src_depth[P.nsrc] = (uint8_t)k;
                    P.src_need_range[P.nsrc] = plan.last_level[a] > (int)lvl ? 1 : 0;
                    P.nsrc++;
                }
        // carried atoms: touched at or before this level and still needed later
        P.ncarry = 0;
        if (!last)
            for (uint32_t a = 0; a < plan.natoms; a++)
                if (plan.first_level[a] <= (int)lvl && plan.last_level[a] > (int)lvl) {
                    const int c = (int)P.ncarry++;
                    P.carry_atom[c] = (uint8_t)a;
                    P.carry_src[c] = -1;
                    for (uint32_t s = 0; s < P.nsrc; s++)
                        if (P.src_atom[s] == a) P.carry_src[c] = (int8_t)s;
                    P.carry_slot[c] = slot_of[a];
                }

        // Phase 1: histogram + prefix
        C = E.array<uint64_t>(nF + 1);
        auto drv = E.array<uint8_t>(nF);
        P.C = (unsigned long long*)C.p;
        P.drv = drv.p;
        // algorithmic bytes of one frontier entry read (values + carried ranges)
        uint32_t nslots_in = 0;
        for (uint32_t a = 0; a < plan.natoms; a++) nslots_in += slot_of[a] >= 0;
        const uint64_t entry_bytes = 4ull * (lvl + 2 * nslots_in);
        E.phase_begin(0);
        {
            KernelScope ks(E, DL_K_JOIN_HIST, (entry_bytes + 9) * nF);
            k_wcoj_hist<<<(unsigned)((nF + 255) / 256), 256, 0, E.stream>>>(P);
            DL_CHECK_LAUNCH();
        }
        scan_u64(E, C.p, nF, true, C.p + nF);
        const uint64_t T = E.readback(C.p + nF, 1)[0];
        if (T == 0) { E.phase_end(0); return; }
        P.T = T;
        const uint64_t ntiles = P.naive ? nF : (T + P.tile - 1) / P.tile;
        if (ntiles >= (1ull << 31)) throw Error(DL_ERR_CAPACITY, "join level exceeds 2^31 tiles");
        auto bc = E.array<uint64_t>(ntiles + 1);
        P.block_count = (unsigned long long*)bc.p;

        if (last && count_sink) {
            auto dg = E.array<uint64_t>(3);
            DL_CUDA(cudaMemsetAsync(dg.p, 0, 24, E.stream));
            P.mode = MODE_COUNT;
            P.digest = (unsigned long long*)dg.p;
            {
                KernelScope ks(E, DL_K_JOIN_COUNT, 4 * T + (entry_bytes + 9) * nF);
                k_wcoj_count<<<(unsigned)ntiles, kJoinThreads, 0, E.stream>>>(P);
                DL_CHECK_LAUNCH();
            }
            const uint64_t* d = E.readback(dg.p, 3);
            head.sink_count += d[0];
            head.sink_digest[0] += d[1];
            head.sink_digest[1] ^= d[2];
            E.count_rows += d[0];
            E.phase_end(0);
            return;
        }

        // Phase 2: count -> exclusive offsets
        P.mode = last ? MODE_HEAD : MODE_FRONTIER;
        {
            KernelScope ks(E, DL_K_JOIN_COUNT, 4 * T + (entry_bytes + 9) * nF);
            k_wcoj_count<<<(unsigned)ntiles, kJoinThreads, 0, E.stream>>>(P);
            DL_CHECK_LAUNCH();
        }
        scan_u64(E, bc.p, ntiles, false, bc.p + ntiles);
        const uint64_t total = E.readback(bc.p + ntiles, 1)[0];
        if (total == 0) { E.phase_end(0); return; }

        // Phase 3: allocate exactly and write
        if (last) {
            if (total >= (1ull << 32)) throw Error(DL_ERR_CAPACITY, "rule output of 2^32 rows or more in one round");
            auto buf = E.make(sizeof(uint32_t) * R.head.arity * total);
            TableView tv;
            memset(&tv, 0, sizeof(tv));
            tv.arity = R.head.arity;
            tv.n = total;
            for (uint32_t c = 0; c < R.head.arity; c++) {
                tv.col[c] = (uint32_t*)buf->ptr + (size_t)c * total;
                P.ocol[c] = tv.col[c];
            }
            {
                KernelScope ks(E, DL_K_JOIN_WRITE, 4 * T + (entry_bytes + 9) * nF + 4ull * R.head.arity * total);
                k_wcoj_write<<<(unsigned)ntiles, kJoinThreads, 0, E.stream>>>(P);
                DL_CHECK_LAUNCH();
            }
            out.parts.push_back(tv);
            out.owners.push_back(buf);
            E.join_rows += total;
            E.phase_end(0);
            return;
        }
        auto vals = E.make(sizeof(uint32_t) * (lvl + 1) * total);
        auto rng = E.make(sizeof(uint32_t) * 2 * std::max<uint32_t>(1, P.ncarry) * total);
        for (uint32_t k = 0; k <= lvl; k++) P.oval[k] = (uint32_t*)vals->ptr + (size_t)k * total;
        for (uint32_t c = 0; c < P.ncarry; c++) {
            P.olo[c] = (uint32_t*)rng->ptr + (size_t)(2 * c) * total;
            P.ohi[c] = (uint32_t*)rng->ptr + (size_t)(2 * c + 1) * total;
        }
        {
            KernelScope ks(E, DL_K_JOIN_WRITE,
                           4 * T + (entry_bytes + 9) * nF + 4ull * (lvl + 1 + 2 * P.ncarry) * total);
            k_wcoj_write<<<(unsigned)ntiles, kJoinThreads, 0, E.stream>>>(P);
            DL_CHECK_LAUNCH();
        }
        E.phase_end(0);
        // the new frontier
        nF = total;
        for (uint32_t k = 0; k <= lvl; k++) f_vals[k] = P.oval[k];
        for (int a = 0; a < kMaxAtoms; a++) slot_of[a] = -1;
        for (uint32_t c = 0; c < P.ncarry; c++) {
            slot_of[P.carry_atom[c]] = (int8_t)c;
            f_lo[c] = P.olo[c];
            f_hi[c] = P.ohi[c];
        }
        f_vals_owner.assign(1, vals);
        f_rng_owner.assign(1, rng);
    }
}

}  // namespace dl
