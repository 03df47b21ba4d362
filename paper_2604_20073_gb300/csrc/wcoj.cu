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

#include "wcoj_kernels.cuh"

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
uint32_t auto_tile(const Engine& E, uint64_t T, uint64_t nF, bool warp_major) {
    const uint64_t waves = 8ull * 8ull * E.sms;
    uint32_t t = 4096;
    while (t < (1u << 16) && T / (2ull * t) >= waves) t *= 2;
    // a thread per unit: keep a tile's entries within the shared-memory stage of entry ends
    if (!warp_major)
        while (t > 4096 && (long double)t * nF > (long double)kStageC * T) t >>= 1;
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
// size bucket of its work (log2 of the units and of the frontier entries), its source count,
// whether it filters, and whether its rows go to a dense bitmap (suffix ":D").
std::string tune_key(const Rule& R, uint32_t lvl, uint64_t T, uint64_t nF, uint32_t nsrc, bool filt, int mode) {
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
    snprintf(buf, sizeof(buf), "%016llx:L%u:T%d:F%d:S%u:f%d%s", (unsigned long long)h, lvl, lg(T), lg(nF), nsrc,
             filt ? 1 : 0, mode == MODE_DENSE ? ":D" : "");
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
    bool dense_sink = false;   // the last level test-and-sets rows in the head's dense bitmap
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
    } else if (last && dense_sink) {
        // rows go straight into the head relation's dense bitmap: no write pass, no raw output
        P.mode = MODE_DENSE;
        P.dense_bits = (uint32_t*)head.dense->ptr;
        P.dense_dirty = (uint8_t*)head.dense_dirty->ptr;
        unsigned long long mul = 1;
        P.dense_lvl_mul = 0;
        P.dense_lvl_dom = UINT32_MAX;
        for (int c = (int)P.head_arity - 1; c >= 0; c--) {
            P.dense_mul[c] = mul;
            P.dense_dom[c] = head.dense_dom[c];
            if (P.head_pos[c] == (int)lvl) {
                P.dense_lvl_mul += mul;
                P.dense_lvl_dom = std::min(P.dense_lvl_dom, head.dense_dom[c]);
            }
            mul *= head.dense_dom[c];
        }
    } else {
        P.mode = last ? MODE_HEAD : MODE_FRONTIER;
    }
    const bool dmode = P.mode == MODE_DENSE;
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
        if (P.mode == MODE_COUNT || dmode) {
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
            else if (wmk) DL_NS_DISPATCH_D(k_wcoj_count_wm, P.nsrc, filt, dmode, (unsigned)r.ntiles, E.stream, P);
            else if (filt && dmode) k_wcoj_count<true, true><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            else if (dmode) k_wcoj_count<false, true><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            else if (filt) k_wcoj_count<true, false><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
            else k_wcoj_count<false, false><<<(unsigned)r.ntiles, kJoinThreads, 0, E.stream>>>(P);
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
        const std::string key = tune_key(R, lvl, T, nF, P.nsrc, filt, P.mode);
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
        // warp-major kernels when entries average >= 32 units (one count per warp)
        const bool wmk = !P.naive && T >= 32 * nF;
        const uint32_t tile = E.tile_units ? E.tile_units : auto_tile(E, T, nF, wmk);
        cr = count_with(tile, wmk, false);
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

    if (dmode) {
        const uint64_t* d = E.readback(cr.dg.p, 3);
        if (d[2]) throw Error(DL_ERR_STATE, "a row lies outside its relation's dense domain");
        E.join_rows += d[0];
        out.dense_rows += d[0];
        out.dense_sunk = true;
        E.phase_end(0);
        return;
    }
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
    J.dense_sink = head.dense && head.dense_dirty && !J.count_sink;
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
    for (uint32_t a = 0; a < J.plan.natoms && a < (uint32_t)kMaxAtoms; a++) P.lazy_pos[a] = (int8_t)J.plan.lazy_pos[a];
    Frontier root;   // the empty prefix
    J.level(0, root, 0, 1);
}

}  // namespace dl
