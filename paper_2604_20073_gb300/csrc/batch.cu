// Batches of different programs (dl_program_* and dl_fixpoint_batch).
//
// A program is a description (relations, rules, host facts) that is not bound to device
// memory until a batch runs.  dl_fixpoint_batch groups the programs by shape (the same
// relations, sinks and rules; facts may differ) and evaluates each group in the batched form
// of the engine (the instance id as the leading join variable of every atom), so that every
// evaluation stage of a group is one launch over all of its programs, whatever their sizes
// (the work histogram balances them).  Groups run one after another on the parent engine's
// stream.  Results stay on the device in the group's engine until the last program of the
// group is destroyed; results and round counts equal those of each program run alone.
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dl.h"
#include "engine.h"

namespace {

struct AtomCopy {
    dl_rel_id rel = 0;
    std::vector<dl_term> terms;
};

struct RuleCopy {
    AtomCopy head;
    std::vector<AtomCopy> body, neg;
    std::vector<dl_cmp> cmps;
    std::vector<uint32_t> order;
};

struct RelDecl {
    std::string name;
    uint32_t arity = 0, sink = DL_SINK_STORE;
};

struct GroupEngine {
    dl_engine* eng = nullptr;
    dl_stats stats{};
    ~GroupEngine() {
        if (eng) dl_engine_destroy(eng);
    }
};

AtomCopy copy_atom(const dl_atom& a) {
    AtomCopy c;
    c.rel = a.rel;
    if (a.terms) c.terms.assign(a.terms, a.terms + a.arity);
    return c;
}

dl_atom view_atom(const AtomCopy& c) {
    dl_atom a;
    a.rel = c.rel;
    a.arity = (uint32_t)c.terms.size();
    a.terms = c.terms.data();
    return a;
}

}  // namespace

struct dl_program {
    dl_engine* parent = nullptr;
    std::vector<RelDecl> rels;
    std::vector<RuleCopy> rules;
    std::vector<std::pair<dl_rel_id, std::vector<uint32_t>>> facts;   // column-major host copies
    std::vector<uint64_t> fact_rows;
    std::shared_ptr<GroupEngine> group;   // set by dl_fixpoint_batch
    uint32_t inst = 0;
    std::string err;

    // Shape key: relations (arity, sink) and rules; programs with equal keys share launches.
    std::string key() const {
        std::string k;
        auto put = [&k](uint64_t v) { k.append(reinterpret_cast<const char*>(&v), sizeof(v)); };
        put(rels.size());
        for (const RelDecl& r : rels) {
            put(r.arity);
            put(r.sink);
        }
        put(rules.size());
        auto atom = [&](const AtomCopy& a) {
            put(a.rel);
            put(a.terms.size());
            for (const dl_term& t : a.terms) {
                put(t.kind);
                put(t.id);
            }
        };
        for (const RuleCopy& r : rules) {
            atom(r.head);
            put(r.body.size());
            for (const AtomCopy& a : r.body) atom(a);
            put(r.neg.size());
            for (const AtomCopy& a : r.neg) atom(a);
            put(r.cmps.size());
            for (const dl_cmp& c : r.cmps) {
                put(c.op);
                put(c.a.kind);
                put(c.a.id);
                put(c.b.kind);
                put(c.b.id);
            }
            put(r.order.size());
            for (uint32_t v : r.order) put(v);
        }
        return k;
    }
};

namespace {

int fail(dl_program* p, int code, const std::string& msg) {
    p->err = msg;
    return code;
}

// Evaluate one group of same-shape programs in one batched engine.
int run_group(dl_engine* parent, const std::vector<dl_program*>& g) {
    dl::Engine& P = *reinterpret_cast<dl::Engine*>(parent);
    dl_config c;
    memset(&c, 0, sizeof(c));
    c.device = P.device;
    c.stream = P.stream;
    c.arena_bytes = P.budget > P.used ? P.budget - P.used : 1;
    c.flags = P.flags;
    c.tile_units = P.tile_units;
    c.instances = (uint32_t)g.size();
    c.chunk_rows = P.chunk_rows;
    c.hub_rows = P.hub_rows;
    c.frontier_bytes = P.frontier_bytes;
    c.head_percent = P.head_percent;
    auto ge = std::make_shared<GroupEngine>();
    int rc = dl_engine_create(&c, &ge->eng);
    if (rc != DL_OK) return rc;
    const dl_program& p0 = *g[0];
    auto report = [&](int code) {
        const std::string msg = dl_last_error(ge->eng);
        for (dl_program* p : g) p->err = msg;
        return code;
    };
    for (const RelDecl& r : p0.rels) {
        dl_rel_id id;
        if ((rc = dl_relation_create(ge->eng, r.name.c_str(), r.arity, &id)) != DL_OK) return report(rc);
        if (r.sink != DL_SINK_STORE && (rc = dl_relation_set_sink(ge->eng, id, r.sink)) != DL_OK) return report(rc);
    }
    for (const RuleCopy& r : p0.rules) {
        const dl_atom head = view_atom(r.head);
        std::vector<dl_atom> body, neg;
        for (const AtomCopy& a : r.body) body.push_back(view_atom(a));
        for (const AtomCopy& a : r.neg) neg.push_back(view_atom(a));
        dl_rule_id rid;
        rc = dl_rule_add_ex(ge->eng, &head, body.data(), (uint32_t)body.size(), neg.data(), (uint32_t)neg.size(),
                            r.cmps.data(), (uint32_t)r.cmps.size(), r.order.data(), (uint32_t)r.order.size(), &rid);
        if (rc != DL_OK) return report(rc);
    }
    for (uint32_t i = 0; i < g.size(); i++) {
        const dl_program& p = *g[i];
        for (size_t f = 0; f < p.facts.size(); f++) {
            const uint64_t n = p.fact_rows[f];
            if (!n) continue;
            const uint32_t a = p.rels[p.facts[f].first].arity;
            std::vector<const uint32_t*> cols(a);
            for (uint32_t k = 0; k < a; k++) cols[k] = p.facts[f].second.data() + (size_t)k * n;
            if ((rc = dl_load_facts_instance(ge->eng, p.facts[f].first, i, cols.data(), n)) != DL_OK) return report(rc);
        }
    }
    if ((rc = dl_fixpoint(ge->eng, &ge->stats)) != DL_OK) return report(rc);
    for (uint32_t i = 0; i < g.size(); i++) {
        g[i]->group = ge;
        g[i]->inst = i;
        g[i]->err.clear();
    }
    return DL_OK;
}

}  // namespace

extern "C" {

int dl_program_create(dl_engine* e, dl_program** out) {
    if (!e || !out) return DL_ERR_ARG;
    *out = new (std::nothrow) dl_program();
    if (!*out) return DL_ERR_CAPACITY;
    (*out)->parent = e;
    return DL_OK;
}

void dl_program_destroy(dl_program* p) { delete p; }

const char* dl_program_last_error(const dl_program* p) { return p ? p->err.c_str() : "null program"; }

int dl_program_relation(dl_program* p, const char* name, uint32_t arity, uint32_t sink, dl_rel_id* out) {
    if (!p) return DL_ERR_ARG;
    if (!name || !*name) return fail(p, DL_ERR_ARG, "empty relation name");
    if (arity < 1 || arity + 1 > DL_MAX_ARITY) return fail(p, DL_ERR_ARG, "arity out of range");
    if (sink != DL_SINK_STORE && sink != DL_SINK_COUNT) return fail(p, DL_ERR_ARG, "bad sink");
    for (const RelDecl& r : p->rels)
        if (r.name == name) return fail(p, DL_ERR_ARG, std::string("duplicate relation name ") + name);
    p->rels.push_back({name, arity, sink});
    if (out) *out = (dl_rel_id)(p->rels.size() - 1);
    return DL_OK;
}

int dl_program_rule(dl_program* p, const dl_atom* head, const dl_atom* body, uint32_t nbody, const dl_atom* neg,
                    uint32_t nneg, const dl_cmp* cmps, uint32_t ncmp, const uint32_t* var_order, uint32_t nvars) {
    if (!p) return DL_ERR_ARG;
    if (!head || !body || nbody == 0 || (nneg && !neg) || (ncmp && !cmps) || !var_order)
        return fail(p, DL_ERR_ARG, "null or empty rule parts");
    auto known = [&](const dl_atom& a) { return a.rel < p->rels.size() && a.arity == p->rels[a.rel].arity && a.terms; };
    if (!known(*head)) return fail(p, DL_ERR_ARG, "bad head atom");
    RuleCopy r;
    r.head = copy_atom(*head);
    for (uint32_t b = 0; b < nbody; b++) {
        if (!known(body[b])) return fail(p, DL_ERR_ARG, "bad body atom");
        r.body.push_back(copy_atom(body[b]));
    }
    for (uint32_t b = 0; b < nneg; b++) {
        if (!known(neg[b])) return fail(p, DL_ERR_ARG, "bad negated atom");
        r.neg.push_back(copy_atom(neg[b]));
    }
    r.cmps.assign(cmps, cmps + ncmp);
    r.order.assign(var_order, var_order + nvars);
    p->rules.push_back(std::move(r));   // checked in full when the batch declares it
    return DL_OK;
}

int dl_program_load_facts(dl_program* p, dl_rel_id rel, const uint32_t* const* cols, uint64_t nrows) {
    if (!p) return DL_ERR_ARG;
    if (rel >= p->rels.size()) return fail(p, DL_ERR_ARG, "bad relation id");
    if (nrows == 0) return DL_OK;
    if (!cols) return fail(p, DL_ERR_ARG, "null column array");
    const uint32_t a = p->rels[rel].arity;
    std::vector<uint32_t> data((size_t)a * nrows);
    for (uint32_t c = 0; c < a; c++) {
        if (!cols[c]) return fail(p, DL_ERR_ARG, "null column pointer");
        memcpy(data.data() + (size_t)c * nrows, cols[c], sizeof(uint32_t) * nrows);
    }
    p->facts.push_back({rel, std::move(data)});
    p->fact_rows.push_back(nrows);
    return DL_OK;
}

int dl_fixpoint_batch(dl_engine* e, dl_program* const* progs, uint32_t n, dl_stats* per_prog) {
    if (!e || (n && !progs)) return DL_ERR_ARG;
    std::map<std::string, std::vector<dl_program*>> groups;
    std::vector<std::string> order;
    for (uint32_t i = 0; i < n; i++) {
        if (!progs[i] || progs[i]->parent != e) return DL_ERR_ARG;
        progs[i]->group.reset();
        const std::string k = progs[i]->key();
        if (!groups.count(k)) order.push_back(k);
        groups[k].push_back(progs[i]);
    }
    int status = DL_OK;
    for (const std::string& k : order) {
        const int rc = run_group(e, groups[k]);
        if (rc != DL_OK && status == DL_OK) status = rc;
    }
    if (per_prog)
        for (uint32_t i = 0; i < n; i++) {
            if (progs[i]->group) per_prog[i] = progs[i]->group->stats;
            else memset(&per_prog[i], 0, sizeof(dl_stats));
        }
    return status;
}

int dl_program_fetch(dl_program* p, dl_rel_id rel, uint32_t* const* cols_out, uint64_t cap_rows, uint64_t* nrows_out) {
    if (!p) return DL_ERR_ARG;
    if (!p->group) return fail(p, DL_ERR_STATE, "the program has not been evaluated");
    const int rc = dl_fetch_instance(p->group->eng, rel, p->inst, cols_out, cap_rows, nrows_out);
    if (rc != DL_OK) p->err = dl_last_error(p->group->eng);
    return rc;
}

int dl_program_digest(dl_program* p, dl_rel_id rel, uint64_t* count, uint64_t digest[2]) {
    if (!p) return DL_ERR_ARG;
    if (!p->group) return fail(p, DL_ERR_STATE, "the program has not been evaluated");
    const int rc = dl_instance_digest(p->group->eng, rel, p->inst, count, digest);
    if (rc != DL_OK) p->err = dl_last_error(p->group->eng);
    return rc;
}

int dl_program_rounds(dl_program* p, uint32_t* rounds, uint32_t cap, uint32_t* nstrata) {
    if (!p) return DL_ERR_ARG;
    if (!p->group) return fail(p, DL_ERR_STATE, "the program has not been evaluated");
    const int rc = dl_instance_rounds(p->group->eng, p->inst, rounds, cap, nstrata);
    if (rc != DL_OK) p->err = dl_last_error(p->group->eng);
    return rc;
}

int dl_program_stratum(dl_program* p, uint32_t s, dl_rel_id* rels, uint32_t cap, uint32_t* nrels) {
    if (!p) return DL_ERR_ARG;
    if (!p->group) return fail(p, DL_ERR_STATE, "the program has not been evaluated");
    const int rc = dl_stratum_info(p->group->eng, s, rels, cap, nrels, nullptr);
    if (rc != DL_OK) p->err = dl_last_error(p->group->eng);
    return rc;
}

}  // extern "C"
