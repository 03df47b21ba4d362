// Serving loop (dl_server_*): admission of many independent programs by device-memory
// budget, one worker thread and CUDA stream per slot, results resident until released.
//
// Each admitted request gets its own engine on its slot's stream; engines of concurrent
// requests run their kernels on different streams, so their work overlaps on the GPU.  All
// device memory comes from one server-owned stream-ordered pool through the engines'
// allocator hooks; each engine's budget is its request's share, so a request that outgrows
// its share fails alone (DL_ERR_CAPACITY) while the server's total stays within budget.
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

struct RuleCopy {
    dl_atom head;
    std::vector<dl_term> head_terms;
    std::vector<dl_atom> body, neg;
    std::vector<std::vector<dl_term>> body_terms, neg_terms;
    std::vector<dl_cmp> cmps;
    std::vector<uint32_t> order;
};

struct FactCopy {
    uint32_t rel;
    std::vector<uint32_t> rows;
    uint64_t nrows;
};

struct Ticket {
    uint64_t id = 0;
    std::vector<std::string> names;
    std::vector<uint32_t> arity, sink;
    std::vector<RuleCopy> rules;
    std::vector<FactCopy> facts;
    uint64_t share = 0;
    uint32_t grows = 0;               // re-evaluations with a doubled share so far
    bool admitted = false;            // its share was added to the server's reservation
    int state = DL_REQ_QUEUED;
    int status = DL_OK;
    dl_engine* eng = nullptr;
};

}  // namespace

struct dl_server {
    int device = 0;
    uint64_t budget = 0, reserved = 0, peak_reserved = 0, default_share = 1ull << 30;
    uint32_t flags = 0;
    uint32_t grow_retries = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<Ticket*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    uint64_t submitted = 0, admitted = 0, completed = 0, failed = 0, regrown = 0;
    uint32_t running = 0;
};

namespace {

void* pool_alloc(uint64_t bytes, void* stream, void* user) {
    dl_server* s = (dl_server*)user;
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, s->pool, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void* p, uint64_t, void* stream, void*) { cudaFreeAsync(p, (cudaStream_t)stream); }

int evaluate(dl_server* s, cudaStream_t stream, Ticket* t) {
    dl_config c;
    memset(&c, 0, sizeof(c));
    c.device = s->device;
    c.stream = stream;
    c.arena_bytes = t->share;
    c.alloc = pool_alloc;
    c.free = pool_free;
    c.alloc_user = s;
    c.flags = s->flags;
    dl_engine* e = nullptr;
    int rc = dl_engine_create(&c, &e);
    if (rc != DL_OK) return rc;
    t->eng = e;
    for (size_t i = 0; i < t->names.size(); i++) {
        dl_rel_id id;
        if ((rc = dl_relation_create(e, t->names[i].c_str(), t->arity[i], &id)) != DL_OK) return rc;
        if (t->sink[i] != DL_SINK_STORE && (rc = dl_relation_set_sink(e, id, t->sink[i])) != DL_OK) return rc;
    }
    for (RuleCopy& r : t->rules) {
        r.head.terms = r.head_terms.data();
        for (size_t b = 0; b < r.body.size(); b++) r.body[b].terms = r.body_terms[b].data();
        for (size_t b = 0; b < r.neg.size(); b++) r.neg[b].terms = r.neg_terms[b].data();
        dl_rule_id rid;
        rc = dl_rule_add_ex(e, &r.head, r.body.data(), (uint32_t)r.body.size(), r.neg.data(), (uint32_t)r.neg.size(),
                            r.cmps.data(), (uint32_t)r.cmps.size(), r.order.data(), (uint32_t)r.order.size(), &rid);
        if (rc != DL_OK) return rc;
    }
    for (FactCopy& f : t->facts)
        if ((rc = dl_load_facts_rows(e, f.rel, f.rows.data(), f.nrows)) != DL_OK) return rc;
    if (t->grows >= s->grow_retries) {   // no re-evaluation can follow: drop the host copy
        t->facts.clear();
        t->facts.shrink_to_fit();
    }
    return dl_fixpoint(e, nullptr);
}

void worker_loop(dl_server* s, size_t slot) {
    cudaSetDevice(s->device);
    cudaStream_t stream = s->streams[slot];
    for (;;) {
        Ticket* t = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                return s->stop || (!s->queue.empty() && s->reserved + s->queue.front()->share <= s->budget);
            });
            if (s->stop && s->queue.empty()) return;
            if (s->stop) {  // drain: fail what was never admitted
                Ticket* q = s->queue.front();
                s->queue.pop_front();
                q->state = DL_REQ_DONE;
                q->status = DL_ERR_STATE;
                s->cv.notify_all();
                continue;
            }
            t = s->queue.front();
            s->queue.pop_front();
            s->reserved += t->share;
            t->admitted = true;
            s->peak_reserved = std::max(s->peak_reserved, s->reserved);
            s->admitted++;
            s->running++;
            t->state = DL_REQ_RUNNING;
        }
        const int rc = evaluate(s, stream, t);
        // outgrew its share: start again from scratch with twice the share, ahead of later
        // arrivals (the failed engine's memory goes back to the pool first)
        const bool regrow = rc == DL_ERR_CAPACITY && t->grows < s->grow_retries && t->share < s->budget;
        if (regrow && t->eng) {
            dl_engine_destroy(t->eng);
            t->eng = nullptr;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->running--;
            if (regrow) {
                s->reserved -= t->share;
                t->admitted = false;
                t->share = std::min(s->budget, 2 * t->share);
                t->grows++;
                t->state = DL_REQ_QUEUED;
                s->queue.push_front(t);
                s->regrown++;
            } else {
                t->status = rc;
                t->state = DL_REQ_DONE;
                s->completed++;
                if (rc != DL_OK) s->failed++;
            }
        }
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

int dl_server_create(const dl_server_config* cfg, dl_server** out) {
    if (!out) return DL_ERR_ARG;
    *out = nullptr;
    dl_server_config c;
    memset(&c, 0, sizeof(c));
    c.device = -1;
    if (cfg) c = *cfg;
    auto s = std::make_unique<dl_server>();
    if (c.device < 0) {
        if (cudaGetDevice(&s->device) != cudaSuccess) return DL_ERR_CUDA;
    } else {
        s->device = c.device;
    }
    if (cudaSetDevice(s->device) != cudaSuccess) return DL_ERR_CUDA;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return DL_ERR_CUDA;
    s->budget = c.budget_bytes ? c.budget_bytes : (uint64_t)(fr * 0.9);
    s->flags = c.flags;
    if (c.default_share) s->default_share = c.default_share;
    s->grow_retries = c.grow_retries;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) return DL_ERR_CUDA;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    const uint32_t slots = c.max_slots ? c.max_slots : 8;
    s->streams.resize(slots);
    for (uint32_t i = 0; i < slots; i++)
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) return DL_ERR_CUDA;
    dl_server* raw = s.get();
    for (uint32_t i = 0; i < slots; i++) raw->workers.emplace_back(worker_loop, raw, (size_t)i);
    *out = s.release();
    return DL_OK;
}

void dl_server_destroy(dl_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto& w : s->workers) w.join();
    cudaSetDevice(s->device);
    for (auto& kv : s->tickets)
        if (kv.second->eng) dl_engine_destroy(kv.second->eng);
    s->tickets.clear();
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

int dl_server_submit(dl_server* s, const dl_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || (req->nrel && (!req->rel_names || !req->rel_arity))) return DL_ERR_ARG;
    if ((req->nrules && !req->rules) || (req->nfacts && !req->facts)) return DL_ERR_ARG;
    auto t = std::make_unique<Ticket>();
    for (uint32_t i = 0; i < req->nrel; i++) {
        if (!req->rel_names[i]) return DL_ERR_ARG;
        t->names.push_back(req->rel_names[i]);
        t->arity.push_back(req->rel_arity[i]);
        t->sink.push_back(req->rel_sink ? req->rel_sink[i] : DL_SINK_STORE);
    }
    for (uint32_t r = 0; r < req->nrules; r++) {
        const dl_rule_spec& rs = req->rules[r];
        if (!rs.head.terms || (rs.nbody && !rs.body) || (rs.nvars && !rs.var_order)) return DL_ERR_ARG;
        RuleCopy rc;
        rc.head = rs.head;
        rc.head_terms.assign(rs.head.terms, rs.head.terms + rs.head.arity);
        for (uint32_t b = 0; b < rs.nbody; b++) {
            if (!rs.body[b].terms) return DL_ERR_ARG;
            rc.body.push_back(rs.body[b]);
            rc.body_terms.emplace_back(rs.body[b].terms, rs.body[b].terms + rs.body[b].arity);
        }
        if ((rs.nneg && !rs.neg) || (rs.ncmp && !rs.cmps)) return DL_ERR_ARG;
        for (uint32_t b = 0; b < rs.nneg; b++) {
            if (!rs.neg[b].terms) return DL_ERR_ARG;
            rc.neg.push_back(rs.neg[b]);
            rc.neg_terms.emplace_back(rs.neg[b].terms, rs.neg[b].terms + rs.neg[b].arity);
        }
        if (rs.ncmp) rc.cmps.assign(rs.cmps, rs.cmps + rs.ncmp);
        rc.order.assign(rs.var_order, rs.var_order + rs.nvars);
        t->rules.push_back(std::move(rc));
    }
    for (uint32_t f = 0; f < req->nfacts; f++) {
        const dl_fact_spec& fs = req->facts[f];
        if (fs.rel >= req->nrel || (fs.nrows && !fs.rows)) return DL_ERR_ARG;
        FactCopy fc;
        fc.rel = fs.rel;
        fc.nrows = fs.nrows;
        fc.rows.assign(fs.rows, fs.rows + fs.nrows * req->rel_arity[fs.rel]);
        t->facts.push_back(std::move(fc));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    t->share = req->share_bytes ? req->share_bytes : s->default_share;
    if (t->share > s->budget) return DL_ERR_ARG;
    t->id = s->next_id++;
    *ticket = t->id;
    s->queue.push_back(t.get());
    s->tickets[t->id] = std::move(t);
    s->submitted++;
    s->cv.notify_all();
    return DL_OK;
}

int dl_server_poll(dl_server* s, uint64_t ticket, int* state, int* status) {
    if (!s) return DL_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return DL_ERR_ARG;
    if (state) *state = it->second->state;
    if (status) *status = it->second->status;
    return DL_OK;
}

int dl_server_wait(dl_server* s, uint64_t ticket, int* status) {
    if (!s) return DL_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return DL_ERR_ARG;
    Ticket* t = it->second.get();
    s->cv.wait(lk, [&] { return t->state == DL_REQ_DONE; });
    if (status) *status = t->status;
    return DL_OK;
}

int dl_server_result(dl_server* s, uint64_t ticket, dl_engine** engine) {
    if (!s || !engine) return DL_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return DL_ERR_ARG;
    if (it->second->state != DL_REQ_DONE || !it->second->eng) return DL_ERR_STATE;
    *engine = it->second->eng;
    return DL_OK;
}

int dl_server_release(dl_server* s, uint64_t ticket) {
    if (!s) return DL_ERR_ARG;
    std::unique_ptr<Ticket> t;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return DL_ERR_ARG;
        if (it->second->state != DL_REQ_DONE) return DL_ERR_STATE;
        t = std::move(it->second);
        s->tickets.erase(it);
    }
    if (t->eng) {
        cudaSetDevice(s->device);
        dl_engine_destroy(t->eng);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (t->admitted) s->reserved -= t->share;   // a request drained at stop was never admitted
    }
    s->cv.notify_all();
    return DL_OK;
}

int dl_server_get_stats(dl_server* s, dl_server_stats* out) {
    if (!s || !out) return DL_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->reserved_bytes = s->reserved;
    out->peak_reserved_bytes = s->peak_reserved;
    out->running = s->running;
    out->queued = (uint32_t)s->queue.size();
    out->regrown = s->regrown;
    return DL_OK;
}

}  // extern "C"
