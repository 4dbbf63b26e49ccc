// Many-product batch call and the continuous-batching serving loop, both on
// the task engine (engine.h).
//
// Serving: a worker thread owns the context while the server lives.  Between
// waves it admits queued requests while the HBM budget holds the engine's
// batch buffers (reserved once, at their size for the highest admitted level)
// plus every admitted request's result chunks and mask (operands and keys are
// already resident), plans them into the engine, and runs the next wave, so
// requests that arrive while others are on the GPU join the same batches.  A
// request's completion is the CUDA event recorded after its last
// accumulation; the worker polls these events and timestamps completions.  A
// wave that fails does not fail the requests in it: completed ones keep their
// results and the rest run again alone, so only a request that fails by
// itself reports an error.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <set>
#include <thread>

#include "engine.h"
#include "handles.h"

namespace spfhe {

static double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

static void job_from_req(Job &job, const spfhe_matmul_req &r, size_t n_c)
{
    if (!r.keys || !r.A_csr || !r.B_csc || !r.A_chunks || !r.B_chunks) throw Error(SPFHE_EINVAL, "null request field");
    validate_pair(*r.A_csr, *r.B_csc);
    std::vector<Ct *> a(r.n_a), b(r.n_b);
    for (size_t i = 0; i < r.n_a; ++i) a[i] = r.A_chunks[i] ? r.A_chunks[i]->c : nullptr;
    for (size_t i = 0; i < r.n_b; ++i) b[i] = r.B_chunks[i] ? r.B_chunks[i]->c : nullptr;
    fill_job(job, *r.keys->k, *r.A_csr, a.data(), r.n_a, *r.B_csc, b.data(), r.n_b, r.mask0 ? r.mask0->p : nullptr,
             n_c);
}

size_t result_chunks(const Ctx &ctx, const spfhe_matmul_req &r)
{
    if (!r.A_csr || !r.B_csc) throw Error(SPFHE_EINVAL, "null metadata");
    return chunks_for((long long)r.A_csr->rows * r.B_csc->cols, ctx.S);
}

void sparse_matmul_batch(Ctx &ctx, size_t n_req, const spfhe_matmul_req *reqs, Ct **C, size_t n_c_total,
                         spfhe_stats *stats)
{
    const uint64_t launches0 = ctx.launches;
    size_t want = 0;
    for (size_t r = 0; r < n_req; ++r) want += result_chunks(ctx, reqs[r]);
    if (want != n_c_total) throw Error(SPFHE_EINVAL, "result array size != sum of ceil(rows*cols / S)");
    std::vector<Job> jobs(n_req);
    for (size_t r = 0; r < n_req; ++r) job_from_req(jobs[r], reqs[r], result_chunks(ctx, reqs[r]));
    for (size_t i = 0; i < n_c_total; ++i) C[i] = nullptr;
    Engine eng(ctx);
    try {
        for (auto &j : jobs) eng.add(&j);
        eng.run_all();
        ctx_sync(ctx);
    } catch (...) {
        for (auto &j : jobs) release_job(ctx, j, true);
        throw;
    }
    size_t o = 0;
    for (size_t r = 0; r < n_req; ++r) {
        Job &j = jobs[r];
        for (Ct *c : j.C) C[o++] = c;
        release_job(ctx, j, false);
        if (stats) {
            stats[r].matches = j.st_matches;
            stats[r].ks_relin = j.st_relin;
            stats[r].ks_align = j.st_align;
            stats[r].ks_final = j.st_final;
            stats[r].rescales = j.st_rescales;
            stats[r].launches = ctx.launches - launches0;   // launches of the whole batch
        }
    }
}

// ---------------------------------------------------------------------------
struct Server {
    Ctx &ctx;
    uint64_t budget;
    uint64_t in_use = 0;       // footprints of admitted, unfinished requests
    uint64_t ws_reserved = 0;  // the engine's batch buffers at the highest admitted level
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    struct Entry {
        Job job;
        uint64_t footprint = 0;
        double t_submit = 0, t_done = 0;
        spfhe_status status = SPFHE_OK;
        std::string err;
        bool done = false;
    };
    std::map<uint64_t, std::unique_ptr<Entry>> entries;   // guarded by mu
    std::deque<uint64_t> queue;      // submitted, not yet admitted
    uint64_t next_ticket = 1;
    uint64_t retried = 0;            // requests re-run alone after a failed wave
    std::set<uint64_t> poisoned;     // future tickets marked for fault injection
    std::thread worker;

    Server(Ctx &c, uint64_t b) : ctx(c), budget(b) { worker = std::thread([this] { loop(); }); }

    // device memory a request adds while it runs: its result chunks and its
    // mask (a private copy of the caller's, or the level's library mask if
    // none exists yet); the shared batch buffers are reserved separately
    uint64_t footprint_of(const Job &j) const
    {
        const int ell = j.Ach.empty() || !j.Ach[0] ? ctx.L : j.Ach[0]->level;
        return (uint64_t)j.n_c * 2ull * (uint64_t)std::max(ell - 2, 1) * ctx.n * sizeof(u64) +
               job_mask_bytes(ctx, j);
    }

    static int level_of(const Ctx &c, const Job &j) { return j.Ach.empty() || !j.Ach[0] ? c.L : j.Ach[0]->level; }

    void complete(Entry &e)
    {
        std::lock_guard<std::mutex> lk(mu);
        e.t_done = now_ms();
        e.done = true;
        in_use -= e.footprint;
        cv_done.notify_all();
    }

    // a failed wave: requests whose last task had completed keep their
    // results; every other running request is run again alone in a fresh
    // engine (its results reallocated and zeroed), so only a request that also
    // fails alone is reported failed
    void recover(std::vector<Entry *> &running)
    {
        cudaStreamSynchronize(ctx.stream);
        cudaGetLastError();
        std::vector<Entry *> redo;
        for (Entry *e : running) {
            if (e->job.finished && e->job.done_ev && cudaEventQuery(e->job.done_ev) == cudaSuccess)
                complete(*e);
            else
                redo.push_back(e);
        }
        running.clear();
        cudaGetLastError();
        for (Entry *e : redo) {
            release_job(ctx, e->job, true);
            reset_job(e->job);
            ++retried;
            try {
                Engine solo(ctx);
                solo.add(&e->job);
                solo.run_all();
                SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
                complete(*e);
            } catch (const Error &err) {
                finish_failed(*e, err.code, err.what());
            } catch (const std::exception &err) {
                finish_failed(*e, SPFHE_EINVAL, err.what());
            } catch (...) {
                finish_failed(*e, SPFHE_EINVAL, "unknown error");
            }
        }
    }

    void loop()
    {
        cudaSetDevice(ctx.device);
        std::unique_ptr<Engine> eng(new Engine(ctx));
        std::vector<Entry *> running;   // admitted, event not yet complete
        int ws_level = 0;               // level the workspace reservation covers
        for (;;) {
            std::vector<Entry *> admit;
            {
                std::unique_lock<std::mutex> lk(mu);
                while (!queue.empty()) {
                    Entry *e = entries.at(queue.front()).get();
                    // computed here: only this thread touches the context
                    // (its level masks) while the server lives
                    e->footprint = footprint_of(e->job);
                    const int lv = std::max(ws_level, level_of(ctx, e->job));
                    const uint64_t ws = engine_workspace_bound(ctx, lv);
                    // a request is admitted whatever its size when nothing else
                    // runs (nothing else could free memory for it)
                    if (in_use + ws + e->footprint > budget && !(running.empty() && admit.empty())) break;
                    in_use += e->footprint;
                    ws_level = lv;
                    ws_reserved = ws;
                    admit.push_back(e);
                    queue.pop_front();
                }
                if (admit.empty() && running.empty() && eng->idle()) {
                    if (stop) break;
                    cv_work.wait_for(lk, std::chrono::milliseconds(50));
                    continue;
                }
            }
            for (Entry *e : admit) {
                try {
                    SPFHE_CHECK_CUDA(cudaEventCreateWithFlags(&e->job.done_ev, cudaEventDisableTiming));
                    eng->add(&e->job);
                    running.push_back(e);
                } catch (const Error &err) {
                    finish_failed(*e, err.code, err.what());
                } catch (const std::exception &err) {
                    finish_failed(*e, SPFHE_EINVAL, err.what());
                } catch (...) {
                    finish_failed(*e, SPFHE_EINVAL, "unknown error");
                }
            }
            bool worked = false, failed = false;
            try {
                worked = eng->step();
                eng->take_finished();
            } catch (...) {
                failed = true;
            }
            if (failed) {
                recover(running);
                eng.reset(new Engine(ctx));
                continue;
            }
            if (!worked && !running.empty()) std::this_thread::sleep_for(std::chrono::microseconds(200));
            // completions
            for (size_t i = 0; i < running.size();) {
                Entry *e = running[i];
                if (e->job.finished && cudaEventQuery(e->job.done_ev) == cudaSuccess) {
                    complete(*e);
                    running.erase(running.begin() + i);
                } else {
                    ++i;
                }
            }
        }
    }

    void finish_failed(Entry &e, spfhe_status code, const std::string &msg)
    {
        std::lock_guard<std::mutex> lk(mu);
        release_job(ctx, e.job, true);
        if (e.job.done_ev) cudaEventDestroy(e.job.done_ev);
        e.job.done_ev = nullptr;
        e.status = code;
        e.err = msg;
        e.t_done = now_ms();
        e.done = true;
        in_use -= e.footprint;
        cv_done.notify_all();
    }
};

}  // namespace spfhe

using namespace spfhe;

struct spfhe_server {
    Server *s;
};

extern "C" {

spfhe_status spfhe_sparse_matmul_batch(spfhe_ctx *ctx, size_t n_req, const spfhe_matmul_req *reqs,
                                       spfhe_ct **C_chunks, size_t n_c_total, spfhe_stats *stats)
{
    try {
        if (!ctx || (n_req && (!reqs || !C_chunks))) throw Error(SPFHE_EINVAL, "null argument");
        Ctx &c = ctx->c;
        SPFHE_CHECK_CUDA(cudaSetDevice(c.device));
        std::vector<Ct *> out(n_c_total, nullptr);
        sparse_matmul_batch(c, n_req, reqs, out.data(), n_c_total, stats);
        for (size_t i = 0; i < n_c_total; ++i) {
            spfhe_ct *h = new spfhe_ct;
            h->c = out[i];
            C_chunks[i] = h;
        }
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return SPFHE_EINVAL;
    }
}

spfhe_status spfhe_server_create(spfhe_ctx *ctx, uint64_t hbm_budget_bytes, spfhe_server **out)
{
    try {
        if (!ctx || !out) throw Error(SPFHE_EINVAL, "null argument");
        SPFHE_CHECK_CUDA(cudaSetDevice(ctx->c.device));
        *out = new spfhe_server{new Server(ctx->c, hbm_budget_bytes)};
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}

spfhe_status spfhe_server_submit(spfhe_server *srv, const spfhe_matmul_req *req, uint64_t *ticket)
{
    try {
        if (!srv || !req || !ticket) throw Error(SPFHE_EINVAL, "null argument");
        Server &s = *srv->s;
        auto e = std::make_unique<Server::Entry>();
        job_from_req(e->job, *req, result_chunks(s.ctx, *req));
        e->t_submit = now_ms();
        std::lock_guard<std::mutex> lk(s.mu);
        const uint64_t t = s.next_ticket++;
        if (s.poisoned.erase(t)) e->job.inject_fault = true;
        s.entries[t] = std::move(e);
        s.queue.push_back(t);
        *ticket = t;
        s.cv_work.notify_all();
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return SPFHE_EINVAL;
    }
}

spfhe_status spfhe_server_wait(spfhe_server *srv, uint64_t ticket, spfhe_ct **C_chunks, size_t n_c,
                               spfhe_stats *stats, double *latency_ms)
{
    try {
        if (!srv || !C_chunks) throw Error(SPFHE_EINVAL, "null argument");
        Server &s = *srv->s;
        std::unique_lock<std::mutex> lk(s.mu);
        auto it = s.entries.find(ticket);
        if (it == s.entries.end()) throw Error(SPFHE_EINVAL, "unknown ticket");
        Server::Entry &e = *it->second;
        s.cv_done.wait(lk, [&] { return e.done; });
        if (e.status != SPFHE_OK) {
            const spfhe_status st = e.status;
            const std::string msg = e.err;
            s.entries.erase(it);
            throw Error(st, msg);
        }
        if (n_c != e.job.C.size()) throw Error(SPFHE_EINVAL, "result array size mismatch");
        for (size_t i = 0; i < n_c; ++i) {
            spfhe_ct *h = new spfhe_ct;
            h->c = e.job.C[i];
            C_chunks[i] = h;
        }
        if (stats) {
            stats->matches = e.job.st_matches;
            stats->ks_relin = e.job.st_relin;
            stats->ks_align = e.job.st_align;
            stats->ks_final = e.job.st_final;
            stats->rescales = e.job.st_rescales;
            stats->launches = 0;
        }
        if (latency_ms) *latency_ms = e.t_done - e.t_submit;
        if (e.job.done_ev) cudaEventDestroy(e.job.done_ev);
        release_job(s.ctx, e.job, false);
        s.entries.erase(it);
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}

spfhe_status spfhe_server_inject_fault(spfhe_server *srv, uint64_t ticket)
{
    try {
        if (!srv) throw Error(SPFHE_EINVAL, "null argument");
        Server &s = *srv->s;
        std::lock_guard<std::mutex> lk(s.mu);
        if (ticket >= s.next_ticket) {   // a request not submitted yet
            s.poisoned.insert(ticket);
            return SPFHE_OK;
        }
        auto it = s.entries.find(ticket);
        if (it == s.entries.end()) throw Error(SPFHE_EINVAL, "unknown ticket");
        if (std::find(s.queue.begin(), s.queue.end(), ticket) == s.queue.end())
            throw Error(SPFHE_EINVAL, "request already admitted");
        it->second->job.inject_fault = true;
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}

spfhe_status spfhe_server_info(spfhe_server *srv, uint64_t *workspace_reserved, uint64_t *in_use,
                               uint64_t *retried)
{
    try {
        if (!srv) throw Error(SPFHE_EINVAL, "null argument");
        Server &s = *srv->s;
        std::lock_guard<std::mutex> lk(s.mu);
        if (workspace_reserved) *workspace_reserved = s.ws_reserved;
        if (in_use) *in_use = s.in_use;
        if (retried) *retried = s.retried;
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}

spfhe_status spfhe_server_destroy(spfhe_server *srv)
{
    if (!srv) return SPFHE_OK;
    Server *s = srv->s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->ctx.device);
    cudaStreamSynchronize(s->ctx.stream);
    for (auto &kv : s->entries) {
        if (kv.second->job.done_ev) cudaEventDestroy(kv.second->job.done_ev);
        release_job(s->ctx, kv.second->job, true);
    }
    delete s;
    delete srv;
    return SPFHE_OK;
}

}  // extern "C"
