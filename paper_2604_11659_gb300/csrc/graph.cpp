// Encrypted products captured once into a CUDA graph and launched as one
// unit (the batch-launch pattern: the plan, every wave and every batch of the
// product become the nodes of one graph; a launch replays all of them).
//
// While the graph is captured, the library's calls run on a private stream
// in relaxed capture mode and see ctx.cap: device buffers come from
// cudaMalloc and live as long as the graph (workspaces included: the graph
// has its own), metadata uploads go to an append-only pinned/device pair that
// the captured copies read at every launch, and the products skip their final
// host wait.  Result ciphertexts are allocated inside and zeroed by the graph
// at every launch; the operands and keys are read at every launch, so they
// must outlive the graph (their contents may change between launches).
#include "engine.h"
#include "handles.h"

using namespace spfhe;

struct spfhe_graph {
    spfhe_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Capture cap;
    std::vector<Ct *> results;          // every request's chunks, request after request
    std::vector<spfhe_stats> stats;     // one entry per request
    uint64_t launches = 0;              // kernels one launch replays
};

namespace {

void release_capture(Ctx &c, Capture &cap)
{
    cudaStreamSynchronize(c.stream);
    for (void *p : cap.device) cudaFree(p);
    for (void *p : cap.host) cudaFreeHost(p);
    for (void *p : cap.deferred) cudaFreeAsync(p, c.stream);
    cap = Capture{};
}

}  // namespace

extern "C" {

spfhe_status spfhe_matmul_graph_create_batch(spfhe_ctx *ctx, size_t n_req, const spfhe_matmul_req *reqs,
                                             int variant, spfhe_graph **out)
{
    spfhe_graph *g = nullptr;
    try {
        if (!ctx || !reqs || !out || n_req == 0) throw Error(SPFHE_EINVAL, "null argument or no request");
        if (variant != 0 && variant != 1) throw Error(SPFHE_EINVAL, "variant must be 0 (Alg. 2) or 1 (grouped)");
        Ctx &c = ctx->c;
        if (c.cap) throw Error(SPFHE_EINVAL, "a graph is already being captured on this context");
        SPFHE_CHECK_CUDA(cudaSetDevice(c.device));
        std::vector<size_t> n_c(n_req), off(n_req + 1, 0);
        for (size_t r = 0; r < n_req; ++r) {
            if (!reqs[r].keys) throw Error(SPFHE_EINVAL, "null request field");
            n_c[r] = result_chunks(c, reqs[r]);
            off[r + 1] = off[r] + n_c[r];
        }
        // host-synchronous set-up the products may need, before the capture
        ensure_cos_table(c);
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        g = new spfhe_graph;
        g->ctx = ctx;
        g->results.assign(off[n_req], nullptr);
        g->stats.assign(n_req, spfhe_stats{});
        const bool prof_on = c.prof.on;
        c.prof.on = false;
        // captured on a private stream (the context's may be the legacy
        // default stream, which cannot be captured); launched on the context's
        cudaStream_t own = c.stream, cs = nullptr;
        SPFHE_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        c.stream = cs;
        c.cap = &g->cap;
        auto restore = [&] {
            c.cap = nullptr;
            c.stream = own;
            c.prof.on = prof_on;
            cudaStreamDestroy(cs);
        };
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            restore();
            throw Error(SPFHE_ECUDA, "stream capture could not start");
        }
        const uint64_t launches0 = c.launches;
        try {
            if (variant == 0 && n_req > 1) {
                // one task engine over every request: their waves share launches
                sparse_matmul_batch(c, n_req, reqs, g->results.data(), off[n_req], g->stats.data());
            } else {
                for (size_t r = 0; r < n_req; ++r) {
                    const spfhe_matmul_req &q = reqs[r];
                    if (!q.A_csr || !q.B_csc || !q.A_chunks || !q.B_chunks) throw Error(SPFHE_EINVAL, "null request field");
                    std::vector<Ct *> a(q.n_a), b(q.n_b);
                    for (size_t i = 0; i < q.n_a; ++i) a[i] = q.A_chunks[i] ? q.A_chunks[i]->c : nullptr;
                    for (size_t i = 0; i < q.n_b; ++i) b[i] = q.B_chunks[i] ? q.B_chunks[i]->c : nullptr;
                    const Pt *mask0 = q.mask0 ? q.mask0->p : nullptr;
                    Ct **res = g->results.data() + off[r];
                    if (variant == 0)
                        spmspm_ct_ct(c, *q.keys->k, *q.A_csr, a.data(), a.size(), *q.B_csc, b.data(), b.size(),
                                     mask0, res, n_c[r], &g->stats[r]);
                    else
                        spmspm_ct_ct_grouped(c, *q.keys->k, *q.A_csr, a.data(), a.size(), *q.B_csc, b.data(),
                                             b.size(), mask0, true, res, n_c[r], &g->stats[r]);
                }
            }
        } catch (...) {
            cudaGraph_t dropped = nullptr;
            cudaStreamEndCapture(cs, &dropped);
            if (dropped) cudaGraphDestroy(dropped);
            cudaGetLastError();
            restore();
            throw;
        }
        g->launches = c.launches - launches0;
        c.launches = launches0;   // counted again at every launch of the graph
        const cudaError_t ee = cudaStreamEndCapture(cs, &g->graph);
        restore();
        if (ee != cudaSuccess) throw Error(SPFHE_ECUDA, std::string("stream capture: ") + cudaGetErrorString(ee));
        SPFHE_CHECK_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
        *out = g;
        return SPFHE_OK;
    } catch (const Error &e) {
        if (g) {
            if (g->exec) cudaGraphExecDestroy(g->exec);
            if (g->graph) cudaGraphDestroy(g->graph);
            release_capture(ctx->c, g->cap);
            for (Ct *r : g->results) delete r;
            delete g;
        }
        set_last_error(e.what());
        return e.code;
    }
}

spfhe_status spfhe_matmul_graph_create(spfhe_ctx *ctx, const spfhe_matmul_req *req, int variant, spfhe_graph **out)
{
    if (!req) {
        set_last_error("null argument");
        return SPFHE_EINVAL;
    }
    return spfhe_matmul_graph_create_batch(ctx, 1, req, variant, out);
}

spfhe_status spfhe_matmul_graph_launch(spfhe_graph *g)
{
    if (!g) {
        set_last_error("null graph");
        return SPFHE_EINVAL;
    }
    Ctx &c = g->ctx->c;
    cudaSetDevice(c.device);
    const cudaError_t e = cudaGraphLaunch(g->exec, c.stream);
    if (e != cudaSuccess) {
        set_last_error(std::string("graph launch: ") + cudaGetErrorString(e));
        return SPFHE_ECUDA;
    }
    c.launches += g->launches;
    return SPFHE_OK;
}

spfhe_status spfhe_matmul_graph_results(spfhe_graph *g, spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats)
{
    if (!g || !C_chunks || n_c != g->results.size()) {
        set_last_error(!g || !C_chunks ? "null argument" : "result chunk count differs from the graph's total");
        return SPFHE_EINVAL;
    }
    for (size_t i = 0; i < n_c; ++i) {
        spfhe_ct *h = new spfhe_ct;
        h->c = g->results[i];
        h->borrowed = true;
        C_chunks[i] = h;
    }
    if (stats)
        for (size_t r = 0; r < g->stats.size(); ++r) stats[r] = g->stats[r];
    return SPFHE_OK;
}

void spfhe_matmul_graph_free(spfhe_graph *g)
{
    if (!g) return;
    Ctx &c = g->ctx->c;
    cudaSetDevice(c.device);
    cudaStreamSynchronize(c.stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    release_capture(c, g->cap);
    for (Ct *r : g->results) delete r;
    delete g;
}

}  // extern "C"
