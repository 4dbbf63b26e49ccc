// Launch bookkeeping and the optional per-kernel-class profiler: when
// enabled, every launch is bracketed by two CUDA events on the context
// stream and credited with the algorithmic bytes and work its shapes imply.
#include "kernels.h"

namespace spfhe {

const char *kernel_class_name(int cls)
{
    static const char *names[K_NCLASS] = {"ntt_fwd", "ntt_inv", "modup_bconv", "ks_inner_product",
                                          "moddown_bconv", "moddown_final", "tensor", "rescale",
                                          "automorph", "mask_mul", "accumulate", "other", "ks_ntt_fwd",
                                          "ks_ntt_inv"};
    return (cls >= 0 && cls < K_NCLASS) ? names[cls] : "?";
}

// per-thread depth of live ProfSuppress guards
static thread_local int tl_prof_suppress = 0;

ProfSuppress::ProfSuppress() { ++tl_prof_suppress; }
ProfSuppress::~ProfSuppress() { --tl_prof_suppress; }

cudaEvent_t prof_begin(Ctx &ctx)
{
    Prof &p = ctx.prof;
    if (!p.on || tl_prof_suppress) return nullptr;
    if (p.used + 2 > p.pool.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            SPFHE_CHECK_CUDA(cudaEventCreate(&e));
            p.pool.push_back(e);
        }
    }
    cudaEvent_t a = p.pool[p.used++];
    SPFHE_CHECK_CUDA(cudaEventRecord(a, ctx.stream));
    return a;
}

void prof_end(Ctx &ctx, cudaEvent_t start, int cls, double bytes, double work, const char *what)
{
    ++ctx.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(SPFHE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    Prof &p = ctx.prof;
    p.launches[cls] += 1;
    p.bytes[cls] += bytes;
    p.work[cls] += work;
    if (!p.on || !start) return;
    cudaEvent_t b = p.pool[p.used++];
    SPFHE_CHECK_CUDA(cudaEventRecord(b, ctx.stream));
    p.recs.push_back(ProfRec{cls, start, b});
}

void prof_limbs(Ctx &ctx, int cls, int kind, double limbs)
{
    if (cls >= 0 && cls < K_NCLASS && kind >= 0 && kind < 3) ctx.prof.limbs[cls][kind] += limbs;
}

void prof_reset(Ctx &ctx, bool on)
{
    Prof &p = ctx.prof;
    p.on = on;
    p.used = 0;
    p.recs.clear();
    p.ks_calls = 0;
    p.ks_bytes = 0;
    for (int c = 0; c < K_NCLASS; ++c) {
        p.launches[c] = 0;
        p.bytes[c] = p.work[c] = p.ms[c] = 0;
        p.limbs[c][0] = p.limbs[c][1] = p.limbs[c][2] = 0;
        p.timed[c] = 0;
    }
}

void prof_collect(Ctx &ctx)
{
    Prof &p = ctx.prof;
    SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
    for (const ProfRec &r : p.recs) {
        float ms = 0;
        SPFHE_CHECK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        p.ms[r.cls] += ms;
        ++p.timed[r.cls];
    }
    p.recs.clear();
    p.used = 0;
}

void prof_destroy(Ctx &ctx)
{
    for (cudaEvent_t e : ctx.prof.pool) cudaEventDestroy(e);
    ctx.prof.pool.clear();
}

}  // namespace spfhe
