// Rescale that allocates nothing.
//
// Some callers cannot allocate device memory while they run: code that sits
// inside an application's own fixed memory budget (a serving process that
// hands this library pre-sized buffers and forbids the driver allocator
// afterwards), or a host whose allocator must not be re-entered.  For them
// spfhe_rescale_noalloc takes caller-owned device input and output buffers and
// keeps its scratch (one polynomial's top limb in coefficient form and one
// limb of the rounded correction) in a file-scope device array instead of the
// context's stream-ordered pool.
//
// The array is reserved in every process that loads the library, on every
// GPU it touches, until exit: 2 * 2^17 words = 2 MiB, enough for the largest
// ring (n = 2^17) the library builds.  All calls on a GPU share it and it
// keeps the last call's contents; nothing in it needs to start at zero (every
// word a call reads was written earlier in the same call).  Two calls whose
// work overlaps on the GPU (different streams or contexts of the same device)
// race on it; calls on one stream are ordered and safe.
#include <mutex>

#include "handles.h"
#include "kernels.h"

namespace spfhe {
namespace {

constexpr size_t kNoAllocWords = (size_t)2 << 17;
constexpr int kMaxDevices = 64;

__device__ __align__(256) u64 g_noalloc_scratch[kNoAllocWords];

std::mutex g_mu;
u64 *g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (the current device).  The
// host-side symbol is only a stand-in: its device address is looked up once
// per device and cached.
u64 *scratch_on_device(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) throw Error(SPFHE_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            throw Error(SPFHE_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_dev_ptr[dev] = static_cast<u64 *>(p);
    }
    return g_dev_ptr[dev];
}

__global__ void k_na_copy(int n, const u64 *src, u64 *dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = src[k];
}

// dst = [r]_{q_i} with r the centred top-limb residue (coefficient rep.)
__global__ void k_na_spread(int n, const u64 *top, u64 qt, u64 qt_mod_qi, ModConst m, u64 *dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const u64 c = top[k];
    u64 r = mul_shoup(redc(U128{c, 0}, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
    if (c > (qt >> 1)) r = sub_mod(r, qt_mod_qi, m.q);
    dst[k] = r;
}

// out = (c - r) q_t^{-1} mod q_i (evaluation rep.)
__global__ void k_na_final(int n, const u64 *c, const u64 *r, u64 inv, u64 invp, u64 q, u64 *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = mul_shoup(sub_mod(c[k], r[k], q), inv, invp, q);
}

}  // namespace
}  // namespace spfhe

using namespace spfhe;

extern "C" spfhe_status spfhe_rescale_noalloc(spfhe_ctx *ctx, const uint64_t *in, uint32_t level, uint64_t *out)
{
    try {
        if (!ctx || !in || !out) throw Error(SPFHE_EINVAL, "null argument");
        Ctx &c = ctx->c;
        SPFHE_CHECK_CUDA(cudaSetDevice(c.device));
        const int ell = (int)level;
        if (ell < 2 || ell > c.L) throw Error(SPFHE_ELEVEL, "rescale needs 2 <= level <= L");
        const size_t n = c.n;
        if (2 * n > kNoAllocWords)
            throw Error(SPFHE_EINVAL, "ring degree " + std::to_string(n) + " needs " + std::to_string(2 * n) +
                                          " scratch words; the fixed scratch holds " + std::to_string(kNoAllocWords));
        u64 *top = scratch_on_device(c.device);
        u64 *spread = top + n;
        // the profiler would create CUDA events: none are recorded for this
        // call's launches (a per-thread guard; the context's own profiler
        // switch, which another thread may be reading, is not touched)
        ProfSuppress quiet;
        const int threads = 256, blocks = (int)((n + threads - 1) / threads);
        const u64 qt = c.mods[ell - 1];
        for (int b = 0; b < 2; ++b) {
            const u64 *cin = reinterpret_cast<const u64 *>(in) + (size_t)b * ell * n;
            u64 *cout = reinterpret_cast<u64 *>(out) + (size_t)b * (ell - 1) * n;
            k_na_copy<<<blocks, threads, 0, c.stream>>>((int)n, cin + (size_t)(ell - 1) * n, top);
            prof_end(c, nullptr, K_RESCALE, 16.0 * n, 0.0, "rescale (no alloc) copy");
            LimbMap tm;
            tm.nl = 1;
            tm.off[0] = 0;
            tm.mi[0] = ell - 1;
            ntt_inverse(c, Batch{top, 0, 1, nullptr}, tm);
            for (int i = 0; i < ell - 1; ++i) {
                const ModConst &m = c.mc[i];
                const u64 qi = c.mods[i];
                const u64 qt_mod = qt % qi;
                const u64 inv = invmod_host(qt_mod, qi);
                k_na_spread<<<blocks, threads, 0, c.stream>>>((int)n, top, qt, qt_mod, m, spread);
                prof_end(c, nullptr, K_RESCALE, 16.0 * n, 1.0 * n, "rescale (no alloc) spread");
                LimbMap sm;
                sm.nl = 1;
                sm.off[0] = 0;
                sm.mi[0] = i;
                ntt_forward(c, Batch{spread, 0, 1, nullptr}, sm);
                k_na_final<<<blocks, threads, 0, c.stream>>>((int)n, cin + (size_t)i * n, spread, inv,
                                                             shoup_pre(inv, qi), qi, cout + (size_t)i * n);
                prof_end(c, nullptr, K_RESCALE, 24.0 * n, 1.0 * n, "rescale (no alloc) final");
            }
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
