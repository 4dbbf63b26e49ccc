// Device memory for a context: stream-ordered allocations from the device's
// memory pool (kept cached by a high release threshold, so steady-state calls
// do not reach the driver), a per-context workspace cache for the large
// per-batch buffers, and a pinned ring that uploads small per-launch tables
// (pointer arrays, Galois elements) without stalling the stream.
#include <algorithm>
#include <cstring>

#include "runtime.h"

namespace spfhe {

void ctx_sync(Ctx &ctx)
{
    if (!ctx.cap) SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
}

void *dev_alloc(Ctx &ctx, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 8;
    if (ctx.cap) {
        // outside the graph: the buffer lives as long as the graph
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            throw Error(SPFHE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
        ctx.cap->device.push_back(p);
        return p;
    }
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(SPFHE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return p;
}

void dev_free(Ctx &ctx, void *p)
{
    if (!p) return;
    if (ctx.cap) {
        // a buffer of the capture is freed with the graph; one from before
        // the capture may still be used by captured work: freed after it
        for (void *q : ctx.cap->device)
            if (q == p) return;
        ctx.cap->deferred.push_back(p);
        return;
    }
    cudaFreeAsync(p, ctx.stream);
}

void configure_pool(int device)
{
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

u64 *Runtime::workspace(int slot, size_t words)
{
    if (slot < 0 || slot >= kWorkspaceSlots) throw Error(SPFHE_EINVAL, "bad workspace slot");
    if (Capture *c = ctx.cap) {
        if (c->ws.empty()) {
            c->ws.assign(kWorkspaceSlots, nullptr);
            c->ws_words.assign(kWorkspaceSlots, 0);
        }
        if (c->ws_words[slot] < words) {
            c->ws[slot] = static_cast<u64 *>(dev_alloc(ctx, words * sizeof(u64)));
            c->ws_words[slot] = words;
        }
        return c->ws[slot];
    }
    Buf &b = ws[slot];
    if (b.words < words) {
        if (b.p) dev_free(ctx, b.p);
        b.p = static_cast<u64 *>(dev_alloc(ctx, words * sizeof(u64)));
        b.words = words;
    }
    return b.p;
}

void *Runtime::upload(const void *host, size_t bytes)
{
    const size_t padded = (bytes + 255) & ~(size_t)255;
    if (Capture *c = ctx.cap) {
        if (c->up_off + padded > c->up_cap) {
            const size_t blk = std::max(padded, (size_t)kRingBytes);
            char *h = nullptr;
            SPFHE_CHECK_CUDA(cudaMallocHost(&h, blk));
            c->host.push_back(h);
            c->up_host = h;
            c->up_dev = static_cast<char *>(dev_alloc(ctx, blk));
            c->up_off = 0;
            c->up_cap = blk;
        }
        std::memcpy(c->up_host + c->up_off, host, bytes);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(c->up_dev + c->up_off, c->up_host + c->up_off, bytes,
                                         cudaMemcpyHostToDevice, ctx.stream));
        void *d = c->up_dev + c->up_off;
        c->up_off += padded;
        return d;
    }
    if (padded > kRingBytes) throw Error(SPFHE_EINVAL, "metadata upload too large");
    if (!ring_host) {
        SPFHE_CHECK_CUDA(cudaMallocHost(&ring_host, kRingBytes));
        ring_dev = static_cast<char *>(dev_alloc(ctx, kRingBytes));
        ring_off = 0;
    }
    if (ring_off + padded > kRingBytes) {
        // every earlier copy out of the ring must have landed before reuse
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
        ring_off = 0;
    }
    std::memcpy(ring_host + ring_off, host, bytes);
    SPFHE_CHECK_CUDA(cudaMemcpyAsync(ring_dev + ring_off, ring_host + ring_off, bytes, cudaMemcpyHostToDevice,
                                     ctx.stream));
    void *d = ring_dev + ring_off;
    ring_off += padded;
    return d;
}

void Runtime::release()
{
    for (Buf &b : ws) {
        if (b.p) dev_free(ctx, b.p);
        b = Buf{};
    }
    if (ring_dev) dev_free(ctx, ring_dev);
    ring_dev = nullptr;
    if (ring_host) {
        cudaStreamSynchronize(ctx.stream);
        cudaFreeHost(ring_host);
    }
    ring_host = nullptr;
}

}  // namespace spfhe
