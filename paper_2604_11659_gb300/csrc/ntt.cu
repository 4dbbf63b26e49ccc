// Negacyclic NTT over Z_q[X]/(X^n + 1), 64-bit residues, sm_103a.
//
// Forward: merged-psi Cooley-Tukey, natural-order input, bit-reversed output
//   out[k] = a(psi^(2 brv(k) + 1)).  Stage s (0 <= s < log_n) pairs x and
//   x + t, t = n >> (s+1), inside group x >> (log_n - s), twiddle
//   psi^brv(2^s + group).
// Inverse: Gentleman-Sande with psi^-1 in the reverse stage order, times n^-1.
//
// Two passes per transform, each staged in shared memory:
//   pass A covers stages [0, PA): the 2^PA elements c + r * 2^(log_n-PA)
//     (r = 0..2^PA-1) of a column c only interact with each other; a CTA
//     takes 16 adjacent columns so every row read is a 128-byte segment;
//   pass B covers stages [PA, log_n): contiguous tiles of 2^(log_n-PA).
// Residues are kept fully reduced in [0, q) between stages.
#include "kernels.h"

namespace spfhe {

namespace {

constexpr int kThreads = 256;

struct NttArgs {
    u64 *base;
    long long stride;
    const int *ids;
    LimbMap map;
};

__device__ __forceinline__ u64 *limb_ptr(const NttArgs &a, int n, int &mi)
{
    const int slot = blockIdx.y;
    const long long item = a.ids ? a.ids[blockIdx.z] : blockIdx.z;
    mi = a.map.mi[slot];
    return a.base + item * a.stride + (long long)a.map.off[slot] * n;
}

__global__ void __launch_bounds__(kThreads) k_fwd_a(NttArgs a, const ModConst *__restrict__ mc,
                                                    const u64 *__restrict__ tw, const u64 *__restrict__ twp,
                                                    int log_n, int PA)
{
    extern __shared__ u64 sm[];
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const u64 q = mc[mi].q;
    const u64 *w = tw + (size_t)mi * n;
    const u64 *wp = twp + (size_t)mi * n;
    const int rows = 1 << PA;
    const int lg_ncols = log_n - PA;
    const int lgC = lg_ncols < 4 ? lg_ncols : 4;
    const int C = 1 << lgC;
    const int c0 = blockIdx.x * C;
    for (int idx = threadIdx.x; idx < rows * C; idx += blockDim.x) {
        const int r = idx >> lgC, cc = idx & (C - 1);
        sm[idx] = p[((size_t)r << lg_ncols) + c0 + cc];
    }
    __syncthreads();
    for (int s = 0; s < PA; ++s) {
        const int lgt = PA - s - 1;        // half distance in rows: t = 2^lgt
        const int t = 1 << lgt;
        for (int u = threadIdx.x; u < (rows >> 1) * C; u += blockDim.x) {
            const int cc = u & (C - 1), v = u >> lgC;
            const int g = v >> lgt;
            const int jr = (g << (lgt + 1)) + (v & (t - 1));
            const int ti = (1 << s) + g;
            const u64 W = __ldg(w + ti), Wp = __ldg(wp + ti);
            const u64 x = sm[(jr << lgC) + cc];
            const u64 y = mul_shoup(sm[((jr + t) << lgC) + cc], W, Wp, q);
            sm[(jr << lgC) + cc] = add_mod(x, y, q);
            sm[((jr + t) << lgC) + cc] = sub_mod(x, y, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < rows * C; idx += blockDim.x) {
        const int r = idx >> lgC, cc = idx & (C - 1);
        p[((size_t)r << lg_ncols) + c0 + cc] = sm[idx];
    }
}

__global__ void __launch_bounds__(kThreads) k_fwd_b(NttArgs a, const ModConst *__restrict__ mc,
                                                    const u64 *__restrict__ tw, const u64 *__restrict__ twp,
                                                    int log_n, int PA, int lg_tile_elems)
{
    extern __shared__ u64 sm[];
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const u64 q = mc[mi].q;
    const u64 *w = tw + (size_t)mi * n;
    const u64 *wp = twp + (size_t)mi * n;
    const int PB = log_n - PA;               // tile = 2^PB contiguous elements
    const int E = 1 << lg_tile_elems;        // elements per CTA (several tiles)
    const size_t e0 = (size_t)blockIdx.x * E;
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) sm[idx] = p[e0 + idx];
    __syncthreads();
    const int b0 = (int)(e0 >> PB);           // first tile index
    for (int s = PA; s < log_n; ++s) {
        const int lgt = log_n - s - 1;
        const int t = 1 << lgt;
        for (int u = threadIdx.x; u < (E >> 1); u += blockDim.x) {
            const int tile = u >> (PB - 1), v = u & ((1 << (PB - 1)) - 1);
            const int gl = v >> lgt;
            const int j = (tile << PB) + (gl << (lgt + 1)) + (v & (t - 1));
            const int g = ((b0 + tile) << (s - PA)) + gl;
            const int ti = (1 << s) + g;
            const u64 W = __ldg(w + ti), Wp = __ldg(wp + ti);
            const u64 x = sm[j];
            const u64 y = mul_shoup(sm[j + t], W, Wp, q);
            sm[j] = add_mod(x, y, q);
            sm[j + t] = sub_mod(x, y, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) p[e0 + idx] = sm[idx];
}

__global__ void __launch_bounds__(kThreads) k_inv_b(NttArgs a, const ModConst *__restrict__ mc,
                                                    const u64 *__restrict__ itw, const u64 *__restrict__ itwp,
                                                    int log_n, int PA, int lg_tile_elems)
{
    extern __shared__ u64 sm[];
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const u64 q = mc[mi].q;
    const u64 *w = itw + (size_t)mi * n;
    const u64 *wp = itwp + (size_t)mi * n;
    const int PB = log_n - PA;
    const int E = 1 << lg_tile_elems;
    const size_t e0 = (size_t)blockIdx.x * E;
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) sm[idx] = p[e0 + idx];
    __syncthreads();
    const int b0 = (int)(e0 >> PB);
    for (int s = log_n - 1; s >= PA; --s) {
        const int lgt = log_n - s - 1;
        const int t = 1 << lgt;
        for (int u = threadIdx.x; u < (E >> 1); u += blockDim.x) {
            const int tile = u >> (PB - 1), v = u & ((1 << (PB - 1)) - 1);
            const int gl = v >> lgt;
            const int j = (tile << PB) + (gl << (lgt + 1)) + (v & (t - 1));
            const int g = ((b0 + tile) << (s - PA)) + gl;
            const int ti = (1 << s) + g;
            const u64 W = __ldg(w + ti), Wp = __ldg(wp + ti);
            const u64 x = sm[j], y = sm[j + t];
            sm[j] = add_mod(x, y, q);
            sm[j + t] = mul_shoup(sub_mod(x, y, q), W, Wp, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) p[e0 + idx] = sm[idx];
}

__global__ void __launch_bounds__(kThreads) k_inv_a(NttArgs a, const ModConst *__restrict__ mc,
                                                    const u64 *__restrict__ itw, const u64 *__restrict__ itwp,
                                                    int log_n, int PA)
{
    extern __shared__ u64 sm[];
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const ModConst m = mc[mi];
    const u64 q = m.q;
    const u64 *w = itw + (size_t)mi * n;
    const u64 *wp = itwp + (size_t)mi * n;
    const int rows = 1 << PA;
    const int lg_ncols = log_n - PA;
    const int lgC = lg_ncols < 4 ? lg_ncols : 4;
    const int C = 1 << lgC;
    const int c0 = blockIdx.x * C;
    for (int idx = threadIdx.x; idx < rows * C; idx += blockDim.x) {
        const int r = idx >> lgC, cc = idx & (C - 1);
        sm[idx] = p[((size_t)r << lg_ncols) + c0 + cc];
    }
    __syncthreads();
    for (int s = PA - 1; s >= 0; --s) {
        const int lgt = PA - s - 1;
        const int t = 1 << lgt;
        for (int u = threadIdx.x; u < (rows >> 1) * C; u += blockDim.x) {
            const int cc = u & (C - 1), v = u >> lgC;
            const int g = v >> lgt;
            const int jr = (g << (lgt + 1)) + (v & (t - 1));
            const int ti = (1 << s) + g;
            const u64 W = __ldg(w + ti), Wp = __ldg(wp + ti);
            const u64 x = sm[(jr << lgC) + cc], y = sm[((jr + t) << lgC) + cc];
            sm[(jr << lgC) + cc] = add_mod(x, y, q);
            sm[((jr + t) << lgC) + cc] = mul_shoup(sub_mod(x, y, q), W, Wp, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < rows * C; idx += blockDim.x) {
        const int r = idx >> lgC, cc = idx & (C - 1);
        p[((size_t)r << lg_ncols) + c0 + cc] = mul_shoup(sm[idx], m.n_inv, m.n_inv_p, q);
    }
}

struct Geometry {
    int PA, lg_cols, lgC, lgE;
    size_t smem_a, smem_b;
    int grid_a, grid_b;
};

Geometry geometry(int log_n)
{
    Geometry g;
    g.PA = log_n / 2;
    g.lg_cols = log_n - g.PA;
    g.lgC = g.lg_cols < 4 ? g.lg_cols : 4;
    const int PB = log_n - g.PA;
    g.lgE = PB > 11 ? PB : 11;                 // at least one whole tile, 2048 elements if n allows
    if (g.lgE > log_n) g.lgE = log_n;
    g.smem_a = ((size_t)1 << (g.PA + g.lgC)) * sizeof(u64);
    g.smem_b = ((size_t)1 << g.lgE) * sizeof(u64);
    g.grid_a = 1 << (g.lg_cols - g.lgC);
    g.grid_b = 1 << (log_n - g.lgE);
    return g;
}

void launch_checks(const Batch &b, const LimbMap &map)
{
    if (map.nl <= 0 || b.items <= 0) return;
    if (map.nl > kMaxLimbSlots) throw Error(SPFHE_EINVAL, "too many limbs in one NTT launch");
    if (b.items > 65535) throw Error(SPFHE_EINVAL, "too many items in one NTT launch");
}

}  // namespace

LimbMap limb_range(int first_off, int count, int first_mi)
{
    LimbMap m;
    m.nl = count;
    for (int i = 0; i < count; ++i) {
        m.off[i] = first_off + i;
        m.mi[i] = first_mi + i;
    }
    return m;
}

void ntt_forward(Ctx &ctx, Batch b, const LimbMap &map)
{
    launch_checks(b, map);
    if (map.nl <= 0 || b.items <= 0) return;
    Geometry g = geometry(ctx.log_n);
    NttArgs a{b.base, b.stride, b.ids, map};
    dim3 ga(g.grid_a, map.nl, b.items), gb(g.grid_b, map.nl, b.items);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_fwd_a<<<ga, kThreads, g.smem_a, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.tw, ctx.dt.twp, ctx.log_n, g.PA);
        prof_end(ctx, t0_, ctx.in_keyswitch ? K_KS_NTT_FWD : K_NTT_FWD, 16.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * g.PA * map.nl * b.items, "ntt fwd A");
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_fwd_b<<<gb, kThreads, g.smem_b, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.tw, ctx.dt.twp, ctx.log_n, g.PA, g.lgE);
        prof_end(ctx, t0_, ctx.in_keyswitch ? K_KS_NTT_FWD : K_NTT_FWD, 16.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * (ctx.log_n - g.PA) * map.nl * b.items, "ntt fwd B");
    }
}

void ntt_inverse(Ctx &ctx, Batch b, const LimbMap &map)
{
    launch_checks(b, map);
    if (map.nl <= 0 || b.items <= 0) return;
    Geometry g = geometry(ctx.log_n);
    NttArgs a{b.base, b.stride, b.ids, map};
    dim3 ga(g.grid_a, map.nl, b.items), gb(g.grid_b, map.nl, b.items);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_inv_b<<<gb, kThreads, g.smem_b, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.itw, ctx.dt.itwp, ctx.log_n, g.PA, g.lgE);
        prof_end(ctx, t0_, ctx.in_keyswitch ? K_KS_NTT_INV : K_NTT_INV, 16.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * (ctx.log_n - g.PA) * map.nl * b.items, "ntt inv B");
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_inv_a<<<ga, kThreads, g.smem_a, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.itw, ctx.dt.itwp, ctx.log_n, g.PA);
        prof_end(ctx, t0_, ctx.in_keyswitch ? K_KS_NTT_INV : K_NTT_INV, 16.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * g.PA * map.nl * b.items, "ntt inv A");
    }
}

}  // namespace spfhe
