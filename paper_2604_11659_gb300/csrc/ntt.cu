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
//
// Algorithmic bytes credited to the profiler: a transform reads its limb once
// and writes it once (8 B per residue each way), split as the read in the
// first pass and the write in the second; the round trip between the passes
// is implementation traffic and is not credited.  A fused epilogue adds the
// limbs it reads and writes.
#include <atomic>

#include "kernels.h"

namespace spfhe {

namespace {

constexpr int kThreads = 256;

struct NttArgs {
    u64 *base;
    long long stride;
    const int *ids;
    LimbMap map;
    // inverse transforms: 1 = leave out the final factor n^{-1} (the output is
    // n x, not reduced below q; for consumers that fold n^{-1} into their own
    // constants, the base conversions of key switching)
    int unscaled = 0;
    // inverse radix-16 transforms without item list: when set, the first
    // pass reads item z's limbs from src[z] (same limb offsets) instead of
    // the batch, which receives the result (an out-of-place transform)
    const u64 *const *src = nullptr;
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
        p[((size_t)r << lg_ncols) + c0 + cc] = a.unscaled ? sm[idx] : mul_shoup(sm[idx], m.n_inv, m.n_inv_p, q);
    }
}

// ---------------------------------------------------------------------------
// Register-resident radix-16 transforms for n >= 2^12.
//
// A pass of P stages (6 <= P <= 9) runs on tiles of 2^P elements (pass A: one
// column of 2^P rows, stride n >> P; pass B: 2^P contiguous elements).  A CTA
// of 256 threads owns 4096 elements (4096 >> P tiles); every thread holds 16
// elements of one tile in registers.  Round r covers the pass-local stages
// [4r, 4r + Q), Q = min(4, P - 4r): the 16 registers hold 2^(4-Q) groups of
// 2^Q elements whose tile indices differ only in the Q bits that these stages
// pair, so each round is 4 (or Q) butterfly stages without any exchange;
// rounds are separated by one shared-memory transpose.
//   round r < last (Q = 4, a0 = P - 4r - 4 > 0):
//       j = (t & (2^a0 - 1)) | (i << a0) | ((t >> a0) << (a0 + 4))
//   last round (bit 0 is paired):  j = 16 t + i
// (t = thread index within its tile, i = register index).
// ---------------------------------------------------------------------------
constexpr int kElems = 4096;

template <int P, int RND> __device__ __forceinline__ int r16_index(int t, int i)
{
    constexpr int s0 = 4 * RND;
    constexpr int Q = (P - s0) < 4 ? (P - s0) : 4;
    constexpr int a0 = P - s0 - Q;
    if constexpr (a0 == 0) {
        return (t << 4) | i;
    } else {
        return (t & ((1 << a0) - 1)) | (i << a0) | ((t >> a0) << (a0 + 4));
    }
}

template <int P, int RND> constexpr int r16_q() { return (P - 4 * RND) < 4 ? (P - 4 * RND) : 4; }

// twiddle index of the butterfly whose lower element is tile index j at
// pass-local stage ls: group G = j >> (P - ls); pass A (stage0 = 0):
// 2^ls + G; pass B (stage0 = PA, tile b): 2^(PA + ls) + (b << ls) + G.
template <int P> __device__ __forceinline__ int r16_tw(int j, int ls, int stage0, int btile)
{
    return (1 << (stage0 + ls)) + (btile << ls) + (j >> (P - ls));
}

// Stage l of a round pairs register bit Q-1-l; the twiddle of a butterfly
// depends on the register index only through i >> (Q - l), so each stage
// loads its 16 >> (Q - l) distinct (twiddle, companion) pairs once, from
// global memory or (SM, pass B) from the CTA's shared-memory copy.
//
// Shared-memory twiddles of pass B: the CTA's T = 4096 >> P tiles need, at
// pass-local stage ls, the contiguous entries 2^(PA+ls) + b0 2^ls + [0, T 2^ls)
// (b0 = the CTA's first tile); they are kept at offset T (2^ls - 1).
template <int P> __host__ __device__ constexpr int r16_tw_smem_entries() { return (kElems >> P) * ((1 << P) - 1); }

template <int P, int RND, int Q, int l, bool SM>
__device__ __forceinline__ void r16_load_tw(ulonglong2 (&wt)[16], int t, const ulonglong2 *__restrict__ w2,
                                            int stage0, int btile, const ulonglong2 *smt, int ltile)
{
    constexpr int G = 16 >> (Q - l);
    constexpr int ls = 4 * RND + l;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = r16_index<P, RND>(t, g << (Q - l));
        if constexpr (SM) wt[g] = smt[(kElems >> P) * ((1 << ls) - 1) + (ltile << ls) + (j >> (P - ls))];
        else wt[g] = __ldg(w2 + r16_tw<P>(j, ls, stage0, btile));
    }
}

// Products w*y are taken in [0, 3q) for any y < 2^64 (mul_shoup3).
// LAZY (q < 2^58): no reduction of x at all; every stage raises the bound on
// all values by 3q, so after the log_n <= 17 stages of both passes they lie
// in [0, 52q) (< 2^64) and pass B reduces them once at the end.  Otherwise
// values stay in [0, 6q): x is first brought to [0, 3q).
template <int P, int RND, int l, bool LAZY, bool SM, int AR = 0>
__device__ __forceinline__ void r16_fwd_stage(u64 (&v)[16], int t, const ulonglong2 *__restrict__ w2, u64 q,
                                              int stage0, int btile, const ulonglong2 *smt, int ltile)
{
    constexpr int Q = r16_q<P, RND>();
    constexpr int half = 1 << (Q - 1 - l);
    const u64 qb = shoup_bound<AR>() * q, nq = 0 - q;
    ulonglong2 wt[16];
    r16_load_tw<P, RND, Q, l, SM>(wt, t, w2, stage0, btile, smt, ltile);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (i & half) continue;
        const ulonglong2 w = wt[i >> (Q - l)];
        const u64 x = LAZY ? v[i] : csub(v[i], qb);
        const u64 y = mul_shoup_ar<AR>(v[i + half], w.x, w.y, nq);
        v[i] = x + y;
        v[i + half] = x - y + qb;
    }
}

// PRE: the stage's twiddles were loaded ahead into `pre`
template <int P, int RND, int l, bool SM, bool PRE = false, int AR = 0>
__device__ __forceinline__ void r16_inv_stage(u64 (&v)[16], int t, const ulonglong2 *__restrict__ w2, u64 q,
                                              int stage0, int btile, const ulonglong2 *smt, int ltile,
                                              const ulonglong2 (*pre)[16] = nullptr)
{
    constexpr int Q = r16_q<P, RND>();
    constexpr int half = 1 << (Q - 1 - l);
    const u64 qb = shoup_bound<AR>() * q, nq = 0 - q;
    ulonglong2 wt[16];
    if constexpr (PRE) {
#pragma unroll
        for (int g = 0; g < (16 >> (Q - l)); ++g) wt[g] = (*pre)[g];
    } else {
        r16_load_tw<P, RND, Q, l, SM>(wt, t, w2, stage0, btile, smt, ltile);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (i & half) continue;
        const ulonglong2 w = wt[i >> (Q - l)];
        const u64 x = v[i], y = v[i + half];
        v[i] = csub(x + y, qb);
        v[i + half] = mul_shoup_ar<AR>(x - y + qb, w.x, w.y, nq);
    }
}

// Lazy butterflies (Harvey's scheme with the [0, 3q) products of
// mul_shoup3): forward values stay below 6q (52q on the reduction-free path),
// inverse values in [0, 3q); only the last pass reduces to [0, q).
template <int P, int RND, bool LAZY, bool SM = false, int AR = 0>
__device__ __forceinline__ void r16_fwd_round(u64 (&v)[16], int t, const ulonglong2 *__restrict__ w2, u64 q,
                                              int stage0, int btile, const ulonglong2 *smt = nullptr,
                                              int ltile = 0)
{
    constexpr int Q = r16_q<P, RND>();
    r16_fwd_stage<P, RND, 0, LAZY, SM, AR>(v, t, w2, q, stage0, btile, smt, ltile);
    if constexpr (Q > 1) r16_fwd_stage<P, RND, 1, LAZY, SM, AR>(v, t, w2, q, stage0, btile, smt, ltile);
    if constexpr (Q > 2) r16_fwd_stage<P, RND, 2, LAZY, SM, AR>(v, t, w2, q, stage0, btile, smt, ltile);
    if constexpr (Q > 3) r16_fwd_stage<P, RND, 3, LAZY, SM, AR>(v, t, w2, q, stage0, btile, smt, ltile);
}

// moduli below this take the reduction-free forward butterflies: values grow
// by shoup_bound<AR>() q per stage from [0, q), so after the 17 stages of the
// largest transform they stay below 52q (AR 0, 1) or 69q (AR 2) < 2^64
template <int AR> constexpr u64 lazy_fwd_bound() { return AR == 2 ? 1ull << 57 : 1ull << 58; }

// PRE: the twiddles of the round's first stage (l = Q - 1) are in `pre`
template <int P, int RND, bool SM = false, bool PRE = false, int AR = 0>
__device__ __forceinline__ void r16_inv_round(u64 (&v)[16], int t, const ulonglong2 *__restrict__ w2, u64 q,
                                              int stage0, int btile, const ulonglong2 *smt = nullptr,
                                              int ltile = 0, const ulonglong2 (*pre)[16] = nullptr)
{
    constexpr int Q = r16_q<P, RND>();
    if constexpr (Q > 3) r16_inv_stage<P, RND, 3, SM, PRE, AR>(v, t, w2, q, stage0, btile, smt, ltile, pre);
    if constexpr (Q > 2) r16_inv_stage<P, RND, 2, SM, PRE && Q == 3, AR>(v, t, w2, q, stage0, btile, smt, ltile, pre);
    if constexpr (Q > 1) r16_inv_stage<P, RND, 1, SM, PRE && Q == 2, AR>(v, t, w2, q, stage0, btile, smt, ltile, pre);
    r16_inv_stage<P, RND, 0, SM, PRE && Q == 1, AR>(v, t, w2, q, stage0, btile, smt, ltile, pre);
}

// shared-memory slot of tile element j (pass B layout; pad one word per 16)
template <int P> __device__ __forceinline__ int r16_slot_b(int tile, int j)
{
    return tile * ((1 << P) + (1 << (P - 4))) + j + (j >> 4);
}
// pass A layout: [row][column], 8 words of padding per 16 rows
template <int P> __device__ __forceinline__ int r16_slot_a(int col, int row)
{
    return row * (kElems >> P) + col + ((row >> 4) << 3);
}
template <int P> constexpr int r16_smem_words_a() { return kElems + (((1 << P) >> 4) << 3); }
template <int P> constexpr int r16_smem_words_b() { return kElems + (kElems >> 4); }

// Kernel variants (picked per context, see spfhe_ctx_set_ntt_variant):
//   0: twiddles loaded per stage from global memory, 3 CTAs per SM;
//   1: the same with the register budget of 2 CTAs per SM;
//   2: as 1, and pass B copies its CTA's twiddles into shared memory with
//      asynchronous copies issued before its data loads;
//   3: as 0 with the register budget of 4 CTAs per SM;
//   4: as 3 with the Shoup products split into single-word halves
//      (mul_shoup3s; the same bits);
//   5: as 4 with the quotient's low middle halves dropped (mul_shoup4s,
//      products in [0, 4q); the transforms' outputs are the same residues);
//   6: as 5 with pass B synchronising warps instead of the CTA (r16_sync).
template <int V> constexpr int r16_min_blocks() { return V == 0 ? 3 : (V >= 3 ? 4 : 2); }
template <int V> constexpr int r16_arith() { return V >= 5 ? 2 : (V == 4 ? 1 : 0); }
template <int V> constexpr bool r16_warp_local() { return V == 6; }
// variants that carry the merged relinearise-rescale transform (kFuseRelinRescale)
template <int V> constexpr bool r16_relin_rescale() { return V == 5 || V == 6; }

// Pass B, V = 2: start the asynchronous copy of the CTA's twiddles.
template <int P>
__device__ __forceinline__ void r16_prefetch_tw(ulonglong2 *smt, const ulonglong2 *__restrict__ w2, int PA, int b0)
{
    constexpr int T = kElems >> P;
#pragma unroll 1
    for (int ls = 0; ls < P; ++ls) {
        const ulonglong2 *src = w2 + ((size_t)1 << (PA + ls)) + ((size_t)b0 << ls);
        ulonglong2 *dst = smt + T * ((1 << ls) - 1);
        for (int x = threadIdx.x; x < (T << ls); x += 256) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + x);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + x) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void r16_prefetch_wait()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
}

// Pass B exchanges data only inside a tile, and a tile (2^P elements, 16
// per thread) never spans two warps: with WL ("warp-local") the transposes
// synchronise the warp instead of the CTA, and every warp stages and stores
// its own 512 contiguous elements, so pass B has no CTA-wide barrier.
template <bool WL> __device__ __forceinline__ void r16_sync()
{
    if constexpr (WL) __syncwarp();
    else __syncthreads();
}
// loop over the CTA's elements (all of them, or the calling warp's 512)
template <bool WL> __device__ __forceinline__ int r16_first()
{
    return WL ? (int)(threadIdx.x & ~31u) * 16 + (int)(threadIdx.x & 31u) : (int)threadIdx.x;
}
template <bool WL> __device__ __forceinline__ int r16_end() { return WL ? (int)(threadIdx.x & ~31u) * 16 + 512 : kElems; }
template <bool WL> constexpr int r16_step() { return WL ? 32 : 256; }

template <int P, bool LAZY, int MODE, int AR = 0>
__device__ __forceinline__ void fwd16_a_body(u64 *sm, u64 *p, u64 q, const ulonglong2 *__restrict__ w2, int log_n,
                                             const FuseArgs &f, const ModConst *__restrict__ mc)
{
    constexpr int TPC = kElems >> P;   // columns per CTA
    constexpr int R = (P + 3) / 4;
    const int lg_ncols = log_n - P;
    const int col = threadIdx.x % TPC, t = threadIdx.x / TPC;
    const int gcol = blockIdx.x * TPC + col;
    u64 v[16];
    if constexpr (MODE == kFuseRescale || MODE == kFuseRelinRescale) {
        // the limb [r]_{q_i} of the centred top limb r, read from the top limb itself
        const int slot = blockIdx.y, it = blockIdx.z;
        const int b = slot / (f.ell - 1), i = slot % (f.ell - 1);
        const u64 *top = f.top + ((size_t)it * f.polys + b) * ((size_t)1 << log_n);
        const ModConst m = mc[i];
        const u64 qt_half = mc[f.ell - 1].q >> 1, qt_mod = __ldg(f.qt_mod + i);
#pragma unroll
        for (int x = 0; x < 16; ++x) {
            const u64 c = top[((size_t)r16_index<P, 0>(t, x) << lg_ncols) + gcol];
            u64 r = mul_shoup(redc(U128{c, 0}, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
            if (c > qt_half) r = sub_mod(r, qt_mod, m.q);
            v[x] = r;
        }
        if constexpr (MODE == kFuseRelinRescale) {
            // plus P^{-1} times ModDown's conversion of limb i (coefficient rep.)
            const u64 *cv = f.conv + it * f.conv_stride + ((size_t)b * f.ell + i) * ((size_t)1 << log_n);
            const u64 pinv = __ldg(f.pinv + i), pinvp = __ldg(f.pinvp + i);
#pragma unroll
            for (int x = 0; x < 16; ++x)
                v[x] = add_mod(v[x], mul_shoup(cv[((size_t)r16_index<P, 0>(t, x) << lg_ncols) + gcol], pinv, pinvp, m.q),
                               m.q);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = p[((size_t)r16_index<P, 0>(t, i) << lg_ncols) + gcol];
    }
    r16_fwd_round<P, 0, LAZY, false, AR>(v, t, w2, q, 0, 0);
    if constexpr (R > 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_a<P>(col, r16_index<P, 0>(t, i))] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_a<P>(col, r16_index<P, 1>(t, i))];
        r16_fwd_round<P, 1, LAZY, false, AR>(v, t, w2, q, 0, 0);
    }
    if constexpr (R > 2) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_a<P>(col, r16_index<P, 1>(t, i))] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_a<P>(col, r16_index<P, 2>(t, i))];
        r16_fwd_round<P, 2, LAZY, false, AR>(v, t, w2, q, 0, 0);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) p[((size_t)r16_index<P, R - 1>(t, i) << lg_ncols) + gcol] = v[i];
}

template <int P, int V, int MODE = kFuseNone>
__global__ void __launch_bounds__(256, r16_min_blocks<V>()) k_fwd16_a(NttArgs a, const ModConst *__restrict__ mc,
                                                                      const ulonglong2 *__restrict__ tw2, int log_n,
                                                                      FuseArgs f)
{
    __shared__ u64 sm[r16_smem_words_a<P>()];
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const u64 q = mc[mi].q;
    const ulonglong2 *w2 = tw2 + (size_t)mi * n;
    constexpr int AR = r16_arith<V>();
    if (q < lazy_fwd_bound<AR>()) fwd16_a_body<P, true, MODE, AR>(sm, p, q, w2, log_n, f, mc);
    else fwd16_a_body<P, false, MODE, AR>(sm, p, q, w2, log_n, f, mc);
}

template <int P, bool LAZY, bool SM, int MODE = kFuseNone, int AR = 0, bool WL = false>
__device__ __forceinline__ void fwd16_b_body(u64 *sm, u64 *p, const ModConst &m, const ulonglong2 *__restrict__ w2,
                                             int PA, const ulonglong2 *smt, const FuseArgs &f = FuseArgs{},
                                             int log_n = 0)
{
    constexpr int TPT = 1 << (P - 4);  // threads per tile
    constexpr int R = (P + 3) / 4;
    const u64 q = m.q;
    const int tile = threadIdx.x / TPT, t = threadIdx.x % TPT;
    const size_t e0 = (size_t)blockIdx.x * kElems;
    const int btile = (int)(e0 >> P) + tile;
    u64 *tp = p + e0 + ((size_t)tile << P);
    u64 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = tp[r16_index<P, 0>(t, i)];
    if constexpr (SM) r16_prefetch_wait();
    r16_fwd_round<P, 0, LAZY, SM, AR>(v, t, w2, q, PA, btile, smt, tile);
    if constexpr (R > 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_b<P>(tile, r16_index<P, 0>(t, i))] = v[i];
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_b<P>(tile, r16_index<P, 1>(t, i))];
        r16_fwd_round<P, 1, LAZY, SM, AR>(v, t, w2, q, PA, btile, smt, tile);
    }
    if constexpr (R > 2) {
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_b<P>(tile, r16_index<P, 1>(t, i))] = v[i];
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_b<P>(tile, r16_index<P, 2>(t, i))];
        r16_fwd_round<P, 2, LAZY, SM, AR>(v, t, w2, q, PA, btile, smt, tile);
    }
    // the last round holds 16 contiguous elements per thread: stage through
    // shared memory so the global stores are coalesced
    r16_sync<WL>();
#pragma unroll
    for (int i = 0; i < 16; ++i) sm[r16_slot_b<P>(tile, r16_index<P, R - 1>(t, i))] = v[i];
    r16_sync<WL>();
    if constexpr (MODE == kFuseNone) {
        for (int x = r16_first<WL>(); x < r16_end<WL>(); x += r16_step<WL>()) {
            const u64 y = sm[r16_slot_b<P>(x >> P, x & ((1 << P) - 1))];
            p[e0 + x] = reduce_any(y, q, m.one_p);
        }
    } else if constexpr (MODE == kFuseModDown) {
        // out_b[i] = base_b[sigma(k)] + (acc_b[i] - conv_b[i]) P^{-1} (conv = this transform)
        const int slot = blockIdx.y, it = blockIdx.z;
        const int b = slot / f.ell, i = slot % f.ell;
        const int next = f.ell + f.K;
        const u64 pinv = __ldg(f.pinv + i), pinvp = __ldg(f.pinvp + i);
        const u64 *__restrict__ acc = f.acc + it * f.acc_stride + ((size_t)b * next + i) * ((size_t)1 << log_n);
        const bool add_base = f.base && (b == 0 || f.base_c1);
        const u64 *__restrict__ base =
            add_base ? f.base[it] + ((size_t)b * f.ell + i) * ((size_t)1 << log_n) : nullptr;
        const unsigned g = f.base_g ? (unsigned)f.base_g[it] : 1u;
        u64 *__restrict__ out = f.out + it * f.out_stride + ((size_t)b * f.ell + i) * ((size_t)1 << log_n);
        // eight elements per thread at a time: all their loads in flight together
        for (int x0 = r16_first<WL>(); x0 < r16_end<WL>(); x0 += 8 * r16_step<WL>()) {
            u64 av[8], bv[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const size_t k = e0 + x0 + r * r16_step<WL>();
                av[r] = acc[k];
                bv[r] = add_base ? base[f.base_g ? perm_index((int)k, g, log_n) : (int)k] : 0;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int x = x0 + r * r16_step<WL>();
                const u64 c = reduce_any(sm[r16_slot_b<P>(x >> P, x & ((1 << P) - 1))], q, m.one_p);
                u64 v = mul_shoup(sub_mod(av[r], c, q), pinv, pinvp, q);
                if (add_base) v = add_mod(v, bv[r], q);
                out[e0 + x] = v;
            }
        }
    } else if constexpr (MODE == kFuseRelinRescale) {
        // out_b[i] = (P^{-1} acc_b[i] + base_b[i] - X) q_t^{-1}, X = this
        // transform of P^{-1} conv_b[i] + [t_b]_{q_i}: ModDown's output
        // rescaled, by linearity of the transform
        const int slot = blockIdx.y, it = blockIdx.z;
        const int b = slot / (f.ell - 1), i = slot % (f.ell - 1);
        const int next = f.ell + f.K;
        const u64 pinv = __ldg(f.pinv + i), pinvp = __ldg(f.pinvp + i);
        const u64 inv = __ldg(f.inv + i), invp = __ldg(f.invp + i);
        const u64 *__restrict__ acc = f.acc + it * f.acc_stride + ((size_t)b * next + i) * ((size_t)1 << log_n);
        const u64 *__restrict__ base = f.base[it] + ((size_t)b * f.ell + i) * ((size_t)1 << log_n);
        u64 *__restrict__ out = f.out + it * f.out_stride + ((size_t)b * (f.ell - 1) + i) * ((size_t)1 << log_n);
        // optional mask product (Alg. 2's mask multiply after this rescale):
        // the Montgomery-form mask limb read through sigma_{mask_g}
        const u64 *__restrict__ mk = f.mask ? f.mask[it] + ((size_t)i << log_n) : nullptr;
        const unsigned mg = f.mask ? (unsigned)f.mask_g[it] : 1u;
        for (int x0 = r16_first<WL>(); x0 < r16_end<WL>(); x0 += 8 * r16_step<WL>()) {
            u64 av[8], bv[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const size_t k = e0 + x0 + r * r16_step<WL>();
                av[r] = acc[k];
                bv[r] = base[k];
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int x = x0 + r * r16_step<WL>();
                const u64 X = reduce_any(sm[r16_slot_b<P>(x >> P, x & ((1 << P) - 1))], q, m.one_p);
                const u64 y = add_mod(mul_shoup(av[r], pinv, pinvp, q), bv[r], q);
                u64 v = mul_shoup(sub_mod(y, X, q), inv, invp, q);
                if (mk) v = redc(mul_wide(v, mk[perm_index((int)(e0 + x), mg, log_n)]), q, m.qneg_inv);
                out[e0 + x] = v;
            }
        }
    } else if constexpr (MODE == kFuseRotAccum) {
        // target it: outp[it] += sum_j sigma_{g_j}(c0_j) (polynomial 0)
        //                      + P^{-1} (sum_j acc_j - X), X = this transform of
        // the target's summed conv: the rotated sources' ModDown outputs,
        // summed (the transform is linear, so one serves them all)
        const int slot = blockIdx.y, it = blockIdx.z;
        const int b = slot / f.ell, i = slot % f.ell;
        const int next = f.ell + f.K;
        const size_t n = (size_t)1 << log_n;
        const u64 pinv = __ldg(f.pinv + i), pinvp = __ldg(f.pinvp + i);
        u64 *__restrict__ out = f.outp[it] + ((size_t)b * f.ell + i) * n;
        const int j0 = f.seg[it], j1 = f.seg[it + 1];
        for (int x0 = r16_first<WL>(); x0 < r16_end<WL>(); x0 += 8 * r16_step<WL>()) {
            u64 sa[8], sc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) sa[r] = sc[r] = 0;
            for (int j = j0; j < j1; ++j) {
                const u64 *__restrict__ a = f.acc + (long long)f.item[j] * f.acc_stride + ((size_t)b * next + i) * n;
                u64 av[8], cv[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) av[r] = a[e0 + x0 + r * r16_step<WL>()];
                if (b == 0) {
                    const u64 *__restrict__ c0 = f.base[j] + (size_t)i * n;
                    const unsigned g = (unsigned)f.base_g[j];
#pragma unroll
                    for (int r = 0; r < 8; ++r) cv[r] = c0[perm_index((int)(e0 + x0 + r * r16_step<WL>()), g, log_n)];
#pragma unroll
                    for (int r = 0; r < 8; ++r) sc[r] = add_mod(sc[r], cv[r], q);
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) sa[r] = add_mod(sa[r], av[r], q);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int x = x0 + r * r16_step<WL>();
                const u64 X = reduce_any(sm[r16_slot_b<P>(x >> P, x & ((1 << P) - 1))], q, m.one_p);
                const u64 v = mul_shoup(sub_mod(sa[r], X, q), pinv, pinvp, q);
                out[e0 + x] = add_mod(add_mod(v, sc[r], q), out[e0 + x], q);
            }
        }
    } else {
        // rescale: out_b[i] = (in_b[i] - [r]_{q_i}) q_t^{-1} ([r]_{q_i} = this transform)
        const int slot = blockIdx.y, it = blockIdx.z;
        const int b = slot / (f.ell - 1), i = slot % (f.ell - 1);
        const u64 inv = __ldg(f.inv + i), invp = __ldg(f.invp + i);
        const u64 *__restrict__ in = f.in[it] + ((size_t)b * f.ell + i) * ((size_t)1 << log_n);
        u64 *__restrict__ out = f.out + it * f.out_stride + ((size_t)b * (f.ell - 1) + i) * ((size_t)1 << log_n);
        for (int x0 = r16_first<WL>(); x0 < r16_end<WL>(); x0 += 8 * r16_step<WL>()) {
            u64 cv[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) cv[r] = in[e0 + x0 + r * r16_step<WL>()];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int x = x0 + r * r16_step<WL>();
                const u64 rr = reduce_any(sm[r16_slot_b<P>(x >> P, x & ((1 << P) - 1))], q, m.one_p);
                out[e0 + x] = mul_shoup(sub_mod(cv[r], rr, q), inv, invp, q);
            }
        }
    }
}

template <int P, int V, int MODE = kFuseNone>
__global__ void __launch_bounds__(256, r16_min_blocks<V>()) k_fwd16_b(NttArgs a, const ModConst *__restrict__ mc,
                                                                      const ulonglong2 *__restrict__ tw2, int log_n,
                                                                      int PA, FuseArgs f)
{
    __shared__ u64 sm[r16_smem_words_b<P>()];
    extern __shared__ __align__(16) ulonglong2 smt[];   // V == 2: [r16_tw_smem_entries<P>()]
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const ModConst m = mc[mi];
    const ulonglong2 *w2 = tw2 + (size_t)mi * n;
    constexpr int AR = r16_arith<V>();
    constexpr bool WL = r16_warp_local<V>();
    constexpr u64 LB = lazy_fwd_bound<AR>();
    if constexpr (MODE != kFuseNone) {
        if (m.q < LB) fwd16_b_body<P, true, false, MODE, AR, WL>(sm, p, m, w2, PA, nullptr, f, log_n);
        else fwd16_b_body<P, false, false, MODE, AR, WL>(sm, p, m, w2, PA, nullptr, f, log_n);
    } else if constexpr (V == 2) {
        r16_prefetch_tw<P>(smt, w2, PA, (int)(((size_t)blockIdx.x * kElems) >> P));
        if (m.q < LB) fwd16_b_body<P, true, true>(sm, p, m, w2, PA, smt);
        else fwd16_b_body<P, false, true>(sm, p, m, w2, PA, smt);
    } else {
        if (m.q < LB) fwd16_b_body<P, true, false, kFuseNone, AR, WL>(sm, p, m, w2, PA, nullptr);
        else fwd16_b_body<P, false, false, kFuseNone, AR, WL>(sm, p, m, w2, PA, nullptr);
    }
}

template <int P, int V>
__global__ void __launch_bounds__(256, r16_min_blocks<V>()) k_inv16_b(NttArgs a, const ModConst *__restrict__ mc,
                                                                      const ulonglong2 *__restrict__ tw2, int log_n,
                                                                      int PA)
{
    __shared__ u64 sm[r16_smem_words_b<P>()];
    extern __shared__ __align__(16) ulonglong2 smt[];   // V == 2: [r16_tw_smem_entries<P>()]
    constexpr bool SM = V == 2;
    constexpr int AR = r16_arith<V>();
    constexpr bool WL = r16_warp_local<V>();
    constexpr int TPT = 1 << (P - 4);
    constexpr int R = (P + 3) / 4;
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const u64 *ps = a.src ? a.src[blockIdx.z] + (long long)a.map.off[blockIdx.y] * n : p;
    const u64 q = mc[mi].q;
    const ulonglong2 *w2 = tw2 + (size_t)mi * n;
    const int tile = threadIdx.x / TPT, t = threadIdx.x % TPT;
    const size_t e0 = (size_t)blockIdx.x * kElems;
    const int btile = (int)(e0 >> P) + tile;
    // the first stage's twiddles are requested before the data, so their
    // latency overlaps the data loads
    constexpr int Q1 = r16_q<P, R - 1>();
    ulonglong2 wpre[16];
    if constexpr (SM) r16_prefetch_tw<P>(smt, w2, PA, (int)(e0 >> P));
    else r16_load_tw<P, R - 1, Q1, Q1 - 1, false>(wpre, t, w2, PA, btile, nullptr, 0);
    // loads before stores, eight at a time (the stores into shared memory
    // would otherwise wait for each load in turn)
    for (int x0 = r16_first<WL>(); x0 < r16_end<WL>(); x0 += 8 * r16_step<WL>()) {
        u64 tmp[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) tmp[r] = ps[e0 + x0 + r * r16_step<WL>()];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = x0 + r * r16_step<WL>();
            sm[r16_slot_b<P>(x >> P, x & ((1 << P) - 1))] = tmp[r];
        }
    }
    if constexpr (SM) r16_prefetch_wait();
    else r16_sync<WL>();
    u64 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_b<P>(tile, r16_index<P, R - 1>(t, i))];
    r16_inv_round<P, R - 1, SM, !SM, AR>(v, t, w2, q, PA, btile, smt, tile, &wpre);
    if constexpr (R > 2) {
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_b<P>(tile, r16_index<P, R - 1>(t, i))] = v[i];
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_b<P>(tile, r16_index<P, R - 2>(t, i))];
        r16_inv_round<P, R - 2, SM, false, AR>(v, t, w2, q, PA, btile, smt, tile);
    }
    if constexpr (R > 1) {
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_b<P>(tile, r16_index<P, 1>(t, i))] = v[i];
        r16_sync<WL>();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_b<P>(tile, r16_index<P, 0>(t, i))];
        r16_inv_round<P, 0, SM, false, AR>(v, t, w2, q, PA, btile, smt, tile);
    }
    u64 *tp = p + e0 + ((size_t)tile << P);
#pragma unroll
    for (int i = 0; i < 16; ++i) tp[r16_index<P, 0>(t, i)] = v[i];
}

template <int P, int V>
__global__ void __launch_bounds__(256, r16_min_blocks<V>()) k_inv16_a(NttArgs a, const ModConst *__restrict__ mc,
                                                                      const ulonglong2 *__restrict__ tw2, int log_n)
{
    __shared__ u64 sm[r16_smem_words_a<P>()];
    constexpr int TPC = kElems >> P;
    constexpr int R = (P + 3) / 4;
    const int n = 1 << log_n;
    int mi;
    u64 *p = limb_ptr(a, n, mi);
    const ModConst m = mc[mi];
    const u64 q = m.q;
    const ulonglong2 *w2 = tw2 + (size_t)mi * n;
    const int lg_ncols = log_n - P;
    const int col = threadIdx.x % TPC, t = threadIdx.x / TPC;
    const int gcol = blockIdx.x * TPC + col;
    constexpr int AR = r16_arith<V>();
    u64 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = p[((size_t)r16_index<P, R - 1>(t, i) << lg_ncols) + gcol];
    r16_inv_round<P, R - 1, false, false, AR>(v, t, w2, q, 0, 0);
    if constexpr (R > 2) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_a<P>(col, r16_index<P, R - 1>(t, i))] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_a<P>(col, r16_index<P, R - 2>(t, i))];
        r16_inv_round<P, R - 2, false, false, AR>(v, t, w2, q, 0, 0);
        __syncthreads();
    }
    if constexpr (R > 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r16_slot_a<P>(col, r16_index<P, 1>(t, i))] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[r16_slot_a<P>(col, r16_index<P, 0>(t, i))];
        r16_inv_round<P, 0, false, false, AR>(v, t, w2, q, 0, 0);
    }
    if (a.unscaled) {
#pragma unroll
        for (int i = 0; i < 16; ++i) p[((size_t)r16_index<P, 0>(t, i) << lg_ncols) + gcol] = v[i];
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            p[((size_t)r16_index<P, 0>(t, i) << lg_ncols) + gcol] = mul_shoup(v[i], m.n_inv, m.n_inv_p, q);
    }
}

// dynamic shared memory of pass B for variant V (opted in once per kernel and
// device: the attribute belongs to the kernel's instance on the current
// device; DIR tells the forward and inverse kernels apart, their types are
// equal)
template <int P, int V, int DIR, typename K> size_t r16_b_smem(K kernel)
{
    if constexpr (V != 2) {
        (void)kernel;
        return 0;
    } else {
        const size_t bytes = (size_t)r16_tw_smem_entries<P>() * sizeof(ulonglong2);
        static std::atomic<uint64_t> done{0};   // bit d: set on device d (d < 64)
        int dev = 0;
        SPFHE_CHECK_CUDA(cudaGetDevice(&dev));
        const uint64_t bit = dev < 64 ? 1ull << dev : 0;
        if (!bit || !(done.load() & bit)) {
            SPFHE_CHECK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
            done.fetch_or(bit);
        }
        return bytes;
    }
}

template <int P, int V> struct R16LaunchV {
    static void fwd_a(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c)
    {
        k_fwd16_a<P, V><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, FuseArgs{});
    }
    static void fwd_b(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int PA)
    {
        const size_t smem = r16_b_smem<P, V, 0>(k_fwd16_b<P, V>);
        k_fwd16_b<P, V><<<g, 256, smem, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, PA, FuseArgs{});
    }
    static void inv_a(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c)
    {
        k_inv16_a<P, V><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.itw2, c.log_n);
    }
    static void inv_b(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int PA)
    {
        const size_t smem = r16_b_smem<P, V, 1>(k_inv16_b<P, V>);
        k_inv16_b<P, V><<<g, 256, smem, s>>>(a, c.dt.mc, c.dt.itw2, c.log_n, PA);
    }
};

// transforms with a fused prologue / epilogue (kernel variants 0 and 3 to 6)
template <int P, int V> struct R16FusedV {
    static void fwd_a(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int mode, const FuseArgs &f)
    {
        if (mode == kFuseRescale) k_fwd16_a<P, V, kFuseRescale><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, f);
        else if (mode == kFuseRelinRescale) {
            if constexpr (r16_relin_rescale<V>())
                k_fwd16_a<P, V, kFuseRelinRescale><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, f);
            else throw Error(SPFHE_EINVAL, "no merged relinearise-rescale transform for this NTT variant");
        } else k_fwd16_a<P, V><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, f);
    }
    static void fwd_b(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int PA, int mode, const FuseArgs &f)
    {
        if (mode == kFuseRescale) k_fwd16_b<P, V, kFuseRescale><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, PA, f);
        else if (mode == kFuseRelinRescale) {
            if constexpr (r16_relin_rescale<V>())
                k_fwd16_b<P, V, kFuseRelinRescale><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, PA, f);
            else throw Error(SPFHE_EINVAL, "no merged relinearise-rescale transform for this NTT variant");
        } else if (mode == kFuseRotAccum) {
            if constexpr (r16_relin_rescale<V>())
                k_fwd16_b<P, V, kFuseRotAccum><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, PA, f);
            else throw Error(SPFHE_EINVAL, "no fused rotate-accumulate transform for this NTT variant");
        } else k_fwd16_b<P, V, kFuseModDown><<<g, 256, 0, s>>>(a, c.dt.mc, c.dt.tw2, c.log_n, PA, f);
    }
};
template <int P> struct R16Fused {
    static void fwd_a(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int mode, const FuseArgs &f)
    {
        if (c.ntt_variant == 6) R16FusedV<P, 6>::fwd_a(g, s, a, c, mode, f);
        else if (c.ntt_variant == 5) R16FusedV<P, 5>::fwd_a(g, s, a, c, mode, f);
        else if (c.ntt_variant == 4) R16FusedV<P, 4>::fwd_a(g, s, a, c, mode, f);
        else if (c.ntt_variant == 3) R16FusedV<P, 3>::fwd_a(g, s, a, c, mode, f);
        else R16FusedV<P, 0>::fwd_a(g, s, a, c, mode, f);
    }
    static void fwd_b(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int PA, int mode, const FuseArgs &f)
    {
        if (c.ntt_variant == 6) R16FusedV<P, 6>::fwd_b(g, s, a, c, PA, mode, f);
        else if (c.ntt_variant == 5) R16FusedV<P, 5>::fwd_b(g, s, a, c, PA, mode, f);
        else if (c.ntt_variant == 4) R16FusedV<P, 4>::fwd_b(g, s, a, c, PA, mode, f);
        else if (c.ntt_variant == 3) R16FusedV<P, 3>::fwd_b(g, s, a, c, PA, mode, f);
        else R16FusedV<P, 0>::fwd_b(g, s, a, c, PA, mode, f);
    }
};

template <int P> struct R16Launch {
    template <typename F> static void variant(int v, F &&f)
    {
        switch (v) {
        case 0: f(R16LaunchV<P, 0>{}); break;
        case 1: f(R16LaunchV<P, 1>{}); break;
        case 2: f(R16LaunchV<P, 2>{}); break;
        case 3: f(R16LaunchV<P, 3>{}); break;
        case 4: f(R16LaunchV<P, 4>{}); break;
        case 5: f(R16LaunchV<P, 5>{}); break;
        case 6: f(R16LaunchV<P, 6>{}); break;
        default: throw Error(SPFHE_EINVAL, "no such NTT variant");
        }
    }
    static void fwd_a(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c)
    {
        variant(c.ntt_variant, [&](auto L) { decltype(L)::fwd_a(g, s, a, c); });
    }
    static void fwd_b(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int PA)
    {
        variant(c.ntt_variant, [&](auto L) { decltype(L)::fwd_b(g, s, a, c, PA); });
    }
    static void inv_a(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c)
    {
        variant(c.ntt_variant, [&](auto L) { decltype(L)::inv_a(g, s, a, c); });
    }
    static void inv_b(dim3 g, cudaStream_t s, const NttArgs &a, const Ctx &c, int PA)
    {
        variant(c.ntt_variant, [&](auto L) { decltype(L)::inv_b(g, s, a, c, PA); });
    }
};

template <typename F> void r16_fused_dispatch(int P, F &&f)
{
    switch (P) {
    case 6: f(R16Fused<6>{}); break;
    case 7: f(R16Fused<7>{}); break;
    case 8: f(R16Fused<8>{}); break;
    case 9: f(R16Fused<9>{}); break;
    default: throw Error(SPFHE_EINVAL, "no radix-16 pass for this size");
    }
}

template <typename F> void r16_dispatch(int P, F &&f)
{
    switch (P) {
    case 6: f(R16Launch<6>{}); break;
    case 7: f(R16Launch<7>{}); break;
    case 8: f(R16Launch<8>{}); break;
    case 9: f(R16Launch<9>{}); break;
    default: throw Error(SPFHE_EINVAL, "no radix-16 pass for this size");
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

// Split a transform batch into launch pairs of at most ctx.ntt_chunk limbs,
// so that pass B finds pass A's output in L2 (0 = one pair for the batch).
template <typename F> void for_chunks(const Ctx &ctx, const Batch &b, const LimbMap &map, F &&f)
{
    const int chunk = ctx.ntt_chunk;
    if (chunk <= 0 || (long long)map.nl * b.items <= chunk) {
        f(b, map);
        return;
    }
    auto item_batch = [&](int i0, int cnt) {
        Batch s = b;
        s.items = cnt;
        if (b.ids) s.ids = b.ids + i0;
        else s.base = b.base + (long long)i0 * b.stride;
        return s;
    };
    if (map.nl <= chunk) {
        const int per = chunk / map.nl;
        for (int i0 = 0; i0 < b.items; i0 += per) f(item_batch(i0, std::min(per, b.items - i0)), map);
        return;
    }
    for (int i0 = 0; i0 < b.items; ++i0)
        for (int s0 = 0; s0 < map.nl; s0 += chunk) {
            LimbMap m;
            m.nl = std::min(chunk, map.nl - s0);
            for (int k = 0; k < m.nl; ++k) {
                m.off[k] = map.off[s0 + k];
                m.mi[k] = map.mi[s0 + k];
            }
            f(item_batch(i0, 1), m);
        }
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

// stages in pass A of the radix-16 transforms (the rest run in pass B)
static int pass_a_stages(const Ctx &ctx) { return ctx.ntt_pa ? ctx.ntt_pa : ctx.log_n / 2; }

void ntt_forward(Ctx &ctx, Batch b, const LimbMap &map)
{
    launch_checks(b, map);
    if (map.nl <= 0 || b.items <= 0) return;
    Geometry g = geometry(ctx.log_n);
    NttArgs a{b.base, b.stride, b.ids, map};
    const int cls = ctx.in_keyswitch ? K_KS_NTT_FWD : K_NTT_FWD;
    if (ctx.log_n >= 12) {
        const int PA = pass_a_stages(ctx), PB = ctx.log_n - PA;
        for_chunks(ctx, b, map, [&](const Batch &cb, const LimbMap &cm) {
            NttArgs ca{cb.base, cb.stride, cb.ids, cm};
            dim3 grid(ctx.n / kElems, cm.nl, cb.items);
            {
                cudaEvent_t t0_ = prof_begin(ctx);
                r16_dispatch(PA, [&](auto L) { decltype(L)::fwd_a(grid, ctx.stream, ca, ctx); });
                prof_end(ctx, t0_, cls, 8.0 * ctx.n * cm.nl * cb.items, 0.5 * ctx.n * PA * cm.nl * cb.items, "ntt fwd A");
                prof_limbs(ctx, cls, 0, (double)cm.nl * cb.items);
            }
            {
                cudaEvent_t t0_ = prof_begin(ctx);
                r16_dispatch(PB, [&](auto L) { decltype(L)::fwd_b(grid, ctx.stream, ca, ctx, PA); });
                prof_end(ctx, t0_, cls, 8.0 * ctx.n * cm.nl * cb.items, 0.5 * ctx.n * PB * cm.nl * cb.items, "ntt fwd B");
                prof_limbs(ctx, cls, 1, (double)cm.nl * cb.items);
            }
        });
        return;
    }
    dim3 ga(g.grid_a, map.nl, b.items), gb(g.grid_b, map.nl, b.items);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_fwd_a<<<ga, kThreads, g.smem_a, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.tw, ctx.dt.twp, ctx.log_n, g.PA);
        prof_end(ctx, t0_, cls, 8.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * g.PA * map.nl * b.items, "ntt fwd A");
        prof_limbs(ctx, cls, 0, (double)map.nl * b.items);
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_fwd_b<<<gb, kThreads, g.smem_b, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.tw, ctx.dt.twp, ctx.log_n, g.PA, g.lgE);
        prof_end(ctx, t0_, cls, 8.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * (ctx.log_n - g.PA) * map.nl * b.items, "ntt fwd B");
        prof_limbs(ctx, cls, 1, (double)map.nl * b.items);
    }
}

bool ntt_forward_fused(Ctx &ctx, Batch b, const LimbMap &map, int mode, const FuseArgs &f)
{
    if (ctx.log_n < 12 || ctx.ntt_variant == 1 || ctx.ntt_variant == 2 || b.ids)
        return false;
    if ((mode == kFuseRelinRescale || mode == kFuseRotAccum) && ctx.ntt_variant != 5 && ctx.ntt_variant != 6)
        return false;
    launch_checks(b, map);
    if (map.nl <= 0 || b.items <= 0) return true;
    NttArgs a{b.base, b.stride, b.ids, map};
    const int cls = ctx.in_keyswitch ? K_KS_NTT_FWD : K_NTT_FWD;
    const int PA = pass_a_stages(ctx), PB = ctx.log_n - PA;
    dim3 grid(ctx.n / kElems, map.nl, b.items);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        r16_fused_dispatch(PA, [&](auto L) { decltype(L)::fwd_a(grid, ctx.stream, a, ctx, mode, f); });
        // the merged relinearise-rescale pass also reads ModDown's conversion
        prof_end(ctx, t0_, cls, (mode == kFuseRelinRescale ? 16.0 : 8.0) * ctx.n * map.nl * b.items,
                 0.5 * ctx.n * PA * map.nl * b.items,
                 mode == kFuseRescale ? "ntt fwd A + rescale spread"
                 : mode == kFuseRelinRescale ? "ntt fwd A + relinearised spread" : "ntt fwd A");
        prof_limbs(ctx, cls, 0, (double)map.nl * b.items);
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        r16_fused_dispatch(PB, [&](auto L) { decltype(L)::fwd_b(grid, ctx.stream, a, ctx, PA, mode, f); });
        // epilogue: ModDown reads acc, the base limbs it adds (both
        // polynomials, or only c0 for a rotation) and writes out; the rescale
        // reads its input limb and writes out
        const double base_limbs = !f.base ? 0.0 : (f.base_c1 ? 1.0 : 0.5) * map.nl;
        // rotate-accumulate: per source its acc limbs and (polynomial 0) its
        // c0 limbs, per target the result read and written
        const double sources = mode == kFuseRotAccum ? (double)f.polys : 0.0;
        const double epi = mode == kFuseModDown        ? (16.0 * ctx.n * map.nl + 8.0 * ctx.n * base_limbs) * b.items
                           : mode == kFuseRelinRescale ? 24.0 * ctx.n * map.nl * b.items
                           : mode == kFuseRotAccum     ? 8.0 * ctx.n * map.nl * (1.5 * sources + 2.0 * b.items)
                                                       : 16.0 * ctx.n * map.nl * b.items;
        prof_end(ctx, t0_, cls, epi,
                 0.5 * ctx.n * PB * map.nl * b.items,
                 mode == kFuseRescale ? "ntt fwd B + rescale final"
                 : mode == kFuseRelinRescale ? "ntt fwd B + relinearise-rescale final"
                 : mode == kFuseRotAccum ? "ntt fwd B + rotation sums" : "ntt fwd B + moddown final");
        prof_limbs(ctx, cls, 2, (double)map.nl * b.items);
    }
    return true;
}

void ntt_inverse(Ctx &ctx, Batch b, const LimbMap &map, bool scale)
{
    launch_checks(b, map);
    if (map.nl <= 0 || b.items <= 0) return;
    Geometry g = geometry(ctx.log_n);
    NttArgs a{b.base, b.stride, b.ids, map, scale ? 0 : 1};
    const int cls = ctx.in_keyswitch ? K_KS_NTT_INV : K_NTT_INV;
    if (ctx.log_n >= 12) {
        const int PA = pass_a_stages(ctx), PB = ctx.log_n - PA;
        for_chunks(ctx, b, map, [&](const Batch &cb, const LimbMap &cm) {
            NttArgs ca{cb.base, cb.stride, cb.ids, cm, scale ? 0 : 1};
            dim3 grid(ctx.n / kElems, cm.nl, cb.items);
            {
                cudaEvent_t t0_ = prof_begin(ctx);
                r16_dispatch(PB, [&](auto L) { decltype(L)::inv_b(grid, ctx.stream, ca, ctx, PA); });
                prof_end(ctx, t0_, cls, 8.0 * ctx.n * cm.nl * cb.items, 0.5 * ctx.n * PB * cm.nl * cb.items, "ntt inv B");
                prof_limbs(ctx, cls, 0, (double)cm.nl * cb.items);
            }
            {
                cudaEvent_t t0_ = prof_begin(ctx);
                r16_dispatch(PA, [&](auto L) { decltype(L)::inv_a(grid, ctx.stream, ca, ctx); });
                prof_end(ctx, t0_, cls, 8.0 * ctx.n * cm.nl * cb.items, 0.5 * ctx.n * PA * cm.nl * cb.items, "ntt inv A");
                prof_limbs(ctx, cls, 1, (double)cm.nl * cb.items);
            }
        });
        return;
    }
    dim3 ga(g.grid_a, map.nl, b.items), gb(g.grid_b, map.nl, b.items);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_inv_b<<<gb, kThreads, g.smem_b, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.itw, ctx.dt.itwp, ctx.log_n, g.PA, g.lgE);
        prof_end(ctx, t0_, cls, 8.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * (ctx.log_n - g.PA) * map.nl * b.items, "ntt inv B");
        prof_limbs(ctx, cls, 0, (double)map.nl * b.items);
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_inv_a<<<ga, kThreads, g.smem_a, ctx.stream>>>(a, ctx.dt.mc, ctx.dt.itw, ctx.dt.itwp, ctx.log_n, g.PA);
        prof_end(ctx, t0_, cls, 8.0 * ctx.n * map.nl * b.items, 0.5 * ctx.n * g.PA * map.nl * b.items, "ntt inv A");
        prof_limbs(ctx, cls, 1, (double)map.nl * b.items);
    }
}

bool ntt_inverse_from(Ctx &ctx, Batch dst, const u64 *const *src, const LimbMap &map, bool scale)
{
    if (ctx.log_n < 12 || dst.ids || ctx.ntt_chunk > 0) return false;
    launch_checks(dst, map);
    if (map.nl <= 0 || dst.items <= 0) return true;
    NttArgs a{dst.base, dst.stride, nullptr, map, scale ? 0 : 1, src};
    NttArgs a2{dst.base, dst.stride, nullptr, map, scale ? 0 : 1};
    const int cls = ctx.in_keyswitch ? K_KS_NTT_INV : K_NTT_INV;
    const int PA = pass_a_stages(ctx), PB = ctx.log_n - PA;
    dim3 grid(ctx.n / kElems, map.nl, dst.items);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        r16_dispatch(PB, [&](auto L) { decltype(L)::inv_b(grid, ctx.stream, a, ctx, PA); });
        prof_end(ctx, t0_, cls, 8.0 * ctx.n * map.nl * dst.items, 0.5 * ctx.n * PB * map.nl * dst.items, "ntt inv B");
        prof_limbs(ctx, cls, 0, (double)map.nl * dst.items);
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        r16_dispatch(PA, [&](auto L) { decltype(L)::inv_a(grid, ctx.stream, a2, ctx); });
        prof_end(ctx, t0_, cls, 8.0 * ctx.n * map.nl * dst.items, 0.5 * ctx.n * PA * map.nl * dst.items, "ntt inv A");
        prof_limbs(ctx, cls, 1, (double)map.nl * dst.items);
    }
    return true;
}

}  // namespace spfhe
