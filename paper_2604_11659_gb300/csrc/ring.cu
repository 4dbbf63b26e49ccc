// Elementwise and basis-conversion kernels of RNS-CKKS on sm_103a.
// Layouts: a polynomial at level ell is [ell][n] u64 (limb-major), a
// ciphertext [2][ell][n]; batches place items `stride` words apart.
#include <cmath>
#include <type_traits>

#include "kernels.h"

namespace spfhe {

namespace {
constexpr int kT = 256;

inline dim3 grid_n(int n, int y, int z) { return dim3((n + kT - 1) / kT, y, z); }


__global__ void k_tensor(int ell, int n, const u64 *const *pa, const u64 *const *pb, u64 *d,
                         const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y, it = blockIdx.z;
    const ModConst m = mc[l];
    const u64 *a = pa[it], *b = pb[it];
    const size_t o0 = (size_t)l * n + k, o1 = (size_t)(ell + l) * n + k;
    const u64 a0 = a[o0], a1 = a[o1], b0 = b[o0], b1 = b[o1];
    u64 *out = d + (size_t)it * 3 * ell * n;
    out[(size_t)l * n + k] = mul_mod(a0, b0, m);
    U128 t = mul_wide(a0, b1);
    add_wide(t, mul_wide(a1, b0));
    out[(size_t)(ell + l) * n + k] = mul_shoup(redc(t, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
    out[(size_t)(2 * ell + l) * n + k] = mul_mod(a1, b1, m);
}

__global__ void k_automorph(int polys, int ell, int log_n, const u64 *const *in, u64 *out, long long out_stride,
                            const int *g)
{
    const int n = 1 << log_n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int pl = blockIdx.y, it = blockIdx.z;   // pl over polys * ell
    const int src = perm_index(k, (unsigned)g[it], log_n);
    out[it * out_stride + (size_t)pl * n + k] = in[it][(size_t)pl * n + src];
    (void)polys;
    (void)ell;
}

// Base-conversion constant rows in shared memory: for every target modulus a
// row of RL words [c_0 .. c_{NS-1}, c_corr, q, -q^{-1} mod 2^64 (, pad)]
// (c's split, Montgomery form), RL even so rows are 16-byte aligned.
template <int NS> constexpr int bconv_row() { return (NS + 3 + 1) & ~1; }

template <int NS>
__device__ __forceinline__ u64 bconv_out(const u64 *row, const uint32_t (&y0)[NS], const uint32_t (&y1)[NS],
                                         uint32_t v)
{
    constexpr int RL = bconv_row<NS>();
    const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(row);
    Acc30K a;
    acc30k_zero(a);
    u64 q = 0, qi = 0;
#pragma unroll
    for (int p = 0; p < RL / 2; ++p) {
        const ulonglong2 w = r2[p];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = 2 * p + h;
            const u64 c = h ? w.y : w.x;
            if (e < NS) acc30k_mac(a, y0[e < NS ? e : 0], y1[e < NS ? e : 0], c);
            else if (e == NS) acc30k_mac_small(a, v, c);
            else if (e == NS + 1) q = c;
            else if (e == NS + 2) qi = c;
        }
    }
    return redc(acc30k_value(a), q, qi);
}

// ModUp: for digit j (blockIdx.y) with source limbs [lo, hi) of the
// coefficient-domain input, write the centred representative of the digit
// value modulo D = prod q_i into every extended limb t outside [lo, hi):
//   y_i = [x_i (D/q_i)^{-1}]_{q_i},  v = round(sum_i y_i / q_i) (fma chain),
//   out_t = sum_i y_i (D/q_i) - v D  mod m_t,
// one carry-free accumulation (Acc30K: three 32x32 products per term) of NS + 1
// products with Montgomery-form
// constants (the last one v * (-D mod m_t)) and one REDC per output.
// Extended limb t < ell is q_t, t >= ell is p_{t-ell} (modulus L + t - ell).
template <int NS>
__global__ void __launch_bounds__(256, 4) k_modup_bconv(int digit0, int ell, int L, int K, int alpha, int M, int n,
                                                     const u64 *coef, long long coef_stride, u64 *ext,
                                                     long long ext_stride, const ModConst *__restrict__ mc,
                                                     const u64 *__restrict__ hinv, const u64 *__restrict__ hinvp,
                                                     const u64 *__restrict__ hsplit, const u64 *__restrict__ negd,
                                                     const double *__restrict__ inv_q)
{
    constexpr int RL = bconv_row<NS>();
    extern __shared__ __align__(16) u64 sh[];   // [M][RL]
    const int j = digit0 + blockIdx.y, it = blockIdx.z;
    const int lo = j * alpha, hi = lo + NS;
    const size_t row0 = (size_t)(hi - 1) * alpha;
    for (int x = threadIdx.x; x < M * RL; x += blockDim.x) {
        const int gm = x / RL, c = x - gm * RL;
        u64 w = 0;
        if (c < NS) w = hsplit[(row0 + c) * M + gm];
        else if (c == NS) w = negd[(size_t)(hi - 1) * M + gm];
        else if (c == NS + 1) w = mc[gm].q;
        else if (c == NS + 2) w = mc[gm].qneg_inv;
        sh[x] = w;
    }
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t y0[NS], y1[NS];
    double f = 0.0;
    const u64 *src = coef + it * coef_stride;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const u64 q = mc[lo + i].q;
        const u64 y = mul_shoup(src[(size_t)(lo + i) * n + k], __ldg(hinv + row0 + i), __ldg(hinvp + row0 + i), q);
        f = fma((double)y, __ldg(inv_q + lo + i), f);
        split30(y, y0[i], y1[i]);
    }
    const uint32_t v = (uint32_t)rint(f);
    const int next = ell + K;
    u64 *dst = ext + it * ext_stride + (size_t)j * next * n + k;
    // global stores (st.global): the shared-memory constant loads need not
    // wait for them
    for (int t = 0; t < lo; ++t) __stcg(dst + (size_t)t * n, bconv_out<NS>(sh + t * RL, y0, y1, v));
    for (int t = hi; t < ell; ++t) __stcg(dst + (size_t)t * n, bconv_out<NS>(sh + t * RL, y0, y1, v));
    for (int t = ell; t < next; ++t)
        __stcg(dst + (size_t)t * n, bconv_out<NS>(sh + (L + t - ell) * RL, y0, y1, v));
}

// Inner product with the switching key: acc_b[t] = sum_j E_j[t] k_{j,b}[t].
// Items of one group share a key; keys are in Montgomery form so a single
// REDC of the 128-bit sum yields the standard residue.
struct IpGroup {
    const u64 *key;
    int first, count;
};

constexpr int kMaxIpGroups = 48;
struct IpGroups {
    IpGroup g[kMaxIpGroups];
};

// BETA = number of digits at this level (compile-time, so the per-thread key
// values stay in registers); BETA = 0 selects a generic loop for larger counts.
// Products are summed carry-free (Acc30) and reduced by one REDC.
template <int BETA>
__global__ void __launch_bounds__(256) k_ip(int ell, int L, int K, int alpha, int M, int n, const u64 *const *in,
                                            const u64 *__restrict__ ext, long long ext_stride, IpGroups groups,
                                            u64 *__restrict__ acc, long long acc_stride,
                                            const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int t = blockIdx.y;
    const IpGroup gr = groups.g[blockIdx.z];
    const int next = ell + K;
    const int gm = t < ell ? t : L + (t - ell);
    const ModConst m = mc[gm];
    // digit holding limb t (t < ell), -1 for special-prime limbs
    const int own = t < ell ? t / alpha : -1;
    if constexpr (BETA > 0) {
        u64 k0[BETA], k1[BETA];   // key values, split
#pragma unroll
        for (int j = 0; j < BETA; ++j) {
            uint32_t a0, a1;
            split30(__ldg(gr.key + (((size_t)j * 2 + 0) * M + gm) * n + k), a0, a1);
            k0[j] = (u64)a0 | ((u64)a1 << 32);
            split30(__ldg(gr.key + (((size_t)j * 2 + 1) * M + gm) * n + k), a0, a1);
            k1[j] = (u64)a0 | ((u64)a1 << 32);
        }
        for (int it = gr.first; it < gr.first + gr.count; ++it) {
            Acc30 a0, a1;
            acc30_zero(a0);
            acc30_zero(a1);
            const u64 *e_it = ext + it * ext_stride + (size_t)t * n + k;
#pragma unroll
            for (int j = 0; j < BETA; ++j) {
                const u64 e = (j == own) ? in[it][(size_t)t * n + k] : e_it[(size_t)j * next * n];
                uint32_t e0, e1;
                split30(e, e0, e1);
                acc30_mac(a0, e0, e1, k0[j]);
                acc30_mac(a1, e0, e1, k1[j]);
            }
            u64 *o = acc + it * acc_stride;
            o[(size_t)t * n + k] = redc(acc30_value(a0), m.q, m.qneg_inv);
            o[((size_t)next + t) * n + k] = redc(acc30_value(a1), m.q, m.qneg_inv);
        }
    } else {
        const int beta = (ell + alpha - 1) / alpha;
        for (int it = gr.first; it < gr.first + gr.count; ++it) {
            U128 a0 = {0, 0}, a1 = {0, 0};
            for (int j = 0; j < beta; ++j) {
                const u64 e = (j == own) ? in[it][(size_t)t * n + k]
                                         : ext[it * ext_stride + ((size_t)j * next + t) * n + k];
                mac_wide(a0, e, __ldg(gr.key + (((size_t)j * 2 + 0) * M + gm) * n + k));
                mac_wide(a1, e, __ldg(gr.key + (((size_t)j * 2 + 1) * M + gm) * n + k));
            }
            u64 *o = acc + it * acc_stride;
            o[(size_t)t * n + k] = redc(a0, m.q, m.qneg_inv);
            o[((size_t)next + t) * n + k] = redc(a1, m.q, m.qneg_inv);
        }
    }
}

// Hoisted inner product: item it reads the extension of source src_of[it]
// and its own limbs in[it] through the automorphism X -> X^perm_g[it]
// (evaluation rep.: slot k reads slot perm_index(k, g)); one key per group.
__global__ void __launch_bounds__(256) k_ip_hoisted(int ell, int L, int K, int alpha, int M, int log_n,
                                                    const u64 *const *in, const u64 *__restrict__ ext,
                                                    long long ext_stride, IpGroups groups, u64 *__restrict__ acc,
                                                    long long acc_stride, const ModConst *__restrict__ mc,
                                                    const int *__restrict__ src_of, const int *__restrict__ perm_g)
{
    const int n = 1 << log_n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int t = blockIdx.y;
    const IpGroup gr = groups.g[blockIdx.z];
    const int next = ell + K;
    const int gm = t < ell ? t : L + (t - ell);
    const ModConst m = mc[gm];
    const int own = t < ell ? t / alpha : -1;
    const int beta = (ell + alpha - 1) / alpha;
    for (int it = gr.first; it < gr.first + gr.count; ++it) {
        const int ks = perm_index(k, (unsigned)perm_g[it], log_n);
        const u64 *e_it = ext + src_of[it] * ext_stride + (size_t)t * n + ks;
        Acc30 a0, a1;
        acc30_zero(a0);
        acc30_zero(a1);
        for (int j = 0; j < beta; ++j) {
            const u64 e = (j == own) ? in[it][(size_t)t * n + ks] : e_it[(size_t)j * next * n];
            uint32_t e0, e1, q0, q1;
            split30(e, e0, e1);
            split30(__ldg(gr.key + (((size_t)j * 2 + 0) * M + gm) * n + k), q0, q1);
            acc30_mac(a0, e0, e1, (u64)q0 | ((u64)q1 << 32));
            split30(__ldg(gr.key + (((size_t)j * 2 + 1) * M + gm) * n + k), q0, q1);
            acc30_mac(a1, e0, e1, (u64)q0 | ((u64)q1 << 32));
        }
        u64 *o = acc + it * acc_stride;
        o[(size_t)t * n + k] = redc(acc30_value(a0), m.q, m.qneg_inv);
        o[((size_t)next + t) * n + k] = redc(acc30_value(a1), m.q, m.qneg_inv);
    }
}

// ModDown basis conversion P -> Q_ell of the CENTRED representative of the
// accumulator modulo P: with y_k = [acc_k (P/p_k)^{-1}]_{p_k},
//   sum_k y_k (P/p_k) = (acc mod P) + u P,  u = floor(sum_k y_k / p_k),
// and v = round(sum_k y_k / p_k) (fma chain over k ascending, 1/p_k as a
// correctly rounded double) replaces u, so
// conv = sum_k y_k (P/p_k) - v P lies in [-P/2, P/2) and the final
// (acc - conv) / P is acc / P rounded to nearest: a zero-mean error
// (Halevi-Polyakov-Shoup floating-point correction, CT-RSA 2019).
// One carry-free accumulation of KK + 1 products (the last v * (-P mod q_t))
// and one REDC per output.
// in = acc (coefficient rep. on the P limbs), out conv [items][2][ell][n].
template <int KK>
__global__ void __launch_bounds__(256, 4) k_moddown_bconv(int ell, int L, int M, int n, const u64 *acc,
                                                       long long acc_stride, u64 *conv, const ModConst *__restrict__ mc,
                                                       const u64 *__restrict__ hinv, const u64 *__restrict__ hinvp,
                                                       const u64 *__restrict__ hsplit, const u64 *__restrict__ negp,
                                                       const double *__restrict__ inv_q)
{
    constexpr int RL = bconv_row<KK>();
    extern __shared__ __align__(16) u64 sh[];   // [ell][RL]
    for (int x = threadIdx.x; x < ell * RL; x += blockDim.x) {
        const int t = x / RL, c = x - t * RL;
        u64 w = 0;
        if (c < KK) w = hsplit[(size_t)c * M + t];
        else if (c == KK) w = negp[t];
        else if (c == KK + 1) w = mc[t].q;
        else if (c == KK + 2) w = mc[t].qneg_inv;
        sh[x] = w;
    }
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = blockIdx.y, it = blockIdx.z;
    const int next = ell + KK;
    const u64 *src = acc + it * acc_stride + ((size_t)b * next + ell) * n;
    uint32_t y0[KK], y1[KK];
    double f = 0.0;
#pragma unroll
    for (int i = 0; i < KK; ++i) {
        const u64 p = mc[L + i].q;
        const u64 y = mul_shoup(src[(size_t)i * n + k], __ldg(hinv + i), __ldg(hinvp + i), p);
        f = fma((double)y, __ldg(inv_q + L + i), f);
        split30(y, y0[i], y1[i]);
    }
    const uint32_t v = (uint32_t)rint(f);
    u64 *dst = conv + ((size_t)it * 2 + b) * ell * n + k;
    for (int t = 0; t < ell; ++t) __stcg(dst + (size_t)t * n, bconv_out<KK>(sh + t * RL, y0, y1, v));
}

// out_b[i] = base_b[sigma(i)] + (acc_b[i] - conv_b[i]) P^{-1} mod q_i
// base_c1 = false: only poly 0 gets the base added (rotation: c0 part).
__global__ void k_moddown_final(int ell, int K, int log_n, const u64 *acc, long long acc_stride, const u64 *conv,
                                const u64 *const *base, const int *base_g, int base_c1, u64 *out,
                                long long out_stride, const ModConst *__restrict__ mc,
                                const u64 *__restrict__ pinv, const u64 *__restrict__ pinvp)
{
    const int n = 1 << log_n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y, it = blockIdx.z;   // bi over 2 * ell
    const int b = bi / ell, i = bi % ell;
    const int next = ell + K;
    const u64 q = mc[i].q;
    const u64 a = acc[it * acc_stride + ((size_t)b * next + i) * n + k];
    const u64 c = conv[((size_t)it * 2 + b) * ell * n + (size_t)i * n + k];
    u64 v = mul_shoup(sub_mod(a, c, q), __ldg(pinv + i), __ldg(pinvp + i), q);
    if (base && (b == 0 || base_c1)) {
        const int src = base_g ? perm_index(k, (unsigned)base_g[it], log_n) : k;
        v = add_mod(v, base[it][((size_t)b * ell + i) * n + src], q);
    }
    out[it * out_stride + ((size_t)b * ell + i) * n + k] = v;
}

// Rescale, step 1: r = centred top limb (coefficient rep., [items][polys][n]),
// spread into tmp [items][polys][ell-1][n] as [r]_{q_i}.
__global__ void k_rescale_spread(int polys, int ell, int n, const u64 *top, u64 *tmp, const ModConst *__restrict__ mc,
                                 const u64 *__restrict__ qt_mod)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y, it = blockIdx.z;   // over polys * (ell-1)
    const int b = bi / (ell - 1), i = bi % (ell - 1);
    const u64 qt = mc[ell - 1].q;
    const u64 c = top[((size_t)it * polys + b) * n + k];
    const ModConst m = mc[i];
    // c mod q_i: REDC(c) = c 2^-64, then times 2^64 mod q_i
    u64 r = mul_shoup(redc(U128{c, 0}, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
    if (c > (qt >> 1)) r = sub_mod(r, __ldg(qt_mod + i), m.q);   // r = c - q_t (negative representative)
    tmp[(((size_t)it * polys + b) * (ell - 1) + i) * n + k] = r;
}

__global__ void k_rescale_final(int polys, int ell, int n, const u64 *const *in, const u64 *tmp, u64 *out,
                                long long out_stride, const ModConst *__restrict__ mc, const u64 *__restrict__ inv,
                                const u64 *__restrict__ invp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y, it = blockIdx.z;
    const int b = bi / (ell - 1), i = bi % (ell - 1);
    const u64 q = mc[i].q;
    const u64 c = in[it][((size_t)b * ell + i) * n + k];
    const u64 r = tmp[(((size_t)it * polys + b) * (ell - 1) + i) * n + k];
    out[it * out_stride + ((size_t)b * (ell - 1) + i) * n + k] = mul_shoup(sub_mod(c, r, q), __ldg(inv + i), __ldg(invp + i), q);
}

__global__ void k_copy_top(int polys, int ell, int n, const u64 *const *in, u64 *top)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = blockIdx.y, it = blockIdx.z;
    top[((size_t)it * polys + b) * n + k] = in[it][((size_t)b * ell + ell - 1) * n + k];
}

// Relinearised top limb in coefficient rep. (modulus q_t = q_{ell-1}):
// top[it][b] = [(acc_b[t] - conv_b[t]) P^{-1} + top[it][b]]_{q_t}, with
// acc_b[t] and the base's top limb (top on entry) already inverse transformed.
__global__ void k_relin_top(int ell, int K, int n, const u64 *acc, long long acc_stride, const u64 *conv, u64 *top,
                            const ModConst *__restrict__ mc, const u64 *__restrict__ pinv,
                            const u64 *__restrict__ pinvp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = blockIdx.y, it = blockIdx.z, t = ell - 1;
    const u64 q = mc[t].q;
    const u64 a = acc[it * acc_stride + ((size_t)b * (ell + K) + t) * n + k];
    const u64 c = conv[((size_t)it * 2 + b) * ell * n + (size_t)t * n + k];
    u64 *o = top + ((size_t)it * 2 + b) * n + k;
    *o = add_mod(mul_shoup(sub_mod(a, c, q), __ldg(pinv + t), __ldg(pinvp + t), q), *o, q);
}

__global__ void k_mul_plain_perm(int ell, int log_n, u64 *ct, long long stride, const u64 *const *mask, const int *g,
                                 const ModConst *__restrict__ mc)
{
    const int n = 1 << log_n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y, it = blockIdx.z;
    const int i = bi % ell;
    const ModConst m = mc[i];
    const int src = perm_index(k, (unsigned)g[it], log_n);
    const u64 w = mask[it][(size_t)i * n + src];
    u64 *p = ct + it * stride + (size_t)bi * n + k;
    *p = redc(mul_wide(*p, w), m.q, m.qneg_inv);
}

__global__ void k_accumulate(int ell, int n, u64 *res, const u64 *x, long long stride, const int *ids, int count,
                             const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y;   // over 2 * ell
    const u64 q = mc[bi % ell].q;
    const size_t off = (size_t)bi * n + k;
    u64 acc = res[off];
    for (int c = 0; c < count; ++c) acc = add_mod(acc, x[(long long)ids[c] * stride + off], q);
    res[off] = acc;
}

// Segmented sums: target g (blockIdx.z) receives the sum over its segment
// [seg[g], seg[g+1]) of source items, plus its own value when `into`; each
// item is `limbs` limbs (polynomials x ell), limb l has modulus l % ell.
__global__ void k_accumulate_seg(int limbs, int ell, int n, u64 *const *tgt, const u64 *const *src, const int *seg,
                                 int into, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y, g = blockIdx.z;
    const u64 q = mc[l % ell].q;
    const size_t off = (size_t)l * n + k;
    u64 acc = into ? tgt[g][off] : 0;
    for (int c = seg[g]; c < seg[g + 1]; ++c) acc = add_mod(acc, src[c][off], q);
    tgt[g][off] = acc;
}

__global__ void k_add(int polys, int ell, int n, const u64 *a, const u64 *b, u64 *out, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y;
    const u64 q = mc[bi % ell].q;
    const size_t o = (size_t)bi * n + k;
    out[o] = add_mod(a[o], b[o], q);
    (void)polys;
}

__global__ void k_mul_ct_pt(int ell, int n, const u64 *ct, const u64 *pt, u64 *out, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int bi = blockIdx.y;
    const int i = bi % ell;
    const size_t o = (size_t)bi * n + k;
    out[o] = mul_mod(ct[o], pt[(size_t)i * n + k], mc[i]);
}

struct MiList {
    int mi[kMaxMods];
};

__global__ void k_to_mont(int n, u64 *x, MiList ml, int limbs, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y, rep = blockIdx.z;
    const ModConst m = mc[ml.mi[l]];
    u64 *p = x + ((size_t)rep * limbs + l) * n + k;
    *p = to_mont(*p, m);
}

// x -> x 2^-64 mod q (out of Montgomery form), x < q
__global__ void k_from_mont(int n, u64 *x, MiList ml, int limbs, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y, rep = blockIdx.z;
    const ModConst m = mc[ml.mi[l]];
    u64 *p = x + ((size_t)rep * limbs + l) * n + k;
    *p = redc(U128{*p, 0}, m.q, m.qneg_inv);
}

__global__ void k_from_signed(int n, const long long *coef, u64 *out, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y;
    const u64 q = mc[l].q;
    const long long c = coef[k];
    // |c| < 2^62 assumed; reduce |c| then negate
    const u64 a = (u64)(c < 0 ? -c : c);
    const ModConst m = mc[l];
    u64 r = mul_shoup(redc(U128{a, 0}, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
    if (c < 0) r = neg_mod(r, q);
    out[(size_t)l * n + k] = r;
}

__global__ void k_decrypt(int ell, int n, const u64 *ct, const u64 *s_mont, u64 *out, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = blockIdx.y;
    const ModConst m = mc[i];
    const u64 c0 = ct[(size_t)i * n + k], c1 = ct[((size_t)ell + i) * n + k];
    const u64 s = s_mont[(size_t)i * n + k];
    out[(size_t)i * n + k] = add_mod(c0, redc(mul_wide(c1, s), m.q, m.qneg_inv), m.q);
}

// ---- ChaCha20 (RFC 8439 block function) --------------------------------
__device__ __forceinline__ unsigned rotl32(unsigned x, int r) { return (x << r) | (x >> (32 - r)); }

__device__ __forceinline__ void qr(unsigned &a, unsigned &b, unsigned &c, unsigned &d)
{
    a += b; d ^= a; d = rotl32(d, 16);
    c += d; b ^= c; b = rotl32(b, 12);
    a += b; d ^= a; d = rotl32(d, 8);
    c += d; b ^= c; b = rotl32(b, 7);
}

// 16 output words for (key from seed, block counter, nonce = stream id)
__device__ void chacha_block(uint64_t seed, uint64_t stream_id, unsigned counter, unsigned out[16])
{
    unsigned st[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                       (unsigned)seed, (unsigned)(seed >> 32), 0x9e3779b9u, 0x7f4a7c15u,
                       0xbf58476du, 0x1ce4e5b9u, 0x94d049bbu, 0x13311eb1u,
                       counter, (unsigned)stream_id, (unsigned)(stream_id >> 32), 0u};
    unsigned x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = st[i];
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        qr(x[0], x[4], x[8], x[12]);
        qr(x[1], x[5], x[9], x[13]);
        qr(x[2], x[6], x[10], x[14]);
        qr(x[3], x[7], x[11], x[15]);
        qr(x[0], x[5], x[10], x[15]);
        qr(x[1], x[6], x[11], x[12]);
        qr(x[2], x[7], x[8], x[13]);
        qr(x[3], x[4], x[9], x[14]);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = x[i] + st[i];
}

// Uniform residues: each block gives 4 coefficients of 128 random bits;
// value = floor(X q / 2^128).
__global__ void k_sample_uniform(int n, u64 *out, MiList ml, uint64_t seed, uint64_t stream_id,
                                 const ModConst *__restrict__ mc)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;   // group of 4 coefficients
    if (g * 4 >= n) return;
    const int l = blockIdx.y;
    const u64 q = mc[ml.mi[l]].q;
    unsigned w[16];
    chacha_block(seed, stream_id, (unsigned)(l * (n / 4) + g), w);
    for (int c = 0; c < 4; ++c) {
        const u64 lo = (u64)w[4 * c] | ((u64)w[4 * c + 1] << 32);
        const u64 hi = (u64)w[4 * c + 2] | ((u64)w[4 * c + 3] << 32);
        const u64 a_lo = hi * q, a_hi = __umul64hi(hi, q);
        const u64 b = __umul64hi(lo, q);
        const u64 s = a_lo + b;
        out[(size_t)l * n + g * 4 + c] = a_hi + (s < a_lo ? 1ull : 0ull);
    }
}

__global__ void k_sample_ternary(int n, long long *out, uint64_t seed, uint64_t stream_id)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;   // 8 coefficients per block
    if (g * 8 >= n) return;
    unsigned w[16];
    chacha_block(seed, stream_id, (unsigned)g, w);
    for (int c = 0; c < 8 && g * 8 + c < n; ++c) {
        const u64 x = (u64)w[2 * c] | ((u64)w[2 * c + 1] << 32);
        out[g * 8 + c] = (long long)__umul64hi(x, 3ull) - 1;
    }
}

// Rounded Gaussian, sigma = 3.2, |e| <= 19 (6 sigma), by Box-Muller.
__global__ void k_sample_gaussian(int n, long long *out, uint64_t seed, uint64_t stream_id)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;   // 8 coefficients per block
    if (g * 8 >= n) return;
    unsigned w[16];
    chacha_block(seed, stream_id, (unsigned)g, w);
    for (int c = 0; c < 8 && g * 8 + c < n; c += 2) {
        const u64 x1 = (u64)w[2 * c] | ((u64)w[2 * c + 1] << 32);
        const u64 x2 = (u64)w[2 * c + 2] | ((u64)w[2 * c + 3] << 32);
        const double u1 = ((double)(x1 >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = (double)(x2 >> 11) * 0x1.0p-53;
        const double r = 3.2 * sqrt(-2.0 * log(u1));
        double s, co;
        sincospi(2.0 * u2, &s, &co);
        for (int h = 0; h < 2 && g * 8 + c + h < n; ++h) {
            double z = rint(r * (h == 0 ? co : s));
            z = fmin(19.0, fmax(-19.0, z));
            out[g * 8 + c + h] = (long long)z;
        }
    }
}

__global__ void k_rlwe_b(int n, MiList ml, const u64 *a, const u64 *s_mont, const u64 *e, const u64 *extra, u64 *out,
                         const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y;
    const int gm = ml.mi[l];
    const ModConst m = mc[gm];
    const size_t o = (size_t)l * n + k;
    const u64 as = redc(mul_wide(a[o], s_mont[(size_t)gm * n + k]), m.q, m.qneg_inv);
    u64 v = sub_mod(e[o], as, m.q);
    if (extra) v = add_mod(v, extra[o], m.q);
    out[o] = v;
}

struct GadgetConsts {
    u64 p[16], pp[16];
};

__global__ void k_add_gadget(int n, u64 *out, const u64 *sp, int lo, GadgetConsts gc, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = lo + blockIdx.y;
    const u64 q = mc[i].q;
    const size_t o = (size_t)i * n + k;
    out[o] = add_mod(out[o], mul_shoup(sp[o], gc.p[blockIdx.y], gc.pp[blockIdx.y], q), q);
}

__global__ void k_gather(int words_per_item, const u64 *const *in, u64 *out, long long stride)
{
    const int it = blockIdx.y;
    const u64 *src = in[it];
    u64 *dst = out + it * stride;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < words_per_item; x += gridDim.x * blockDim.x)
        dst[x] = src[x];
}

__global__ void k_scatter(int words_per_item, const u64 *src, long long stride, u64 *const *out)
{
    const int it = blockIdx.y;
    const u64 *s = src + it * stride;
    u64 *d = out[it];
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < words_per_item; x += gridDim.x * blockDim.x)
        d[x] = s[x];
}

__global__ void k_mul_poly(int n, const u64 *a, const u64 *b, u64 *out, const ModConst *__restrict__ mc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int l = blockIdx.y;
    const size_t o = (size_t)l * n + k;
    out[o] = mul_mod(a[o], b[o], mc[l]);
}

}  // namespace


void tensor(Ctx &ctx, int items, int ell, const u64 *const *pa, const u64 *const *pb, u64 *d)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_tensor<<<grid_n(ctx.n, ell, items), kT, 0, ctx.stream>>>(ell, ctx.n, pa, pb, d, ctx.dt.mc);
        prof_end(ctx, t0_, K_TENSOR, 56.0 * ctx.n * items * ell, 4.0 * ctx.n * items * ell, "tensor");
    }
}

void automorph(Ctx &ctx, int items, int polys, int ell, const u64 *const *in, long long, u64 *out,
               long long out_stride, const int *g)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_automorph<<<grid_n(ctx.n, polys * ell, items), kT, 0, ctx.stream>>>(polys, ell, ctx.log_n, in, out,
                                                                             out_stride, g);
        prof_end(ctx, t0_, K_AUTOMORPH, 16.0 * ctx.n * items * polys * ell, 0.0, "automorph");
    }
}

template <typename F> static void ns_dispatch(int ns, F &&f)
{
    switch (ns) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: f(std::integral_constant<int, 9>{}); break;
    case 10: f(std::integral_constant<int, 10>{}); break;
    case 11: f(std::integral_constant<int, 11>{}); break;
    case 12: f(std::integral_constant<int, 12>{}); break;
    case 13: f(std::integral_constant<int, 13>{}); break;
    case 14: f(std::integral_constant<int, 14>{}); break;
    case 15: f(std::integral_constant<int, 15>{}); break;
    default: throw Error(SPFHE_EPARAM, "digit width out of range");
    }
}

void modup_bconv(Ctx &ctx, int items, int ell, const u64 *coef, long long coef_stride, u64 *ext,
                 long long ext_stride)
{
    const int beta = (ell + ctx.alpha - 1) / ctx.alpha;
    const int full = ell / ctx.alpha;            // digits of width alpha
    const int last = ell - full * ctx.alpha;     // width of a truncated last digit (0: none)
    auto launch = [&](int digit0, int ndig, int ns) {
        const size_t smem = (size_t)((ns + 4) & ~1) * ctx.M * sizeof(u64);
        const dim3 grid((ctx.n + kT - 1) / kT, ndig, items);
        cudaEvent_t t0_ = prof_begin(ctx);
        ns_dispatch(ns, [&](auto NS) {
            k_modup_bconv<decltype(NS)::value><<<grid, kT, smem, ctx.stream>>>(
                digit0, ell, ctx.L, ctx.K, ctx.alpha, ctx.M, ctx.n, coef, coef_stride, ext, ext_stride, ctx.dt.mc,
                ctx.dt.mu_hat_inv_n, ctx.dt.mu_hat_inv_n_p, ctx.dt.mu_hat_split, ctx.dt.mu_negd_split, ctx.dt.inv_q);
        });
        double macs = 0;
        for (int d = digit0; d < digit0 + ndig; ++d) macs += (double)ns * (ell + ctx.K - ns);
        prof_end(ctx, t0_, K_MODUP, 8.0 * ctx.n * items * ndig * (ell + ctx.K), macs * ctx.n * items, "modup bconv");
    };
    if (full > 0) launch(0, full, ctx.alpha);
    if (last > 0) launch(full, 1, last);
    (void)beta;
}

LimbMap modup_ntt_map(const Ctx &ctx, int ell)
{
    LimbMap m;
    m.nl = 0;
    const int beta = (ell + ctx.alpha - 1) / ctx.alpha;
    const int next = ell + ctx.K;
    for (int j = 0; j < beta; ++j) {
        const int lo = j * ctx.alpha, hi = std::min(lo + ctx.alpha, ell);
        for (int t = 0; t < next; ++t) {
            if (t >= lo && t < hi) continue;
            if (m.nl >= kMaxLimbSlots) throw Error(SPFHE_EPARAM, "too many extended limbs");
            m.off[m.nl] = j * next + t;
            m.mi[m.nl] = t < ell ? t : ctx.L + (t - ell);
            ++m.nl;
        }
    }
    return m;
}

void ks_inner_product(Ctx &ctx, int items, int ell, const u64 *const *in, const u64 *ext, long long ext_stride,
                      const std::vector<KeyGroup> &groups, u64 *acc, long long acc_stride, const int *src_of,
                      const int *perm_g)
{
    for (size_t g0 = 0; g0 < groups.size(); g0 += kMaxIpGroups) {
        const int cnt = (int)std::min<size_t>(kMaxIpGroups, groups.size() - g0);
        IpGroups hg;
        double ip_items = 0;
        for (int i = 0; i < cnt; ++i) {
            hg.g[i] = IpGroup{groups[g0 + i].key, groups[g0 + i].first, groups[g0 + i].count};
            ip_items += groups[g0 + i].count;
        }
        const double beta_ip = (ell + ctx.alpha - 1) / ctx.alpha;
        {
            cudaEvent_t t0_ = prof_begin(ctx);
            const dim3 grid = grid_n(ctx.n, ell + ctx.K, cnt);
#define SPFHE_IP(BB) k_ip<BB><<<grid, kT, 0, ctx.stream>>>(ell, ctx.L, ctx.K, ctx.alpha, ctx.M, ctx.n, in, ext, \
                                                           ext_stride, hg, acc, acc_stride, ctx.dt.mc)
            if (src_of)
                k_ip_hoisted<<<grid, kT, 0, ctx.stream>>>(ell, ctx.L, ctx.K, ctx.alpha, ctx.M, ctx.log_n, in, ext,
                                                          ext_stride, hg, acc, acc_stride, ctx.dt.mc, src_of, perm_g);
            else switch ((int)beta_ip) {
            case 1: SPFHE_IP(1); break;
            case 2: SPFHE_IP(2); break;
            case 3: SPFHE_IP(3); break;
            case 4: SPFHE_IP(4); break;
            case 5: SPFHE_IP(5); break;
            case 6: SPFHE_IP(6); break;
            default: SPFHE_IP(0); break;
            }
#undef SPFHE_IP
            prof_end(ctx, t0_, K_IP, 8.0 * ctx.n * (ip_items * (beta_ip * (ell + ctx.K) + 2.0 * (ell + ctx.K)) + cnt * 2.0 * beta_ip * (ell + ctx.K)), 2.0 * ctx.n * ip_items * beta_ip * (ell + ctx.K), "ks inner product");
        }
    }
    (void)items;
}

void moddown(Ctx &ctx, int items, int ell, u64 *acc, long long acc_stride, u64 *conv, const u64 *const *base,
             const int *base_g, bool base_c1, u64 *out, long long out_stride)
{
    moddown_conv(ctx, items, ell, acc, acc_stride, conv);
    LimbMap qm;
    qm.nl = 2 * ell;
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < ell; ++i) {
            qm.off[b * ell + i] = b * ell + i;
            qm.mi[b * ell + i] = i;
        }
    // the transform of conv writes ModDown's output directly where it can
    FuseArgs fa;
    fa.ell = ell;
    fa.K = ctx.K;
    fa.acc = acc;
    fa.acc_stride = acc_stride;
    fa.base = base;
    fa.base_g = base_g;
    fa.base_c1 = base_c1 ? 1 : 0;
    fa.out = out;
    fa.out_stride = out_stride;
    fa.pinv = ctx.dt.md_pinv;
    fa.pinvp = ctx.dt.md_pinv_p;
    if (ctx.fuse_epilogues && ntt_forward_fused(ctx, Batch{conv, 2LL * ell * ctx.n, items, nullptr}, qm, kFuseModDown, fa))
        return;
    ntt_forward(ctx, Batch{conv, 2LL * ell * ctx.n, items, nullptr}, qm);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_moddown_final<<<grid_n(ctx.n, 2 * ell, items), kT, 0, ctx.stream>>>(
            ell, ctx.K, ctx.log_n, acc, acc_stride, conv, base, base_g, base_c1 ? 1 : 0, out, out_stride, ctx.dt.mc,
            ctx.dt.md_pinv, ctx.dt.md_pinv_p);
        prof_end(ctx, t0_, K_MODDOWN_FINAL, 8.0 * ctx.n * items * ell * (base ? (base_c1 ? 8.0 : 7.0) : 6.0), 2.0 * ctx.n * items * ell, "moddown final");
    }
}

void moddown_conv(Ctx &ctx, int items, int ell, u64 *acc, long long acc_stride, u64 *conv)
{
    const int next = ell + ctx.K;
    // inverse NTT of the P limbs of both accumulators
    LimbMap pm;
    pm.nl = 2 * ctx.K;
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < ctx.K; ++k) {
            pm.off[b * ctx.K + k] = b * next + ell + k;
            pm.mi[b * ctx.K + k] = ctx.L + k;
        }
    // n^{-1} of this transform is folded into the conversion's constants
    ntt_inverse(ctx, Batch{acc, acc_stride, items, nullptr}, pm, false);
    const size_t smem = (size_t)((ctx.K + 4) & ~1) * ell * sizeof(u64);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        ns_dispatch(ctx.K, [&](auto KK) {
            k_moddown_bconv<decltype(KK)::value><<<grid_n(ctx.n, 2, items), kT, smem, ctx.stream>>>(
                ell, ctx.L, ctx.M, ctx.n, acc, acc_stride, conv, ctx.dt.mc, ctx.dt.md_hat_inv_n, ctx.dt.md_hat_inv_n_p,
                ctx.dt.md_hat_split, ctx.dt.md_negp_split, ctx.dt.inv_q);
        });
        prof_end(ctx, t0_, K_MODDOWN_BCONV, 16.0 * ctx.n * items * (ctx.K + ell), 2.0 * ctx.n * items * ctx.K * ell, "moddown bconv");
    }
}

void relin_top(Ctx &ctx, int items, int ell, const u64 *acc, long long acc_stride, const u64 *conv, u64 *top)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_relin_top<<<grid_n(ctx.n, 2, items), kT, 0, ctx.stream>>>(ell, ctx.K, ctx.n, acc, acc_stride, conv, top,
                                                                   ctx.dt.mc, ctx.dt.md_pinv, ctx.dt.md_pinv_p);
        prof_end(ctx, t0_, K_RESCALE, 32.0 * ctx.n * items * 2, 2.0 * ctx.n * items, "relinearised top limb");
    }
}

void copy_top(Ctx &ctx, int items, int ell, int polys, const u64 *const *in, u64 *top)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_copy_top<<<grid_n(ctx.n, polys, items), kT, 0, ctx.stream>>>(polys, ell, ctx.n, in, top);
        prof_end(ctx, t0_, K_RESCALE, 16.0 * ctx.n * items * polys, 0.0, "rescale copy");
    }
}

void rescale(Ctx &ctx, int items, int ell, const u64 *const *in, u64 *tmp, u64 *out, long long out_stride, int polys)
{
    if (ell < 2) throw Error(SPFHE_ELEVEL, "rescale needs two limbs");
    if (polys < 1 || polys > 3) throw Error(SPFHE_EINVAL, "rescale of 1 to 3 polynomials per item");
    const int n = ctx.n;
    // tmp layout: [items][polys][n] top limbs, then [items][polys][ell-1][n]
    u64 *top = tmp;
    u64 *spread = tmp + (size_t)items * polys * n;
    copy_top(ctx, items, ell, polys, in, top);
    LimbMap tm;
    tm.nl = polys;
    for (int b = 0; b < polys; ++b) {
        tm.off[b] = b;
        tm.mi[b] = ell - 1;
    }
    ntt_inverse(ctx, Batch{top, (long long)polys * n, items, nullptr}, tm);
    LimbMap sm;
    sm.nl = polys * (ell - 1);
    for (int b = 0; b < polys; ++b)
        for (int i = 0; i < ell - 1; ++i) {
            sm.off[b * (ell - 1) + i] = b * (ell - 1) + i;
            sm.mi[b * (ell - 1) + i] = i;
        }
    // the transform reads the top limbs and writes the rescaled output where it can
    FuseArgs fa;
    fa.ell = ell;
    fa.polys = polys;
    fa.top = top;
    fa.in = in;
    fa.out = out;
    fa.out_stride = out_stride;
    fa.qt_mod = ctx.dt.rs_qt + (size_t)(ell - 1) * ctx.L;
    fa.inv = ctx.dt.rs_inv + (size_t)(ell - 1) * ctx.L;
    fa.invp = ctx.dt.rs_inv_p + (size_t)(ell - 1) * ctx.L;
    if (ctx.fuse_epilogues && ell >= 2 &&
        ntt_forward_fused(ctx, Batch{spread, (long long)polys * (ell - 1) * n, items, nullptr}, sm, kFuseRescale, fa))
        return;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_rescale_spread<<<grid_n(n, polys * (ell - 1), items), kT, 0, ctx.stream>>>(
            polys, ell, n, top, spread, ctx.dt.mc, ctx.dt.rs_qt + (size_t)(ell - 1) * ctx.L);
        prof_end(ctx, t0_, K_RESCALE, 8.0 * n * items * polys * ell, 1.0 * n * items * polys * (ell - 1), "rescale spread");
    }
    ntt_forward(ctx, Batch{spread, (long long)polys * (ell - 1) * n, items, nullptr}, sm);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_rescale_final<<<grid_n(n, polys * (ell - 1), items), kT, 0, ctx.stream>>>(
            polys, ell, n, in, spread, out, out_stride, ctx.dt.mc, ctx.dt.rs_inv + (size_t)(ell - 1) * ctx.L,
            ctx.dt.rs_inv_p + (size_t)(ell - 1) * ctx.L);
        prof_end(ctx, t0_, K_RESCALE, 24.0 * n * items * polys * (ell - 1), 1.0 * n * items * polys * (ell - 1), "rescale final");
    }
}

void mul_plain_perm(Ctx &ctx, int items, int ell, u64 *ct, long long stride, const u64 *const *mask, const int *g,
                    int polys)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_mul_plain_perm<<<grid_n(ctx.n, polys * ell, items), kT, 0, ctx.stream>>>(ell, ctx.log_n, ct, stride, mask,
                                                                                  g, ctx.dt.mc);
        prof_end(ctx, t0_, K_MASK, 8.0 * ctx.n * (2.0 * polys * items * ell + ell), 1.0 * ctx.n * polys * items * ell, "mask multiply");
    }
}

void accumulate_seg(Ctx &ctx, int polys, int ell, int targets, u64 *const *tgt, const u64 *const *src,
                    const int *seg, int sources, bool into)
{
    if (targets <= 0) return;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_accumulate_seg<<<grid_n(ctx.n, polys * ell, targets), kT, 0, ctx.stream>>>(polys * ell, ell, ctx.n, tgt, src,
                                                                                   seg, into ? 1 : 0, ctx.dt.mc);
        prof_end(ctx, t0_, K_ACCUM, 8.0 * ctx.n * polys * ell * (sources + (into ? 2.0 : 1.0) * targets), 1.0 * ctx.n * polys * ell * sources, "segmented accumulate");
    }
}

void accumulate(Ctx &ctx, int ell, u64 *result, const u64 *x, long long stride, const int *ids, int count)
{
    if (count <= 0) return;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_accumulate<<<grid_n(ctx.n, 2 * ell, 1), kT, 0, ctx.stream>>>(ell, ctx.n, result, x, stride, ids, count,
                                                                       ctx.dt.mc);
        prof_end(ctx, t0_, K_ACCUM, 16.0 * ctx.n * ell * (count + 2.0), 2.0 * ctx.n * ell * count, "accumulate");
    }
}

void add_ct(Ctx &ctx, int polys, int ell, const u64 *a, const u64 *b, u64 *out)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_add<<<grid_n(ctx.n, polys * ell, 1), kT, 0, ctx.stream>>>(polys, ell, ctx.n, a, b, out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 24.0 * ctx.n * polys * ell, 0.0, "add");
    }
}

void mul_ct_pt(Ctx &ctx, int ell, const u64 *ct, const u64 *pt, u64 *out)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_mul_ct_pt<<<grid_n(ctx.n, 2 * ell, 1), kT, 0, ctx.stream>>>(ell, ctx.n, ct, pt, out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 40.0 * ctx.n * ell, 2.0 * ctx.n * ell, "mul ct pt");
    }
}

void to_montgomery(Ctx &ctx, u64 *x, int limbs, const int *mi_host, int reps)
{
    MiList ml;
    for (int l = 0; l < limbs; ++l) ml.mi[l] = mi_host[l];
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_to_mont<<<grid_n(ctx.n, limbs, reps), kT, 0, ctx.stream>>>(ctx.n, x, ml, limbs, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 16.0 * ctx.n * limbs * reps, 1.0 * ctx.n * limbs * reps, "to montgomery");
    }
}

void from_montgomery(Ctx &ctx, u64 *x, int limbs, const int *mi_host, int reps)
{
    MiList ml;
    for (int l = 0; l < limbs; ++l) ml.mi[l] = mi_host[l];
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_from_mont<<<grid_n(ctx.n, limbs, reps), kT, 0, ctx.stream>>>(ctx.n, x, ml, limbs, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 16.0 * ctx.n * limbs * reps, 1.0 * ctx.n * limbs * reps, "from montgomery");
    }
}

void from_signed(Ctx &ctx, const long long *coef, u64 *out, int limbs)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_from_signed<<<grid_n(ctx.n, limbs, 1), kT, 0, ctx.stream>>>(ctx.n, coef, out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 8.0 * ctx.n * (limbs + 1), 0.0, "from signed");
    }
}

void decrypt_core(Ctx &ctx, int ell, const u64 *ct, const u64 *s_mont, u64 *out)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_decrypt<<<grid_n(ctx.n, ell, 1), kT, 0, ctx.stream>>>(ell, ctx.n, ct, s_mont, out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 32.0 * ctx.n * ell, 1.0 * ctx.n * ell, "decrypt");
    }
}

void gather_items(Ctx &ctx, int items, size_t words_per_item, const u64 *const *in, u64 *out, long long stride)
{
    if (items <= 0) return;
    const int blocks = (int)std::min<size_t>(1024, (words_per_item + kT - 1) / kT);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_gather<<<dim3(blocks, items), kT, 0, ctx.stream>>>((int)words_per_item, in, out, stride);
        prof_end(ctx, t0_, K_OTHER, 16.0 * words_per_item * items, 0.0, "gather");
    }
}

void scatter_items(Ctx &ctx, int items, size_t words_per_item, const u64 *src, long long stride, u64 *const *out)
{
    if (items <= 0) return;
    const int blocks = (int)std::min<size_t>(1024, (words_per_item + kT - 1) / kT);
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_scatter<<<dim3(blocks, items), kT, 0, ctx.stream>>>((int)words_per_item, src, stride, out);
        prof_end(ctx, t0_, K_OTHER, 16.0 * words_per_item * items, 0.0, "scatter");
    }
}

void mul_poly(Ctx &ctx, int limbs, const u64 *a, const u64 *b, u64 *out)
{
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_mul_poly<<<grid_n(ctx.n, limbs, 1), kT, 0, ctx.stream>>>(ctx.n, a, b, out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 24.0 * ctx.n * limbs, 1.0 * ctx.n * limbs, "mul poly");
    }
}

void copy_words(Ctx &ctx, u64 *dst, const u64 *src, size_t words)
{
    SPFHE_CHECK_CUDA(cudaMemcpyAsync(dst, src, words * sizeof(u64), cudaMemcpyDeviceToDevice, ctx.stream));
}

void sample_uniform(Ctx &ctx, u64 *out, int limbs, const int *mi_host, uint64_t seed, uint64_t stream_id)
{
    MiList ml;
    for (int l = 0; l < limbs; ++l) ml.mi[l] = mi_host[l];
    const int groups = (ctx.n + 3) / 4;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_sample_uniform<<<dim3((groups + kT - 1) / kT, limbs, 1), kT, 0, ctx.stream>>>(ctx.n, out, ml, seed, stream_id,
                                                                                        ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 8.0 * ctx.n * limbs, 0.0, "sample uniform");
    }
}

void sample_ternary(Ctx &ctx, long long *out, uint64_t seed, uint64_t stream_id)
{
    const int groups = (ctx.n + 7) / 8;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_sample_ternary<<<(groups + kT - 1) / kT, kT, 0, ctx.stream>>>(ctx.n, out, seed, stream_id);
        prof_end(ctx, t0_, K_OTHER, 8.0 * ctx.n, 0.0, "sample ternary");
    }
}

void sample_gaussian(Ctx &ctx, long long *out, uint64_t seed, uint64_t stream_id)
{
    const int groups = (ctx.n + 7) / 8;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_sample_gaussian<<<(groups + kT - 1) / kT, kT, 0, ctx.stream>>>(ctx.n, out, seed, stream_id);
        prof_end(ctx, t0_, K_OTHER, 8.0 * ctx.n, 0.0, "sample gaussian");
    }
}

void rlwe_b(Ctx &ctx, int limbs, const int *mi_host, const u64 *a, const u64 *s_mont, const u64 *e, const u64 *extra,
            u64 *out)
{
    MiList ml;
    for (int l = 0; l < limbs; ++l) ml.mi[l] = mi_host[l];
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_rlwe_b<<<grid_n(ctx.n, limbs, 1), kT, 0, ctx.stream>>>(ctx.n, ml, a, s_mont, e, extra, out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 40.0 * ctx.n * limbs, 1.0 * ctx.n * limbs, "rlwe");
    }
}

void add_gadget(Ctx &ctx, u64 *out, const u64 *sprime, int lo, int hi)
{
    // gadget of digit [lo, hi): P mod q_i on its limbs
    GadgetConsts gc;
    for (int i = lo; i < hi; ++i) {
        u64 P = 1;
        for (int k = 0; k < ctx.K; ++k) P = mulmod_host(P, ctx.mods[ctx.L + k] % ctx.mods[i], ctx.mods[i]);
        gc.p[i - lo] = P;
        gc.pp[i - lo] = shoup_pre(P, ctx.mods[i]);
    }
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_add_gadget<<<grid_n(ctx.n, hi - lo, 1), kT, 0, ctx.stream>>>(ctx.n, out, sprime, lo, gc, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 24.0 * ctx.n * (hi - lo), 1.0 * ctx.n * (hi - lo), "gadget");
    }
}

}  // namespace spfhe
