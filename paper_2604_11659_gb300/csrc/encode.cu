// Canonical-embedding encoding and decoding (host FFT; boundary code, not on
// the timed path) and the device encoder of one-hot plaintexts used for the
// masks of Alg. 2 and the weight plaintexts of the ct x pt product.
//
// Slot i <-> evaluation at zeta^(5^i), zeta = e^(i pi / n).  Encoding of a
// slot vector z: m_j = round_half_away((2 scale / n) Re sum_i z_i zeta^(-5^i j)).
// For z = v e_0 this is round_half_away(v (2 scale / n) cos(pi j / n)); the
// encoding of v e_p is the automorphism X -> X^(5^-p) of it (exactly, since
// the rounding is symmetric and cos(x + pi) = -cos x).
#include <cmath>
#include <complex>

#include "runtime.h"

namespace spfhe {

typedef std::complex<double> cplx;

// in-place radix-2 DFT, sign -1: F[j] = sum_k v[k] e^(-2 pi i k j / n); sign +1 flips the exponent
static void fft(std::vector<cplx> &a, int sign)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = sign * 2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const cplx w = std::polar(1.0, ang * (double)k);
                const cplx u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

static std::vector<long long> slot_exponents(const Ctx &ctx)
{
    std::vector<long long> e(ctx.S);
    long long g = 1;
    for (int i = 0; i < ctx.S; ++i) {
        e[i] = g;
        g = (g * 5) % (2LL * ctx.n);
    }
    return e;
}

static double round_half_away(double x) { return x < 0 ? -std::floor(-x + 0.5) : std::floor(x + 0.5); }

std::vector<long long> encode_host(const Ctx &ctx, const double *re, const double *im, size_t nv, double scale)
{
    const int n = ctx.n;
    if (nv > (size_t)ctx.S) throw Error(SPFHE_EINVAL, "more values than slots");
    std::vector<long long> ex = slot_exponents(ctx);
    std::vector<cplx> v(n, cplx(0, 0));
    for (size_t i = 0; i < nv; ++i) {
        const cplx z(re[i], im ? im[i] : 0.0);
        v[(ex[i] - 1) / 2] = z;
        v[(2LL * n - ex[i] - 1) / 2] = std::conj(z);
    }
    fft(v, -1);
    std::vector<long long> m(n);
    for (int j = 0; j < n; ++j) {
        const cplx zm = std::polar(1.0, -M_PI * (double)j / (double)n);
        const double x = (scale / n) * (zm * v[j]).real();
        const double r = round_half_away(x);
        if (!(std::fabs(r) < 4.6e18)) throw Error(SPFHE_EINVAL, "encoded coefficient exceeds 2^62");
        m[j] = (long long)r;
    }
    return m;
}

void decode_host(const Ctx &ctx, const std::vector<u64> &limb0, double scale, double *re, double *im, size_t nv)
{
    const int n = ctx.n;
    const u64 q0 = ctx.mods[0];
    std::vector<cplx> w(n);
    for (int j = 0; j < n; ++j) {
        const u64 c = limb0[j];
        const double cv = c > q0 / 2 ? -(double)(q0 - c) : (double)c;
        w[j] = cv * std::polar(1.0, M_PI * (double)j / (double)n);
    }
    fft(w, +1);
    std::vector<long long> ex = slot_exponents(ctx);
    for (size_t i = 0; i < nv && i < (size_t)ctx.S; ++i) {
        const cplx z = w[(ex[i] - 1) / 2] / scale;
        re[i] = z.real();
        if (im) im[i] = z.imag();
    }
}

void ensure_cos_table(Ctx &ctx)
{
    if (ctx.cos_tab) return;
    std::vector<double> t(ctx.n);
    for (int j = 0; j < ctx.n; ++j) t[j] = std::cos(M_PI * j / ctx.n);
    SPFHE_CHECK_CUDA(cudaMalloc(&ctx.cos_tab, ctx.n * sizeof(double)));
    SPFHE_CHECK_CUDA(cudaMemcpy(ctx.cos_tab, t.data(), ctx.n * sizeof(double), cudaMemcpyHostToDevice));
}

namespace {
__global__ void k_onehot0(int n, int ell, const double *vals, double c, const double *cos_tab, u64 *out,
                          const ModConst *__restrict__ mc)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int l = blockIdx.y, it = blockIdx.z;
    const double x = (vals[it] * c) * cos_tab[j];
    const double ax = floor(fabs(x) + 0.5);
    const ModConst m = mc[l];
    const u64 a = (u64)ax;
    u64 r = mul_shoup(redc(U128{a, 0}, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
    if (x < 0) r = neg_mod(r, m.q);
    out[((size_t)it * ell + l) * n + j] = r;
}
// Coefficient-domain sums of one-hot encodings: segment s (blockIdx.z) of
// items c = seg[s] .. seg[s+1]-1 gets sum_c sigma_{g_c}(m0(v_c))_j, where
// m0(v) is k_onehot0's slot-0 encoding of v and sigma_g the automorphism
// X -> X^g (coefficient i goes to i g mod 2n, negated past n), i.e. the
// encoding of v_c at slot p_c for g_c = 5^-p_c.  ginv[c] = g_c^{-1} mod 2n.
// The integer sum is exact; then its residue for every limb.
__global__ void k_onehot_sum(int log_n, int ell, const int *seg, const double *vals, const int *ginv, double c,
                             const double *cos_tab, u64 *out, const ModConst *__restrict__ mc)
{
    const int n = 1 << log_n;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int s = blockIdx.z;
    long long acc = 0;
    for (int it = seg[s]; it < seg[s + 1]; ++it) {
        const unsigned i0 = (unsigned)(((unsigned long long)j * (unsigned)ginv[it]) & ((2ull << log_n) - 1));
        const bool neg = i0 >= (unsigned)n;
        const unsigned i = neg ? i0 - n : i0;
        const double x = (vals[it] * c) * cos_tab[i];
        long long a = (long long)floor(fabs(x) + 0.5);
        if ((x < 0) != neg) a = -a;
        acc += a;
    }
    const u64 mag = (u64)(acc < 0 ? -acc : acc);
    for (int l = 0; l < ell; ++l) {
        const ModConst m = mc[l];
        u64 r = mul_shoup(redc(U128{mag, 0}, m.q, m.qneg_inv), m.r_mod, m.r_mod_p, m.q);
        if (acc < 0) r = neg_mod(r, m.q);
        out[((size_t)s * ell + l) * n + j] = r;
    }
}
}  // namespace

void encode_onehot_sums(Ctx &ctx, int segments, const int *d_seg, const double *d_values, const int *d_ginv, int ell,
                        double scale, u64 *out)
{
    ensure_cos_table(ctx);
    const double c = 2.0 * scale / ctx.n;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_onehot_sum<<<dim3((ctx.n + 255) / 256, 1, segments), 256, 0, ctx.stream>>>(ctx.log_n, ell, d_seg, d_values,
                                                                                    d_ginv, c, ctx.cos_tab, out,
                                                                                    ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 8.0 * ctx.n * ell * segments, 0.0, "one-hot sums");
    }
    ntt_forward(ctx, Batch{out, (long long)ell * ctx.n, segments, nullptr}, limb_range(0, ell, 0));
}

void encode_onehot0(Ctx &ctx, const double *d_values, int items, int ell, double scale, u64 *out)
{
    ensure_cos_table(ctx);
    const double c = 2.0 * scale / ctx.n;
    {
        cudaEvent_t t0_ = prof_begin(ctx);
        k_onehot0<<<dim3((ctx.n + 255) / 256, ell, items), 256, 0, ctx.stream>>>(ctx.n, ell, d_values, c, ctx.cos_tab,
                                                                                  out, ctx.dt.mc);
        prof_end(ctx, t0_, K_OTHER, 8.0 * ctx.n * (1.0 + ell * items), 0.0, "onehot encode");
    }
    ntt_forward(ctx, Batch{out, (long long)ell * ctx.n, items, nullptr}, limb_range(0, ell, 0));
}

}  // namespace spfhe
