// Measured arithmetic speed of light for the ALU-bound kernels.
//
// The transforms and base conversions are bound by 64-bit modular
// multiplication on the INT32 multiply pipe, so their roofline is an ALU
// rate, not a bandwidth.  These microbenchmarks measure that rate on the GPU
// at hand, with the launch shape of the transforms (4 CTAs of 256 threads per
// SM) and no memory traffic beyond one store per thread:
//   * lazy forward butterflies (a, b) -> (a + w b, a - w b + Bq) on 8
//     register-resident values per thread, three stages per round, with each
//     of the transforms' truncated-quotient Shoup products: five 64-bit-result
//     multiplies (mul_shoup3), their split halves (mul_shoup3s), and the
//     shorter quotient (mul_shoup4s, B = 4);
//   * independent chains of 32-bit multiply-adds with a 32-bit result
//     (mad.lo.u32), with a 64-bit result (mad.wide.u32), and of high-half
//     multiply-adds (mad.hi.u32).
// Every launch runs a fixed number of rounds and touches only its own output
// word, so it always ends and stays in bounds.
#include "handles.h"
#include "kernels.h"

namespace spfhe {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;
constexpr int kPeakWaves = 4;
// butterfly benchmark: 8 values per thread, 3 stages (12 butterflies) per round
constexpr int kBflyVals = 8;
constexpr int kBflyStages = 3;

template <int AR>
__global__ void __launch_bounds__(kPeakThreads, kPeakCtasPerSm)
    k_peak_bfly(const u64 *__restrict__ seed, int rounds, u64 *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = seed[0], w = seed[1] + (u64)t, wp = seed[2] ^ (u64)t;
    const u64 nq = 0 - q, qb = shoup_bound<AR>() * q;
    u64 v[kBflyVals];
#pragma unroll
    for (int i = 0; i < kBflyVals; ++i) v[i] = seed[3] + (u64)t * kBflyVals + (u64)i;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int l = 0; l < kBflyStages; ++l) {
            const int half = (kBflyVals / 2) >> l;
#pragma unroll
            for (int i = 0; i < kBflyVals; ++i) {
                if (i & half) continue;
                const u64 x = v[i];
                const u64 y = mul_shoup_ar<AR>(v[i + half], w, wp, nq);
                v[i] = x + y;
                v[i + half] = x - y + qb;
            }
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < kBflyVals; ++i) acc ^= v[i];
    out[t] = acc;
}

__global__ void __launch_bounds__(kPeakThreads, kPeakCtasPerSm)
    k_peak_imad(const u64 *__restrict__ seed, int rounds, u64 *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = (uint32_t)seed[0] | 1u, c = (uint32_t)seed[1];
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (uint32_t)seed[3] + (uint32_t)(t * 8 + i);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int i = 0; i < 8; ++i) asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(m), "r"(c));
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i];
    out[t] = acc;
}

__global__ void __launch_bounds__(kPeakThreads, kPeakCtasPerSm)
    k_peak_imad_wide(const u64 *__restrict__ seed, int rounds, u64 *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = (uint32_t)seed[0] | 1u;
    u64 a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed[3] + (u64)(t * 8 + i);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            // a = hi32(a) * m + a: each step's multiplicand depends on the last
            const uint32_t x = (uint32_t)(a[i] >> 32);
            asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a[i]) : "r"(x), "r"(m));
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i];
    out[t] = acc;
}

__global__ void __launch_bounds__(kPeakThreads, kPeakCtasPerSm)
    k_peak_imad_hi(const u64 *__restrict__ seed, int rounds, u64 *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = (uint32_t)seed[0] | 0x80000001u, c = (uint32_t)seed[1] | 1u;
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (uint32_t)seed[3] + (uint32_t)(t * 8 + i) | 0x80000000u;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int i = 0; i < 8; ++i) asm("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(m), "r"(c));
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i];
    out[t] = acc;
}

// Device time of one launch of `launch` (after one untimed warm-up launch).
template <typename F> double time_launch(Ctx &ctx, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    SPFHE_CHECK_CUDA(cudaEventCreate(&a));
    const cudaError_t eb = cudaEventCreate(&b);
    if (eb != cudaSuccess) {
        cudaEventDestroy(a);
        throw Error(SPFHE_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(eb));
    }
    float ms = 0;
    cudaError_t e = cudaSuccess;
    launch();
    if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventRecord(a, ctx.stream)) == cudaSuccess) {
        launch();
        if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventRecord(b, ctx.stream)) == cudaSuccess &&
            (e = cudaEventSynchronize(b)) == cudaSuccess)
            e = cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) throw Error(SPFHE_ECUDA, std::string("ALU microbenchmark: ") + cudaGetErrorString(e));
    ctx.launches += 2;
    return ms * 1e-3;
}

}  // namespace
}  // namespace spfhe

using namespace spfhe;

// rates[0..2]: butterflies/s with mul_shoup3, mul_shoup3s, mul_shoup4s;
// rates[3..5]: mad.lo.u32, mad.wide.u32, mad.hi.u32 per second
static void alu_rates(Ctx &c, double rates[6])
{
    if (c.cap) throw Error(SPFHE_EINVAL, "not available during graph capture");
    SPFHE_CHECK_CUDA(cudaSetDevice(c.device));
    int sms = 0;
    SPFHE_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    const int blocks = sms * kPeakCtasPerSm * kPeakWaves;
    const size_t threads = (size_t)blocks * kPeakThreads;
    // the first modulus and a twiddle of it; the values only feed the arithmetic
    const u64 q = c.mods[0];
    const u64 w = q / 3 + 1;
    const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
    const u64 seed_h[4] = {q, w, wp, 12345};
    u64 *seed = static_cast<u64 *>(dev_alloc(c, sizeof(seed_h)));
    u64 *out = nullptr;
    try {
        out = static_cast<u64 *>(dev_alloc(c, threads * sizeof(u64)));
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(seed, seed_h, sizeof(seed_h), cudaMemcpyHostToDevice, c.stream));
        const int rb = 512, ri = 4096;
        const double t_b0 = time_launch(c, [&] { k_peak_bfly<0><<<blocks, kPeakThreads, 0, c.stream>>>(seed, rb, out); });
        const double t_b1 = time_launch(c, [&] { k_peak_bfly<1><<<blocks, kPeakThreads, 0, c.stream>>>(seed, rb, out); });
        const double t_b2 = time_launch(c, [&] { k_peak_bfly<2><<<blocks, kPeakThreads, 0, c.stream>>>(seed, rb, out); });
        const double t_i = time_launch(c, [&] { k_peak_imad<<<blocks, kPeakThreads, 0, c.stream>>>(seed, ri, out); });
        const double t_w = time_launch(c, [&] { k_peak_imad_wide<<<blocks, kPeakThreads, 0, c.stream>>>(seed, ri, out); });
        const double t_h = time_launch(c, [&] { k_peak_imad_hi<<<blocks, kPeakThreads, 0, c.stream>>>(seed, ri, out); });
        const double bflies = (double)threads * rb * kBflyStages * (kBflyVals / 2);
        const double mads = (double)threads * ri * 8;
        rates[0] = bflies / t_b0;
        rates[1] = bflies / t_b1;
        rates[2] = bflies / t_b2;
        rates[3] = mads / t_i;
        rates[4] = mads / t_w;
        rates[5] = mads / t_h;
    } catch (...) {
        dev_free(c, out);
        dev_free(c, seed);
        throw;
    }
    dev_free(c, out);
    dev_free(c, seed);
    SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
}

extern "C" spfhe_status spfhe_prof_alu_peak(spfhe_ctx *ctx, double *butterflies_per_s,
                                            double *butterflies_split_per_s, double *imad_per_s,
                                            double *imad_wide_per_s)
{
    try {
        if (!ctx) throw Error(SPFHE_EINVAL, "null argument");
        double r[6];
        alu_rates(ctx->c, r);
        if (butterflies_per_s) *butterflies_per_s = r[0];
        if (butterflies_split_per_s) *butterflies_split_per_s = r[1];
        if (imad_per_s) *imad_per_s = r[3];
        if (imad_wide_per_s) *imad_wide_per_s = r[4];
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return SPFHE_EINVAL;
    }
}

extern "C" spfhe_status spfhe_prof_alu_rates(spfhe_ctx *ctx, double *rates, size_t n)
{
    try {
        if (!ctx || !rates || n < 6) throw Error(SPFHE_EINVAL, "null argument or fewer than 6 rates");
        alu_rates(ctx->c, rates);
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return SPFHE_EINVAL;
    }
}
