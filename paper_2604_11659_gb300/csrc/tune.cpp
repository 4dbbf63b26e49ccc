// Tuners.
//
// Rotation-plan base: for a product's Alg. 1 plan, the number of key
// switches its rotations need depends on the base b of the rotation plan
// (one key switch per nonzero base-b digit of each amount), and the key
// memory on the number of keys (every d*b^t < S, 1 <= d < b).  The tuner
// counts both for every power-of-two base and returns the base with the
// fewest key switches whose keys fit the budget.
//
// NTT launch chunk: times the key-switching transforms of one match batch
// (forward NTT of the ModUp extension, inverse NTT of the input limbs) on
// scratch buffers for every candidate chunk and keeps the fastest.
#include "engine.h"
#include "handles.h"
#include "kernels.h"

namespace spfhe {

static uint64_t plan_len(long long r, long long S, long long b)
{
    long long x = ((r % S) + S) % S;
    uint64_t c = 0;
    while (x) {
        if (x % b) ++c;
        x /= b;
    }
    return c;
}

static uint64_t key_count(long long S, long long b)
{
    uint64_t c = 0;
    for (long long w = 1; w < S; w *= b)
        for (long long d = 1; d < b; ++d)
            if (d * w < S) ++c;
    return c;
}

}  // namespace spfhe

using namespace spfhe;

extern "C" spfhe_status spfhe_tune_rotation_base(uint32_t log_n, uint32_t L, uint32_t K, uint32_t dnum,
                                                 const spfhe_sparse_meta *A_csr, const spfhe_sparse_meta *B_csc,
                                                 uint64_t key_budget_bytes, uint32_t *base, uint64_t *key_switches,
                                                 uint64_t *key_bytes)
{
    try {
        if (!A_csr || !B_csc || !base) throw Error(SPFHE_EINVAL, "null argument");
        if (log_n < 2 || log_n > 17 || L < 1 || K < 1 || dnum < 1) throw Error(SPFHE_EINVAL, "bad parameters");
        validate_pair(*A_csr, *B_csc);
        const long long S = 1LL << (log_n - 1);
        const std::vector<MatchRec> ms = plan_alg1(*A_csr, *B_csc);
        // rotation amounts of the plan: distinct alignments and every final rotation
        std::map<std::tuple<int, int, long long>, int> align;
        std::vector<long long> finals;
        for (const MatchRec &m : ms) {
            const long long sa = m.a_pos % S, sb = m.b_pos % S;
            if (sa < sb) align[std::make_tuple(1, (int)(m.b_pos / S), sb - sa)] = 1;
            if (sb < sa) align[std::make_tuple(0, (int)(m.a_pos / S), sa - sb)] = 1;
            const long long t = (long long)m.i * B_csc->cols + m.j;
            finals.push_back(((std::min(sa, sb) - t % S) % S + S) % S);
        }
        const uint64_t per_key = (uint64_t)dnum * 2 * (L + K) * (1ull << log_n) * sizeof(u64);
        uint32_t best = 0;
        uint64_t best_ks = ~0ull, best_bytes = 0;
        for (long long b = 2; b <= S; b *= 2) {
            const uint64_t bytes = key_count(S, b) * per_key;
            if (bytes > key_budget_bytes) continue;
            uint64_t ks = 0;
            for (auto &kv : align) ks += plan_len(std::get<2>(kv.first), S, b);
            for (long long r : finals) ks += plan_len(r, S, b);
            if (ks < best_ks || (ks == best_ks && bytes < best_bytes)) {
                best = (uint32_t)b;
                best_ks = ks;
                best_bytes = bytes;
            }
        }
        if (!best) throw Error(SPFHE_ENOMEM, "no rotation base fits the key budget");
        *base = best;
        if (key_switches) *key_switches = best_ks;
        if (key_bytes) *key_bytes = best_bytes;
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}

extern "C" spfhe_status spfhe_tune_ntt_chunk(spfhe_ctx *ctx, uint32_t ell, uint32_t items, const uint32_t *candidates,
                                            uint32_t n_candidates, uint32_t *best, double *ms)
{
    try {
        if (!ctx || !candidates || !best || n_candidates == 0) throw Error(SPFHE_EINVAL, "null argument");
        Ctx &c = ctx->c;
        if (ell < 1 || (int)ell > c.L || items < 1 || items > 1024) throw Error(SPFHE_EINVAL, "bad shape");
        const int beta = ((int)ell + c.alpha - 1) / c.alpha;
        const int next = (int)ell + c.K;
        const size_t ext_words = (size_t)items * beta * next * c.n;
        const size_t in_words = (size_t)items * ell * c.n;
        Scratch sc(c);
        u64 *ext = sc.words(ext_words);
        u64 *in = sc.words(in_words);
        SPFHE_CHECK_CUDA(cudaMemsetAsync(ext, 0, ext_words * sizeof(u64), c.stream));
        SPFHE_CHECK_CUDA(cudaMemsetAsync(in, 0, in_words * sizeof(u64), c.stream));
        const LimbMap fm = modup_ntt_map(c, (int)ell);
        const LimbMap im = limb_range(0, (int)ell, 0);
        const Batch fb{ext, (long long)beta * next * c.n, (int)items, nullptr};
        const Batch ib{in, (long long)ell * c.n, (int)items, nullptr};
        const int saved = c.ntt_chunk;
        const bool saved_ks = c.in_keyswitch;
        c.in_keyswitch = true;
        cudaEvent_t e0, e1;
        SPFHE_CHECK_CUDA(cudaEventCreate(&e0));
        SPFHE_CHECK_CUDA(cudaEventCreate(&e1));
        float best_ms = 0;
        uint32_t best_c = 0;
        try {
            for (uint32_t k = 0; k < n_candidates; ++k) {
                if (candidates[k] > (1u << 20)) throw Error(SPFHE_EINVAL, "chunk out of range");
                c.ntt_chunk = (int)candidates[k];
                ntt_forward(c, fb, fm);   // warm-up
                ntt_inverse(c, ib, im);
                SPFHE_CHECK_CUDA(cudaEventRecord(e0, c.stream));
                for (int r = 0; r < 3; ++r) {
                    ntt_forward(c, fb, fm);
                    ntt_inverse(c, ib, im);
                }
                SPFHE_CHECK_CUDA(cudaEventRecord(e1, c.stream));
                SPFHE_CHECK_CUDA(cudaEventSynchronize(e1));
                float t = 0;
                SPFHE_CHECK_CUDA(cudaEventElapsedTime(&t, e0, e1));
                t /= 3;
                if (ms) ms[k] = t;
                if (k == 0 || t < best_ms) {
                    best_ms = t;
                    best_c = candidates[k];
                }
            }
        } catch (...) {
            c.ntt_chunk = saved;
            c.in_keyswitch = saved_ks;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c.in_keyswitch = saved_ks;
        c.ntt_chunk = (int)best_c;
        *best = best_c;
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}
