// Batched CKKS evaluator: hybrid key switching, rotations through the
// rotation plan, key generation and encryption, all sequenced on the
// context's stream.
#include <algorithm>
#include <numeric>

#include "runtime.h"

namespace spfhe {

static int beta_of(const Ctx &ctx, int ell) { return (ell + ctx.alpha - 1) / ctx.alpha; }

void keyswitch_batch(Ctx &ctx, int items, int ell, const u64 *const *d_in, const std::vector<KeyGroup> &groups,
                     const u64 *const *d_base, const int *d_base_g, bool base_c1, u64 *out, long long out_stride)
{
    if (items <= 0) return;
    Runtime &rt = *ctx.rt;
    const size_t n = ctx.n;
    const int next = ell + ctx.K, beta = beta_of(ctx, ell);
    const long long coef_stride = (long long)ell * n;
    const long long ext_stride = (long long)beta * next * n;
    const long long acc_stride = 2LL * next * n;
    u64 *coef = rt.workspace(WS_KS_COEF, (size_t)items * coef_stride);
    u64 *ext = rt.workspace(WS_KS_EXT, (size_t)items * ext_stride);
    u64 *acc = rt.workspace(WS_KS_ACC, (size_t)items * acc_stride);
    u64 *conv = rt.workspace(WS_KS_CONV, (size_t)items * 2 * ell * n);
    struct InKs {
        Ctx &c;
        explicit InKs(Ctx &x) : c(x) { ++c.in_keyswitch; }
        ~InKs() { --c.in_keyswitch; }
    } in_ks(ctx);
    ctx.prof.ks_calls += items;
    ctx.prof.ks_bytes += 8.0 * n * (3.0 * ell * items + 2.0 * beta * next * groups.size());
    // ModUp: coefficient representation of every input limb, then one base
    // conversion per digit and forward transforms of the new limbs
    gather_items(ctx, items, (size_t)coef_stride, d_in, coef, coef_stride);
    // n^{-1} of this transform is folded into the ModUp conversion's constants
    ntt_inverse(ctx, Batch{coef, coef_stride, items, nullptr}, limb_range(0, ell, 0), false);
    modup_bconv(ctx, items, ell, coef, coef_stride, ext, ext_stride);
    ntt_forward(ctx, Batch{ext, ext_stride, items, nullptr}, modup_ntt_map(ctx, ell));
    ks_inner_product(ctx, items, ell, d_in, ext, ext_stride, groups, acc, acc_stride);
    moddown(ctx, items, ell, acc, acc_stride, conv, d_base, d_base_g, base_c1, out, out_stride);
}

void rotate_hoisted(Ctx &ctx, const Keys &keys, int ell, const u64 *src, const std::vector<int> &amounts, u64 *out)
{
    const int total = (int)amounts.size();
    if (!total) return;
    Runtime &rt = *ctx.rt;
    const size_t n = ctx.n;
    const int next = ell + ctx.K, beta = beta_of(ctx, ell);
    const long long pstride = (long long)ell * n, cstride = 2 * pstride;
    const long long ext_stride = (long long)beta * next * n;
    const long long acc_stride = 2LL * next * n;
    for (int a : amounts) rotation_key(keys, a);   // EKEY before any launch
    struct InKs {
        Ctx &c;
        explicit InKs(Ctx &x) : c(x) { ++c.in_keyswitch; }
        ~InKs() { --c.in_keyswitch; }
    } in_ks(ctx);
    // ModUp of the source's c1, once
    u64 *coef = rt.workspace(WS_KS_COEF, (size_t)pstride);
    u64 *ext = rt.workspace(WS_HOIST_EXT, (size_t)ext_stride);
    const u64 *c1 = src + pstride;
    copy_words(ctx, coef, c1, (size_t)pstride);
    ntt_inverse(ctx, Batch{coef, pstride, 1, nullptr}, limb_range(0, ell, 0), false);
    modup_bconv(ctx, 1, ell, coef, pstride, ext, ext_stride);
    ntt_forward(ctx, Batch{ext, ext_stride, 1, nullptr}, modup_ntt_map(ctx, ell));
    // per amount: inner product of the permuted extension, ModDown, c0 permuted
    const int B = match_batch_size(ctx);
    for (int a0 = 0; a0 < total; a0 += B) {
        const int items = std::min(B, total - a0);
        u64 *acc = rt.workspace(WS_KS_ACC, (size_t)items * acc_stride);
        u64 *conv = rt.workspace(WS_KS_CONV, (size_t)items * 2 * ell * n);
        std::vector<const u64 *> own(items, c1), base(items, src);
        std::vector<int> srci(items, 0), g(items);
        std::vector<KeyGroup> groups;
        for (int i = 0; i < items; ++i) {
            g[i] = galois_element(ctx, amounts[a0 + i]);
            groups.push_back(KeyGroup{rotation_key(keys, amounts[a0 + i]), i, 1});
        }
        ctx.prof.ks_calls += items;
        ctx.prof.ks_bytes += 8.0 * n * (3.0 * ell * items + 2.0 * beta * next * items);
        const int *d_g = rt.upload_vec(g);
        ks_inner_product(ctx, items, ell, rt.upload_vec(own), ext, ext_stride, groups, acc, acc_stride,
                         rt.upload_vec(srci), d_g);
        moddown(ctx, items, ell, acc, acc_stride, conv, rt.upload_vec(base), d_g, false, out + (long long)a0 * cstride,
                cstride);
    }
}

int galois_element(const Ctx &ctx, int r)
{
    const long long two_n = 2LL * ctx.n;
    long long e = ((long long)r % ctx.S + ctx.S) % ctx.S;
    return (int)powmod_host(5, (u64)e, (u64)two_n);
}

std::vector<int> rotation_plan(const Ctx &ctx, long long r)
{
    long long x = ((r % ctx.S) + ctx.S) % ctx.S;
    std::vector<int> steps;
    long long w = 1;
    while (x) {
        const long long d = x % ctx.rot_base;
        if (d) steps.push_back((int)(d * w));
        x /= ctx.rot_base;
        w *= ctx.rot_base;
    }
    return steps;
}

const u64 *rotation_key(const Keys &keys, int amount)
{
    auto it = keys.rot.find(amount);
    if (it == keys.rot.end()) throw Error(SPFHE_EKEY, "no rotation key for amount " + std::to_string(amount));
    return it->second;
}

void rotate_step_batch(Ctx &ctx, int ell, const std::vector<const u64 *> &in, const std::vector<int> &g,
                       const std::vector<const u64 *> &keys, u64 *out)
{
    const int items = (int)in.size();
    if (!items) return;
    Runtime &rt = *ctx.rt;
    const size_t n = ctx.n;
    const long long pstride = (long long)ell * n;
    std::vector<const u64 *> c1(items), tp(items);
    u64 *tmp = rt.workspace(WS_ROT_TMP, (size_t)items * pstride);
    for (int i = 0; i < items; ++i) {
        c1[i] = in[i] + pstride;
        tp[i] = tmp + i * pstride;
    }
    const u64 *const *d_c1 = rt.upload_vec(c1);
    const u64 *const *d_in = rt.upload_vec(in);
    const u64 *const *d_tp = rt.upload_vec(tp);
    const int *d_g = rt.upload_vec(g);
    automorph(ctx, items, 1, ell, d_c1, 0, tmp, pstride, d_g);
    std::vector<KeyGroup> groups;
    for (int i = 0; i < items; ++i) {
        if (!groups.empty() && groups.back().key == keys[i])
            ++groups.back().count;
        else
            groups.push_back(KeyGroup{keys[i], i, 1});
    }
    keyswitch_batch(ctx, items, ell, d_tp, groups, d_in, d_g, false, out, 2 * pstride);
}

void rotate_batch(Ctx &ctx, const Keys &keys, int ell, const std::vector<const u64 *> &in,
                  const std::vector<int> &r, u64 *out, uint64_t *ks)
{
    rotate_batch(ctx, std::vector<const Keys *>(in.size(), &keys), ell, in, r, out, ks);
}

void rotate_batch(Ctx &ctx, const std::vector<const Keys *> &keys, int ell, const std::vector<const u64 *> &in,
                  const std::vector<int> &r, u64 *out, uint64_t *ks)
{
    Runtime &rt = *ctx.rt;
    const int items = (int)in.size();
    if (!items) return;
    const long long cstride = 2LL * ell * ctx.n;
    std::vector<std::vector<int>> plans(items);
    size_t T = 0;
    for (int i = 0; i < items; ++i) {
        plans[i] = rotation_plan(ctx, r[i]);
        T = std::max(T, plans[i].size());
        for (int a : plans[i]) rotation_key(*keys[i], a);   // EKEY before any launch
    }
    std::vector<const u64 *> cur(in.begin(), in.end());
    // items that need no rotation are copied straight to their output slot
    {
        std::vector<const u64 *> src;
        std::vector<u64 *> dst;
        for (int i = 0; i < items; ++i)
            if (plans[i].empty()) {
                src.push_back(in[i]);
                dst.push_back(out + i * cstride);
            }
        for (size_t k = 0; k < src.size(); ++k) copy_words(ctx, dst[k], src[k], (size_t)cstride);
    }
    u64 *buf[2] = {rt.workspace(WS_ROT_OUT_A, (size_t)items * cstride),
                   rt.workspace(WS_ROT_OUT_B, (size_t)items * cstride)};
    for (size_t s = 0; s < T; ++s) {
        std::vector<int> act;
        for (int i = 0; i < items; ++i)
            if (plans[i].size() > s) act.push_back(i);
        // group equal keys next to each other
        std::stable_sort(act.begin(), act.end(), [&](int a, int b) {
            const u64 *ka = rotation_key(*keys[a], plans[a][s]), *kb = rotation_key(*keys[b], plans[b][s]);
            return ka < kb;
        });
        std::vector<const u64 *> sin, skey;
        std::vector<int> sg;
        for (int i : act) {
            sin.push_back(cur[i]);
            sg.push_back(galois_element(ctx, plans[i][s]));
            skey.push_back(rotation_key(*keys[i], plans[i][s]));
        }
        u64 *dst = buf[s & 1];
        rotate_step_batch(ctx, ell, sin, sg, skey, dst);
        if (ks) *ks += act.size();
        std::vector<const u64 *> fin_src;
        std::vector<u64 *> fin_dst;
        for (size_t k = 0; k < act.size(); ++k) {
            const int i = act[k];
            cur[i] = dst + k * cstride;
            if (plans[i].size() == s + 1) {
                fin_src.push_back(cur[i]);
                fin_dst.push_back(out + i * cstride);
            }
        }
        for (size_t k = 0; k < fin_src.size(); ++k) copy_words(ctx, fin_dst[k], fin_src[k], (size_t)cstride);
    }
}

}  // namespace spfhe
