// Batched CKKS evaluator: hybrid key switching, rotations through the
// rotation plan, key generation and encryption, all sequenced on the
// context's stream.
#include <algorithm>
#include <map>
#include <numeric>

#include "runtime.h"

namespace spfhe {

static int beta_of(const Ctx &ctx, int ell) { return (ell + ctx.alpha - 1) / ctx.alpha; }

namespace {
// Marks the launches of a key switch (their transforms are profiled apart).
struct InKeySwitch {
    Ctx &c;
    explicit InKeySwitch(Ctx &x) : c(x) { ++c.in_keyswitch; }
    ~InKeySwitch() { --c.in_keyswitch; }
};

struct KsBuffers {
    u64 *acc, *conv;
    long long acc_stride;
};

// ModUp and the inner product of a key-switching batch: acc [items][2][ell+K][n]
// (evaluation rep.) and the workspace for ModDown's conversion.
KsBuffers ks_front(Ctx &ctx, int items, int ell, const u64 *const *d_in, const std::vector<KeyGroup> &groups)
{
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
    ctx.prof.ks_calls += items;
    ctx.prof.ks_bytes += 8.0 * n * (3.0 * ell * items + 2.0 * beta * next * groups.size());
    // ModUp: coefficient representation of every input limb, then one base
    // conversion per digit and forward transforms of the new limbs
    // (read straight from the inputs where the transform can; n^{-1} of this
    // transform is folded into the ModUp conversion's constants)
    if (!ntt_inverse_from(ctx, Batch{coef, coef_stride, items, nullptr}, d_in, limb_range(0, ell, 0), false)) {
        gather_items(ctx, items, (size_t)coef_stride, d_in, coef, coef_stride);
        ntt_inverse(ctx, Batch{coef, coef_stride, items, nullptr}, limb_range(0, ell, 0), false);
    }
    modup_bconv(ctx, items, ell, coef, coef_stride, ext, ext_stride);
    ntt_forward(ctx, Batch{ext, ext_stride, items, nullptr}, modup_ntt_map(ctx, ell));
    ks_inner_product(ctx, items, ell, d_in, ext, ext_stride, groups, acc, acc_stride);
    return KsBuffers{acc, conv, acc_stride};
}
}  // namespace

void keyswitch_batch(Ctx &ctx, int items, int ell, const u64 *const *d_in, const std::vector<KeyGroup> &groups,
                     const u64 *const *d_base, const int *d_base_g, bool base_c1, u64 *out, long long out_stride)
{
    if (items <= 0) return;
    InKeySwitch in_ks(ctx);
    const KsBuffers kb = ks_front(ctx, items, ell, d_in, groups);
    moddown(ctx, items, ell, kb.acc, kb.acc_stride, kb.conv, d_base, d_base_g, base_c1, out, out_stride);
}

bool relin_rescale_supported(const Ctx &ctx, int ell)
{
    return ctx.fuse_epilogues && ctx.log_n >= 12 && (ctx.ntt_variant == 5 || ctx.ntt_variant == 6) && ell >= 2;
}

// Relinearisation followed by a rescale (Alg. 2's Relinearize, then
// Rescale) with one transform per output limb instead of two.  ModDown's
// output is o_b[i] = base_b[i] + P^{-1} (acc_b[i] - NTT(conv_b[i])) and the
// rescale turns it into (o_b[i] - NTT([t_b]_{q_i})) q_t^{-1}, t_b the
// coefficients of o_b's top limb.  The transform is linear over Z_{q_i}, so
// (P^{-1} acc_b[i] + base_b[i] - NTT(P^{-1} conv_b[i] + [t_b]_{q_i})) q_t^{-1}
// is the same residue: ModDown's own transforms of conv are left out, and
// t_b = P^{-1} (INTT(acc_b[t]) - conv_b[t]) + INTT(base_b[t]) comes from two
// inverse transforms of top limbs instead of one.
void relin_rescale_batch(Ctx &ctx, int items, int ell, const u64 *const *d_in, const std::vector<KeyGroup> &groups,
                         const u64 *const *d_base, u64 *tmp, u64 *out, long long out_stride, const u64 *const *mask,
                         const int *mask_g)
{
    if (items <= 0) return;
    if (!relin_rescale_supported(ctx, ell)) throw Error(SPFHE_EINVAL, "merged relinearise-rescale unavailable");
    const size_t n = ctx.n;
    const int next = ell + ctx.K;
    KsBuffers kb;
    {
        InKeySwitch in_ks(ctx);
        kb = ks_front(ctx, items, ell, d_in, groups);
        moddown_conv(ctx, items, ell, kb.acc, kb.acc_stride, kb.conv);
    }
    // tmp: top limbs [items][2][n], then the spread buffer [items][2][ell-1][n]
    u64 *top = tmp;
    u64 *spread = tmp + (size_t)items * 2 * n;
    copy_top(ctx, items, ell, 2, d_base, top);
    LimbMap tm;
    tm.nl = 2;
    tm.off[0] = 0;
    tm.off[1] = 1;
    tm.mi[0] = tm.mi[1] = ell - 1;
    ntt_inverse(ctx, Batch{top, 2LL * (long long)n, items, nullptr}, tm);
    LimbMap am;
    am.nl = 2;
    am.off[0] = ell - 1;
    am.off[1] = next + ell - 1;
    am.mi[0] = am.mi[1] = ell - 1;
    ntt_inverse(ctx, Batch{kb.acc, kb.acc_stride, items, nullptr}, am);
    relin_top(ctx, items, ell, kb.acc, kb.acc_stride, kb.conv, top);
    LimbMap sm;
    sm.nl = 2 * (ell - 1);
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < ell - 1; ++i) {
            sm.off[b * (ell - 1) + i] = b * (ell - 1) + i;
            sm.mi[b * (ell - 1) + i] = i;
        }
    FuseArgs fa;
    fa.ell = ell;
    fa.K = ctx.K;
    fa.polys = 2;
    fa.top = top;
    fa.conv = kb.conv;
    fa.conv_stride = 2LL * ell * n;
    fa.acc = kb.acc;
    fa.acc_stride = kb.acc_stride;
    fa.base = d_base;
    fa.out = out;
    fa.out_stride = out_stride;
    fa.pinv = ctx.dt.md_pinv;
    fa.pinvp = ctx.dt.md_pinv_p;
    fa.qt_mod = ctx.dt.rs_qt + (size_t)(ell - 1) * ctx.L;
    fa.inv = ctx.dt.rs_inv + (size_t)(ell - 1) * ctx.L;
    fa.invp = ctx.dt.rs_inv_p + (size_t)(ell - 1) * ctx.L;
    fa.mask = mask;
    fa.mask_g = mask_g;
    if (!ntt_forward_fused(ctx, Batch{spread, 2LL * (ell - 1) * (long long)n, items, nullptr}, sm, kFuseRelinRescale,
                           fa))
        throw Error(SPFHE_EINVAL, "merged relinearise-rescale transform refused");
}

bool rotate_accumulate_supported(const Ctx &ctx)
{
    return ctx.fuse_epilogues && ctx.log_n >= 12 && (ctx.ntt_variant == 5 || ctx.ntt_variant == 6);
}

// One rotation step of every source (Galois element g[j], key keys[j],
// sources with equal keys next to each other) added into tgt[j], which holds
// its initial value.  ModDown's output of source j is
// sigma_g(c0_j) + P^{-1} (acc_j - NTT(conv_j)); the sources of one target
// are summed as sum sigma_g(c0_j) + P^{-1} (sum acc_j - NTT(sum conv_j)),
// the transform being linear over Z_q: one forward transform per target.
void rotate_step_accumulate(Ctx &ctx, int ell, const std::vector<const u64 *> &in, const std::vector<int> &g,
                            const std::vector<const u64 *> &keys, const std::vector<u64 *> &tgt)
{
    if (!rotate_accumulate_supported(ctx)) throw Error(SPFHE_EINVAL, "fused rotate-accumulate unavailable");
    const int A = (int)in.size();
    if (!A) return;
    Runtime &rt = *ctx.rt;
    const size_t n = ctx.n;
    const long long pstride = (long long)ell * n, cstride = 2 * pstride;
    std::vector<const u64 *> c1(A), tp(A);
    std::vector<KeyGroup> groups;
    u64 *tmp = rt.workspace(WS_ROT_TMP, (size_t)A * pstride);
    for (int k = 0; k < A; ++k) {
        c1[k] = in[k] + pstride;
        tp[k] = tmp + k * pstride;
        if (!groups.empty() && groups.back().key == keys[k])
            ++groups.back().count;
        else
            groups.push_back(KeyGroup{keys[k], k, 1});
    }
    automorph(ctx, A, 1, ell, rt.upload_vec(c1), 0, tmp, pstride, rt.upload_vec(g));
    KsBuffers kb;
    {
        InKeySwitch in_ks(ctx);
        kb = ks_front(ctx, A, ell, rt.upload_vec(tp), groups);
        moddown_conv(ctx, A, ell, kb.acc, kb.acc_stride, kb.conv);
    }
    // sources by target
    std::map<u64 *, std::vector<int>> by_t;
    for (int k = 0; k < A; ++k) by_t[tgt[k]].push_back(k);
    const int nt = (int)by_t.size();
    std::vector<u64 *> tptr, sptr;
    std::vector<const u64 *> cptr, c0;
    std::vector<int> seg{0}, item, gj;
    u64 *sconv = rt.workspace(WS_ROT_SUM, (size_t)nt * cstride);
    for (auto &kv : by_t) {
        tptr.push_back(kv.first);
        sptr.push_back(sconv + (long long)(tptr.size() - 1) * cstride);
        for (int k : kv.second) {
            item.push_back(k);
            cptr.push_back(kb.conv + (long long)k * cstride);
            c0.push_back(in[k]);
            gj.push_back(g[k]);
        }
        seg.push_back((int)item.size());
    }
    const int *d_seg = rt.upload_vec(seg);
    accumulate_seg(ctx, 2, ell, nt, rt.upload_vec(sptr), rt.upload_vec(cptr), d_seg, A, false);
    LimbMap qm;
    qm.nl = 2 * ell;
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < ell; ++i) {
            qm.off[b * ell + i] = b * ell + i;
            qm.mi[b * ell + i] = i;
        }
    FuseArgs fa;
    fa.ell = ell;
    fa.K = ctx.K;
    fa.polys = A;   // sources, for the profiler's byte count
    fa.acc = kb.acc;
    fa.acc_stride = kb.acc_stride;
    fa.pinv = ctx.dt.md_pinv;
    fa.pinvp = ctx.dt.md_pinv_p;
    fa.outp = rt.upload_vec(tptr);
    fa.seg = d_seg;
    fa.item = rt.upload_vec(item);
    fa.base = rt.upload_vec(c0);
    fa.base_g = rt.upload_vec(gj);
    if (!ntt_forward_fused(ctx, Batch{sconv, cstride, nt, nullptr}, qm, kFuseRotAccum, fa))
        throw Error(SPFHE_EINVAL, "fused rotate-accumulate transform refused");
}

// Rotations through the plan whose results are only summed into result
// ciphertexts (Alg. 2's EvalRotate then EvalAdd).  Every step but the last
// runs as in rotate_batch.  The last step's ModDown output is
// sigma_g(c0) + P^{-1} (acc - NTT(conv)) (c1's part without sigma_g(c0));
// summed over the sources of one result ciphertext that is
// sum sigma_g(c0) + P^{-1} (sum acc - NTT(sum conv)), the transform being
// linear over Z_q: one forward transform per result ciphertext and batch
// instead of one per source, and no rotated ciphertext written out.  The
// sums are exact residues, so the result is bit for bit rotate_batch's
// outputs added into the targets.
void rotate_accumulate_batch(Ctx &ctx, const std::vector<const Keys *> &keys, int ell,
                             const std::vector<const u64 *> &in, const std::vector<int> &r,
                             const std::vector<u64 *> &tgt, uint64_t *ks)
{
    if (!rotate_accumulate_supported(ctx)) throw Error(SPFHE_EINVAL, "fused rotate-accumulate unavailable");
    Runtime &rt = *ctx.rt;
    const int items = (int)in.size();
    if (!items) return;
    const size_t n = ctx.n;
    const long long pstride = (long long)ell * n, cstride = 2 * pstride;
    std::vector<std::vector<int>> plans(items);
    size_t T = 0;
    for (int i = 0; i < items; ++i) {
        plans[i] = rotation_plan(ctx, r[i]);
        T = std::max(T, plans[i].size());
        for (int a : plans[i]) rotation_key(*keys[i], a);   // EKEY before any launch
    }
    // every step but each item's last; an item whose prefix ends while more
    // prefix steps follow is copied aside (the step buffers alternate)
    std::vector<const u64 *> cur(in.begin(), in.end());
    u64 *buf[2] = {rt.workspace(WS_ROT_OUT_A, (size_t)items * cstride),
                   rt.workspace(WS_ROT_OUT_B, (size_t)items * cstride)};
    u64 *hold = T > 3 ? rt.workspace(WS_MISC, (size_t)items * cstride) : nullptr;
    for (size_t s = 0; s + 1 < T; ++s) {
        std::vector<int> act;
        for (int i = 0; i < items; ++i)
            if (plans[i].size() > s + 1) act.push_back(i);
        std::stable_sort(act.begin(), act.end(), [&](int a, int b) {
            return rotation_key(*keys[a], plans[a][s]) < rotation_key(*keys[b], plans[b][s]);
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
        std::vector<const u64 *> keep_src;
        std::vector<u64 *> keep_dst;
        for (size_t k = 0; k < act.size(); ++k) {
            const int i = act[k];
            cur[i] = dst + k * cstride;
            // its prefix ends here; step s + 2 (if any) writes this buffer again
            if (plans[i].size() == s + 2 && s + 3 < T) {
                keep_src.push_back(cur[i]);
                keep_dst.push_back(hold + i * cstride);
                cur[i] = hold + i * cstride;
            }
        }
        for (size_t k = 0; k < keep_src.size(); ++k) copy_words(ctx, keep_dst[k], keep_src[k], (size_t)cstride);
    }
    // the last step of every rotated item, keys grouped
    std::vector<int> act;
    for (int i = 0; i < items; ++i)
        if (!plans[i].empty()) act.push_back(i);
    std::stable_sort(act.begin(), act.end(), [&](int a, int b) {
        return rotation_key(*keys[a], plans[a].back()) < rotation_key(*keys[b], plans[b].back());
    });
    if (!act.empty()) {
        std::vector<const u64 *> sin, skey;
        std::vector<int> sg;
        std::vector<u64 *> st;
        for (int i : act) {
            sin.push_back(cur[i]);
            sg.push_back(galois_element(ctx, plans[i].back()));
            skey.push_back(rotation_key(*keys[i], plans[i].back()));
            st.push_back(tgt[i]);
        }
        rotate_step_accumulate(ctx, ell, sin, sg, skey, st);
        if (ks) *ks += act.size();
    }
    // items that need no rotation are added as they are
    std::map<u64 *, std::vector<int>> plain;
    for (int i = 0; i < items; ++i)
        if (plans[i].empty()) plain[tgt[i]].push_back(i);
    if (!plain.empty()) {
        std::vector<u64 *> tptr;
        std::vector<const u64 *> src;
        std::vector<int> seg{0};
        for (auto &kv : plain) {
            tptr.push_back(kv.first);
            for (int i : kv.second) src.push_back(in[i]);
            seg.push_back((int)src.size());
        }
        accumulate_seg(ctx, 2, ell, (int)tptr.size(), rt.upload_vec(tptr), rt.upload_vec(src), rt.upload_vec(seg),
                       (int)src.size(), true);
    }
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
