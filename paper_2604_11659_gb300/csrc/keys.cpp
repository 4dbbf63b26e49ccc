// Secret and switching keys: GPU key generation (ChaCha20-driven sampling),
// import of keys computed elsewhere, encryption and decryption.
#include <algorithm>

#include "runtime.h"

namespace spfhe {

size_t Keys::key_words() const { return (size_t)ctx->dnum * 2 * ctx->M * ctx->n; }

static std::vector<int> all_moduli(const Ctx &ctx)
{
    std::vector<int> mi(ctx.M);
    for (int i = 0; i < ctx.M; ++i) mi[i] = i;
    return mi;
}

// Every amount d * b^t < S (1 <= d < b) a rotation plan can request.
std::vector<int> plan_key_amounts(const Ctx &ctx)
{
    std::vector<int> out;
    for (long long w = 1; w < ctx.S; w *= ctx.rot_base)
        for (long long d = 1; d < ctx.rot_base; ++d)
            if (d * w < ctx.S) out.push_back((int)(d * w));
    return out;
}

// Switching key s' -> s, [dnum][2][M][n] standard form into `key` (then
// converted to Montgomery form by the caller).  s_std/s_mont over all M moduli.
static void gen_switch_key(Ctx &ctx, const u64 *s_mont, const u64 *sprime, uint64_t seed, uint64_t stream0, u64 *key)
{
    const size_t n = ctx.n;
    const int M = ctx.M;
    std::vector<int> mi = all_moduli(ctx);
    Scratch sc(ctx);
    long long *ecoef = sc.typed<long long>(n);
    u64 *e = sc.words((size_t)M * n);
    const int used = (ctx.L + ctx.alpha - 1) / ctx.alpha;
    for (int j = 0; j < ctx.dnum; ++j) {
        u64 *k0 = key + ((size_t)j * 2 + 0) * M * n;
        u64 *k1 = key + ((size_t)j * 2 + 1) * M * n;
        sample_uniform(ctx, k1, M, mi.data(), seed, stream0 + 2 * j);
        sample_gaussian(ctx, ecoef, seed, stream0 + 2 * j + 1);
        from_signed(ctx, ecoef, e, M);
        ntt_forward(ctx, Batch{e, 0, 1, nullptr}, limb_range(0, M, 0));
        rlwe_b(ctx, M, mi.data(), k1, s_mont, e, nullptr, k0);
        if (j < used) {
            const int lo = j * ctx.alpha, hi = std::min(lo + ctx.alpha, ctx.L);
            add_gadget(ctx, k0, sprime, lo, hi);
        }
    }
}

static void key_to_mont(Ctx &ctx, u64 *key)
{
    std::vector<int> mi = all_moduli(ctx);
    to_montgomery(ctx, key, ctx.M, mi.data(), 2 * ctx.dnum);
}

Keys *keygen(Ctx &ctx, uint64_t seed)
{
    const size_t n = ctx.n;
    const int M = ctx.M;
    Keys *k = new Keys;
    k->ctx = &ctx;
    try {
        std::vector<int> mi = all_moduli(ctx);
        Scratch sc(ctx);
        long long *sc_coef = sc.typed<long long>(n);
        u64 *s_std = sc.words((size_t)M * n);
        u64 *sp = sc.words((size_t)M * n);
        sample_ternary(ctx, sc_coef, seed, 1);
        k->s_coef.resize(n);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(k->s_coef.data(), sc_coef, n * sizeof(long long), cudaMemcpyDeviceToHost,
                                         ctx.stream));
        from_signed(ctx, sc_coef, s_std, M);
        ntt_forward(ctx, Batch{s_std, 0, 1, nullptr}, limb_range(0, M, 0));
        k->s = static_cast<u64 *>(dev_alloc(ctx, (size_t)M * n * sizeof(u64)));
        copy_words(ctx, k->s, s_std, (size_t)M * n);
        to_montgomery(ctx, k->s, M, mi.data(), 1);
        // relinearisation key: s^2 -> s
        mul_poly(ctx, M, s_std, s_std, sp);
        k->relin = static_cast<u64 *>(dev_alloc(ctx, k->key_words() * sizeof(u64)));
        gen_switch_key(ctx, k->s, sp, seed, 1000, k->relin);
        key_to_mont(ctx, k->relin);
        // rotation keys: sigma_{5^r}(s) -> s for every plan amount
        std::vector<int> amounts = plan_key_amounts(ctx);
        const u64 *s_ptr = s_std;
        const u64 *const *d_sp = ctx.rt->upload_vec(std::vector<const u64 *>{s_ptr});
        for (size_t a = 0; a < amounts.size(); ++a) {
            const int r = amounts[a];
            const int *d_g = ctx.rt->upload_vec(std::vector<int>{galois_element(ctx, r)});
            automorph(ctx, 1, 1, M, d_sp, 0, sp, 0, d_g);
            u64 *key = static_cast<u64 *>(dev_alloc(ctx, k->key_words() * sizeof(u64)));
            k->rot[r] = key;
            gen_switch_key(ctx, k->s, sp, seed, 2000 + 64 * (uint64_t)a, key);
            key_to_mont(ctx, key);
        }
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
    } catch (...) {
        free_keys(k);
        throw;
    }
    return k;
}

void free_keys(Keys *k)
{
    if (!k) return;
    Ctx &ctx = *k->ctx;
    dev_free(ctx, k->s);
    dev_free(ctx, k->relin);
    for (auto &kv : k->rot) dev_free(ctx, kv.second);
    delete k;
}

Keys *keys_import(Ctx &ctx, const int64_t *secret, const u64 *relin, size_t n_rot, const int32_t *amounts,
                  const u64 *const *rot)
{
    const size_t n = ctx.n;
    const int M = ctx.M;
    Keys *k = new Keys;
    k->ctx = &ctx;
    try {
        std::vector<int> mi = all_moduli(ctx);
        for (size_t i = 0; i < n; ++i)
            if (secret[i] < -1 || secret[i] > 1) throw Error(SPFHE_EINVAL, "secret must be ternary");
        k->s_coef.assign(secret, secret + n);
        Scratch sc(ctx);
        long long *coef = sc.typed<long long>(n);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(coef, secret, n * sizeof(long long), cudaMemcpyHostToDevice, ctx.stream));
        k->s = static_cast<u64 *>(dev_alloc(ctx, (size_t)M * n * sizeof(u64)));
        from_signed(ctx, coef, k->s, M);
        ntt_forward(ctx, Batch{k->s, 0, 1, nullptr}, limb_range(0, M, 0));
        to_montgomery(ctx, k->s, M, mi.data(), 1);
        const size_t kw = k->key_words();
        if (relin) {
            k->relin = static_cast<u64 *>(dev_alloc(ctx, kw * sizeof(u64)));
            SPFHE_CHECK_CUDA(cudaMemcpyAsync(k->relin, relin, kw * sizeof(u64), cudaMemcpyHostToDevice, ctx.stream));
            key_to_mont(ctx, k->relin);
        }
        for (size_t i = 0; i < n_rot; ++i) {
            const int r = amounts[i];
            if (r <= 0 || r >= ctx.S) throw Error(SPFHE_EINVAL, "rotation key amount out of [1, S)");
            if (k->rot.count(r)) throw Error(SPFHE_EINVAL, "duplicate rotation key amount");
            u64 *key = static_cast<u64 *>(dev_alloc(ctx, kw * sizeof(u64)));
            k->rot[r] = key;
            SPFHE_CHECK_CUDA(cudaMemcpyAsync(key, rot[i], kw * sizeof(u64), cudaMemcpyHostToDevice, ctx.stream));
            key_to_mont(ctx, key);
        }
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
    } catch (...) {
        free_keys(k);
        throw;
    }
    return k;
}

// The inverse of keys_import: the ternary secret and every switching key in
// standard (not Montgomery) evaluation form, each key converted in a scratch
// copy on the device and copied to the caller's host or device buffer.
void keys_export(Ctx &ctx, const Keys &k, int64_t *secret, u64 *relin, size_t *n_rot, int32_t *amounts,
                 u64 *const *rot)
{
    const size_t n = ctx.n, kw = k.key_words();
    if (amounts && *n_rot < k.rot.size())
        throw Error(SPFHE_EINVAL, "room for " + std::to_string(*n_rot) + " rotation keys, the key set holds " +
                                      std::to_string(k.rot.size()));
    if (relin && !k.relin) throw Error(SPFHE_EKEY, "the key set holds no relinearisation key");
    if (secret) {
        if (k.s_coef.size() != n) throw Error(SPFHE_EINVAL, "the key set holds no secret coefficients");
        for (size_t i = 0; i < n; ++i) secret[i] = (int64_t)k.s_coef[i];
    }
    std::vector<int> mi = all_moduli(ctx);
    Scratch sc(ctx);
    u64 *tmp = (relin || (amounts && rot)) ? sc.words(kw) : nullptr;
    auto put = [&](const u64 *key, u64 *dst) {
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(tmp, key, kw * sizeof(u64), cudaMemcpyDeviceToDevice, ctx.stream));
        from_montgomery(ctx, tmp, ctx.M, mi.data(), 2 * ctx.dnum);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(dst, tmp, kw * sizeof(u64), cudaMemcpyDefault, ctx.stream));
        // tmp is reused by the next key: this copy must have landed first
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
    };
    if (relin) put(k.relin, relin);
    if (amounts) {
        size_t i = 0;
        for (const auto &kv : k.rot) {
            amounts[i] = kv.first;
            if (rot && rot[i]) put(kv.second, rot[i]);
            ++i;
        }
    }
    *n_rot = k.rot.size();
    SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
}

Ct *ct_new(Ctx &ctx, int level, double scale)
{
    Ct *c = new Ct;
    c->ctx = &ctx;
    c->level = level;
    c->scale = scale;
    try {
        c->d = static_cast<u64 *>(dev_alloc(ctx, 2ull * level * ctx.n * sizeof(u64)));
    } catch (...) {
        delete c;
        throw;
    }
    return c;
}

Pt *pt_new(Ctx &ctx, int level, double scale)
{
    Pt *p = new Pt;
    p->ctx = &ctx;
    p->level = level;
    p->scale = scale;
    try {
        p->d = static_cast<u64 *>(dev_alloc(ctx, (size_t)level * ctx.n * sizeof(u64)));
    } catch (...) {
        delete p;
        throw;
    }
    return p;
}

Ct *encrypt(Ctx &ctx, const Keys &keys, const Pt &pt, uint64_t seed)
{
    const int ell = pt.level;
    const size_t n = ctx.n;
    Ct *c = ct_new(ctx, ell, pt.scale);
    std::vector<int> mi(ell);
    for (int i = 0; i < ell; ++i) mi[i] = i;
    Scratch sc(ctx);
    long long *ecoef = sc.typed<long long>(n);
    u64 *e = sc.words((size_t)ell * n);
    u64 *c0 = c->d, *c1 = c->d + (size_t)ell * n;
    sample_uniform(ctx, c1, ell, mi.data(), seed, 1);
    sample_gaussian(ctx, ecoef, seed, 2);
    from_signed(ctx, ecoef, e, ell);
    ntt_forward(ctx, Batch{e, 0, 1, nullptr}, limb_range(0, ell, 0));
    rlwe_b(ctx, ell, mi.data(), c1, keys.s, e, pt.d, c0);
    return c;
}

Pt *decrypt(Ctx &ctx, const Keys &keys, const Ct &ct)
{
    Pt *p = pt_new(ctx, ct.level, ct.scale);
    decrypt_core(ctx, ct.level, ct.d, keys.s, p->d);
    return p;
}

}  // namespace spfhe
