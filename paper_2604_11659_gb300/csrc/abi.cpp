// extern "C" boundary of libspfhe: argument checks, error translation, and the
// single-operation entry points.  Every call returns a status; no C++
// exception crosses this file.
#include <cmath>
#include <cstring>

#include "runtime.h"


#include "engine.h"
#include "handles.h"

using namespace spfhe;

namespace {
thread_local std::string g_err;

spfhe_status fail(spfhe_status s, const std::string &m)
{
    g_err = m;
    return s;
}

template <typename F> spfhe_status guard(F &&f)
{
    try {
        f();
        return SPFHE_OK;
    } catch (const Error &e) {
        return fail(e.code, e.what());
    } catch (const std::bad_alloc &) {
        return fail(SPFHE_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(SPFHE_EINVAL, e.what());
    }
}

void need(bool ok, const char *what)
{
    if (!ok) throw Error(SPFHE_EINVAL, what);
}

spfhe_ct *wrap(Ct *c)
{
    spfhe_ct *h = new spfhe_ct;
    h->c = c;
    return h;
}

spfhe_pt *wrap(Pt *p)
{
    spfhe_pt *h = new spfhe_pt;
    h->p = p;
    return h;
}

void free_ct(Ct *c)
{
    if (!c) return;
    dev_free(*c->ctx, c->d);
    delete c;
}

void free_pt(Pt *p)
{
    if (!p) return;
    dev_free(*p->ctx, p->d);
    delete p;
}

Ctx &C(spfhe_ctx *ctx)
{
    need(ctx != nullptr, "null context");
    SPFHE_CHECK_CUDA(cudaSetDevice(ctx->c.device));
    return ctx->c;
}

void same_scale(double a, double b)
{
    if (std::fabs(a - b) > 1e-9 * std::fabs(a)) throw Error(SPFHE_ESCALE, "operand scales differ");
}
}  // namespace

namespace spfhe {
void set_last_error(const std::string &m) { g_err = m; }
}  // namespace spfhe

extern "C" {

const char *spfhe_last_error(void) { return g_err.c_str(); }

spfhe_status spfhe_ctx_create(const spfhe_params *params, void *cuda_stream, spfhe_ctx **out)
{
    return guard([&] {
        need(params && out, "null argument");
        *out = nullptr;
        spfhe_ctx *h = new spfhe_ctx;
        try {
            Ctx &c = h->c;
            SPFHE_CHECK_CUDA(cudaGetDevice(&c.device));
            c.stream = static_cast<cudaStream_t>(cuda_stream);
            configure_pool(c.device);
            build_params(c, *params);
            upload_tables(c);
            c.rt = new Runtime(c);
        } catch (...) {
            free_tables(h->c);
            delete h;
            throw;
        }
        *out = h;
    });
}

spfhe_status spfhe_ctx_destroy(spfhe_ctx *ctx)
{
    if (!ctx) return SPFHE_OK;
    return guard([&] {
        Ctx &c = ctx->c;
        cudaSetDevice(c.device);
        cudaStreamSynchronize(c.stream);
        if (c.rt) {
            c.rt->release();
            delete c.rt;
        }
        for (auto &kv : c.masks) dev_free(c, kv.second);
        c.masks.clear();
        cudaStreamSynchronize(c.stream);
        if (c.cos_tab) cudaFree(c.cos_tab);
        prof_destroy(c);
        free_tables(c);
        delete ctx;
    });
}

spfhe_status spfhe_ctx_moduli(const spfhe_ctx *ctx, uint64_t *mods, uint64_t *psis)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        for (int i = 0; i < ctx->c.M; ++i) {
            if (mods) mods[i] = ctx->c.mods[i];
            if (psis) psis[i] = ctx->c.psis[i];
        }
    });
}

spfhe_status spfhe_sync(spfhe_ctx *ctx)
{
    return guard([&] { SPFHE_CHECK_CUDA(cudaStreamSynchronize(C(ctx).stream)); });
}

uint64_t spfhe_launch_count(const spfhe_ctx *ctx) { return ctx ? ctx->c.launches : 0; }

spfhe_status spfhe_ctx_set_match_batch(spfhe_ctx *ctx, uint32_t matches)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        need(matches <= 1024, "batch size out of range");
        ctx->c.match_batch = (int)matches;
    });
}

spfhe_status spfhe_ctx_set_ntt_chunk(spfhe_ctx *ctx, uint32_t limbs)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        need(limbs <= (1u << 20), "chunk out of range");
        ctx->c.ntt_chunk = (int)limbs;
    });
}

spfhe_status spfhe_ctx_set_ntt_split(spfhe_ctx *ctx, uint32_t pass_a_stages)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        Ctx &c = ctx->c;
        if (pass_a_stages != 0) {
            const int pb = c.log_n - (int)pass_a_stages;
            need(c.log_n >= 12 && pass_a_stages >= 6 && pass_a_stages <= 9 && pb >= 6 && pb <= 9,
                 "both NTT passes need 6 to 9 stages");
        }
        c.ntt_pa = (int)pass_a_stages;
    });
}

spfhe_status spfhe_ctx_set_fusion(spfhe_ctx *ctx, int enable)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        ctx->c.fuse_epilogues = enable != 0;
    });
}

spfhe_status spfhe_ctx_set_align_budget(spfhe_ctx *ctx, uint64_t bytes)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        ctx->c.align_budget = (size_t)bytes;
    });
}

spfhe_status spfhe_ctx_set_ntt_variant(spfhe_ctx *ctx, uint32_t variant)
{
    return guard([&] {
        need(ctx != nullptr, "null context");
        need(variant <= 6, "NTT variant must be 0 to 6");
        ctx->c.ntt_variant = (int)variant;
    });
}

spfhe_status spfhe_prof_enable(spfhe_ctx *ctx, int enable)
{
    return guard([&] {
        Ctx &c = C(ctx);
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        prof_reset(c, enable != 0);
    });
}

spfhe_status spfhe_prof_read(spfhe_ctx *ctx, int cls, uint64_t *launches, double *ms, double *bytes, double *work)
{
    return guard([&] {
        Ctx &c = C(ctx);
        need(cls >= 0 && cls < K_NCLASS, "kernel class out of range");
        prof_collect(c);
        if (launches) *launches = c.prof.launches[cls];
        if (ms) *ms = c.prof.ms[cls];
        if (bytes) *bytes = c.prof.bytes[cls];
        if (work) *work = c.prof.work[cls];
    });
}

int spfhe_prof_classes(void) { return K_NCLASS; }

spfhe_status spfhe_prof_transform_limbs(spfhe_ctx *ctx, int cls, double *first, double *second,
                                        double *second_fused)
{
    try {
        if (!ctx || cls < 0 || cls >= K_NCLASS) throw Error(SPFHE_EINVAL, "bad argument");
        const Prof &p = ctx->c.prof;
        if (first) *first = p.limbs[cls][0];
        if (second) *second = p.limbs[cls][1];
        if (second_fused) *second_fused = p.limbs[cls][2];
        return SPFHE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}

spfhe_status spfhe_prof_keyswitch(spfhe_ctx *ctx, uint64_t *calls, double *bytes)
{
    return guard([&] {
        Ctx &c = C(ctx);
        if (calls) *calls = c.prof.ks_calls;
        if (bytes) *bytes = c.prof.ks_bytes;
    });
}

const char *spfhe_prof_class_name(int cls) { return kernel_class_name(cls); }

spfhe_status spfhe_keygen(spfhe_ctx *ctx, uint64_t seed, spfhe_keys **out)
{
    return guard([&] {
        need(out != nullptr, "null out");
        *out = nullptr;
        Ctx &c = C(ctx);
        Keys *k = keygen(c, seed);
        *out = new spfhe_keys{k};
    });
}

spfhe_status spfhe_keys_import(spfhe_ctx *ctx, const int64_t *secret, const uint64_t *relin, size_t n_rot,
                               const int32_t *rot_amounts, const uint64_t *const *rot, spfhe_keys **out)
{
    return guard([&] {
        need(out && secret, "null argument");
        need(n_rot == 0 || (rot_amounts && rot), "null rotation keys");
        *out = nullptr;
        Ctx &c = C(ctx);
        Keys *k = keys_import(c, secret, reinterpret_cast<const u64 *>(relin), n_rot, rot_amounts,
                              reinterpret_cast<const u64 *const *>(rot));
        *out = new spfhe_keys{k};
    });
}

spfhe_status spfhe_keys_export(spfhe_ctx *ctx, const spfhe_keys *keys, int64_t *secret, uint64_t *relin,
                               size_t *n_rot, int32_t *rot_amounts, uint64_t *const *rot)
{
    return guard([&] {
        need(keys && n_rot, "null argument");
        Ctx &c = C(ctx);
        need(keys->k->ctx == &c, "the key set belongs to another context");
        keys_export(c, *keys->k, secret, reinterpret_cast<u64 *>(relin), n_rot, rot_amounts,
                    reinterpret_cast<u64 *const *>(rot));
    });
}

void spfhe_keys_free(spfhe_keys *keys)
{
    if (!keys) return;
    try {
        cudaSetDevice(keys->k->ctx->device);
        free_keys(keys->k);
    } catch (...) {
    }
    delete keys;
}

spfhe_status spfhe_encode(spfhe_ctx *ctx, const double *re, const double *im, size_t n_vals, uint32_t level,
                          double scale, spfhe_pt **out)
{
    return guard([&] {
        need(out && (re || n_vals == 0), "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        need(level >= 1 && (int)level <= c.L, "level out of range");
        need(scale > 0, "scale must be positive");
        std::vector<long long> m = encode_host(c, re, im, n_vals, scale);
        Pt *p = pt_new(c, level, scale);
        try {
            Scratch sc(c);
            long long *dm = sc.typed<long long>(c.n);
            SPFHE_CHECK_CUDA(cudaMemcpyAsync(dm, m.data(), c.n * sizeof(long long), cudaMemcpyHostToDevice, c.stream));
            from_signed(c, dm, p->d, level);
            ntt_forward(c, Batch{p->d, 0, 1, nullptr}, limb_range(0, level, 0));
            SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        } catch (...) {
            free_pt(p);
            throw;
        }
        *out = wrap(p);
    });
}

spfhe_status spfhe_pt_import(spfhe_ctx *ctx, const uint64_t *limbs, uint32_t level, double scale, int coeff_domain,
                             spfhe_pt **out)
{
    return guard([&] {
        need(out && limbs, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        need(level >= 1 && (int)level <= c.M, "level out of range");
        Pt *p = pt_new(c, level, scale);
        try {
            SPFHE_CHECK_CUDA(cudaMemcpyAsync(p->d, limbs, (size_t)level * c.n * sizeof(u64), cudaMemcpyDefault, c.stream));
            if (coeff_domain) ntt_forward(c, Batch{p->d, 0, 1, nullptr}, limb_range(0, level, 0));
            SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        } catch (...) {
            free_pt(p);
            throw;
        }
        *out = wrap(p);
    });
}

spfhe_status spfhe_pt_export(spfhe_ctx *ctx, const spfhe_pt *pt, uint64_t *limbs)
{
    return guard([&] {
        need(pt && limbs, "null argument");
        Ctx &c = C(ctx);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(limbs, pt->p->d, (size_t)pt->p->level * c.n * sizeof(u64), cudaMemcpyDefault,
                                         c.stream));
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
    });
}

spfhe_status spfhe_pt_info(const spfhe_pt *pt, uint32_t *level, double *scale)
{
    return guard([&] {
        need(pt != nullptr, "null plaintext");
        if (level) *level = pt->p->level;
        if (scale) *scale = pt->p->scale;
    });
}

void spfhe_pt_free(spfhe_pt *pt)
{
    if (!pt) return;
    free_pt(pt->p);
    delete pt;
}

spfhe_status spfhe_decode(spfhe_ctx *ctx, const spfhe_pt *pt, double *re, double *im, size_t n_vals)
{
    return guard([&] {
        need(pt && (re || n_vals == 0), "null argument");
        Ctx &c = C(ctx);
        Scratch sc(c);
        u64 *t = sc.words(c.n);
        copy_words(c, t, pt->p->d, c.n);
        ntt_inverse(c, Batch{t, 0, 1, nullptr}, limb_range(0, 1, 0));
        std::vector<u64> h(c.n);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(h.data(), t, c.n * sizeof(u64), cudaMemcpyDeviceToHost, c.stream));
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        decode_host(c, h, pt->p->scale, re, im, n_vals);
    });
}

spfhe_status spfhe_encrypt(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_pt *pt, uint64_t seed, spfhe_ct **out)
{
    return guard([&] {
        need(keys && pt && out, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        *out = wrap(encrypt(c, *keys->k, *pt->p, seed));
    });
}

spfhe_status spfhe_decrypt(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_ct *ct, spfhe_pt **out)
{
    return guard([&] {
        need(keys && ct && out, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        *out = wrap(decrypt(c, *keys->k, *ct->c));
    });
}

spfhe_status spfhe_ct_import(spfhe_ctx *ctx, const uint64_t *limbs, uint32_t level, double scale, spfhe_ct **out)
{
    return guard([&] {
        need(out && limbs, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        need(level >= 1 && (int)level <= c.L, "level out of range");
        Ct *ct = ct_new(c, level, scale);
        cudaError_t e = cudaMemcpyAsync(ct->d, limbs, 2ull * level * c.n * sizeof(u64), cudaMemcpyDefault, c.stream);
        if (e != cudaSuccess) {
            free_ct(ct);
            throw Error(SPFHE_ECUDA, cudaGetErrorString(e));
        }
        *out = wrap(ct);
    });
}

spfhe_status spfhe_ct_overwrite(spfhe_ctx *ctx, spfhe_ct *ct, const uint64_t *limbs)
{
    return guard([&] {
        need(ct && limbs, "null argument");
        Ctx &c = C(ctx);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(ct->c->d, limbs, 2ull * ct->c->level * c.n * sizeof(u64), cudaMemcpyDefault,
                                         c.stream));
    });
}

spfhe_status spfhe_ct_export(spfhe_ctx *ctx, const spfhe_ct *ct, uint64_t *limbs)
{
    return guard([&] {
        need(ct && limbs, "null argument");
        Ctx &c = C(ctx);
        SPFHE_CHECK_CUDA(cudaMemcpyAsync(limbs, ct->c->d, 2ull * ct->c->level * c.n * sizeof(u64), cudaMemcpyDefault,
                                         c.stream));
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
    });
}

spfhe_status spfhe_ct_info(const spfhe_ct *ct, uint32_t *level, double *scale)
{
    return guard([&] {
        need(ct != nullptr, "null ciphertext");
        if (level) *level = ct->c->level;
        if (scale) *scale = ct->c->scale;
    });
}

void spfhe_ct_free(spfhe_ct *ct)
{
    if (!ct) return;
    if (!ct->borrowed) free_ct(ct->c);
    delete ct;
}

spfhe_status spfhe_mult_relin(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_ct *a, const spfhe_ct *b,
                              spfhe_ct **out)
{
    return guard([&] {
        need(keys && a && b && out, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        const Ct &x = *a->c, &y = *b->c;
        if (x.level != y.level) throw Error(SPFHE_ELEVEL, "operands at different levels");
        if (!keys->k->relin) throw Error(SPFHE_EKEY, "no relinearisation key");
        const int ell = x.level;
        const size_t n = c.n;
        Runtime &rt = *c.rt;
        Ct *o = ct_new(c, ell, x.scale * y.scale);
        try {
            u64 *D = rt.workspace(WS_TENSOR, 3ull * ell * n);
            tensor(c, 1, ell, rt.upload_vec(std::vector<const u64 *>{x.d}), rt.upload_vec(std::vector<const u64 *>{y.d}), D);
            const u64 *d2 = D + 2ull * ell * n;
            keyswitch_batch(c, 1, ell, rt.upload_vec(std::vector<const u64 *>{d2}), {KeyGroup{keys->k->relin, 0, 1}},
                            rt.upload_vec(std::vector<const u64 *>{D}), nullptr, true, o->d, 2LL * ell * n);
            SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        } catch (...) {
            free_ct(o);
            throw;
        }
        *out = wrap(o);
    });
}

spfhe_status spfhe_rescale(spfhe_ctx *ctx, spfhe_ct *ct)
{
    return guard([&] {
        need(ct != nullptr, "null argument");
        Ctx &c = C(ctx);
        Ct &x = *ct->c;
        if (x.level < 2) throw Error(SPFHE_ELEVEL, "rescale needs two limbs");
        const int ell = x.level;
        const size_t n = c.n;
        Runtime &rt = *c.rt;
        u64 *T = rt.workspace(WS_RS_TMP, 2ull * ell * n);
        u64 *nd = static_cast<u64 *>(dev_alloc(c, 2ull * (ell - 1) * n * sizeof(u64)));
        rescale(c, 1, ell, rt.upload_vec(std::vector<const u64 *>{x.d}), T, nd, 2LL * (ell - 1) * n);
        dev_free(c, x.d);
        x.d = nd;
        x.scale /= (double)c.mods[ell - 1];
        x.level = ell - 1;
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
    });
}

spfhe_status spfhe_rotate(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_ct *ct, int32_t r, spfhe_ct **out)
{
    return guard([&] {
        need(keys && ct && out, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        const Ct &x = *ct->c;
        Ct *o = ct_new(c, x.level, x.scale);
        try {
            rotate_batch(c, *keys->k, x.level, {x.d}, {r}, o->d, nullptr);
            SPFHE_CHECK_CUDA(cudaStreamSynchronize(c.stream));
        } catch (...) {
            free_ct(o);
            throw;
        }
        *out = wrap(o);
    });
}

spfhe_status spfhe_mul_plain(spfhe_ctx *ctx, const spfhe_ct *ct, const spfhe_pt *pt, spfhe_ct **out)
{
    return guard([&] {
        need(ct && pt && out, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        const Ct &x = *ct->c;
        const Pt &p = *pt->p;
        if (x.level != p.level) throw Error(SPFHE_ELEVEL, "ciphertext and plaintext at different levels");
        Ct *o = ct_new(c, x.level, x.scale * p.scale);
        mul_ct_pt(c, x.level, x.d, p.d, o->d);
        *out = wrap(o);
    });
}

spfhe_status spfhe_add(spfhe_ctx *ctx, const spfhe_ct *a, const spfhe_ct *b, spfhe_ct **out)
{
    return guard([&] {
        need(a && b && out, "null argument");
        *out = nullptr;
        Ctx &c = C(ctx);
        const Ct &x = *a->c, &y = *b->c;
        if (x.level != y.level) throw Error(SPFHE_ELEVEL, "operands at different levels");
        same_scale(x.scale, y.scale);
        Ct *o = ct_new(c, x.level, x.scale);
        add_ct(c, 2, x.level, x.d, y.d, o->d);
        *out = wrap(o);
    });
}

spfhe_status spfhe_ntt(spfhe_ctx *ctx, uint64_t *dev_limbs, uint32_t n_limbs, const int32_t *mod_idx, int inverse)
{
    return guard([&] {
        need(dev_limbs && mod_idx, "null argument");
        Ctx &c = C(ctx);
        need(n_limbs >= 1 && n_limbs <= (uint32_t)kMaxLimbSlots, "limb count out of range");
        LimbMap m;
        m.nl = (int)n_limbs;
        for (uint32_t l = 0; l < n_limbs; ++l) {
            need(mod_idx[l] >= 0 && mod_idx[l] < c.M, "modulus index out of range");
            m.off[l] = (int)l;
            m.mi[l] = mod_idx[l];
        }
        Batch b{reinterpret_cast<u64 *>(dev_limbs), 0, 1, nullptr};
        if (inverse)
            ntt_inverse(c, b, m);
        else
            ntt_forward(c, b, m);
    });
}

spfhe_status spfhe_plan_matches(const spfhe_sparse_meta *A_csr, const spfhe_sparse_meta *B_csc, int32_t *out,
                                uint64_t *n_matches)
{
    return guard([&] {
        need(A_csr && B_csc && n_matches, "null argument");
        validate_pair(*A_csr, *B_csc);
        std::vector<MatchRec> m = plan_alg1(*A_csr, *B_csc);
        if (out) {
            need(*n_matches >= m.size(), "output array too small");
            for (size_t x = 0; x < m.size(); ++x) {
                out[5 * x + 0] = m[x].i;
                out[5 * x + 1] = m[x].j;
                out[5 * x + 2] = m[x].k;
                out[5 * x + 3] = m[x].a_pos;
                out[5 * x + 4] = m[x].b_pos;
            }
        }
        *n_matches = m.size();
    });
}

spfhe_status spfhe_sparse_matmul_ct_ct(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_sparse_meta *A_csr,
                                       spfhe_ct *const *A_chunks, size_t n_a, const spfhe_sparse_meta *B_csc,
                                       spfhe_ct *const *B_chunks, size_t n_b, const spfhe_pt *mask0,
                                       spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats)
{
    return guard([&] {
        need(keys && A_csr && B_csc && A_chunks && B_chunks && C_chunks, "null argument");
        Ctx &c = C(ctx);
        std::vector<Ct *> a(n_a), b(n_b), out(n_c, nullptr);
        for (size_t i = 0; i < n_a; ++i) a[i] = A_chunks[i] ? A_chunks[i]->c : nullptr;
        for (size_t i = 0; i < n_b; ++i) b[i] = B_chunks[i] ? B_chunks[i]->c : nullptr;
        spmspm_ct_ct(c, *keys->k, *A_csr, a.data(), n_a, *B_csc, b.data(), n_b, mask0 ? mask0->p : nullptr,
                     out.data(), n_c, stats);
        for (size_t i = 0; i < n_c; ++i) C_chunks[i] = wrap(out[i]);
    });
}

spfhe_status spfhe_naive_matmul_ct_ct(spfhe_ctx *ctx, const spfhe_keys *keys, int mode, int32_t rows,
                                      int32_t inner, int32_t cols, const uint8_t *A_nonzero,
                                      const uint8_t *B_nonzero, spfhe_ct *const *A_chunks, size_t n_a,
                                      spfhe_ct *const *B_chunks, size_t n_b, const spfhe_pt *mask0,
                                      spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats)
{
    return guard([&] {
        need(keys && A_chunks && B_chunks && C_chunks, "null argument");
        Ctx &c = C(ctx);
        std::vector<Ct *> a(n_a), b(n_b), out(n_c, nullptr);
        for (size_t i = 0; i < n_a; ++i) a[i] = A_chunks[i] ? A_chunks[i]->c : nullptr;
        for (size_t i = 0; i < n_b; ++i) b[i] = B_chunks[i] ? B_chunks[i]->c : nullptr;
        naive_ct_ct(c, *keys->k, mode, rows, inner, cols, A_nonzero, B_nonzero, a.data(), n_a, b.data(), n_b,
                    mask0 ? mask0->p : nullptr, out.data(), n_c, stats);
        for (size_t i = 0; i < n_c; ++i) C_chunks[i] = wrap(out[i]);
    });
}

spfhe_status spfhe_sparse_matmul_ct_ct_grouped(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_sparse_meta *A_csr,
                                               spfhe_ct *const *A_chunks, size_t n_a, const spfhe_sparse_meta *B_csc,
                                               spfhe_ct *const *B_chunks, size_t n_b, const spfhe_pt *mask0,
                                               int merge_digits, spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats)
{
    return guard([&] {
        need(keys && A_csr && B_csc && A_chunks && B_chunks && C_chunks, "null argument");
        Ctx &c = C(ctx);
        std::vector<Ct *> a(n_a), b(n_b), out(n_c, nullptr);
        for (size_t i = 0; i < n_a; ++i) a[i] = A_chunks[i] ? A_chunks[i]->c : nullptr;
        for (size_t i = 0; i < n_b; ++i) b[i] = B_chunks[i] ? B_chunks[i]->c : nullptr;
        spmspm_ct_ct_grouped(c, *keys->k, *A_csr, a.data(), n_a, *B_csc, b.data(), n_b, mask0 ? mask0->p : nullptr,
                             merge_digits != 0, out.data(), n_c, stats);
        for (size_t i = 0; i < n_c; ++i) C_chunks[i] = wrap(out[i]);
    });
}

spfhe_status spfhe_sparse_matmul_ct_pt_grouped(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_sparse_meta *A_csr,
                                               spfhe_ct *const *A_chunks, size_t n_a, const spfhe_sparse_meta *B_csc,
                                               const double *B_values, spfhe_pt *const *B_pts, int merge_digits,
                                               spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats)
{
    return guard([&] {
        need(keys && A_csr && B_csc && A_chunks && C_chunks, "null argument");
        need(n_a > 0, "no operand chunks");
        Ctx &c = C(ctx);
        std::vector<Ct *> a(n_a), out(n_c, nullptr);
        for (size_t i = 0; i < n_a; ++i) a[i] = A_chunks[i] ? A_chunks[i]->c : nullptr;
        std::vector<Pt *> bp;
        if (B_pts) {
            bp.resize(B_csc->nnz);
            for (int i = 0; i < B_csc->nnz; ++i) bp[i] = B_pts[i] ? B_pts[i]->p : nullptr;
        }
        spmspm_ct_pt_grouped(c, *keys->k, *A_csr, a.data(), n_a, *B_csc, B_values, B_pts ? bp.data() : nullptr,
                             merge_digits != 0, out.data(), n_c, stats);
        for (size_t i = 0; i < n_c; ++i) C_chunks[i] = wrap(out[i]);
    });
}

spfhe_status spfhe_sparse_matmul_ct_pt(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_sparse_meta *A_csr,
                                       spfhe_ct *const *A_chunks, size_t n_a, const spfhe_sparse_meta *B_csc,
                                       const double *B_values, spfhe_pt *const *B_pts, spfhe_ct **C_chunks,
                                       size_t n_c, spfhe_stats *stats)
{
    return guard([&] {
        need(keys && A_csr && B_csc && A_chunks && C_chunks, "null argument");
        Ctx &c = C(ctx);
        std::vector<Ct *> a(n_a), out(n_c, nullptr);
        for (size_t i = 0; i < n_a; ++i) a[i] = A_chunks[i] ? A_chunks[i]->c : nullptr;
        std::vector<Pt *> bp;
        if (B_pts) {
            bp.resize(B_csc->nnz);
            for (int i = 0; i < B_csc->nnz; ++i) bp[i] = B_pts[i] ? B_pts[i]->p : nullptr;
        }
        spmspm_ct_pt(c, *keys->k, *A_csr, a.data(), n_a, *B_csc, B_values, B_pts ? bp.data() : nullptr, out.data(),
                     n_c, stats);
        for (size_t i = 0; i < n_c; ++i) C_chunks[i] = wrap(out[i]);
    });
}

}  // extern "C"
