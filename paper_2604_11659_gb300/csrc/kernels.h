// Launchers for the sm_103a kernels (declared here, defined in ntt.cu / ring.cu).
#pragma once
#include "internal.h"

namespace spfhe {

// A batch of `items` equally laid-out blocks of limbs.  Item z starts at
// base + (ids ? ids[z] : z) * stride (in u64 words).
struct Batch {
    u64 *base;
    long long stride;
    int items;
    const int *ids;   // device array or nullptr
};

// ---- NTT (ntt.cu) ----
// Forward / inverse negacyclic NTT of the limbs `map` names in every item.
void ntt_forward(Ctx &ctx, Batch b, const LimbMap &map);

// Forward transforms with a fused prologue or epilogue (radix-16 sizes,
// kernel variant 0, 3 or 4, no item list; returns false otherwise and does
// nothing):
//   kFuseModDown: the transform of ModDown's conv [items][2][ell][n] writes
//     out = base[sigma(k)] + (acc - conv) P^{-1} instead of conv;
//   kFuseRescale: pass A reads [r]_{q_i} from the centred top limbs
//     (top [items][polys][n]) instead of a spread buffer, pass B writes
//     out = (in - [r]_{q_i}) q_t^{-1}; the batch is the spread buffer
//     [items][polys][ell-1][n] that holds the intermediate pass;
//   kFuseRelinRescale (variants 5 and 6 only): ModDown's last step and the
//     rescale that follows it in one transform (relin_rescale_batch): pass A
//     reads P^{-1} conv_b[i] + [t_b]_{q_i} (conv [items][2][ell][n]
//     coefficient rep., t_b the relinearised top limb's coefficients, top
//     [items][2][n]), pass B writes
//     out = (P^{-1} acc_b[i] + base_b[i] - X) q_t^{-1}, X the transform.
//     By linearity of the transform this is, residue for residue, ModDown's
//     output rescaled: the transform of conv and the one of [t]_{q_i} are
//     taken together.
//   kFuseRotAccum (variants 5 and 6 only): the last rotation step of
//     several key switches summed into their result ciphertexts
//     (rotate_accumulate_batch): the batch holds, per target t, the sum of
//     its sources' conv [2][ell][n]; pass B adds
//     sum_j sigma_{g_j}(c0_j) (polynomial 0) + P^{-1} (sum_j acc_j - X) to
//     outp[t], j over the sources seg[t] .. seg[t+1]-1 (acc index item[j],
//     c0 base[j], Galois element base_g[j]).
enum { kFuseNone = 0, kFuseModDown = 1, kFuseRescale = 2, kFuseRelinRescale = 3, kFuseRotAccum = 4 };
struct FuseArgs {
    int ell = 0, K = 0, polys = 0, base_c1 = 0;
    const u64 *acc = nullptr;
    const u64 *conv = nullptr;
    long long acc_stride = 0, out_stride = 0, conv_stride = 0;
    u64 *const *outp = nullptr;
    const int *seg = nullptr, *item = nullptr;
    // kFuseRelinRescale: optional per-item mask (Montgomery form, [ell-1][n],
    // read through sigma_{mask_g}) multiplied into the rescaled output
    const u64 *const *mask = nullptr;
    const int *mask_g = nullptr;
    const u64 *const *base = nullptr;
    const int *base_g = nullptr;
    u64 *out = nullptr;
    const u64 *pinv = nullptr, *pinvp = nullptr;
    const u64 *top = nullptr;
    const u64 *const *in = nullptr;
    const u64 *qt_mod = nullptr, *inv = nullptr, *invp = nullptr;
};
bool ntt_forward_fused(Ctx &ctx, Batch b, const LimbMap &map, int mode, const FuseArgs &f);
// scale = false leaves out the final factor n^{-1}: the limbs hold n x,
// below 4q but not reduced (for the key-switching base conversions, whose
// constants carry the n^{-1} instead)
void ntt_inverse(Ctx &ctx, Batch b, const LimbMap &map, bool scale = true);
// Out-of-place inverse transform: item z's limbs are read from src[z]
// (device array of pointers, same limb offsets as `map`) and the result is
// written to dst.  Radix-16 sizes, no item list and no launch chunking only;
// returns false otherwise and does nothing.
bool ntt_inverse_from(Ctx &ctx, Batch dst, const u64 *const *src, const LimbMap &map, bool scale = true);
LimbMap limb_range(int first_off, int count, int first_mi);

// ---- ring kernels (ring.cu) ----
// d[item] = (a0 b0, a0 b1 + a1 b0, a1 b1) with a, b given by per-item
// pointers to [2][ell][n] ciphertexts; d is [items][3][ell][n].
void tensor(Ctx &ctx, int items, int ell, const u64 *const *pa, const u64 *const *pb, u64 *d);

// out[item] = sigma_g(in[item]) in evaluation representation, for `polys`
// polynomials of ell limbs each.  g per item (device array).
void automorph(Ctx &ctx, int items, int polys, int ell, const u64 *const *in, long long in_stride_unused,
               u64 *out, long long out_stride, const int *g);

// ModUp basis conversion: coef [items][ell][n] (coefficient rep. of the
// key-switching input) -> ext [items][beta][ell+K][n] (targets outside each digit).
void modup_bconv(Ctx &ctx, int items, int ell, const u64 *coef, long long coef_stride, u64 *ext,
                 long long ext_stride);
// LimbMap of the ext limbs that need a forward NTT after modup_bconv.
LimbMap modup_ntt_map(const Ctx &ctx, int ell);

// Key-switching inner product.  in: per item the NTT-domain input polynomial
// ([ell][n]); ext: [items][beta][ell+K][n]; key per item group; acc:
// [items][2][ell+K][n].
struct KeyGroup {
    const u64 *key;    // [dnum][2][M][n] Montgomery form
    int first, count;  // items [first, first + count)
};
// Hoisted form (src_of, perm_g device arrays, else nullptr): item it reads
// the extension of source src_of[it] and in[it] through the automorphism
// X -> X^perm_g[it].
void ks_inner_product(Ctx &ctx, int items, int ell, const u64 *const *in, const u64 *ext, long long ext_stride,
                      const std::vector<KeyGroup> &groups, u64 *acc, long long acc_stride,
                      const int *src_of = nullptr, const int *perm_g = nullptr);

// ModDown: acc [items][2][ell+K][n] NTT domain.  P-limbs are inverse
// transformed in place, converted into conv [items][2][ell][n] (coefficient),
// transformed, then out[item][b] = base_b(perm) + (acc_b - conv_b) P^{-1}.
// base: per item [2][ell][n] (or nullptr), read at sigma_g index when g given.
void moddown(Ctx &ctx, int items, int ell, u64 *acc, long long acc_stride, u64 *conv,
             const u64 *const *base, const int *base_g, bool base_c1, u64 *out, long long out_stride);
// ModDown's first half: the P limbs of acc inverse transformed in place and
// converted into conv [items][2][ell][n] (coefficient rep.).
void moddown_conv(Ctx &ctx, int items, int ell, u64 *acc, long long acc_stride, u64 *conv);
// Coefficients of the relinearised ciphertext's top limb (modulus q_{ell-1}):
// top[item][b] = (acc_b[ell-1] - conv_b[ell-1]) P^{-1} + base_b[ell-1], with
// acc's top limbs and base's top limbs (top [items][2][n] on entry) already
// in coefficient rep.
void relin_top(Ctx &ctx, int items, int ell, const u64 *acc, long long acc_stride, const u64 *conv, u64 *top);
// k_copy_top: top[item][b] = in[item][b][ell-1] for b < polys
void copy_top(Ctx &ctx, int items, int ell, int polys, const u64 *const *in, u64 *top);

// Rescale every item [polys][ell][n] -> out [polys][ell-1][n] (polys 1..3);
// tmp holds items * polys * ell * n words.
void rescale(Ctx &ctx, int items, int ell, const u64 *const *in, u64 *tmp, u64 *out, long long out_stride,
             int polys = 2);

// ct[item] (= [polys][ell][n]) *= mask permuted by sigma_{g[item]}; mask
// [ell][n] in Montgomery form.
void mul_plain_perm(Ctx &ctx, int items, int ell, u64 *ct, long long stride, const u64 *const *mask,
                    const int *g, int polys = 2);

// Segmented sums over items of `polys` x ell limbs: tgt[g] (+)= sum of
// src[seg[g]] .. src[seg[g+1]-1]; `into` adds to tgt's own value.
void accumulate_seg(Ctx &ctx, int polys, int ell, int targets, u64 *const *tgt, const u64 *const *src,
                    const int *seg, int sources, bool into);

// result[2][ell][n] += sum over the listed items of x[item]
void accumulate(Ctx &ctx, int ell, u64 *result, const u64 *x, long long stride, const int *ids, int count);

// elementwise helpers
void add_ct(Ctx &ctx, int polys, int ell, const u64 *a, const u64 *b, u64 *out);
void mul_ct_pt(Ctx &ctx, int ell, const u64 *ct, const u64 *pt, u64 *out);           // pt standard form
void to_montgomery(Ctx &ctx, u64 *x, int limbs, const int *mi_host, int reps);         // in place
void from_montgomery(Ctx &ctx, u64 *x, int limbs, const int *mi_host, int reps);       // in place, x 2^-64
void from_signed(Ctx &ctx, const long long *coef, u64 *out, int limbs);                // out[l] = coef mod q_l
void decrypt_core(Ctx &ctx, int ell, const u64 *ct, const u64 *s_mont, u64 *out);      // c0 + c1 s
void copy_words(Ctx &ctx, u64 *dst, const u64 *src, size_t words);
// out + i*stride <- in[i] (words_per_item each); and the reverse
void gather_items(Ctx &ctx, int items, size_t words_per_item, const u64 *const *in, u64 *out, long long stride);
void scatter_items(Ctx &ctx, int items, size_t words_per_item, const u64 *src, long long stride, u64 *const *out);
// out[l] = a[l] * b[l] mod q_l (modulus index = limb index), limbs x n
void mul_poly(Ctx &ctx, int limbs, const u64 *a, const u64 *b, u64 *out);

// sampling (ChaCha20 stream keyed by seed, domain-separated by `stream_id`)
void sample_uniform(Ctx &ctx, u64 *out, int limbs, const int *mi_host, uint64_t seed, uint64_t stream_id);
void sample_ternary(Ctx &ctx, long long *out, uint64_t seed, uint64_t stream_id);
void sample_gaussian(Ctx &ctx, long long *out, uint64_t seed, uint64_t stream_id);
// out[l] = -(a[l] s_l) + e[l] + extra[l] (all evaluation rep.); s in Montgomery form.
void rlwe_b(Ctx &ctx, int limbs, const int *mi_host, const u64 *a, const u64 *s_mont, const u64 *e,
            const u64 *extra, u64 *out);
// out[l] = out[l] + gadget_l * sprime[l], gadget_l = P mod q for l in [lo, hi)
void add_gadget(Ctx &ctx, u64 *out, const u64 *sprime, int lo, int hi);

// launch bookkeeping: t = prof_begin(ctx); kernel<<<...>>>; prof_end(ctx, t, class,
// algorithmic bytes, algorithmic work, name).  prof_end counts the launch and
// turns a launch error into an Error.
cudaEvent_t prof_begin(Ctx &ctx);
void prof_end(Ctx &ctx, cudaEvent_t start, int cls, double bytes, double work, const char *what);
void prof_reset(Ctx &ctx, bool on);
// count `limbs` transformed limbs of pass kind `kind` (see Prof::limbs)
void prof_limbs(Ctx &ctx, int cls, int kind, double limbs);
// While one of these lives, launches made by the constructing thread record no
// profiler events (calls that must create no CUDA events of their own); the
// context's profiler switch itself is left untouched.
struct ProfSuppress {
    ProfSuppress();
    ~ProfSuppress();
    ProfSuppress(const ProfSuppress &) = delete;
    ProfSuppress &operator=(const ProfSuppress &) = delete;
};
void prof_collect(Ctx &ctx);
void prof_destroy(Ctx &ctx);
const char *kernel_class_name(int cls);

}  // namespace spfhe
