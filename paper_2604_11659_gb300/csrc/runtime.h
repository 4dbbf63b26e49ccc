// Runtime services of a context and the batched CKKS evaluator (ckks.cpp).
#pragma once
#include "kernels.h"

namespace spfhe {

void configure_pool(int device);

struct Runtime {
    static constexpr int kWorkspaceSlots = 24;
    static constexpr size_t kRingBytes = 8u << 20;
    struct Buf {
        u64 *p = nullptr;
        size_t words = 0;
    };
    Ctx &ctx;
    Buf ws[kWorkspaceSlots];
    char *ring_host = nullptr;
    char *ring_dev = nullptr;
    size_t ring_off = 0;
    explicit Runtime(Ctx &c) : ctx(c) {}
    // persistent device buffer `slot` of at least `words` u64 (contents not kept on growth)
    u64 *workspace(int slot, size_t words);
    // copy a small host table to device memory valid for work enqueued after it
    void *upload(const void *host, size_t bytes);
    template <typename T> T *upload_vec(const std::vector<T> &v) {
        return static_cast<T *>(upload(v.data(), v.size() * sizeof(T)));
    }
    void release();
};

// workspace slot ids
enum WsSlot {
    WS_KS_COEF = 0,
    WS_KS_EXT,
    WS_KS_ACC,
    WS_KS_CONV,
    WS_ROT_TMP,
    WS_ROT_OUT_A,
    WS_ROT_OUT_B,
    WS_RS_TMP,
    WS_TENSOR,
    WS_RELIN_OUT,
    WS_LEVEL1,
    WS_LEVEL2,
    WS_ALIGN,
    WS_MASK,
    WS_PTS,
    WS_MISC,
    WS_GRP_SUM,
    WS_TREE_ROT,
    WS_HOIST_EXT,
    WS_ROT_SUM,   // per-target sums of the last rotation step's conversions
};

// ---- batched evaluator (ckks.cpp) ----
// Key switch `items` polynomials ([ell][n], evaluation rep., pointers in
// d_in); see moddown() for base/out.
void keyswitch_batch(Ctx &ctx, int items, int ell, const u64 *const *d_in, const std::vector<KeyGroup> &groups,
                     const u64 *const *d_base, const int *d_base_g, bool base_c1, u64 *out, long long out_stride);

// Relinearisation of d_in (the tensor's d2, [ell][n] per item) added to the
// base d_base ((d0, d1), [2][ell][n] per item), then rescaled: out
// [items][2][ell-1][n], bit for bit keyswitch_batch followed by rescale, with
// one forward transform per output limb (ModDown's are folded into the
// rescale's; see ckks.cpp).  tmp holds items * 2 * ell * n words.  Needs
// relin_rescale_supported (fused epilogues, n >= 2^12, NTT variant 5 or 6).
bool relin_rescale_supported(const Ctx &ctx, int ell);
// mask / mask_g (device arrays, or nullptr): the rescaled output is also
// multiplied by mask[item] (Montgomery form, [ell-1][n]) read through
// sigma_{mask_g[item]}, as mul_plain_perm would afterwards.
void relin_rescale_batch(Ctx &ctx, int items, int ell, const u64 *const *d_in, const std::vector<KeyGroup> &groups,
                         const u64 *const *d_base, u64 *tmp, u64 *out, long long out_stride,
                         const u64 *const *mask = nullptr, const int *mask_g = nullptr);

// One rotation step per item: item i of `in` ([2][ell][n]) rotated with
// Galois element g[i] and key keys[i]; out [items][2][ell][n].
void rotate_step_batch(Ctx &ctx, int ell, const std::vector<const u64 *> &in, const std::vector<int> &g,
                       const std::vector<const u64 *> &keys, u64 *out);

// Rotation of item i by r[i] through the plan, added into tgt[i]
// ([2][ell][n], evaluation rep.): bit for bit rotate_batch followed by the
// sums, with the last step's ModDown transforms taken once per target (see
// ckks.cpp).  Uses the WS_ROT_* (WS_ROT_SUM included), WS_KS_* and WS_MISC
// workspaces; needs rotate_accumulate_supported (fused epilogues, n >= 2^12,
// NTT variant 5 or 6).  Counts the key switches in *ks.
bool rotate_accumulate_supported(const Ctx &ctx);
// One rotation step per source (Galois element g[j], key keys[j]; equal keys
// next to each other) added into tgt[j] (which holds its initial value); one
// forward transform per distinct target (see ckks.cpp).
void rotate_step_accumulate(Ctx &ctx, int ell, const std::vector<const u64 *> &in, const std::vector<int> &g,
                            const std::vector<const u64 *> &keys, const std::vector<u64 *> &tgt);
void rotate_accumulate_batch(Ctx &ctx, const std::vector<const Keys *> &keys, int ell,
                             const std::vector<const u64 *> &in, const std::vector<int> &r,
                             const std::vector<u64 *> &tgt, uint64_t *ks);

// Full plan rotation of each item by amount r[i] (left, any integer);
// results in out [items][2][ell][n].  counts the key switches in *ks.
void rotate_batch(Ctx &ctx, const Keys &keys, int ell, const std::vector<const u64 *> &in,
                  const std::vector<int> &r, u64 *out, uint64_t *ks);
// the same with a key set per item
void rotate_batch(Ctx &ctx, const std::vector<const Keys *> &keys, int ell, const std::vector<const u64 *> &in,
                  const std::vector<int> &r, u64 *out, uint64_t *ks);

// Rotations of one ciphertext src ([2][ell][n]) by every amount (each with a
// key of its own, 0 < amount < S) sharing one ModUp of its c1: the
// automorphism is applied to the extended digits in the inner product.
// out [amounts][2][ell][n].
void rotate_hoisted(Ctx &ctx, const Keys &keys, int ell, const u64 *src, const std::vector<int> &amounts, u64 *out);

std::vector<int> rotation_plan(const Ctx &ctx, long long r);
int match_batch_size(const Ctx &ctx);   // matches per batch (engine.cpp)
int galois_element(const Ctx &ctx, int r);   // 5^r mod 2n
const u64 *rotation_key(const Keys &keys, int amount);

// Keys, ciphertexts (keys.cpp)
std::vector<int> plan_key_amounts(const Ctx &ctx);
Keys *keygen(Ctx &ctx, uint64_t seed);
Keys *keys_import(Ctx &ctx, const int64_t *secret, const u64 *relin, size_t n_rot, const int32_t *amounts,
                  const u64 *const *rot);
void keys_export(Ctx &ctx, const Keys &k, int64_t *secret, u64 *relin, size_t *n_rot, int32_t *amounts,
                 u64 *const *rot);
void free_keys(Keys *k);
Ct *ct_new(Ctx &ctx, int level, double scale);
Pt *pt_new(Ctx &ctx, int level, double scale);
Ct *encrypt(Ctx &ctx, const Keys &keys, const Pt &pt, uint64_t seed);
Pt *decrypt(Ctx &ctx, const Keys &keys, const Ct &ct);

// Alg. 1 planner and the encrypted products (spmspm.cpp)
struct MatchRec {
    int i, j, k, a_pos, b_pos;
};
std::vector<MatchRec> plan_alg1(const spfhe_sparse_meta &A, const spfhe_sparse_meta &B);
void validate_pair(const spfhe_sparse_meta &A, const spfhe_sparse_meta &B);
void spmspm_ct_ct(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                  const spfhe_sparse_meta &B, Ct *const *Bch, size_t nB, const Pt *mask0, Ct **C, size_t nC,
                  spfhe_stats *out_stats);
void spmspm_ct_pt(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                  const spfhe_sparse_meta &B, const double *Bvals, Pt *const *Bpts, Ct **C, size_t nC,
                  spfhe_stats *out_stats);

// Encoding helpers (encode.cu)
std::vector<long long> encode_host(const Ctx &ctx, const double *re, const double *im, size_t nv, double scale);
void decode_host(const Ctx &ctx, const std::vector<u64> &limb0, double scale, double *re, double *im, size_t nv);
void ensure_cos_table(Ctx &ctx);
// device: out [items][ell][n] = residues of round_half_away(v_i * (2 scale/n) cos(pi j/n))
void encode_onehot0(Ctx &ctx, const double *d_values, int items, int ell, double scale, u64 *out);
// device: out [segments][ell][n] (evaluation rep.) = per segment, the sum of
// the one-hot encodings of values[c] at slots p_c, each taken as the
// automorphism 5^-p_c of the slot-0 encoding (d_ginv[c] = 5^p_c mod 2n)
void encode_onehot_sums(Ctx &ctx, int segments, const int *d_seg, const double *d_values, const int *d_ginv, int ell,
                        double scale, u64 *out);

}  // namespace spfhe
