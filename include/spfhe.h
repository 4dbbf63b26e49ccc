/*
 * spfhe.h -- C ABI of the GB300 (sm_103a) encrypted sparse x sparse matmul.
 *
 * The library multiplies CKKS-encrypted sparse matrices held in the CSR
 * (left operand) x CSC (right operand) packing of "GPU Acceleration of Sparse
 * Fully Homomorphic Encrypted DNNs" (Sec. 3, Alg. 1 and Alg. 2).  Every ring
 * operation runs in sm_103a CUDA kernels; the host only walks the plaintext
 * sparsity metadata (Sec. 3.2.1: indptr/indices stay in the clear, values are
 * encrypted) and sequences kernel launches.
 *
 * Representation
 *   - Ring R_q = Z_q[X]/(X^n + 1), n = 2^log_n, S = n/2 slots.  Moduli are
 *     q_0 .. q_{L-1} then the special primes p_0 .. p_{K-1} (global modulus
 *     index 0 .. L+K-1), all primes = 1 (mod 2n) below 2^62, chosen by
 *     searching downward from 2^bits in steps of 2n (q_0 first, scaling primes
 *     next, special primes last, all distinct).  psi_q is x^((q-1)/2n) for the
 *     first x = 2, 3, ... with psi^n = -1.
 *   - A polynomial at level ell has ell limbs (q_0 .. q_{ell-1}) of n uint64
 *     residues in [0, q), limb-major.  "Evaluation representation" (the one
 *     every handle stores) is the negacyclic NTT: limb value at index k is
 *     a(psi^(2 brv(k) + 1)) mod q, brv = log_n-bit reversal.
 *   - Ciphertext (c0, c1) is stored as [2][ell][n]; a plaintext as [ell][n].
 *   - Slot i of the canonical embedding is m(zeta^(5^i)), zeta = e^(i pi/n).
 *     Rotation by r (> 0) is a LEFT rotation: slot i + r moves to slot i
 *     (EvalRotate of Alg. 1/Alg. 2), realised as X -> X^(5^r mod 2n) followed
 *     by hybrid key switching.  Amounts are applied through the base-b plan:
 *     r mod S written in base b = rot_base, one key switch with the key for
 *     d*b^t per nonzero digit d, ascending t.
 *
 * Conventions
 *   - Every call returns spfhe_status (0 = OK, < 0 = error).  No exception
 *     crosses the ABI.  spfhe_last_error() returns a thread-local message for
 *     the most recent failing call of the calling thread.
 *   - Handles (ctx, keys, ct, pt) are opaque and owned by the caller, who
 *     frees them with the matching *_free / *_destroy call.  Their device
 *     memory lives on the GPU that was current at spfhe_ctx_create.
 *   - Host arrays passed in (metadata, values, imported limbs) are borrowed
 *     for the duration of the call only.
 *   - Work is enqueued on the context's CUDA stream; results are ready after
 *     spfhe_sync(ctx) (or a synchronisation of that stream).  Calls that
 *     return data to host memory synchronise the stream themselves.
 *   - A context and its handles must not be used from two threads at once.
 */
#ifndef SPFHE_H
#define SPFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPFHE_OK = 0,
    SPFHE_EINVAL = -1,   /* bad argument: null pointer, malformed CSR/CSC, size out of range */
    SPFHE_ENOMEM = -2,   /* device or host allocation failed */
    SPFHE_ELEVEL = -3,   /* not enough levels left for the operation */
    SPFHE_EKEY = -4,     /* a needed switching key is missing */
    SPFHE_ESCALE = -5,   /* operands' scales differ beyond 1e-9 relative */
    SPFHE_ECUDA = -6,    /* a CUDA runtime call failed */
    SPFHE_ETIMEOUT = -7, /* a bounded device-side wait gave up */
    SPFHE_EPARAM = -8    /* parameter set cannot be built (no primes, too many limbs, ...) */
} spfhe_status;

typedef struct spfhe_ctx spfhe_ctx;
typedef struct spfhe_keys spfhe_keys;
typedef struct spfhe_ct spfhe_ct;
typedef struct spfhe_pt spfhe_pt;

/* CKKS parameter set.  The paper states none (Sec. 4 gives matrix sizes
 * only); these fields carry the workload's ring degree, prime sizes, key
 * switching digits and scale. */
typedef struct {
    uint32_t log_n;          /* ring degree n = 2^log_n, 2 <= log_n <= 17 */
    uint32_t L;              /* number of q primes (top level), 3 <= L <= 64 */
    const uint32_t *q_bits;  /* L bit sizes: q_0 then the scaling primes; each in [20, 60] */
    uint32_t K;              /* number of special primes, 1 <= K <= 16 */
    uint32_t p_bits;         /* bit size of each special prime, in [20, 60] */
    uint32_t dnum;           /* key-switching digits; alpha = ceil(L/dnum) limbs per digit */
    double scale;            /* encoding scale Delta of fresh ciphertexts */
    uint32_t rot_base;       /* rotation plan base b (power of two >= 2) */
} spfhe_params;

/* Plaintext sparsity metadata (Sec. 3.2.1 keeps it in the clear).
 * CSR (left operand): rows = matrix rows, cols = inner dimension, indptr has
 * rows+1 entries, indices are column ids sorted ascending within each row.
 * CSC (right operand): rows = inner dimension, cols = matrix columns, indptr
 * has cols+1 column pointers, indices are row ids sorted ascending within
 * each column.  nnz = indptr[last]. */
typedef struct {
    int32_t rows;
    int32_t cols;
    int32_t nnz;
    const int32_t *indptr;
    const int32_t *indices;
} spfhe_sparse_meta;

/* Per-call counters (Sec. 4.3's complexity model counts the matches). */
typedef struct {
    uint64_t matches;     /* (i, j, k) triples with A[i,k] != 0 and B[k,j] != 0 */
    uint64_t ks_relin;    /* relinearisation key switches */
    uint64_t ks_align;    /* key switches spent aligning operands (Alg. 1) */
    uint64_t ks_final;    /* key switches of the final per-match rotations (Alg. 2) */
    uint64_t rescales;    /* ciphertext rescales */
    uint64_t launches;    /* CUDA kernels launched by the call */
} spfhe_stats;

/* ---- errors, context ------------------------------------------------- */
const char *spfhe_last_error(void);

/* Build the primes, NTT tables and base-conversion constants and upload them.
 * cuda_stream: a cudaStream_t to enqueue work on (NULL = the default
 * stream); the stream must outlive the context.  *out receives the context. */
spfhe_status spfhe_ctx_create(const spfhe_params *params, void *cuda_stream, spfhe_ctx **out);
spfhe_status spfhe_ctx_destroy(spfhe_ctx *ctx);

/* Copy the L+K moduli (q's then p's) and their psi roots to host arrays of
 * L+K entries each (either may be NULL). */
spfhe_status spfhe_ctx_moduli(const spfhe_ctx *ctx, uint64_t *mods, uint64_t *psis);

/* Block the host until every operation enqueued on the context is done. */
spfhe_status spfhe_sync(spfhe_ctx *ctx);

/* Matches per batch of the encrypted products (and alignment rotations per
 * wave): 1 .. 1024, or 0 for the default (64).  Larger
 * batches share each relinearisation key stream over more matches and need
 * about 320 MB of batch buffers per match at n = 2^16, L = 24. */
spfhe_status spfhe_ctx_set_match_batch(spfhe_ctx *ctx, uint32_t matches);

/* Limbs per launch pair of the two-pass NTT (n >= 2^12): a batch of
 * transforms is cut into pieces of at most this many limbs, each running
 * both passes before the next piece starts, so that the second pass reads
 * the first pass's output from L2.  0 (default) = one launch pair for the
 * whole batch; 1 .. 2^20 otherwise.  Results do not depend on it. */
spfhe_status spfhe_ctx_set_ntt_chunk(spfhe_ctx *ctx, uint32_t limbs);

/* Stages of the first pass of the two-pass NTT (n >= 2^12; the second pass
 * takes the other log_n - pass_a_stages); both passes must have 6 to 9
 * stages, else EINVAL.  0 (default) = log_n / 2.  Results do not depend on
 * it. */
spfhe_status spfhe_ctx_set_ntt_split(spfhe_ctx *ctx, uint32_t pass_a_stages);

/* Kernel variant of the two-pass NTT (n >= 2^12): 0 = twiddles read per
 * butterfly stage from global memory at 3 CTAs per SM; 1 = the same with the
 * register budget of 2 CTAs per SM; 2 = as 1, with the second pass copying
 * its twiddles into shared memory asynchronously before its data loads
 * (about 64 KB of dynamic shared memory per CTA); 3 = as 0 with the register
 * budget of 4 CTAs per SM; 4 = as 3 with every 32x32-bit partial product of
 * the Shoup multiplications taken as separate low and high halves instead of
 * one 64-bit-result multiply; 5 = as 4 with a shorter quotient estimate
 * (products in [0, 4q), intermediate values kept below 8q); 6 (default) = as
 * 5 with the second pass synchronising warps instead of whole CTAs (a tile
 * of the second pass never spans two warps).  EINVAL otherwise.  Results do
 * not depend on it. */
spfhe_status spfhe_ctx_set_ntt_variant(spfhe_ctx *ctx, uint32_t variant);

/* Device memory (bytes) spfhe_sparse_matmul_ct_ct_grouped may hold in
 * alignment rotations for a whole call (default: no limit but the free
 * memory).  Above it, or when they do not fit in the free memory, each batch
 * of result groups computes the rotations its matches use and frees them
 * afterwards (more key switches, bounded memory).  Results do not depend on
 * it. */
spfhe_status spfhe_ctx_set_align_budget(spfhe_ctx *ctx, uint64_t bytes);

/* enable != 0 (default): ModDown's last step ((acc - conv) P^{-1} + base) and
 * the rescale's spread and last step run inside the forward transforms that
 * feed them (kernel variant 0 or 3 to 6, n >= 2^12); 0: as separate kernels.  Results
 * do not depend on it. */
spfhe_status spfhe_ctx_set_fusion(spfhe_ctx *ctx, int enable);

/* Number of kernels the library has launched since the context was created. */
uint64_t spfhe_launch_count(const spfhe_ctx *ctx);

/* Kernel profiler.  spfhe_prof_enable(ctx, 1) clears the counters and starts
 * bracketing every kernel launch with two CUDA events on the context stream
 * (0 stops it).  spfhe_prof_read(ctx, cls, ...) synchronises the stream and
 * returns for kernel class cls (0 .. spfhe_prof_classes()-1) the launches,
 * the summed device time of the timed launches in milliseconds, and the
 * algorithmic bytes (each input and output limb counted once) and work
 * (butterflies for transforms, modular multiply-accumulates otherwise)
 * implied by the launch shapes.  Any out-pointer may be NULL. */
spfhe_status spfhe_prof_enable(spfhe_ctx *ctx, int enable);
spfhe_status spfhe_prof_read(spfhe_ctx *ctx, int cls, uint64_t *launches, double *ms, double *bytes, double *work);
int spfhe_prof_classes(void);
/* For a transform class: limbs transformed since spfhe_prof_enable by pass
 * kind (the transforms run in two passes over each limb): first passes,
 * second passes, and second passes with a fused epilogue (ModDown's or the
 * rescale's final step).  Counted whether or not the profiler is on. */
spfhe_status spfhe_prof_transform_limbs(spfhe_ctx *ctx, int cls, double *first, double *second,
                                        double *second_fused);
const char *spfhe_prof_class_name(int cls);
/* Key switching as a whole since the last spfhe_prof_enable: number of
 * key-switched polynomials and their algorithmic bytes (input polynomial,
 * output pair, and the switching key once per group of polynomials that
 * share it in one launch). */
spfhe_status spfhe_prof_keyswitch(spfhe_ctx *ctx, uint64_t *calls, double *bytes);
/* Measured arithmetic speed of light of the GPU behind ctx, the ALU roofline
 * of the transforms and base conversions (64-bit modular arithmetic on the
 * INT32 multiply pipe).  Three register-resident microbenchmarks run on the
 * context stream with the transforms' launch shape (4 CTAs of 256 threads per
 * SM, four waves), each timed with CUDA events after one warm-up launch and
 * a few milliseconds long: lazy forward NTT butterflies with the transforms'
 * truncated-quotient Shoup product, its partial products taken as 64-bit
 * results (kernel variants 0-3) and as split 32-bit halves (variant 4)
 * (butterflies per second), and independent
 * chains of 32-bit multiply-adds with a 32-bit (mad.lo) and a 64-bit
 * (mad.wide) result (operations per second).  No memory traffic beyond one
 * store per thread.  A measurement aid: the paper times wall-clock runs
 * only (Sec. 4) and has no counterpart.  Any out-pointer may be NULL;
 * synchronises the stream.  Errors: SPFHE_EINVAL (null ctx, called during
 * graph capture), SPFHE_ENOMEM, SPFHE_ECUDA. */
spfhe_status spfhe_prof_alu_peak(spfhe_ctx *ctx, double *butterflies_per_s, double *butterflies_split_per_s,
                                 double *imad_per_s, double *imad_wide_per_s);
/* The same microbenchmarks with every butterfly form the transforms use:
 * rates[0..2] = butterflies/s with the truncated-quotient Shoup product as
 * wide products, as split halves, and with the shorter quotient (products in
 * [0, 4q)); rates[3..5] = 32-bit multiply-adds per second with a 32-bit
 * result, a 64-bit result, and the high half.  n >= 6. */
spfhe_status spfhe_prof_alu_rates(spfhe_ctx *ctx, double *rates, size_t n);

/* ---- keys ------------------------------------------------------------ */
/* Sample a ternary secret, the relinearisation key and one rotation key per
 * amount the rotation plan can request (d*b^t < S, 1 <= d < b) on the GPU,
 * from a ChaCha20 stream keyed by `seed` (Gaussian errors sigma = 3.2,
 * |e| <= 6 sigma).  Keys stay resident on the device. */
spfhe_status spfhe_keygen(spfhe_ctx *ctx, uint64_t seed, spfhe_keys **out);

/* Import keys computed elsewhere (used to feed identical keys to two
 * implementations).  secret: n int64 coefficients in {-1, 0, 1}.
 * relin: [dnum][2][L+K][n] uint64, evaluation representation, key for
 * s^2 -> s.  rot: n_rot pointers to keys of the same layout for
 * sigma_{5^amount}(s) -> s, amounts in rot_amounts (each in [1, S)).
 * The key of digit j must hold P mod q_i on the limbs q_i of digit j and 0
 * on every other modulus as its gadget, P = prod p_k. */
spfhe_status spfhe_keys_import(spfhe_ctx *ctx, const int64_t *secret, const uint64_t *relin,
                               size_t n_rot, const int32_t *rot_amounts, const uint64_t *const *rot,
                               spfhe_keys **out);
/* Checkpoint of a key set: writes what spfhe_keys_import takes back, so keys
 * made by spfhe_keygen survive the process or move to another context with
 * the same parameters.  The paper describes no key storage; it notes that
 * switching keys take hundreds of MB each (Sec. 1), which is what a restart
 * would otherwise regenerate.  secret: n int64
 * coefficients in {-1, 0, 1}, or NULL.  relin: [dnum][2][L+K][n] uint64,
 * evaluation representation (the import layout), or NULL.  Rotation keys:
 * with rot_amounts = NULL only their count is written to *n_rot; otherwise
 * *n_rot gives the room in rot_amounts (int32, written in ascending order)
 * and rot (NULL, or *n_rot pointers, each NULL or a buffer of the relin
 * layout), and receives the count.  Buffers may be host or device memory;
 * the call synchronises the context stream.  Errors: SPFHE_EINVAL (null
 * ctx/keys/n_rot, keys of another context, room for fewer keys than the set
 * holds), SPFHE_EKEY (relin requested from a set imported without one),
 * SPFHE_ENOMEM, SPFHE_ECUDA. */
spfhe_status spfhe_keys_export(spfhe_ctx *ctx, const spfhe_keys *keys, int64_t *secret, uint64_t *relin,
                               size_t *n_rot, int32_t *rot_amounts, uint64_t *const *rot);
void spfhe_keys_free(spfhe_keys *keys);

/* ---- plaintexts --------------------------------------------------------- */
/* Canonical-embedding encoding of n_vals <= S complex slots (re, im; im may be
 * NULL) at `level` and `scale`: m_j = round_half_away((2 scale/n) Re
 * sum_i z_i zeta^(-5^i j)), reduced into each limb and transformed. */
spfhe_status spfhe_encode(spfhe_ctx *ctx, const double *re, const double *im, size_t n_vals,
                          uint32_t level, double scale, spfhe_pt **out);

/* Import a plaintext given as `level` limbs of n uint64 residues (host
 * memory); coeff_domain != 0 means coefficient representation (the library
 * transforms it), 0 means evaluation representation. */
spfhe_status spfhe_pt_import(spfhe_ctx *ctx, const uint64_t *limbs, uint32_t level, double scale,
                             int coeff_domain, spfhe_pt **out);
/* Copy the evaluation-representation limbs ([level][n]) to host memory. */
spfhe_status spfhe_pt_export(spfhe_ctx *ctx, const spfhe_pt *pt, uint64_t *limbs);
spfhe_status spfhe_pt_info(const spfhe_pt *pt, uint32_t *level, double *scale);
void spfhe_pt_free(spfhe_pt *pt);

/* Decode slots 0 .. n_vals-1 of a plaintext (limb q_0, centred residues),
 * dividing by the plaintext's scale.  re/im host arrays of n_vals (im may be
 * NULL). */
spfhe_status spfhe_decode(spfhe_ctx *ctx, const spfhe_pt *pt, double *re, double *im, size_t n_vals);

/* ---- ciphertexts -------------------------------------------------------- */
/* Secret-key encryption (c0, c1) = (-a s + e + m, a) with a and e drawn on the
 * GPU from a ChaCha20 stream keyed by `seed`. */
spfhe_status spfhe_encrypt(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_pt *pt, uint64_t seed,
                           spfhe_ct **out);
/* m = c0 + c1 s at the ciphertext's level (evaluation representation). */
spfhe_status spfhe_decrypt(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_ct *ct, spfhe_pt **out);

/* Import/export a ciphertext as [2][level][n] uint64 in evaluation
 * representation.  `limbs` may point to host (pageable or pinned) or device
 * memory; the copy is enqueued on the context stream and export waits for it. */
spfhe_status spfhe_ct_import(spfhe_ctx *ctx, const uint64_t *limbs, uint32_t level, double scale,
                             spfhe_ct **out);

/* Replace the contents of ct (its level and scale unchanged) with 2 * level *
 * n words in the layout of spfhe_ct_import, from host or device memory;
 * asynchronous on the context stream (a host buffer must stay unchanged
 * until the copy is done).  Lets a captured graph (spfhe_matmul_graph_*)
 * run on new operands. */
spfhe_status spfhe_ct_overwrite(spfhe_ctx *ctx, spfhe_ct *ct, const uint64_t *limbs);
spfhe_status spfhe_ct_export(spfhe_ctx *ctx, const spfhe_ct *ct, uint64_t *limbs);
spfhe_status spfhe_ct_info(const spfhe_ct *ct, uint32_t *level, double *scale);
void spfhe_ct_free(spfhe_ct *ct);

/* ---- single homomorphic operations (Alg. 2's building blocks) ---------- */
/* EvalMult + Relinearize: tensor product then key switch of the s^2 part
 * (Sec. 3.2.2, Alg. 2).  Operands at the same level; out at that level with
 * scale = product of scales. */
spfhe_status spfhe_mult_relin(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_ct *a, const spfhe_ct *b,
                              spfhe_ct **out);
/* Rescale in place: drop q_{ell-1}, c_i <- (c_i - [r]_{q_i}) q_{ell-1}^{-1} with r
 * the centred residue of limb ell-1; scale /= q_{ell-1} (Sec. 3.2.2). */
spfhe_status spfhe_rescale(spfhe_ctx *ctx, spfhe_ct *ct);
/* EvalRotate (left by r, any integer) through the rotation plan. */
spfhe_status spfhe_rotate(spfhe_ctx *ctx, const spfhe_keys *keys, const spfhe_ct *ct, int32_t r, spfhe_ct **out);
/* Product with a plaintext at the same level; scale = product of scales. */
spfhe_status spfhe_mul_plain(spfhe_ctx *ctx, const spfhe_ct *ct, const spfhe_pt *pt, spfhe_ct **out);
/* EvalAdd: out = a + b (same level, scales equal within 1e-9 relative). */
spfhe_status spfhe_add(spfhe_ctx *ctx, const spfhe_ct *a, const spfhe_ct *b, spfhe_ct **out);

/* In-place negacyclic NTT of n_limbs device-resident limbs (limb l holds n
 * residues for modulus index mod_idx[l], mod_idx a host array).  inverse != 0
 * runs the inverse transform (including the n^{-1} factor). */
spfhe_status spfhe_ntt(spfhe_ctx *ctx, uint64_t *dev_limbs, uint32_t n_limbs, const int32_t *mod_idx,
                       int inverse);

/* Rescale that allocates nothing (the paper has no counterpart: this is a
 * service for callers that cannot allocate device memory while they run, e.g.
 * a process that owns a fixed GPU memory budget and hands the library
 * pre-sized buffers).  Same result as spfhe_rescale, bit for bit.
 * in:  device pointer to a ciphertext [2][level][n] (evaluation rep.);
 * out: device pointer receiving [2][level-1][n]; must not overlap `in`.
 * Both stay owned by the caller.  The call enqueues its work on the context
 * stream and returns; synchronise before reading `out`.
 * Scratch lives in a fixed 2 MiB device array (2 * 2^17 words) that every
 * process loading the library reserves on each GPU it uses until exit; all
 * calls on a GPU share it, so calls that overlap on the GPU (different
 * streams) race on it.  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  No
 * cudaMalloc/cudaFree or other allocating routine is called.
 * Errors: SPFHE_EINVAL (null pointer, ring needing more than the fixed
 * scratch), SPFHE_ELEVEL (level < 2 or > L), SPFHE_ECUDA. */
spfhe_status spfhe_rescale_noalloc(spfhe_ctx *ctx, const uint64_t *in, uint32_t level, uint64_t *out);

/* ---- Alg. 1 planner ------------------------------------------------------ */
/* Alg. 1's merge over every (i, j): returns the matches in Alg. 1 order as
 * (i, j, k, a_pos, b_pos) rows.  Call with out = NULL to get the count in
 * *n_matches; then with out pointing at 5 * count int32. */
spfhe_status spfhe_plan_matches(const spfhe_sparse_meta *A_csr, const spfhe_sparse_meta *B_csc,
                                int32_t *out, uint64_t *n_matches);

/* ---- encrypted sparse x sparse matmul ------------------------------------- */
/* C = A B with both operands encrypted (Alg. 1 + Alg. 2).
 * A_chunks: ceil(nnz_A / S) ciphertexts at level L, scale Delta, with CSR
 * data[p] in slot p mod S of chunk p / S (zero padding elsewhere).
 * B_chunks: the same for B's CSC data.  mask0: NULL, or a plaintext at level
 * L-1 encoding the one-hot slot-0 vector at scale q_{L-2} (the library then
 * derives every mask from it; when NULL it encodes its own).
 * C_chunks (out): caller array of n_c = ceil(rows*cols / S) handle slots that
 * receive the result chunks at level L-2, scale Delta^2/q_{L-1}: C[i,j] in
 * slot t mod S of chunk t / S, t = i*cols + j.  stats may be NULL.
 * Requires L >= 3.  Missing rotation keys give SPFHE_EKEY. */
spfhe_status spfhe_sparse_matmul_ct_ct(spfhe_ctx *ctx, const spfhe_keys *keys,
                                       const spfhe_sparse_meta *A_csr, spfhe_ct *const *A_chunks, size_t n_a,
                                       const spfhe_sparse_meta *B_csc, spfhe_ct *const *B_chunks, size_t n_b,
                                       const spfhe_pt *mask0, spfhe_ct **C_chunks, size_t n_c,
                                       spfhe_stats *stats);

/* ---- the paper's element-wise baselines (Sec. 4) ------------------------ */
/* Naive Dense multiplies every element pair individually; Naive Sparse is
 * element-wise too but skips pairs by the zero pattern (the paper's prior
 * method).  SPFHE_NAIVE_SPARSE skips a pair when either value is zero (the
 * exact product with the fewest products: the pairs Alg. 1 matches);
 * SPFHE_NAIVE_SPARSE_LITERAL skips it only when both are zero, as printed. */
typedef enum { SPFHE_NAIVE_DENSE = 0, SPFHE_NAIVE_SPARSE = 1, SPFHE_NAIVE_SPARSE_LITERAL = 2 } spfhe_naive_mode;
/* C = A B through an element-wise baseline over densely packed operands:
 * A (rows x inner) row-major, element (i, k) in slot (i*inner + k) mod S of
 * chunk (i*inner + k) / S, n_a = ceil(rows*inner / S) ciphertexts; B (inner x
 * cols) row-major the same way, n_b = ceil(inner*cols / S).  A_nonzero /
 * B_nonzero: host arrays of rows*inner / inner*cols bytes, nonzero where the
 * element is nonzero (plaintext structure, like the CSR/CSC metadata of the
 * sparse product; read during the call only).  For every pair (i, j, k) the
 * mode keeps, in the order i, j, k, both ciphertexts are rotated so the two
 * elements sit in slot 0 (one rotation per operand, none when already
 * there), then Alg. 2's chain runs with the mask at slot 0 and the final
 * rotation to t = i*cols + j.  mask0, C_chunks (n_c = ceil(rows*cols / S)),
 * levels, scales and errors as in spfhe_sparse_matmul_ct_ct; stats.matches
 * counts the pairs computed. */
spfhe_status spfhe_naive_matmul_ct_ct(spfhe_ctx *ctx, const spfhe_keys *keys, int mode, int32_t rows,
                                      int32_t inner, int32_t cols, const uint8_t *A_nonzero,
                                      const uint8_t *B_nonzero, spfhe_ct *const *A_chunks, size_t n_a,
                                      spfhe_ct *const *B_chunks, size_t n_b, const spfhe_pt *mask0,
                                      spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats);

/* C = A B with A encrypted (packed as above) and B a plaintext (CSC).  Per
 * match the weight plaintext encodes B[k,j] in A's slot at scale q_{L-1}
 * (alignment of B becomes re-encoding, the mask merges into it), then
 * product, rescale, final rotation, add: depth 1.  B_values: nnz_B doubles
 * in CSC order.  B_pts: NULL, or nnz_B plaintexts at level L encoding
 * B[k,j] * e_0 at scale q_{L-1} (used in place of the library's own
 * encodings).  C_chunks at level L-1, scale Delta. */
spfhe_status spfhe_sparse_matmul_ct_pt(spfhe_ctx *ctx, const spfhe_keys *keys,
                                       const spfhe_sparse_meta *A_csr, spfhe_ct *const *A_chunks, size_t n_a,
                                       const spfhe_sparse_meta *B_csc, const double *B_values,
                                       spfhe_pt *const *B_pts, spfhe_ct **C_chunks, size_t n_c,
                                       spfhe_stats *stats);

/* Lazy-accumulation variant of spfhe_sparse_matmul_ct_ct (a library
 * extension that reorders Alg. 2; the paper has no counterpart).  Alignment
 * rotations and tensor products are Alg. 2's; each tensor product is
 * multiplied by its mask and summed into the group of matches sharing the
 * result chunk and the final rotation amount r; each group is rescaled,
 * relinearised (at level L-1), rescaled again and rotated, by the lowest
 * base-b digit of r when
 * merge_digits != 0 (the rotated groups are then summed per remaining amount
 * and rotated digit by digit) or by the whole of r otherwise.  The result
 * decrypts like Alg. 2's product (relinearisation and rotation are linear),
 * with one relinearisation per group instead of per match and fewer
 * final-rotation key switches; its ciphertext bits differ from Alg. 2's.
 * Arguments as spfhe_sparse_matmul_ct_ct, except mask0: NULL or the slot-0
 * one-hot plaintext at the operands' level L (not L-1), scale q_{L-2}.
 * stats: ks_relin counts groups, rescales two per group.  Every distinct alignment rotation is held in device memory for
 * the whole call: SPFHE_ENOMEM (before any launch) when it and the digit
 * tree's accumulators do not fit.  Blocks until the result is ready. */
spfhe_status spfhe_sparse_matmul_ct_ct_grouped(spfhe_ctx *ctx, const spfhe_keys *keys,
                                               const spfhe_sparse_meta *A_csr, spfhe_ct *const *A_chunks, size_t n_a,
                                               const spfhe_sparse_meta *B_csc, spfhe_ct *const *B_chunks, size_t n_b,
                                               const spfhe_pt *mask0, int merge_digits, spfhe_ct **C_chunks,
                                               size_t n_c, spfhe_stats *stats);

/* Lazy-accumulation variant of spfhe_sparse_matmul_ct_pt (a library
 * extension that reorders the ct x pt products; the paper has no
 * counterpart).  The weight plaintexts B[k, j] e_{a_slot} of the matches that
 * share the result chunk and the final rotation amount r are summed per A
 * chunk, each sum multiplies its chunk, a group's products are added,
 * rescaled once and rotated as in spfhe_sparse_matmul_ct_ct_grouped (digit by
 * digit when merge_digits != 0).  Arguments, result level and scale as
 * spfhe_sparse_matmul_ct_pt; stats: rescales counts groups.  Blocks until the
 * result is ready. */
spfhe_status spfhe_sparse_matmul_ct_pt_grouped(spfhe_ctx *ctx, const spfhe_keys *keys,
                                               const spfhe_sparse_meta *A_csr, spfhe_ct *const *A_chunks, size_t n_a,
                                               const spfhe_sparse_meta *B_csc, const double *B_values,
                                               spfhe_pt *const *B_pts, int merge_digits, spfhe_ct **C_chunks,
                                               size_t n_c, spfhe_stats *stats);

/* NTT launch-chunk tuner (library extension; the paper has no tuner).  Times
 * the key-switching transforms of one match batch at level ell (forward NTT
 * of the ModUp extension of `items` polynomials, inverse NTT of their ell
 * input limbs) on scratch device buffers, three repetitions after one
 * warm-up, for each of the n_candidates chunk sizes (see
 * spfhe_ctx_set_ntt_chunk), sets the fastest on the context and returns it
 * in *best; ms (n_candidates entries, may be NULL) receives the time per
 * repetition.  Blocks the host; allocates and frees its buffers on the
 * context stream.  EINVAL for bad shapes or candidates, ENOMEM when the
 * buffers do not fit. */
spfhe_status spfhe_tune_ntt_chunk(spfhe_ctx *ctx, uint32_t ell, uint32_t items, const uint32_t *candidates,
                                  uint32_t n_candidates, uint32_t *best, double *ms);

/* Rotation-plan base tuner (host only, no GPU work).  For the product A x B
 * (Alg. 1's plan on the metadata) at ring degree 2^log_n with L, K, dnum,
 * returns in *base the power of two b whose rotation plan needs the fewest
 * key switches (distinct alignment rotations plus every final rotation; one
 * key switch per nonzero base-b digit) among the bases whose rotation keys
 * (every d*b^t < S, 1 <= d < b, each dnum*2*(L+K)*n words) fit
 * key_budget_bytes; ties go to the smaller key set.  key_switches and
 * key_bytes (may be NULL) receive that base's counts.  SPFHE_ENOMEM if no
 * base fits. */
spfhe_status spfhe_tune_rotation_base(uint32_t log_n, uint32_t L, uint32_t K, uint32_t dnum,
                                      const spfhe_sparse_meta *A_csr, const spfhe_sparse_meta *B_csc,
                                      uint64_t key_budget_bytes, uint32_t *base, uint64_t *key_switches,
                                      uint64_t *key_bytes);

/* ---- many products in one call, and the serving loop -------------------- */
/* One encrypted product request (ct x ct, Alg. 1 + Alg. 2).  Fields as in
 * spfhe_sparse_matmul_ct_ct; the operand chunks may sit at any level >= 3
 * (all chunks of one request at the same level); results come back at that
 * level - 2.  keys may differ between requests. */
typedef struct {
    const spfhe_keys *keys;
    const spfhe_sparse_meta *A_csr;
    spfhe_ct *const *A_chunks;
    size_t n_a;
    const spfhe_sparse_meta *B_csc;
    spfhe_ct *const *B_chunks;
    size_t n_b;
    const spfhe_pt *mask0;   /* NULL: the library's own mask */
} spfhe_matmul_req;

/* n_req products in one call: their alignment rotations and matches are
 * planned together and executed in shared batches (requests at the same
 * level share launches; each relinearisation key stream serves every match
 * of a batch that uses it).  C_chunks receives, request after request, each
 * request's ceil(rows*cols / S) result chunks (n_c_total in all).  Every
 * result is bit-identical to the one spfhe_sparse_matmul_ct_ct returns for the
 * same request alone.  stats: NULL or n_req entries (launches counts the whole
 * call). */
spfhe_status spfhe_sparse_matmul_batch(spfhe_ctx *ctx, size_t n_req, const spfhe_matmul_req *reqs,
                                       spfhe_ct **C_chunks, size_t n_c_total, spfhe_stats *stats);

/* Continuous-batching server.  A worker thread owns the context until
 * spfhe_server_destroy: do not use the context (or its handles) from other
 * threads meanwhile, except through the server calls.  Between waves of
 * work the worker admits submitted requests in arrival order while
 * hbm_budget_bytes holds the engine's shared batch buffers (their size at the
 * highest level admitted so far) plus, for every admitted unfinished request,
 * its result chunks and its mask (the private copy of a caller's mask, or the
 * library's mask for its level when the context has none yet); a request is
 * always admitted when nothing else runs.  Admitted work is mixed into the
 * running batches; results are bit-identical to running each request alone.
 * A wave that fails does not fail the requests in it: those whose last kernel
 * had completed keep their results, the others are run again one at a time,
 * each alone, and only a request that fails by itself reports its error.
 * Operands and keys of a submitted request must stay alive until
 * spfhe_server_wait returns for it; its metadata is copied at submission. */
typedef struct spfhe_server spfhe_server;
spfhe_status spfhe_server_create(spfhe_ctx *ctx, uint64_t hbm_budget_bytes, spfhe_server **out);
spfhe_status spfhe_server_submit(spfhe_server *srv, const spfhe_matmul_req *req, uint64_t *ticket);
/* Block until request `ticket` is done; hand its n_c result chunks to the
 * caller; latency_ms = completion (its last kernel observed done) minus
 * submission, host clock.  Errors of the request (EKEY, ELEVEL, ...) are
 * returned here. */
spfhe_status spfhe_server_wait(spfhe_server *srv, uint64_t ticket, spfhe_ct **C_chunks, size_t n_c,
                               spfhe_stats *stats, double *latency_ms);
/* Finish every submitted request, stop the worker, free unclaimed results. */
spfhe_status spfhe_server_destroy(spfhe_server *srv);
/* Host-side fault injection for tests of the failure handling above: every
 * wave that would run work of request `ticket` fails with SPFHE_ECUDA before
 * launching anything (no GPU fault is involved).  `ticket` may name a request
 * not submitted yet (tickets are handed out 1, 2, 3, ... per server) or one
 * still queued; EINVAL for a request already admitted or no longer known. */
spfhe_status spfhe_server_inject_fault(spfhe_server *srv, uint64_t ticket);
/* Admission bookkeeping: bytes reserved for the shared batch buffers, bytes
 * held by admitted unfinished requests, and the number of requests re-run
 * alone after a failed wave.  Any pointer may be NULL. */
spfhe_status spfhe_server_info(spfhe_server *srv, uint64_t *workspace_reserved, uint64_t *in_use,
                               uint64_t *retried);

/* ---- products captured as one CUDA graph --------------------------------- */
/* A product planned and captured once into a CUDA graph, launched as one unit
 * (library extension for the batch-launch pattern; the paper has no
 * counterpart).  variant 0 = spfhe_sparse_matmul_ct_ct (Alg. 2), 1 =
 * spfhe_sparse_matmul_ct_ct_grouped with merge_digits.  The request's keys,
 * operand chunks and mask are read at every launch: they must outlive the
 * graph, and their contents may change between launches (same levels,
 * scales and sparsity).  The graph owns its device buffers (a workspace set
 * of its own, every scratch buffer, the result chunks) until
 * spfhe_matmul_graph_free.  Creation does no arithmetic; it blocks while it
 * plans and captures.  EINVAL for bad requests or a capture already running
 * on the context, EKEY/ELEVEL/ESCALE as the product, ENOMEM, ECUDA. */
typedef struct spfhe_graph spfhe_graph;
spfhe_status spfhe_matmul_graph_create(spfhe_ctx *ctx, const spfhe_matmul_req *req, int variant,
                                       spfhe_graph **out);
/* n_req >= 1 products captured into one graph.  variant 0: planned together
 * as spfhe_sparse_matmul_batch does (requests at the same level share
 * launches); variant 1: the grouped products one after another.  Each
 * request's results are bit-identical to its single call's.  Buffers the
 * products free while they are captured stay with the graph until
 * spfhe_matmul_graph_free, so the graph holds the sum of the products'
 * working sets (ENOMEM when they do not fit).  spfhe_matmul_graph_create is
 * this call with one request. */
spfhe_status spfhe_matmul_graph_create_batch(spfhe_ctx *ctx, size_t n_req, const spfhe_matmul_req *reqs,
                                             int variant, spfhe_graph **out);
/* Enqueue one launch of the graph on the context stream (asynchronous):
 * zeroes the result chunks and recomputes the product into them. */
spfhe_status spfhe_matmul_graph_launch(spfhe_graph *g);
/* Handles of the graph's n_c result chunks (valid after a launch completes;
 * n_c = the sum over its requests, request after request) and the products'
 * counters (stats: NULL or one entry per request); spfhe_ct_free on these
 * handles frees only the handle, the chunks belong to the graph. */
spfhe_status spfhe_matmul_graph_results(spfhe_graph *g, spfhe_ct **C_chunks, size_t n_c, spfhe_stats *stats);
/* Wait for the context stream and free the graph and everything it owns. */
void spfhe_matmul_graph_free(spfhe_graph *g);

#ifdef __cplusplus
}
#endif
#endif /* SPFHE_H */
