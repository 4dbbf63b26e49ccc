/*
 * Plain CPU reference ("oracle") for the RNS-CKKS ring arithmetic that the
 * encrypted sparse x sparse matmul of "GPU Acceleration of Sparse Fully
 * Homomorphic Encrypted DNNs" (Alg. 1 and Alg. 2) issues.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Conventions
 *   - Every polynomial is held in the COEFFICIENT domain, one limb per modulus,
 *     residues in [0, q).  Ring R_q = Z_q[X]/(X^n + 1).
 *   - Arithmetic is exact: 128-bit products reduced with the '%' operator.
 *   - Moduli are NTT-friendly primes q = 1 (mod 2n) below 2^62.
 *
 * Nothing here is blocked, fused or reordered for speed: each routine is the
 * definition of the operation, with a radix-2 NTT used as the polynomial
 * multiplication primitive (itself pinned against the O(n^2) definitions
 * or_ntt_direct and or_negacyclic_schoolbook by the tests).  Loops over
 * independent limbs may run on several OpenMP threads (OMP_NUM_THREADS);
 * every limb is computed by the same code either way.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic                                           */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - b) % q); }

u64 or_powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime q (Fermat) */
u64 or_invmod(u64 a, u64 q) { return or_powmod(a, q - 2, q); }

/* Deterministic Miller-Rabin: the first 12 primes as bases are enough for
 * every n < 3.3e24, hence for every 64-bit n. */
int or_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Primes q = 1 (mod 2n) below 2^bits, searched downward from 2^bits in steps
 * of 2n (candidates 2^bits + 1 - 2n*k, k = 1, 2, ...), skipping any value
 * listed in `exclude`.  Returns the number written (== count on success). */
int or_gen_primes(int log_n, int bits, int count, const u64 *exclude, int n_ex, u64 *out)
{
    u64 two_n = (u64)2 << log_n;
    u64 top = (u64)1 << bits;
    int found = 0;
    for (u64 k = 1; found < count; k++) {
        if (k * two_n >= top) break;
        u64 c = top + 1 - k * two_n;
        int skip = 0;
        for (int e = 0; e < n_ex; e++) if (exclude[e] == c) skip = 1;
        for (int e = 0; e < found; e++) if (out[e] == c) skip = 1;
        if (skip) continue;
        if (or_is_prime(c)) out[found++] = c;
    }
    return found;
}

/* psi = x^((q-1)/2n) for the first x = 2, 3, ... with psi^n = -1 (mod q):
 * a primitive 2n-th root of unity. */
u64 or_find_psi(u64 q, int log_n)
{
    u64 n = (u64)1 << log_n;
    for (u64 x = 2; x < q; x++) {
        u64 psi = or_powmod(x, (q - 1) / (2 * n), q);
        if (or_powmod(psi, n, q) == q - 1) return psi;
    }
    return 0;
}

static unsigned brv(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ------------------------------------------------------------------ */
/* negacyclic NTT                                                      */
/* ------------------------------------------------------------------ */
/* tab[k] = x^brv(k) mod q for k in [0, n) */
static void power_table_brv(u64 x, int log_n, u64 q, u64 *tab)
{
    unsigned n = 1u << log_n;
    u64 p = 1;
    for (unsigned j = 0; j < n; j++) {
        tab[brv(j, log_n)] = p;
        p = mulmod(p, x, q);
    }
}

/* Definition (O(n^2)): out[k] = sum_j a[j] * psi^((2*brv(k)+1)*j) mod q,
 * i.e. the evaluation of a(X) at the odd powers of psi, in bit-reversed
 * order of k. */
void or_ntt_direct(const u64 *a, u64 *out, int log_n, u64 q, u64 psi)
{
    unsigned n = 1u << log_n;
    for (unsigned k = 0; k < n; k++) {
        u64 x = or_powmod(psi, 2 * (u64)brv(k, log_n) + 1, q);
        u64 acc = 0, xp = 1;
        for (unsigned j = 0; j < n; j++) {
            acc = addmod(acc, mulmod(a[j], xp, q), q);
            xp = mulmod(xp, x, q);
        }
        out[k] = acc;
    }
}

/* Textbook radix-2 Cooley-Tukey transform with psi merged into the twiddles
 * (bit-reversed output).  Produces exactly or_ntt_direct's result. */
void or_ntt_fwd(u64 *a, int log_n, u64 q, u64 psi)
{
    unsigned n = 1u << log_n;
    u64 *psi_rev = (u64 *)malloc(sizeof(u64) * n);
    power_table_brv(psi, log_n, q, psi_rev);
    unsigned t = n;
    for (unsigned m = 1; m < n; m <<= 1) {
        t >>= 1;
        for (unsigned i = 0; i < m; i++) {
            u64 w = psi_rev[m + i];
            for (unsigned j = 2 * i * t; j < 2 * i * t + t; j++) {
                u64 u = a[j];
                u64 v = mulmod(a[j + t], w, q);
                a[j] = addmod(u, v, q);
                a[j + t] = submod(u, v, q);
            }
        }
    }
    free(psi_rev);
}

/* Gentleman-Sande inverse of or_ntt_fwd (bit-reversed input, natural output),
 * including the final multiplication by n^{-1}. */
void or_ntt_inv(u64 *a, int log_n, u64 q, u64 psi)
{
    unsigned n = 1u << log_n;
    u64 psi_inv = or_invmod(psi, q);
    u64 *ipsi_rev = (u64 *)malloc(sizeof(u64) * n);
    power_table_brv(psi_inv, log_n, q, ipsi_rev);
    unsigned t = 1;
    for (unsigned m = n >> 1; m >= 1; m >>= 1) {
        for (unsigned i = 0; i < m; i++) {
            u64 w = ipsi_rev[m + i];
            for (unsigned j = 2 * i * t; j < 2 * i * t + t; j++) {
                u64 u = a[j];
                u64 v = a[j + t];
                a[j] = addmod(u, v, q);
                a[j + t] = mulmod(submod(u, v, q), w, q);
            }
        }
        t <<= 1;
    }
    u64 n_inv = or_invmod(n % q, q);
    for (unsigned j = 0; j < n; j++) a[j] = mulmod(a[j], n_inv, q);
    free(ipsi_rev);
}

/* Schoolbook product in Z_q[X]/(X^n + 1) (O(n^2) definition). */
void or_negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *out, int n, u64 q)
{
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            u64 p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);   /* X^n = -1 */
        }
}

/* Ring product a*b in R_q through the NTT: INTT(NTT(a) . NTT(b)). */
void or_polymul(const u64 *a, const u64 *b, u64 *out, int log_n, u64 q, u64 psi)
{
    unsigned n = 1u << log_n;
    u64 *fa = (u64 *)malloc(sizeof(u64) * n), *fb = (u64 *)malloc(sizeof(u64) * n);
    memcpy(fa, a, sizeof(u64) * n);
    memcpy(fb, b, sizeof(u64) * n);
    or_ntt_fwd(fa, log_n, q, psi);
    or_ntt_fwd(fb, log_n, q, psi);
    for (unsigned k = 0; k < n; k++) out[k] = mulmod(fa[k], fb[k], q);
    or_ntt_inv(out, log_n, q, psi);
    free(fa);
    free(fb);
}

/* Galois automorphism sigma_g: a(X) -> a(X^g), g odd, in the coefficient
 * domain: X^j -> X^(j*g mod 2n), and X^(n+i) = -X^i. */
void or_automorphism(const u64 *a, u64 *out, int n, u64 g, u64 q)
{
    u64 two_n = 2 * (u64)n;
    for (int j = 0; j < n; j++) {
        u64 t = ((u64)j * g) % two_n;
        if (t < (u64)n) out[t] = a[j];
        else out[t - n] = a[j] == 0 ? 0 : q - a[j];
    }
}

/* Fast (approximate) basis conversion from the moduli src[0..ns) to each
 * modulus dst[t], coefficient-wise, without the overflow correction:
 *   D = prod src,  y_i = [x_i * (D/src_i)^{-1}]_{src_i},
 *   out_t = sum_i y_i * (D/src_i mod dst_t)  mod dst_t.
 * The output represents x + u*D for some 0 <= u < ns.
 * x: ns limbs of n coefficients; out: nd limbs of n coefficients. */
void or_bconv(const u64 *x, const u64 *src, int ns, u64 *out, const u64 *dst, int nd, int n)
{
    u64 *hat_inv = (u64 *)malloc(sizeof(u64) * ns);   /* (D/src_i)^{-1} mod src_i */
    u64 *hat_mod = (u64 *)malloc(sizeof(u64) * ns * nd); /* D/src_i mod dst_t */
    for (int i = 0; i < ns; i++) {
        u64 h = 1;
        for (int k = 0; k < ns; k++) if (k != i) h = mulmod(h, src[k] % src[i], src[i]);
        hat_inv[i] = or_invmod(h, src[i]);
        for (int t = 0; t < nd; t++) {
            u64 ht = 1 % dst[t];
            for (int k = 0; k < ns; k++) if (k != i) ht = mulmod(ht, src[k] % dst[t], dst[t]);
            hat_mod[i * nd + t] = ht;
        }
    }
    u64 *y = (u64 *)malloc(sizeof(u64) * ns);
    for (int c = 0; c < n; c++) {
        for (int i = 0; i < ns; i++) y[i] = mulmod(x[(size_t)i * n + c], hat_inv[i], src[i]);
        for (int t = 0; t < nd; t++) {
            u64 acc = 0;
            for (int i = 0; i < ns; i++)
                acc = addmod(acc, mulmod(y[i] % dst[t], hat_mod[i * nd + t], dst[t]), dst[t]);
            out[(size_t)t * n + c] = acc;
        }
    }
    free(y);
    free(hat_inv);
    free(hat_mod);
}

/* Conversion of x (limbs over the moduli src[0..ns)) to its CENTRED
 * representative [x]_D in [-D/2, D/2), D = prod src, reduced mod dst[t]:
 *   y_i = [x_i * (D/src_i)^{-1}]_{src_i},
 *   v   = round(f),  f = fma(y_i, 1/src_i, f) over i ascending from f = 0
 *         (IEEE double; 1/src_i the correctly rounded reciprocal),
 *   out_t = sum_i y_i * (D/src_i) - v * D   mod dst_t.
 * sum_i y_i (D/src_i) equals x mod D plus u*D with u = floor(sum_i y_i/src_i);
 * subtracting round(.) instead removes that overflow and centres the result
 * (the floating-point correction of Halevi, Polyakov and Shoup, "An Improved
 * RNS Variant of the BFV Homomorphic Encryption Scheme", CT-RSA 2019).  A
 * fractional part within ~2^-50 of one half may round the other way, giving
 * the other representative; the value is then off by D on that coefficient. */
void or_bconv_centred(const u64 *x, const u64 *src, int ns, u64 *out, const u64 *dst, int nd, int n)
{
    u64 *hat_inv = (u64 *)malloc(sizeof(u64) * ns);
    u64 *hat_mod = (u64 *)malloc(sizeof(u64) * ns * nd);
    u64 *D_mod = (u64 *)malloc(sizeof(u64) * nd);
    for (int i = 0; i < ns; i++) {
        u64 h = 1;
        for (int k = 0; k < ns; k++) if (k != i) h = mulmod(h, src[k] % src[i], src[i]);
        hat_inv[i] = or_invmod(h, src[i]);
        for (int t = 0; t < nd; t++) {
            u64 ht = 1 % dst[t];
            for (int k = 0; k < ns; k++) if (k != i) ht = mulmod(ht, src[k] % dst[t], dst[t]);
            hat_mod[i * nd + t] = ht;
        }
    }
    for (int t = 0; t < nd; t++) {
        u64 d = 1 % dst[t];
        for (int k = 0; k < ns; k++) d = mulmod(d, src[k] % dst[t], dst[t]);
        D_mod[t] = d;
    }
    u64 *y = (u64 *)malloc(sizeof(u64) * ns);
    double *inv = (double *)malloc(sizeof(double) * ns);
    for (int i = 0; i < ns; i++) inv[i] = 1.0 / (double)src[i];
    for (int c = 0; c < n; c++) {
        double f = 0.0;
        for (int i = 0; i < ns; i++) {
            y[i] = mulmod(x[(size_t)i * n + c], hat_inv[i], src[i]);
            f = fma((double)y[i], inv[i], f);
        }
        u64 v = (u64)nearbyint(f);
        for (int t = 0; t < nd; t++) {
            u64 acc = 0;
            for (int i = 0; i < ns; i++) acc = addmod(acc, mulmod(y[i], hat_mod[i * nd + t], dst[t]), dst[t]);
            out[(size_t)t * n + c] = submod(acc, mulmod(v, D_mod[t], dst[t]), dst[t]);
        }
    }
    free(y);
    free(inv);
    free(D_mod);
    free(hat_inv);
    free(hat_mod);
}

/* ------------------------------------------------------------------ */
/* CKKS over a fixed parameter set                                     */
/* ------------------------------------------------------------------ */
/* Moduli are indexed q_0..q_{L-1} then p_0..p_{K-1} (mods[L+k] = p_k).
 * A polynomial "at level ell" has ell limbs q_0..q_{ell-1}.  The extended
 * basis of key switching at level ell is Q_ell u P, ordered q_0..q_{ell-1},
 * p_0..p_{K-1}. */
typedef struct {
    int log_n, L, K, dnum;
    u64 mods[96];
    u64 psis[96];
} or_params;

static int ext_mod_index(const or_params *P, int ell, int t) { return t < ell ? t : P->L + (t - ell); }

/* Hybrid key switching of one polynomial c (ell limbs) with the switching
 * key ksk = {(k0_j, k1_j)}_j stored as [dnum][2][L+K][n] (coefficient
 * domain, limbs over the full basis q_0..q_{L-1}, p_0..p_{K-1}).
 *   digits: consecutive groups of alpha = ceil(L/dnum) limbs of Q_ell
 *   ModUp:  digit j -> Q_ell u P: the centred representative of the digit
 *           value modulo its modulus Q_j (or_bconv_centred) is converted to
 *           every other modulus; the digit's own limbs are kept as they are
 *   IP:     acc_b = sum_j ext_j * k_b,j  (ring products, limb by limb)
 *   ModDown: out_b = (acc_b|Q - [acc_b]_P) * P^{-1}  mod q_i with [.]_P the
 *            centred representative (or_bconv_centred), i.e. out_b is
 *            acc_b / P rounded to the nearest integer, coefficient-wise
 * out0, out1: ell limbs each. */
/* ModUp of every digit of c (ell limbs, coefficient domain): ext receives
 * [beta][ell + K][n], digit j's own limbs copied, every other limb the
 * centred base conversion of the digit (reading R12). */
void or_modup(const or_params *P, const u64 *c, int ell, u64 *ext)
{
    int n = 1 << P->log_n, L = P->L, K = P->K, dnum = P->dnum;
    int alpha = (L + dnum - 1) / dnum;
    int n_ext = ell + K;
    int beta = (ell + alpha - 1) / alpha;
    size_t ln = (size_t)n;
    u64 ext_mods[96];
    for (int t = 0; t < n_ext; t++) ext_mods[t] = P->mods[ext_mod_index(P, ell, t)];
    for (int j = 0; j < beta; j++) {
        int lo = j * alpha, hi = (j + 1) * alpha < ell ? (j + 1) * alpha : ell;
        u64 *e = ext + (size_t)j * n_ext * ln;
#pragma omp parallel for schedule(dynamic)
        for (int t = 0; t < n_ext; t++) {
            if (t >= lo && t < hi) memcpy(e + t * ln, c + t * ln, sizeof(u64) * ln);
            else or_bconv_centred(c + lo * ln, P->mods + lo, hi - lo, e + t * ln, &ext_mods[t], 1, n);
        }
    }
}

/* Inner product of the ModUp digits (or_modup's layout), each limb first
 * mapped by the automorphism X -> X^g (g = 1: unchanged), with the
 * switching key, then ModDown to ell limbs: out0, out1. */
void or_ks_ext(const or_params *P, const u64 *ext, int ell, const u64 *ksk, uint64_t g, u64 *out0, u64 *out1)
{
    int n = 1 << P->log_n, L = P->L, K = P->K, dnum = P->dnum;
    int alpha = (L + dnum - 1) / dnum;
    int n_ext = ell + K;
    int beta = (ell + alpha - 1) / alpha;
    size_t ln = (size_t)n;
    u64 *acc[2];
    acc[0] = (u64 *)calloc(n_ext * ln, sizeof(u64));
    acc[1] = (u64 *)calloc(n_ext * ln, sizeof(u64));
    for (int j = 0; j < beta; j++) {
        const u64 *e = ext + (size_t)j * n_ext * ln;
#pragma omp parallel for collapse(2) schedule(dynamic)
        for (int b = 0; b < 2; b++) {
            for (int t = 0; t < n_ext; t++) {
                int mi = ext_mod_index(P, ell, t);
                const u64 *key = ksk + (((size_t)j * 2 + b) * (L + K) + mi) * ln;
                u64 *pr = (u64 *)malloc(sizeof(u64) * ln);
                const u64 *src = e + t * ln;
                u64 *perm = NULL;
                if (g != 1) {
                    perm = (u64 *)malloc(sizeof(u64) * ln);
                    or_automorphism(src, perm, n, g, P->mods[mi]);
                    src = perm;
                }
                or_polymul(src, key, pr, P->log_n, P->mods[mi], P->psis[mi]);
                for (int k = 0; k < n; k++)
                    acc[b][t * ln + k] = addmod(acc[b][t * ln + k], pr[k], P->mods[mi]);
                free(pr);
                free(perm);
            }
        }
    }
    /* ModDown */
    u64 Pmod_inv[96];
    for (int i = 0; i < ell; i++) {
        u64 pm = 1;
        for (int k = 0; k < K; k++) pm = mulmod(pm, P->mods[L + k] % P->mods[i], P->mods[i]);
        Pmod_inv[i] = or_invmod(pm, P->mods[i]);
    }
    u64 *conv = (u64 *)malloc(sizeof(u64) * ell * ln);
    for (int b = 0; b < 2; b++) {
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < ell; i++)
            or_bconv_centred(acc[b] + (size_t)ell * ln, P->mods + L, K, conv + (size_t)i * ln, P->mods + i, 1, n);
        u64 *out = b == 0 ? out0 : out1;
        for (int i = 0; i < ell; i++)
            for (int k = 0; k < n; k++)
                out[i * ln + k] = mulmod(submod(acc[b][i * ln + k], conv[i * ln + k], P->mods[i]),
                                         Pmod_inv[i], P->mods[i]);
    }
    free(conv);
    free(acc[0]);
    free(acc[1]);
}

/* Hybrid key switching of c (ell limbs, coefficient domain) with ksk
 * ([dnum][2][L+K][n]): ModUp, inner product, ModDown. */
void or_keyswitch(const or_params *P, const u64 *c, int ell, const u64 *ksk, u64 *out0, u64 *out1)
{
    int L = P->L, K = P->K, dnum = P->dnum;
    int alpha = (L + dnum - 1) / dnum;
    int beta = (ell + alpha - 1) / alpha;
    size_t words = (size_t)beta * (ell + K) * ((size_t)1 << P->log_n);
    u64 *ext = (u64 *)malloc(sizeof(u64) * words);
    or_modup(P, c, ell, ext);
    or_ks_ext(P, ext, ell, ksk, 1, out0, out1);
    free(ext);
}

/* Rescale one polynomial in place from ell to ell-1 limbs by the top prime
 * q_t = q_{ell-1}: r = centred residue of limb ell-1 in (-q_t/2, q_t/2],
 * then c_i <- (c_i - [r]_{q_i}) * q_t^{-1} mod q_i. */
void or_rescale(const or_params *P, u64 *poly, int ell)
{
    int n = 1 << P->log_n;
    size_t ln = (size_t)n;
    u64 qt = P->mods[ell - 1];
    const u64 *top = poly + (size_t)(ell - 1) * ln;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < ell - 1; i++) {
        u64 qi = P->mods[i];
        u64 qt_inv = or_invmod(qt % qi, qi);
        for (int k = 0; k < n; k++) {
            u64 r = top[k];
            u64 r_mod;
            if (r > qt / 2) r_mod = submod(0, (qt - r) % qi, qi);  /* negative representative */
            else r_mod = r % qi;
            poly[i * ln + k] = mulmod(submod(poly[i * ln + k], r_mod, qi), qt_inv, qi);
        }
    }
}

/* Limb-wise ring product of two RNS polynomials of nl limbs over the moduli
 * with indices mi[0..nl). */
void or_rns_polymul(const or_params *P, const u64 *a, const u64 *b, u64 *out, int nl, const int *mi)
{
    size_t ln = (size_t)1 << P->log_n;
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nl; l++)
        or_polymul(a + l * ln, b + l * ln, out + l * ln, P->log_n, P->mods[mi[l]], P->psis[mi[l]]);
}

/* Limb-wise NTT (forward) of an RNS polynomial: used only to express
 * coefficient-domain results in the evaluation representation. */
void or_rns_ntt_fwd(const or_params *P, u64 *a, int nl, const int *mi)
{
    size_t ln = (size_t)1 << P->log_n;
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nl; l++) or_ntt_fwd(a + l * ln, P->log_n, P->mods[mi[l]], P->psis[mi[l]]);
}

void or_rns_ntt_inv(const or_params *P, u64 *a, int nl, const int *mi)
{
    size_t ln = (size_t)1 << P->log_n;
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nl; l++) or_ntt_inv(a + l * ln, P->log_n, P->mods[mi[l]], P->psis[mi[l]]);
}

/* OpenMP threads used by the limb loops (0 = leave unchanged); returns the
 * current maximum. */
int or_threads(int nthreads)
{
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
}

/* a*b mod q for numpy callers (vectorised over cnt elements) */
void or_mulmod_vec(const u64 *a, const u64 *b, u64 *out, size_t cnt, u64 q)
{
    for (size_t i = 0; i < cnt; i++) out[i] = mulmod(a[i], b[i], q);
}

/* a*s mod q for a scalar s */
void or_mulmod_scalar(const u64 *a, u64 s, u64 *out, size_t cnt, u64 q)
{
    for (size_t i = 0; i < cnt; i++) out[i] = mulmod(a[i], s, q);
}
