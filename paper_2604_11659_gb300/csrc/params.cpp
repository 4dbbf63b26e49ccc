// Parameter set construction: NTT-friendly primes, 2n-th roots, NTT twiddle
// tables and the constants of base conversion and rescale, uploaded once per
// context.  (CKKS parameters are not fixed by the paper; see spfhe.h for the
// selection rules.)
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace spfhe {

typedef unsigned __int128 u128;

u64 mulmod_host(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }

u64 powmod_host(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q, x = a % q;
    for (; e; e >>= 1) {
        if (e & 1) r = mulmod_host(r, x, q);
        x = mulmod_host(x, x, q);
    }
    return r;
}

u64 invmod_host(u64 a, u64 q) { return powmod_host(a, q - 2, q); }

u64 shoup_pre(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// x < 2^60 as two 30-bit halves: low half in the low 32-bit word
static u64 split30_host(u64 x) { return (x & 0x3fffffffull) | ((x >> 30) << 32); }

// Miller-Rabin with the first twelve prime bases (exact for 64-bit inputs).
static bool is_prime64(u64 n)
{
    const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : small) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++r;
    }
    for (u64 a : small) {
        u64 x = powmod_host(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; ++i) {
            x = mulmod_host(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Largest prime q = 1 mod 2n below 2^bits that is not in `taken`.
static u64 next_prime_below(int bits, int log_n, const std::vector<u64> &taken)
{
    const u64 step = (u64)2 << log_n;
    const u64 top = (u64)1 << bits;
    for (u64 c = top + 1 - step; c > step; c -= step) {
        if (std::find(taken.begin(), taken.end(), c) != taken.end()) continue;
        if (is_prime64(c)) return c;
    }
    throw Error(SPFHE_EPARAM, "no NTT-friendly prime of " + std::to_string(bits) + " bits");
}

static u64 primitive_2n_root(u64 q, int log_n)
{
    const u64 n = (u64)1 << log_n;
    for (u64 x = 2; x < q; ++x) {
        u64 w = powmod_host(x, (q - 1) / (2 * n), q);
        if (powmod_host(w, n, q) == q - 1) return w;
    }
    throw Error(SPFHE_EPARAM, "no primitive 2n-th root");
}

static u64 neg_inv64(u64 q)
{
    u64 x = q;  // q * q = 1 mod 8 for odd q
    for (int i = 0; i < 5; ++i) x *= 2 - q * x;
    return (u64)0 - x;
}

void build_params(Ctx &ctx, const spfhe_params &p)
{
    if (p.log_n < 2 || p.log_n > 17) throw Error(SPFHE_EPARAM, "log_n must be in [2, 17]");
    if (p.L < 3 || p.L > 64 || !p.q_bits) throw Error(SPFHE_EPARAM, "L must be in [3, 64] with q_bits");
    if (p.K < 1 || p.K > 16 || p.L + p.K > (uint32_t)kMaxMods) throw Error(SPFHE_EPARAM, "K out of range");
    if (p.dnum < 1 || p.dnum > p.L) throw Error(SPFHE_EPARAM, "dnum must be in [1, L]");
    if (p.p_bits < 20 || p.p_bits > 60) throw Error(SPFHE_EPARAM, "p_bits must be in [20, 60]");
    if (p.rot_base < 2 || (p.rot_base & (p.rot_base - 1))) throw Error(SPFHE_EPARAM, "rot_base must be a power of two");
    if (!(p.scale > 1.0)) throw Error(SPFHE_EPARAM, "scale must exceed 1");
    for (uint32_t i = 0; i < p.L; ++i)
        if (p.q_bits[i] < 20 || p.q_bits[i] > 60) throw Error(SPFHE_EPARAM, "q_bits must be in [20, 60]");
    ctx.log_n = p.log_n;
    ctx.n = 1 << p.log_n;
    ctx.S = ctx.n / 2;
    ctx.L = p.L;
    ctx.K = p.K;
    ctx.M = p.L + p.K;
    ctx.dnum = p.dnum;
    ctx.alpha = (p.L + p.dnum - 1) / p.dnum;
    if (ctx.alpha > 15) throw Error(SPFHE_EPARAM, "more than 15 limbs per digit");
    if (ctx.K > 15) throw Error(SPFHE_EPARAM, "more than 15 special primes");
    ctx.scale = p.scale;
    ctx.rot_base = p.rot_base;
    ctx.mods.clear();
    for (uint32_t i = 0; i < p.L; ++i) ctx.mods.push_back(next_prime_below(p.q_bits[i], p.log_n, ctx.mods));
    for (uint32_t k = 0; k < p.K; ++k) ctx.mods.push_back(next_prime_below(p.p_bits, p.log_n, ctx.mods));
    ctx.psis.clear();
    ctx.mc.clear();
    for (u64 q : ctx.mods) {
        ctx.psis.push_back(primitive_2n_root(q, p.log_n));
        ModConst m{};
        m.q = q;
        m.qneg_inv = neg_inv64(q);
        m.r_mod = (u64)(((u128)1 << 64) % q);
        m.r_mod_p = shoup_pre(m.r_mod, q);
        m.r2_mod = mulmod_host(m.r_mod, m.r_mod, q);
        m.n_inv = invmod_host((u64)ctx.n % q, q);
        m.n_inv_p = shoup_pre(m.n_inv, q);
        m.one_p = shoup_pre(1, q);
        ctx.mc.push_back(m);
    }
}

static unsigned brv_host(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

template <typename T> static T *upload(const std::vector<T> &v)
{
    T *d = nullptr;
    SPFHE_CHECK_CUDA(cudaMalloc(&d, std::max<size_t>(1, v.size()) * sizeof(T)));
    SPFHE_CHECK_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

void upload_tables(Ctx &ctx)
{
    const int n = ctx.n, M = ctx.M, L = ctx.L, K = ctx.K, A = ctx.alpha;
    DevTables &t = ctx.dt;
    t.mc = upload(ctx.mc);

    std::vector<u64> tw((size_t)M * n), twp((size_t)M * n), itw((size_t)M * n), itwp((size_t)M * n);
    for (int mi = 0; mi < M; ++mi) {
        const u64 q = ctx.mods[mi], psi = ctx.psis[mi], ipsi = invmod_host(psi, q);
        u64 pw = 1, ipw = 1;
        for (int j = 0; j < n; ++j) {
            const size_t k = (size_t)mi * n + brv_host(j, ctx.log_n);
            tw[k] = pw;
            twp[k] = shoup_pre(pw, q);
            itw[k] = ipw;
            itwp[k] = shoup_pre(ipw, q);
            pw = mulmod_host(pw, psi, q);
            ipw = mulmod_host(ipw, ipsi, q);
        }
    }
    t.tw = upload(tw);
    t.twp = upload(twp);
    t.itw = upload(itw);
    t.itwp = upload(itwp);
    std::vector<ulonglong2> tw2((size_t)M * n), itw2((size_t)M * n);
    for (size_t k = 0; k < tw2.size(); ++k) {
        tw2[k] = make_ulonglong2(tw[k], twp[k]);
        itw2[k] = make_ulonglong2(itw[k], itwp[k]);
    }
    t.tw2 = upload(tw2);
    t.itw2 = upload(itw2);

    // ModUp: one table per digit source set [lo, hi)
    std::vector<u64> hinv((size_t)L * A), hinvp((size_t)L * A), hmont((size_t)L * A * M);
    for (int hi = 1; hi <= L; ++hi) {
        const int lo = ((hi - 1) / A) * A;
        for (int i = lo; i < hi; ++i) {
            const size_t row = (size_t)(hi - 1) * A + (i - lo);
            const u64 qi = ctx.mods[i];
            u64 d = 1;
            for (int k = lo; k < hi; ++k)
                if (k != i) d = mulmod_host(d, ctx.mods[k] % qi, qi);
            hinv[row] = invmod_host(d, qi);
            hinvp[row] = shoup_pre(hinv[row], qi);
            for (int tt = 0; tt < M; ++tt) {
                const u64 m = ctx.mods[tt];
                u64 dm = 1 % m;
                for (int k = lo; k < hi; ++k)
                    if (k != i) dm = mulmod_host(dm, ctx.mods[k] % m, m);
                hmont[row * M + tt] = mulmod_host(dm, ctx.mc[tt].r_mod, m);
            }
        }
    }
    std::vector<u64> negd((size_t)L * M);
    for (int hi = 1; hi <= L; ++hi) {
        const int lo = ((hi - 1) / A) * A;
        for (int tt = 0; tt < M; ++tt) {
            const u64 m = ctx.mods[tt];
            u64 d = 1 % m;
            for (int k = lo; k < hi; ++k) d = mulmod_host(d, ctx.mods[k] % m, m);
            negd[(size_t)(hi - 1) * M + tt] = split30_host(mulmod_host((m - d) % m, ctx.mc[tt].r_mod, m));
        }
    }
    for (u64 &x : hmont) x = split30_host(x);
    t.mu_negd_split = upload(negd);
    std::vector<double> invq(M);
    for (int i = 0; i < M; ++i) invq[i] = 1.0 / (double)ctx.mods[i];
    t.inv_q = upload(invq);
    t.mu_hat_inv = upload(hinv);
    t.mu_hat_inv_p = upload(hinvp);
    t.mu_hat_split = upload(hmont);
    // hat_inv times n^{-1}: for inputs from inverse transforms that leave it out
    std::vector<u64> hinvn(hinv.size()), hinvnp(hinv.size());
    for (int hi = 1; hi <= L; ++hi) {
        const int lo = ((hi - 1) / A) * A;
        for (int i = lo; i < hi; ++i) {
            const size_t row = (size_t)(hi - 1) * A + (i - lo);
            const u64 qi = ctx.mods[i];
            hinvn[row] = mulmod_host(hinv[row], ctx.mc[i].n_inv, qi);
            hinvnp[row] = shoup_pre(hinvn[row], qi);
        }
    }
    t.mu_hat_inv_n = upload(hinvn);
    t.mu_hat_inv_n_p = upload(hinvnp);

    // ModDown P -> Q
    std::vector<u64> dinv(K), dinvp(K), dmont((size_t)K * M), pinv(L), pinvp(L), negp(L);
    for (int k = 0; k < K; ++k) {
        const u64 pk = ctx.mods[L + k];
        u64 d = 1;
        for (int j = 0; j < K; ++j)
            if (j != k) d = mulmod_host(d, ctx.mods[L + j] % pk, pk);
        dinv[k] = invmod_host(d, pk);
        dinvp[k] = shoup_pre(dinv[k], pk);
        for (int tt = 0; tt < M; ++tt) {
            const u64 m = ctx.mods[tt];
            u64 dm = 1 % m;
            for (int j = 0; j < K; ++j)
                if (j != k) dm = mulmod_host(dm, ctx.mods[L + j] % m, m);
            dmont[(size_t)k * M + tt] = split30_host(mulmod_host(dm, ctx.mc[tt].r_mod, m));
        }
    }
    for (int i = 0; i < L; ++i) {
        const u64 qi = ctx.mods[i];
        u64 P = 1;
        for (int k = 0; k < K; ++k) P = mulmod_host(P, ctx.mods[L + k] % qi, qi);
        pinv[i] = invmod_host(P, qi);
        pinvp[i] = shoup_pre(pinv[i], qi);
        negp[i] = split30_host(mulmod_host((qi - P) % qi, ctx.mc[i].r_mod, qi));
    }
    t.md_hat_inv = upload(dinv);
    t.md_hat_inv_p = upload(dinvp);
    std::vector<u64> dinvn(K), dinvnp(K);
    for (int k = 0; k < K; ++k) {
        const u64 pk = ctx.mods[L + k];
        dinvn[k] = mulmod_host(dinv[k], ctx.mc[L + k].n_inv, pk);
        dinvnp[k] = shoup_pre(dinvn[k], pk);
    }
    t.md_hat_inv_n = upload(dinvn);
    t.md_hat_inv_n_p = upload(dinvnp);
    t.md_hat_split = upload(dmont);
    t.md_pinv = upload(pinv);
    t.md_pinv_p = upload(pinvp);
    t.md_negp_split = upload(negp);

    // Rescale
    std::vector<u64> rinv((size_t)L * L, 0), rinvp((size_t)L * L, 0), rqt((size_t)L * L, 0);
    for (int tt = 1; tt < L; ++tt)
        for (int i = 0; i < tt; ++i) {
            const u64 qi = ctx.mods[i], qt = ctx.mods[tt] % qi;
            rinv[(size_t)tt * L + i] = invmod_host(qt, qi);
            rinvp[(size_t)tt * L + i] = shoup_pre(rinv[(size_t)tt * L + i], qi);
            rqt[(size_t)tt * L + i] = qt;
        }
    t.rs_inv = upload(rinv);
    t.rs_inv_p = upload(rinvp);
    t.rs_qt = upload(rqt);
}

void free_tables(Ctx &ctx)
{
    DevTables &t = ctx.dt;
    u64 *ptrs[] = {t.tw, t.twp, t.itw, t.itwp, t.mu_hat_inv, t.mu_hat_inv_p, t.mu_hat_split,
                   t.mu_hat_inv_n, t.mu_hat_inv_n_p, t.md_hat_inv_n, t.md_hat_inv_n_p,
                   t.md_hat_inv, t.md_hat_inv_p, t.md_hat_split, t.md_pinv, t.md_pinv_p,
                   t.md_negp_split, t.mu_negd_split, t.rs_inv, t.rs_inv_p, t.rs_qt};
    for (u64 *p : ptrs)
        if (p) cudaFree(p);
    if (t.mc) cudaFree(t.mc);
    if (t.inv_q) cudaFree(t.inv_q);
    if (t.tw2) cudaFree(t.tw2);
    if (t.itw2) cudaFree(t.itw2);
    t = DevTables{};
}

}  // namespace spfhe
