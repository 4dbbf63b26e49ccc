// Encrypted sparse x sparse matmul (Alg. 1 + Alg. 2 of "GPU Acceleration of
// Sparse Fully Homomorphic Encrypted DNNs").
//
// Host side: Alg. 1's CSR x CSC merge over the plaintext metadata produces the
// match list; every match names the operand to rotate (only one, by the slot
// difference; none when the slots agree, Sec. 3.2.2), the mask slot
// min(a_slot, b_slot) and the final rotation min_slot - (i*cols + j).
//
// Device side: distinct alignment rotations are computed once each (a
// rotation is a deterministic function of (operand, amount), so reuse gives
// the same bits as recomputing it per match) in waves of up to `G`
// ciphertexts; the matches of a wave then run Alg. 2 in batches of `Bm`
// matches, every stage one launch over the whole batch:
//   tensor -> relinearise (one key stream serves the batch) -> rescale ->
//   mask (one NTT-domain mask, permuted per match) -> rescale ->
//   final rotation (plan steps batched across matches) -> accumulate.
// Modular sums are exact, so the accumulation order does not change the
// result.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <tuple>

#include "engine.h"

namespace spfhe {

void validate_meta(const spfhe_sparse_meta &m, const char *what)
{
    const std::string w(what);
    if (m.rows < 0 || m.cols < 0 || m.nnz < 0) throw Error(SPFHE_EINVAL, w + ": negative size");
    if (!m.indptr) throw Error(SPFHE_EINVAL, w + ": null indptr");
    if (m.nnz > 0 && !m.indices) throw Error(SPFHE_EINVAL, w + ": null indices");
    // CSR: `rows` compressed lines of column ids in [0, cols); CSC: `cols`
    // compressed lines of row ids in [0, rows).  The caller passes which.
    (void)w;
}

static void validate_lines(const int32_t *indptr, const int32_t *indices, int lines, int range, int nnz,
                           const std::string &w)
{
    if (indptr[0] != 0) throw Error(SPFHE_EINVAL, w + ": indptr[0] != 0");
    for (int l = 0; l < lines; ++l) {
        if (indptr[l + 1] < indptr[l]) throw Error(SPFHE_EINVAL, w + ": indptr not monotone");
        for (int p = indptr[l]; p < indptr[l + 1]; ++p) {
            if (p >= nnz) throw Error(SPFHE_EINVAL, w + ": indptr beyond nnz");
            if (indices[p] < 0 || indices[p] >= range) throw Error(SPFHE_EINVAL, w + ": index out of range");
            if (p > indptr[l] && indices[p] <= indices[p - 1])
                throw Error(SPFHE_EINVAL, w + ": indices not strictly ascending");
        }
    }
    if (indptr[lines] != nnz) throw Error(SPFHE_EINVAL, w + ": indptr[last] != nnz");
}

void validate_pair(const spfhe_sparse_meta &A, const spfhe_sparse_meta &B)
{
    validate_meta(A, "A (CSR)");
    validate_meta(B, "B (CSC)");
    if (A.cols != B.rows) throw Error(SPFHE_EINVAL, "inner dimensions differ");
    validate_lines(A.indptr, A.indices, A.rows, A.cols, A.nnz, "A (CSR)");
    validate_lines(B.indptr, B.indices, B.cols, B.rows, B.nnz, "B (CSC)");
}

// Alg. 1: for every (i, j), two-pointer walk over row i of A and column j of B.
std::vector<MatchRec> plan_alg1(const spfhe_sparse_meta &A, const spfhe_sparse_meta &B)
{
    std::vector<MatchRec> out;
    for (int i = 0; i < A.rows; ++i) {
        const int a_start = A.indptr[i], a_end = A.indptr[i + 1];
        if (a_start == a_end) continue;
        for (int j = 0; j < B.cols; ++j) {
            int a_pos = a_start, b_pos = B.indptr[j];
            const int b_end = B.indptr[j + 1];
            while (a_pos < a_end && b_pos < b_end) {
                const int a_col = A.indices[a_pos], b_row = B.indices[b_pos];
                if (a_col == b_row) {
                    out.push_back(MatchRec{i, j, a_col, a_pos, b_pos});
                    ++a_pos;
                    ++b_pos;
                } else if (a_col < b_row) {
                    ++a_pos;
                } else {
                    ++b_pos;
                }
            }
        }
    }
    return out;
}

static void check_chunks(Ct *const *ch, size_t n, int level, const char *what)
{
    for (size_t c = 0; c < n; ++c) {
        if (!ch[c] || !ch[c]->d) throw Error(SPFHE_EINVAL, std::string(what) + ": null chunk");
        if (ch[c]->level != level) throw Error(SPFHE_ELEVEL, std::string(what) + ": chunk not at the top level");
        if (std::fabs(ch[c]->scale - ch[0]->scale) > 1e-9 * std::fabs(ch[0]->scale))
            throw Error(SPFHE_ESCALE, std::string(what) + ": chunk scales differ");
    }
}

void fill_job(Job &job, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
              const spfhe_sparse_meta &B, Ct *const *Bch, size_t nB, const Pt *mask0, size_t nC)
{
    job.keys = &keys;
    job.A = A;
    job.B = B;
    job.aip.assign(A.indptr, A.indptr + A.rows + 1);
    if (A.nnz > 0) job.aix.assign(A.indices, A.indices + A.nnz);
    job.bip.assign(B.indptr, B.indptr + B.cols + 1);
    if (B.nnz > 0) job.bix.assign(B.indices, B.indices + B.nnz);
    job.Ach.assign(Ach, Ach + nA);
    job.Bch.assign(Bch, Bch + nB);
    job.mask0 = mask0;
    job.n_c = nC;
}

void release_job(Ctx &ctx, Job &job, bool free_results)
{
    if (job.own_mask) dev_free(ctx, job.own_mask);
    job.own_mask = nullptr;
    if (free_results)
        for (Ct *&c : job.C)
            if (c) {
                dev_free(ctx, c->d);
                delete c;
                c = nullptr;
            }
}

void reset_job(Job &job)
{
    job.C.clear();
    job.mask = nullptr;
    job.own_mask = nullptr;
    job.ell = 0;
    job.tasks_left = 0;
    job.st_matches = job.st_relin = job.st_align = job.st_final = job.st_rescales = job.st_launches = 0;
    job.finished = false;
}

struct Stats {
    uint64_t matches = 0, ks_relin = 0, ks_align = 0, ks_final = 0, rescales = 0;
};

// Shared tail of both variants for one batch: rescaled products `prod`
// ([m][2][ell][n]) are rotated to their target slots and added into their
// result chunks.
static void rotate_and_accumulate(Ctx &ctx, const Keys &keys, int ell, u64 *prod, int m, const std::vector<int> &rf,
                                  const std::vector<int> &rc, Ct **C, size_t nC, Stats &st)
{
    Runtime &rt = *ctx.rt;
    const long long cs = 2LL * ell * ctx.n;
    std::vector<const u64 *> in(m);
    for (int i = 0; i < m; ++i) in[i] = prod + i * cs;
    u64 *W = rt.workspace(WS_MISC, (size_t)m * cs);
    rotate_batch(ctx, keys, ell, in, rf, W, &st.ks_final);
    for (size_t c = 0; c < nC; ++c) {
        std::vector<int> ids;
        for (int i = 0; i < m; ++i)
            if (rc[i] == (int)c) ids.push_back(i);
        if (ids.empty()) continue;
        const int *d_ids = rt.upload_vec(ids);
        accumulate(ctx, ell, C[c]->d, W, cs, d_ids, (int)ids.size());
    }
}

void spmspm_ct_ct(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                  const spfhe_sparse_meta &B, Ct *const *Bch, size_t nB, const Pt *mask0, Ct **C, size_t nC,
                  spfhe_stats *out_stats)
{
    const uint64_t launches0 = ctx.launches;
    validate_pair(A, B);
    for (size_t c = 0; c < nC; ++c) C[c] = nullptr;
    Job job;
    fill_job(job, keys, A, Ach, nA, B, Bch, nB, mask0, nC);
    Engine eng(ctx);
    try {
        eng.add(&job);
        eng.run_all();
        ctx_sync(ctx);
    } catch (...) {
        release_job(ctx, job, true);
        throw;
    }
    for (size_t c = 0; c < nC; ++c) C[c] = job.C[c];
    release_job(ctx, job, false);
    if (out_stats) {
        out_stats->matches = job.st_matches;
        out_stats->ks_relin = job.st_relin;
        out_stats->ks_align = job.st_align;
        out_stats->ks_final = job.st_final;
        out_stats->rescales = job.st_rescales;
        out_stats->launches = ctx.launches - launches0;
    }
}

void naive_ct_ct(Ctx &ctx, const Keys &keys, int mode, int rows, int inner, int cols, const uint8_t *a_nz,
                 const uint8_t *b_nz, Ct *const *Ach, size_t nA, Ct *const *Bch, size_t nB, const Pt *mask0, Ct **C,
                 size_t nC, spfhe_stats *out_stats)
{
    const uint64_t launches0 = ctx.launches;
    if (mode < SPFHE_NAIVE_DENSE || mode > SPFHE_NAIVE_SPARSE_LITERAL) throw Error(SPFHE_EINVAL, "unknown mode");
    if (rows < 1 || inner < 1 || cols < 1) throw Error(SPFHE_EINVAL, "empty dimension");
    if ((long long)rows * inner > (1LL << 30) || (long long)inner * cols > (1LL << 30) ||
        (long long)rows * cols > (1LL << 30))
        throw Error(SPFHE_EINVAL, "dimensions too large");
    if (!a_nz || !b_nz) throw Error(SPFHE_EINVAL, "null zero pattern");
    for (size_t c = 0; c < nC; ++c) C[c] = nullptr;
    Job job;
    job.keys = &keys;
    job.naive = mode;
    job.rows = rows;
    job.inner = inner;
    job.cols = cols;
    job.a_nz.assign(a_nz, a_nz + (size_t)rows * inner);
    job.b_nz.assign(b_nz, b_nz + (size_t)inner * cols);
    job.Ach.assign(Ach, Ach + nA);
    job.Bch.assign(Bch, Bch + nB);
    job.mask0 = mask0;
    job.n_c = nC;
    Engine eng(ctx);
    try {
        eng.add(&job);
        eng.run_all();
        ctx_sync(ctx);
    } catch (...) {
        release_job(ctx, job, true);
        throw;
    }
    for (size_t c = 0; c < nC; ++c) C[c] = job.C[c];
    release_job(ctx, job, false);
    if (out_stats) {
        out_stats->matches = job.st_matches;
        out_stats->ks_relin = job.st_relin;
        out_stats->ks_align = job.st_align;
        out_stats->ks_final = job.st_final;
        out_stats->rescales = job.st_rescales;
        out_stats->launches = ctx.launches - launches0;
    }
}

void spmspm_ct_pt(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                  const spfhe_sparse_meta &B, const double *Bvals, Pt *const *Bpts, Ct **C, size_t nC,
                  spfhe_stats *out_stats)
{
    const uint64_t launches0 = ctx.launches;
    validate_pair(A, B);
    const int S = ctx.S, L = ctx.L;
    const size_t n = ctx.n;
    if (L < 2) throw Error(SPFHE_ELEVEL, "ct x pt needs L >= 2");
    if (nA != chunks_for(A.nnz, S)) throw Error(SPFHE_EINVAL, "operand chunk count != ceil(nnz / S)");
    if (nC != chunks_for((long long)A.rows * B.cols, S)) throw Error(SPFHE_EINVAL, "result chunk count != ceil(rows*cols / S)");
    if (!Bvals && !Bpts && B.nnz > 0) throw Error(SPFHE_EINVAL, "B values missing");
    check_chunks(Ach, nA, L, "A");
    for (size_t c = 0; c < nC; ++c) C[c] = nullptr;
    const std::vector<MatchRec> matches = plan_alg1(A, B);
    const double wscale = (double)ctx.mods[L - 1];
    const double rscale = Ach[0]->scale * wscale / (double)ctx.mods[L - 1];
    const int ellC = L - 1;
    Stats st;
    std::vector<int> mi(L);
    for (int i = 0; i < L; ++i) mi[i] = i;
    try {
        for (size_t c = 0; c < nC; ++c) {
            C[c] = ct_new(ctx, ellC, rscale);
            SPFHE_CHECK_CUDA(cudaMemsetAsync(C[c]->d, 0, 2ull * ellC * n * sizeof(u64), ctx.stream));
        }
        if (!matches.empty()) {
            Runtime &rt = *ctx.rt;
            std::vector<int> order(matches.size());
            for (size_t x = 0; x < order.size(); ++x) order[x] = (int)x;
            std::stable_sort(order.begin(), order.end(),
                             [&](int a, int b) { return matches[a].b_pos < matches[b].b_pos; });
            for (auto &mt : matches) {
                const long long t = (long long)mt.i * B.cols + mt.j;
                for (int a : rotation_plan(ctx, ((mt.a_pos % S - t % S) % S + S) % S)) rotation_key(keys, a);
            }
            const int Bm = match_batch_size(ctx);
            const long long csL = 2LL * L * n;
            const long long plimb = (long long)L * n;
            for (size_t b0 = 0; b0 < order.size(); b0 += Bm) {
                const int m = (int)std::min<size_t>(Bm, order.size() - b0);
                // distinct B nonzeros of this batch -> weight plaintexts at slot 0
                std::vector<int> bpos;
                for (int i = 0; i < m; ++i) {
                    const int bp = matches[order[b0 + i]].b_pos;
                    if (bpos.empty() || bpos.back() != bp) bpos.push_back(bp);
                }
                const int np = (int)bpos.size();
                u64 *pts = rt.workspace(WS_PTS, (size_t)np * plimb);
                if (Bpts) {
                    for (int p = 0; p < np; ++p) {
                        const Pt *bp = Bpts[bpos[p]];
                        if (!bp || bp->level != L) throw Error(SPFHE_ELEVEL, "B plaintexts must be at level L");
                        copy_words(ctx, pts + p * plimb, bp->d, (size_t)plimb);
                    }
                } else {
                    std::vector<double> vals(np);
                    for (int p = 0; p < np; ++p) vals[p] = Bvals[bpos[p]];
                    const double *d_vals = rt.upload_vec(vals);
                    encode_onehot0(ctx, d_vals, np, L, wscale, pts);
                }
                to_montgomery(ctx, pts, L, mi.data(), np);
                std::vector<const u64 *> src(m), ptp(m), x1(m);
                std::vector<int> g(m), rf(m), rc(m);
                u64 *X = rt.workspace(WS_RELIN_OUT, (size_t)m * csL);
                u64 *Y = rt.workspace(WS_LEVEL1, (size_t)m * 2 * (L - 1) * n);
                u64 *T = rt.workspace(WS_RS_TMP, (size_t)m * 2 * L * n);
                int p = 0;
                for (int i = 0; i < m; ++i) {
                    const MatchRec &mt = matches[order[b0 + i]];
                    while (bpos[p] != mt.b_pos) ++p;
                    const int ca = mt.a_pos / S, sa = mt.a_pos % S;
                    src[i] = Ach[ca]->d;
                    ptp[i] = pts + p * plimb;
                    x1[i] = X + i * csL;
                    g[i] = galois_element(ctx, -sa);
                    const long long t = (long long)mt.i * B.cols + mt.j;
                    rc[i] = (int)(t / S);
                    rf[i] = (int)(((sa - t % S) % S + S) % S);
                }
                gather_items(ctx, m, (size_t)csL, rt.upload_vec(src), X, csL);
                mul_plain_perm(ctx, m, L, X, csL, rt.upload_vec(ptp), rt.upload_vec(g));
                rescale(ctx, m, L, rt.upload_vec(x1), T, Y, 2LL * (L - 1) * n);
                st.rescales += m;
                rotate_and_accumulate(ctx, keys, L - 1, Y, m, rf, rc, C, nC, st);
                st.matches += m;
            }
        }
        ctx_sync(ctx);
    } catch (...) {
        for (size_t c = 0; c < nC; ++c)
            if (C[c]) {
                dev_free(ctx, C[c]->d);
                delete C[c];
                C[c] = nullptr;
            }
        throw;
    }
    if (out_stats) {
        out_stats->matches = st.matches;
        out_stats->ks_relin = 0;
        out_stats->ks_align = 0;
        out_stats->ks_final = st.ks_final;
        out_stats->rescales = st.rescales;
        out_stats->launches = ctx.launches - launches0;
    }
}

}  // namespace spfhe
