// Task engine: waves of alignment rotations and batches of Alg. 2 match
// chains that may mix products (see engine.h).
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace spfhe {

static int env_int(const char *name, int dflt)
{
    const char *v = std::getenv(name);
    if (!v || !*v) return dflt;
    const int x = std::atoi(v);
    return x > 0 ? x : dflt;
}

int match_batch_size(const Ctx &ctx)
{
    if (ctx.match_batch > 0) return ctx.match_batch;
    const int dflt = 64;   // measured at n = 2^16: 64 matches 2 % faster than 32, 48 in between
    return std::max(1, std::min(env_int("SPFHE_MATCH_BATCH", dflt), 1024));
}

size_t chunks_for(long long count, int S) { return (size_t)std::max(1LL, (count + S - 1) / S); }

uint64_t engine_workspace_bound(const Ctx &ctx, int ell)
{
    // limbs per batch item of every workspace slot a wave at level ell uses
    // (run_wave, run_matches, rotate_batch, keyswitch_batch)
    const uint64_t B = (uint64_t)match_batch_size(ctx);
    const uint64_t l = (uint64_t)ell, K = (uint64_t)ctx.K;
    const uint64_t beta = (l + ctx.alpha - 1) / ctx.alpha;
    const uint64_t limbs = 2 * l        // WS_ALIGN (G + 1 = B + 1 alignment outputs)
                           + 3 * l      // WS_TENSOR
                           + 2 * l      // WS_RELIN_OUT
                           + 2 * l      // WS_LEVEL1 (2 (ell-1), rounded up)
                           + 2 * l      // WS_LEVEL2
                           + 2 * l      // WS_RS_TMP
                           + 2 * l      // WS_MISC
                           + l          // WS_KS_COEF
                           + beta * (l + K)   // WS_KS_EXT
                           + 2 * (l + K)      // WS_KS_ACC
                           + 2 * l      // WS_KS_CONV
                           + l          // WS_ROT_TMP
                           + 4 * l      // WS_ROT_OUT_A, WS_ROT_OUT_B
                           + 2 * l;     // WS_ROT_SUM (at most one target per item)
    return (B * limbs + 2 * l) * (uint64_t)ctx.n * sizeof(u64);
}

uint64_t job_mask_bytes(const Ctx &ctx, const Job &job)
{
    const int ell = job.Ach.empty() || !job.Ach[0] ? ctx.L : job.Ach[0]->level;
    const uint64_t mask = (uint64_t)std::max(ell - 1, 1) * ctx.n * sizeof(u64);
    if (job.mask0) return mask;
    return ctx.masks.count(ell) ? 0 : mask;
}

Engine::Engine(Ctx &ctx) : ctx_(ctx) {}

Engine::~Engine() = default;

bool Engine::idle() const
{
    for (const auto &kv : levels_)
        if (!kv.second.rots.empty() || !kv.second.free_matches.empty()) return false;
    return true;
}

std::vector<Job *> Engine::take_finished()
{
    std::vector<Job *> out;
    out.swap(finished_);
    return out;
}

const u64 *Engine::level_mask(int ell)
{
    auto it = ctx_.masks.find(ell);
    if (it != ctx_.masks.end()) return it->second;
    const int ml = ell - 1;
    const size_t words = (size_t)ml * ctx_.n;
    u64 *m = static_cast<u64 *>(dev_alloc(ctx_, words * sizeof(u64)));
    const double one = 1.0;
    const double *d_one = static_cast<const double *>(ctx_.rt->upload(&one, sizeof(double)));
    // one-hot of slot 0 at level ell-1, scale q_{ell-2}: the prime the second rescale removes
    encode_onehot0(ctx_, d_one, 1, ml, (double)ctx_.mods[ell - 2], m);
    std::vector<int> mi(ml);
    for (int i = 0; i < ml; ++i) mi[i] = i;
    to_montgomery(ctx_, m, ml, mi.data(), 1);
    // a mask made while a graph is captured belongs to that graph
    if (!ctx_.cap) ctx_.masks[ell] = m;
    return m;
}

int check_ct_ct(const Ctx &ctx, const spfhe_sparse_meta &A, const std::vector<Ct *> &Ach,
                const spfhe_sparse_meta &B, const std::vector<Ct *> &Bch, size_t n_c, double *rscale)
{
    const int S = ctx.S;
    validate_pair(A, B);
    if (Ach.empty() || Bch.empty()) throw Error(SPFHE_EINVAL, "no operand chunks");
    if (Ach.size() != chunks_for(A.nnz, S) || Bch.size() != chunks_for(B.nnz, S))
        throw Error(SPFHE_EINVAL, "operand chunk count != ceil(nnz / S)");
    if (n_c != chunks_for((long long)A.rows * B.cols, S))
        throw Error(SPFHE_EINVAL, "result chunk count != ceil(rows*cols / S)");
    const int ell = Ach[0] ? Ach[0]->level : 0;
    for (Ct *c : Ach)
        if (!c || !c->d || c->level != ell) throw Error(SPFHE_ELEVEL, "A chunks must share one level");
    for (Ct *c : Bch)
        if (!c || !c->d || c->level != ell) throw Error(SPFHE_ELEVEL, "B chunks must share A's level");
    if (ell < 3) throw Error(SPFHE_ELEVEL, "ct x ct needs operands at level >= 3");
    const double sa = Ach[0]->scale, sb = Bch[0]->scale;
    for (Ct *c : Ach)
        if (std::fabs(c->scale - sa) > 1e-9 * sa) throw Error(SPFHE_ESCALE, "A chunk scales differ");
    for (Ct *c : Bch)
        if (std::fabs(c->scale - sb) > 1e-9 * sb) throw Error(SPFHE_ESCALE, "B chunk scales differ");
    if (std::fabs(sa - sb) > 1e-9 * sa) throw Error(SPFHE_ESCALE, "A and B scales differ");
    *rscale = sa * sb / (double)ctx.mods[ell - 1];
    return ell;
}

// checks shared by the ct x ct products on levels and scales; returns the
// operands' level and their product's result scale
static int check_levels_scales(const Ctx &ctx, const std::vector<Ct *> &Ach, const std::vector<Ct *> &Bch,
                               double *rscale)
{
    if (Ach.empty() || Bch.empty()) throw Error(SPFHE_EINVAL, "no operand chunks");
    const int ell = Ach[0] ? Ach[0]->level : 0;
    for (Ct *c : Ach)
        if (!c || !c->d || c->level != ell) throw Error(SPFHE_ELEVEL, "A chunks must share one level");
    for (Ct *c : Bch)
        if (!c || !c->d || c->level != ell) throw Error(SPFHE_ELEVEL, "B chunks must share A's level");
    if (ell < 3) throw Error(SPFHE_ELEVEL, "ct x ct needs operands at level >= 3");
    const double sa = Ach[0]->scale, sb = Bch[0]->scale;
    for (Ct *c : Ach)
        if (std::fabs(c->scale - sa) > 1e-9 * sa) throw Error(SPFHE_ESCALE, "A chunk scales differ");
    for (Ct *c : Bch)
        if (std::fabs(c->scale - sb) > 1e-9 * sb) throw Error(SPFHE_ESCALE, "B chunk scales differ");
    if (std::fabs(sa - sb) > 1e-9 * sa) throw Error(SPFHE_ESCALE, "A and B scales differ");
    *rscale = sa * sb / (double)ctx.mods[ell - 1];
    return ell;
}

void Engine::add(Job *job)
{
    Ctx &ctx = ctx_;
    const int S = ctx.S;
    const size_t n = ctx.n;
    if (!job->keys) throw Error(SPFHE_EINVAL, "null keys");
    struct Plan {
        int src_a, src_b, min_slot, rf, rc;
    };
    std::vector<Plan> plan;
    // rotation tasks of this job: (operand, chunk, amount), and for the
    // element-wise baselines the task rotating the other operand of the same
    // product (-1: none)
    std::vector<std::tuple<int, int, int>> local_list;
    std::vector<int> partner;
    int ell = 0;
    if (job->naive < 0) {
        job->A.indptr = job->aip.data();
        job->A.indices = job->aix.empty() ? nullptr : job->aix.data();
        job->B.indptr = job->bip.data();
        job->B.indices = job->bix.empty() ? nullptr : job->bix.data();
        ell = check_ct_ct(ctx, job->A, job->Ach, job->B, job->Bch, job->n_c, &job->rscale);
        const std::vector<MatchRec> ms = plan_alg1(job->A, job->B);
        std::map<std::tuple<int, int, int>, int> local_rot;
        auto rot_of = [&](int op, int chunk, int amt) {
            auto key = std::make_tuple(op, chunk, amt);
            auto it = local_rot.find(key);
            if (it != local_rot.end()) return it->second;
            const int id = (int)local_list.size();
            local_rot[key] = id;
            local_list.push_back(key);
            partner.push_back(-1);
            return id;
        };
        plan.resize(ms.size());
        for (size_t x = 0; x < ms.size(); ++x) {
            const MatchRec &mt = ms[x];
            const int ca = mt.a_pos / S, sa_ = mt.a_pos % S, cb = mt.b_pos / S, sb_ = mt.b_pos % S;
            Plan p{-(ca + 1), -(cb + 1), sa_, 0, 0};
            if (sa_ < sb_)
                p.src_b = rot_of(1, cb, sb_ - sa_);
            else if (sb_ < sa_) {
                p.src_a = rot_of(0, ca, sa_ - sb_);
                p.min_slot = sb_;
            }
            const long long t = (long long)mt.i * job->B.cols + mt.j;
            p.rc = (int)(t / S);
            p.rf = (int)(((p.min_slot - t % S) % S + S) % S);
            plan[x] = p;
        }
    } else {
        // element-wise baselines over row-major dense packing: every kept
        // product (i, j, k) rotates both operands so its two elements sit in
        // slot 0 (no reuse between products), then runs Alg. 2's chain
        const int rows = job->rows, inner = job->inner, cols = job->cols;
        if (job->Ach.size() != chunks_for((long long)rows * inner, S) ||
            job->Bch.size() != chunks_for((long long)inner * cols, S))
            throw Error(SPFHE_EINVAL, "operand chunk count != ceil(elements / S)");
        if (job->n_c != chunks_for((long long)rows * cols, S))
            throw Error(SPFHE_EINVAL, "result chunk count != ceil(rows*cols / S)");
        ell = check_levels_scales(ctx, job->Ach, job->Bch, &job->rscale);
        auto new_rot = [&](int op, int chunk, int amt) {
            local_list.push_back(std::make_tuple(op, chunk, amt));
            partner.push_back(-1);
            return (int)local_list.size() - 1;
        };
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < cols; ++j)
                for (int k = 0; k < inner; ++k) {
                    const bool a = job->a_nz[(size_t)i * inner + k] != 0, b = job->b_nz[(size_t)k * cols + j] != 0;
                    if (job->naive == SPFHE_NAIVE_SPARSE && !(a && b)) continue;
                    if (job->naive == SPFHE_NAIVE_SPARSE_LITERAL && !(a || b)) continue;
                    const long long pa = (long long)i * inner + k, pb = (long long)k * cols + j;
                    const int ca = (int)(pa / S), sa_ = (int)(pa % S), cb = (int)(pb / S), sb_ = (int)(pb % S);
                    Plan p{-(ca + 1), -(cb + 1), 0, 0, 0};
                    if (sa_) p.src_a = new_rot(0, ca, sa_);
                    if (sb_) p.src_b = new_rot(1, cb, sb_);
                    if (p.src_a >= 0 && p.src_b >= 0) {
                        partner[p.src_a] = p.src_b;
                        partner[p.src_b] = p.src_a;
                    }
                    const long long t = (long long)i * cols + j;
                    p.rc = (int)(t / S);
                    p.rf = (int)((S - t % S) % S);
                    plan.push_back(p);
                }
    }
    job->ell = ell;
    job->id = next_id_++;
    // keys first: nothing is allocated or launched for a job that would fail
    if (!plan.empty() && !job->keys->relin) throw Error(SPFHE_EKEY, "no relinearisation key");
    for (auto &r : local_list)
        for (int a : rotation_plan(ctx, std::get<2>(r))) rotation_key(*job->keys, a);
    for (auto &p : plan)
        for (int a : rotation_plan(ctx, p.rf)) rotation_key(*job->keys, a);

    // results and mask
    job->C.assign(job->n_c, nullptr);
    try {
        for (size_t c = 0; c < job->n_c; ++c) {
            job->C[c] = ct_new(ctx, ell - 2, job->rscale);
            SPFHE_CHECK_CUDA(cudaMemsetAsync(job->C[c]->d, 0, 2ull * (ell - 2) * n * sizeof(u64), ctx.stream));
        }
        if (!plan.empty()) {
            if (job->mask0) {
                if (job->mask0->level != ell - 1) throw Error(SPFHE_ELEVEL, "mask must be at the operands' level - 1");
                const size_t words = (size_t)(ell - 1) * n;
                job->own_mask = static_cast<u64 *>(dev_alloc(ctx, words * sizeof(u64)));
                copy_words(ctx, job->own_mask, job->mask0->d, words);
                std::vector<int> mi(ell - 1);
                for (int i = 0; i < ell - 1; ++i) mi[i] = i;
                to_montgomery(ctx, job->own_mask, ell - 1, mi.data(), 1);
                job->mask = job->own_mask;
            } else {
                job->mask = level_mask(ell);
            }
        }
    } catch (...) {
        for (Ct *&c : job->C)
            if (c) {
                dev_free(ctx, c->d);
                delete c;
                c = nullptr;
            }
        if (job->own_mask) dev_free(ctx, job->own_mask);
        job->own_mask = nullptr;
        throw;
    }

    // tasks
    LevelQueue &q = levels_[ell];
    const int rot0 = (int)rots_.size();
    for (size_t r = 0; r < local_list.size(); ++r)
        rots_.push_back(RotTask{job, std::get<0>(local_list[r]), std::get<1>(local_list[r]), std::get<2>(local_list[r]),
                                {}, partner[r] >= 0 ? rot0 + partner[r] : -1});
    for (auto &p : plan) {
        const int id = (int)matches_.size();
        MatchTask mt{job, p.src_a >= 0 ? rot0 + p.src_a : p.src_a, p.src_b >= 0 ? rot0 + p.src_b : p.src_b,
                     p.min_slot, p.rf, p.rc};
        matches_.push_back(mt);
        // a product whose operands are both rotated waits for the second of
        // the pair (the two always run in the same wave)
        if (mt.src_b >= 0)
            rots_[mt.src_b].deps.push_back(id);
        else if (mt.src_a >= 0)
            rots_[mt.src_a].deps.push_back(id);
        else
            q.free_matches.push_back(id);
    }
    for (size_t r = 0; r < local_list.size(); ++r) q.rots.push_back(rot0 + (int)r);
    job->tasks_left = local_list.size() + plan.size();
    order_.push_back(job);
    if (job->tasks_left == 0) task_done(job, 0);
}

void Engine::task_done(Job *job, uint64_t count)
{
    job->tasks_left -= count;
    if (job->tasks_left == 0 && !job->finished) {
        job->finished = true;
        if (job->done_ev) SPFHE_CHECK_CUDA(cudaEventRecord(job->done_ev, ctx_.stream));
        finished_.push_back(job);
    }
}

bool Engine::step()
{
    // oldest job with pending work decides the level
    while (!order_.empty() && order_.front()->finished) order_.pop_front();
    for (Job *j : order_) {
        if (j->finished) continue;
        auto it = levels_.find(j->ell);
        if (it == levels_.end()) continue;
        LevelQueue &q = it->second;
        if (q.rots.empty() && q.free_matches.empty()) continue;
        run_wave(j->ell, q);
        return true;
    }
    return false;
}

void Engine::run_wave(int ell, LevelQueue &q)
{
    Ctx &ctx = ctx_;
    for (Job *j : order_)
        if (j->inject_fault && !j->finished && j->ell == ell)
            throw Error(SPFHE_ECUDA, "injected fault (host-side test hook) in a wave of job " + std::to_string(j->id));
    Runtime &rt = *ctx.rt;
    const int Bm = match_batch_size(ctx);
    const int G = Bm;
    const long long csL = 2LL * ell * ctx.n;
    std::vector<int> R;
    while (!q.rots.empty() && (int)R.size() < G) {
        const int r = q.rots.front();
        R.push_back(r);
        q.rots.pop_front();
        // the partner of a pair (queued right after it) joins the same wave
        if (rots_[r].partner > r && !q.rots.empty() && q.rots.front() == rots_[r].partner) {
            R.push_back(q.rots.front());
            q.rots.pop_front();
        }
    }
    u64 *align = nullptr;
    std::map<int, int> slot_of;
    std::vector<int> M;
    if (!R.empty()) {
        align = rt.workspace(WS_ALIGN, (size_t)(G + 1) * csL);
        std::vector<const Keys *> kk;
        std::vector<const u64 *> in;
        std::vector<int> amt;
        for (size_t i = 0; i < R.size(); ++i) {
            const RotTask &t = rots_[R[i]];
            kk.push_back(t.job->keys);
            in.push_back((t.op == 0 ? t.job->Ach[t.chunk] : t.job->Bch[t.chunk])->d);
            amt.push_back(t.amount);
            slot_of[R[i]] = (int)i;
            t.job->st_align += rotation_plan(ctx, t.amount).size();
        }
        rotate_batch(ctx, kk, ell, in, amt, align, nullptr);
        for (int r : R) {
            for (int m : rots_[r].deps) M.push_back(m);
            task_done(rots_[r].job, 1);
        }
    }
    // fill the last batch with matches that need no alignment
    const size_t want = R.empty() ? (size_t)4 * Bm : ((M.size() + Bm - 1) / Bm) * Bm;
    while (!q.free_matches.empty() && M.size() < std::max<size_t>(want, 1)) {
        M.push_back(q.free_matches.front());
        q.free_matches.pop_front();
    }
    for (size_t b0 = 0; b0 < M.size(); b0 += Bm) {
        std::vector<int> ids(M.begin() + b0, M.begin() + std::min(M.size(), b0 + Bm));
        run_matches(ell, ids, align, 0, slot_of);
    }
}

void Engine::run_matches(int ell, const std::vector<int> &ids, const u64 *align, int, const std::map<int, int> &slot_of)
{
    Ctx &ctx = ctx_;
    Runtime &rt = *ctx.rt;
    const size_t n = ctx.n;
    const int m = (int)ids.size();
    if (!m) return;
    const long long csL = 2LL * ell * n;
    const long long cs1 = 2LL * (ell - 1) * n, cs2 = 2LL * (ell - 2) * n;
    // items with equal relinearisation keys next to each other (stable)
    std::vector<int> order(ids);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return matches_[a].job->keys->relin < matches_[b].job->keys->relin; });
    auto operand = [&](Job *j, int src, bool a_side) -> const u64 * {
        if (src < 0) return (a_side ? j->Ach[-src - 1] : j->Bch[-src - 1])->d;
        return align + (long long)slot_of.at(src) * csL;
    };
    std::vector<const u64 *> pa(m), pb(m), d2(m), dbase(m), x1(m), x2(m), mk(m);
    std::vector<int> gm(m), rf(m);
    std::vector<const Keys *> kk(m);
    u64 *D = rt.workspace(WS_TENSOR, (size_t)m * 3 * ell * n);
    u64 *X = rt.workspace(WS_RELIN_OUT, (size_t)m * csL);
    u64 *Y = rt.workspace(WS_LEVEL1, (size_t)m * cs1);
    u64 *Z = rt.workspace(WS_LEVEL2, (size_t)m * cs2);
    u64 *T = rt.workspace(WS_RS_TMP, (size_t)m * 2 * ell * n);
    for (int i = 0; i < m; ++i) {
        const MatchTask &t = matches_[order[i]];
        pa[i] = operand(t.job, t.src_a, true);
        pb[i] = operand(t.job, t.src_b, false);
        dbase[i] = D + (size_t)i * 3 * ell * n;
        d2[i] = dbase[i] + 2 * ell * n;
        x1[i] = X + i * csL;
        x2[i] = Y + i * cs1;
        mk[i] = t.job->mask;
        // the mask for slot p is sigma_h of the slot-0 mask, h = 5^-p
        gm[i] = galois_element(ctx, -t.min_slot);
        rf[i] = t.rf;
        kk[i] = t.job->keys;
    }
    tensor(ctx, m, ell, rt.upload_vec(pa), rt.upload_vec(pb), D);
    std::vector<KeyGroup> groups;
    for (int i = 0; i < m; ++i) {
        const u64 *key = kk[i]->relin;
        if (!groups.empty() && groups.back().key == key && groups.back().count < kRelinShare)
            ++groups.back().count;
        else
            groups.push_back(KeyGroup{key, i, 1});
    }
    if (relin_rescale_supported(ctx, ell)) {
        // the mask product rides on the rescale's last pass
        relin_rescale_batch(ctx, m, ell, rt.upload_vec(d2), groups, rt.upload_vec(dbase), T, Y, cs1,
                            rt.upload_vec(mk), rt.upload_vec(gm));
    } else {
        keyswitch_batch(ctx, m, ell, rt.upload_vec(d2), groups, rt.upload_vec(dbase), nullptr, true, X, csL);
        rescale(ctx, m, ell, rt.upload_vec(x1), T, Y, cs1);
        mul_plain_perm(ctx, m, ell - 1, Y, cs1, rt.upload_vec(mk), rt.upload_vec(gm));
    }
    // Relinearize after a plaintext product has nothing to switch
    rescale(ctx, m, ell - 1, rt.upload_vec(x2), T, Z, cs2);
    // final rotations into target slots, then accumulation per result chunk
    std::vector<const u64 *> zin(m);
    for (int i = 0; i < m; ++i) zin[i] = Z + i * cs2;
    if (rotate_accumulate_supported(ctx)) {
        std::vector<u64 *> tg(m);
        for (int i = 0; i < m; ++i) {
            const MatchTask &t = matches_[order[i]];
            tg[i] = t.job->C[t.rc]->d;
        }
        rotate_accumulate_batch(ctx, kk, ell - 2, zin, rf, tg, nullptr);
    } else {
        u64 *W = rt.workspace(WS_MISC, (size_t)m * cs2);
        rotate_batch(ctx, kk, ell - 2, zin, rf, W, nullptr);
        std::map<u64 *, std::vector<int>> by_target;
        for (int i = 0; i < m; ++i) {
            const MatchTask &t = matches_[order[i]];
            by_target[t.job->C[t.rc]->d].push_back(i);
        }
        for (auto &kv : by_target)
            accumulate(ctx, ell - 2, kv.first, W, cs2, rt.upload_vec(kv.second), (int)kv.second.size());
    }
    for (int i = 0; i < m; ++i) {
        const MatchTask &t = matches_[order[i]];
        Job *j = t.job;
        ++j->st_matches;
        ++j->st_relin;
        j->st_rescales += 2;
        j->st_final += rotation_plan(ctx, t.rf).size();
        task_done(j, 1);
    }
}

}  // namespace spfhe
