// Lazy-accumulation variant of the encrypted ct x ct product: a reordering
// of Alg. 2 (not the paper's op order).
//
// Alignment rotations and tensor products are Alg. 2's.  Every tensor product
// (three polynomials at the operands' level ell) is multiplied by its mask
// e_{min_slot} (level ell, scale q_{ell-2}) and summed into the group of
// matches sharing the result chunk and the final rotation amount r.  Each
// group is then rescaled (three polynomials, level ell-1), relinearised at
// level ell-1, rescaled again (level ell-2) and rotated:
//   merge_digits: by the lowest base-b digit of r; the rotated groups are
//     summed per (chunk, remaining amount) and each sum is rotated by its next
//     digit, digit by digit, until nothing remains;
//   otherwise: by the whole of r (its rotation plan);
// and what remains is added into the result chunks.  Relinearisation and
// rotation are linear, so the product decrypts like Alg. 2's; the number of
// relinearisations drops from #matches to #groups and the final-rotation key
// switches from the sum of the plan lengths to the digit tree's.
//
// Memory: every distinct alignment rotation is kept for the whole call (the
// groups meet them in any order); groups run in batches; with merge_digits
// the accumulators of the second tree level are all live.  Both are checked
// against the free device memory before any launch (ENOMEM otherwise).
#include <algorithm>
#include <cstring>
#include <map>

#include "engine.h"

namespace spfhe {

namespace {

struct GMatch {
    int src_a, src_b;   // >= 0: alignment store slot; < 0: -(chunk + 1)
    int min_slot;
};

struct Group {
    int rc, r;
    std::vector<int> matches;
};

// digit of r at weight w in base b
int digit_at(long long r, long long w, long long b) { return (int)((r / w) % b); }

void need_memory(size_t bytes, const char *what)
{
    size_t free_b = 0, total_b = 0;
    SPFHE_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t margin = (size_t)4 << 30;
    if (bytes + margin > free_b)
        throw Error(SPFHE_ENOMEM, std::string(what) + " needs " + std::to_string(bytes >> 20) + " MiB, " +
                                      std::to_string(free_b >> 20) + " MiB free");
}

}  // namespace

void spmspm_ct_ct_grouped(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                          const spfhe_sparse_meta &B, Ct *const *Bch, size_t nB, const Pt *mask0, bool merge,
                          Ct **C, size_t nC, spfhe_stats *out_stats)
{
    const uint64_t launches0 = ctx.launches;
    Runtime &rt = *ctx.rt;
    const int S = ctx.S;
    const size_t n = ctx.n;
    const long long b = ctx.rot_base;
    for (size_t c = 0; c < nC; ++c) C[c] = nullptr;
    std::vector<Ct *> av(Ach, Ach + nA), bv(Bch, Bch + nB);
    double rscale = 0;
    const int ell = check_ct_ct(ctx, A, av, B, bv, nC, &rscale);
    if (mask0 && mask0->level != ell) throw Error(SPFHE_ELEVEL, "the grouped product's mask is at the operands' level");
    const long long csL = 2LL * ell * n, cs1 = 2LL * (ell - 1) * n, cs2 = 2LL * (ell - 2) * n;
    const long long t3L = 3LL * ell * n, t31 = 3LL * (ell - 1) * n;

    // ---- plan: alignments, matches, groups ----
    const std::vector<MatchRec> ms = plan_alg1(A, B);
    if (!ms.empty() && !keys.relin) throw Error(SPFHE_EKEY, "no relinearisation key");
    std::map<std::tuple<int, int, int>, int> align_id;
    std::vector<std::tuple<int, int, int>> aligns;
    std::vector<GMatch> gm(ms.size());
    std::map<std::pair<int, int>, int> group_id;
    std::vector<Group> groups;
    for (size_t x = 0; x < ms.size(); ++x) {
        const MatchRec &mt = ms[x];
        const int ca = mt.a_pos / S, sa = mt.a_pos % S, cb = mt.b_pos / S, sb = mt.b_pos % S;
        GMatch g{-(ca + 1), -(cb + 1), std::min(sa, sb)};
        auto slot = [&](int op, int chunk, int amt) {
            const auto key = std::make_tuple(op, chunk, amt);
            auto it = align_id.find(key);
            if (it != align_id.end()) return it->second;
            const int id = (int)aligns.size();
            align_id[key] = id;
            aligns.push_back(key);
            return id;
        };
        if (sa < sb) g.src_b = slot(1, cb, sb - sa);
        else if (sb < sa) g.src_a = slot(0, ca, sa - sb);
        gm[x] = g;
        const long long t = (long long)mt.i * B.cols + mt.j;
        const int rc = (int)(t / S), r = (int)(((g.min_slot - t % S) % S + S) % S);
        auto it = group_id.find({rc, r});
        int gid;
        if (it == group_id.end()) {
            gid = (int)groups.size();
            group_id[{rc, r}] = gid;
            groups.push_back(Group{rc, r, {}});
        } else {
            gid = it->second;
        }
        groups[gid].matches.push_back((int)x);
    }
    // groups in (chunk, amount) order
    std::vector<int> gorder;
    for (auto &kv : group_id) gorder.push_back(kv.second);
    // every key the call will use, before anything is launched
    for (auto &a : aligns)
        for (int s : rotation_plan(ctx, std::get<2>(a))) rotation_key(keys, s);
    std::map<std::pair<int, long long>, int> stage1;   // (chunk, remaining) -> accumulator index
    for (const Group &g : groups) {
        if (merge) {
            const int d0 = (int)(g.r % b);
            if (d0) rotation_key(keys, d0);
            stage1.emplace(std::make_pair(g.rc, (long long)g.r - d0), 0);
            for (long long w = b; w < S; w *= b) {
                const int d = digit_at(g.r, w, b);
                if (d) rotation_key(keys, (int)(d * w));
            }
        } else {
            for (int s : rotation_plan(ctx, g.r)) rotation_key(keys, s);
        }
    }
    need_memory(aligns.size() * (size_t)csL * sizeof(u64) + (merge ? stage1.size() * (size_t)cs2 * sizeof(u64) : 0),
                "the alignment store and digit-tree accumulators");

    Scratch sc(ctx);
    uint64_t st_align = 0, st_final = 0, st_relin = 0, st_rescales = 0;
    std::vector<Ct *> res(nC, nullptr);
    try {
        for (size_t c = 0; c < nC; ++c) {
            res[c] = ct_new(ctx, ell - 2, rscale);
            SPFHE_CHECK_CUDA(cudaMemsetAsync(res[c]->d, 0, (size_t)cs2 * sizeof(u64), ctx.stream));
        }
        if (!ms.empty()) {
            // ---- mask at level ell, Montgomery form ----
            u64 *mask = sc.words((size_t)ell * n);
            if (mask0) {
                copy_words(ctx, mask, mask0->d, (size_t)ell * n);
            } else {
                const double one = 1.0;
                const double *d_one = static_cast<const double *>(rt.upload(&one, sizeof(double)));
                encode_onehot0(ctx, d_one, 1, ell, (double)ctx.mods[ell - 2], mask);
            }
            std::vector<int> mi(ell);
            for (int i = 0; i < ell; ++i) mi[i] = i;
            to_montgomery(ctx, mask, ell, mi.data(), 1);

            // ---- alignment store ----
            const int Bm = match_batch_size(ctx);
            u64 *store = aligns.empty() ? nullptr : sc.words(aligns.size() * (size_t)csL);
            for (size_t a0 = 0; a0 < aligns.size(); a0 += Bm) {
                const size_t a1 = std::min(aligns.size(), a0 + Bm);
                std::vector<const u64 *> in;
                std::vector<int> amt;
                for (size_t a = a0; a < a1; ++a) {
                    const int op = std::get<0>(aligns[a]), chunk = std::get<1>(aligns[a]);
                    in.push_back((op == 0 ? Ach[chunk] : Bch[chunk])->d);
                    amt.push_back(std::get<2>(aligns[a]));
                }
                rotate_batch(ctx, keys, ell, in, amt, store + (long long)a0 * csL, &st_align);
            }
            auto operand = [&](int src, bool a_side) -> const u64 * {
                if (src < 0) return (a_side ? Ach[-src - 1] : Bch[-src - 1])->d;
                return store + (long long)src * csL;
            };

            // ---- tree accumulators of the second level ----
            std::vector<u64 *> acc1;
            if (merge) {
                int k = 0;
                for (auto &kv : stage1) {
                    kv.second = k++;
                    u64 *p = sc.words((size_t)cs2);
                    SPFHE_CHECK_CUDA(cudaMemsetAsync(p, 0, (size_t)cs2 * sizeof(u64), ctx.stream));
                    acc1.push_back(p);
                }
            }

            // ---- groups in batches of up to Bm ----
            const size_t max_matches = (size_t)2 * Bm;
            for (size_t gi = 0; gi < gorder.size(); gi += Bm) {
                std::vector<int> bg(gorder.begin() + gi, gorder.begin() + std::min(gorder.size(), gi + Bm));
                const int k = (int)bg.size();
                u64 *G = rt.workspace(WS_GRP_SUM, (size_t)k * t3L);
                u64 *R1 = rt.workspace(WS_LEVEL1, (size_t)k * t31);
                u64 *R2 = rt.workspace(WS_LEVEL2, (size_t)k * cs1);
                u64 *T = rt.workspace(WS_RS_TMP, (size_t)k * t3L);
                u64 *X = rt.workspace(WS_RELIN_OUT, (size_t)k * cs2);
                u64 *Y = rt.workspace(WS_MISC, (size_t)k * cs2);
                // tensor products and masks of the batch's matches, at most
                // max_matches at a time, summed into their groups
                std::vector<std::pair<int, int>> flat;   // (group in batch, match)
                for (int g = 0; g < k; ++g)
                    for (int x : groups[bg[g]].matches) flat.push_back({g, x});
                std::vector<char> started(k, 0);
                for (size_t f0 = 0; f0 < flat.size(); f0 += max_matches) {
                    const size_t f1 = std::min(flat.size(), f0 + max_matches);
                    const int m = (int)(f1 - f0);
                    u64 *D = rt.workspace(WS_TENSOR, (size_t)m * t3L);
                    std::vector<const u64 *> pa, pb, mk, dsrc;
                    std::vector<int> gal;
                    for (size_t f = f0; f < f1; ++f) {
                        const int x = flat[f].second;
                        pa.push_back(operand(gm[x].src_a, true));
                        pb.push_back(operand(gm[x].src_b, false));
                        mk.push_back(mask);
                        // the mask for slot p is sigma_h of the slot-0 mask, h = 5^-p
                        gal.push_back(galois_element(ctx, -gm[x].min_slot));
                        dsrc.push_back(D + (long long)(f - f0) * t3L);
                    }
                    tensor(ctx, m, ell, rt.upload_vec(pa), rt.upload_vec(pb), D);
                    mul_plain_perm(ctx, m, ell, D, t3L, rt.upload_vec(mk), rt.upload_vec(gal), 3);
                    // segments: runs of equal group (flat is in group order); a
                    // group continued from the previous piece adds to its sum
                    std::vector<u64 *> fresh_t, cont_t;
                    std::vector<const u64 *> fresh_s, cont_s;
                    std::vector<int> fresh_seg{0}, cont_seg{0};
                    for (size_t f = f0; f < f1;) {
                        const int g = flat[f].first;
                        size_t e = f;
                        while (e < f1 && flat[e].first == g) ++e;
                        auto &tt = started[g] ? cont_t : fresh_t;
                        auto &ss = started[g] ? cont_s : fresh_s;
                        auto &sg = started[g] ? cont_seg : fresh_seg;
                        tt.push_back(G + (long long)g * t3L);
                        for (size_t q = f; q < e; ++q) ss.push_back(dsrc[q - f0]);
                        sg.push_back((int)ss.size());
                        started[g] = 1;
                        f = e;
                    }
                    if (!fresh_t.empty())
                        accumulate_seg(ctx, 3, ell, (int)fresh_t.size(), rt.upload_vec(fresh_t),
                                       rt.upload_vec(fresh_s), rt.upload_vec(fresh_seg), (int)fresh_s.size(), false);
                    if (!cont_t.empty())
                        accumulate_seg(ctx, 3, ell, (int)cont_t.size(), rt.upload_vec(cont_t), rt.upload_vec(cont_s),
                                       rt.upload_vec(cont_seg), (int)cont_s.size(), true);
                }
                // rescale of the three polynomials, relinearisation at level
                // ell-1 (key switch of the s^2 part, added to the first two),
                // rescale of the ciphertext
                std::vector<const u64 *> g0(k), d2(k), base(k), x1(k);
                for (int g = 0; g < k; ++g) {
                    g0[g] = G + (long long)g * t3L;
                    base[g] = R1 + (long long)g * t31;
                    d2[g] = base[g] + 2LL * (ell - 1) * n;
                    x1[g] = R2 + (long long)g * cs1;
                }
                rescale(ctx, k, ell, rt.upload_vec(g0), T, R1, t31, 3);
                std::vector<KeyGroup> kg;
                for (int g = 0; g < k; g += 4) kg.push_back(KeyGroup{keys.relin, g, std::min(4, k - g)});
                keyswitch_batch(ctx, k, ell - 1, rt.upload_vec(d2), kg, rt.upload_vec(base), nullptr, true, R2, cs1);
                st_relin += k;
                rescale(ctx, k, ell - 1, rt.upload_vec(x1), T, X, cs2, 2);
                st_rescales += 2ull * k;
                // rotation by the lowest digit (merge) or the whole amount
                std::vector<const u64 *> src(k);
                for (int g = 0; g < k; ++g) src[g] = X + (long long)g * cs2;
                if (merge) {
                    std::vector<const u64 *> rin, rkey;
                    std::vector<int> rg, rid;
                    for (int g = 0; g < k; ++g) {
                        const int d0 = (int)(groups[bg[g]].r % b);
                        if (!d0) continue;
                        rin.push_back(src[g]);
                        rg.push_back(galois_element(ctx, d0));
                        rkey.push_back(rotation_key(keys, d0));
                        rid.push_back(g);
                    }
                    // equal keys next to each other for the inner product
                    std::vector<int> ord(rid.size());
                    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
                    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return rkey[x] < rkey[y]; });
                    std::vector<const u64 *> sin, skey;
                    std::vector<int> sg;
                    for (int i : ord) {
                        sin.push_back(rin[i]);
                        sg.push_back(rg[i]);
                        skey.push_back(rkey[i]);
                    }
                    rotate_step_batch(ctx, ell - 2, sin, sg, skey, Y);
                    st_final += sin.size();
                    for (size_t i = 0; i < ord.size(); ++i) src[rid[ord[i]]] = Y + (long long)i * cs2;
                    // sums per (chunk, remaining amount)
                    std::map<int, std::vector<int>> by_acc;
                    for (int g = 0; g < k; ++g) {
                        const Group &gr = groups[bg[g]];
                        by_acc[stage1.at({gr.rc, (long long)gr.r - gr.r % b})].push_back(g);
                    }
                    std::vector<u64 *> tg;
                    std::vector<const u64 *> ss;
                    std::vector<int> sg2{0};
                    for (auto &kv : by_acc) {
                        tg.push_back(acc1[kv.first]);
                        for (int g : kv.second) ss.push_back(src[g]);
                        sg2.push_back((int)ss.size());
                    }
                    accumulate_seg(ctx, 2, ell - 2, (int)tg.size(), rt.upload_vec(tg), rt.upload_vec(ss),
                                   rt.upload_vec(sg2), (int)ss.size(), true);
                } else {
                    std::vector<int> amt(k);
                    for (int g = 0; g < k; ++g) amt[g] = groups[bg[g]].r;
                    rotate_batch(ctx, keys, ell - 2, src, amt, Y, &st_final);
                    std::map<int, std::vector<int>> by_chunk;
                    for (int g = 0; g < k; ++g) by_chunk[groups[bg[g]].rc].push_back(g);
                    std::vector<u64 *> tg;
                    std::vector<const u64 *> ss;
                    std::vector<int> sg2{0};
                    for (auto &kv : by_chunk) {
                        tg.push_back(res[kv.first]->d);
                        for (int g : kv.second) ss.push_back(Y + (long long)g * cs2);
                        sg2.push_back((int)ss.size());
                    }
                    accumulate_seg(ctx, 2, ell - 2, (int)tg.size(), rt.upload_vec(tg), rt.upload_vec(ss),
                                   rt.upload_vec(sg2), (int)ss.size(), true);
                }
            }

            // ---- digit tree: rotate each sum by its next digit and merge ----
            if (merge) {
                std::map<std::pair<int, long long>, u64 *> live;
                for (auto &kv : stage1) live[kv.first] = acc1[kv.second];
                for (long long w = b; w < S; w *= b) {
                    bool rest = false;
                    for (auto &kv : live) rest = rest || kv.first.second != 0;
                    if (!rest) break;
                    std::map<std::pair<int, long long>, std::vector<const u64 *>> next_src;
                    std::vector<std::pair<int, long long>> keys_v;
                    for (auto &kv : live) keys_v.push_back(kv.first);
                    for (size_t k0 = 0; k0 < keys_v.size(); k0 += Bm) {
                        const size_t k1 = std::min(keys_v.size(), k0 + Bm);
                        std::vector<const u64 *> sin, skey;
                        std::vector<int> sg;
                        std::vector<size_t> rid;
                        for (size_t x = k0; x < k1; ++x) {
                            const int d = digit_at(keys_v[x].second, w, b);
                            if (!d) continue;
                            sin.push_back(live[keys_v[x]]);
                            sg.push_back(galois_element(ctx, (int)(d * w)));
                            skey.push_back(rotation_key(keys, (int)(d * w)));
                            rid.push_back(x);
                        }
                        if (!sin.empty()) {
                            u64 *out = sc.words(sin.size() * (size_t)cs2);
                            rotate_step_batch(ctx, ell - 2, sin, sg, skey, out);
                            st_final += sin.size();
                            for (size_t i = 0; i < rid.size(); ++i) live[keys_v[rid[i]]] = out + (long long)i * cs2;
                        }
                    }
                    for (auto &kv : live) {
                        const int d = digit_at(kv.first.second, w, b);
                        next_src[{kv.first.first, kv.first.second - d * w}].push_back(kv.second);
                    }
                    std::map<std::pair<int, long long>, u64 *> nl;
                    std::vector<u64 *> tg;
                    std::vector<const u64 *> ss;
                    std::vector<int> sg2{0};
                    for (auto &kv : next_src) {
                        u64 *p = sc.words((size_t)cs2);
                        nl[kv.first] = p;
                        tg.push_back(p);
                        for (const u64 *q : kv.second) ss.push_back(q);
                        sg2.push_back((int)ss.size());
                    }
                    accumulate_seg(ctx, 2, ell - 2, (int)tg.size(), rt.upload_vec(tg), rt.upload_vec(ss),
                                   rt.upload_vec(sg2), (int)ss.size(), false);
                    live.swap(nl);
                }
                std::map<int, std::vector<const u64 *>> by_chunk;
                for (auto &kv : live) by_chunk[kv.first.first].push_back(kv.second);
                std::vector<u64 *> tg;
                std::vector<const u64 *> ss;
                std::vector<int> sg2{0};
                for (auto &kv : by_chunk) {
                    tg.push_back(res[kv.first]->d);
                    for (const u64 *q : kv.second) ss.push_back(q);
                    sg2.push_back((int)ss.size());
                }
                accumulate_seg(ctx, 2, ell - 2, (int)tg.size(), rt.upload_vec(tg), rt.upload_vec(ss),
                               rt.upload_vec(sg2), (int)ss.size(), true);
            }
        }
        SPFHE_CHECK_CUDA(cudaStreamSynchronize(ctx.stream));
    } catch (...) {
        for (Ct *c : res)
            if (c) {
                dev_free(ctx, c->d);
                delete c;
            }
        throw;
    }
    for (size_t c = 0; c < nC; ++c) C[c] = res[c];
    if (out_stats) {
        out_stats->matches = ms.size();
        out_stats->ks_relin = st_relin;
        out_stats->ks_align = st_align;
        out_stats->ks_final = st_final;
        out_stats->rescales = st_rescales;
        out_stats->launches = ctx.launches - launches0;
    }
}

}  // namespace spfhe
