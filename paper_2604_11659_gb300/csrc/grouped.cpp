// Lazy-accumulation variants of the encrypted products: reorderings of
// Alg. 2 (not the paper's op order).
//
// ct x ct: alignment rotations and tensor products are Alg. 2's.  Every
// tensor product (three polynomials at the operands' level ell) is multiplied
// by its mask e_{min_slot} (level ell, scale q_{ell-2}) and summed into the
// group of matches sharing the result chunk and the final rotation amount r.
// Each group is rescaled (three polynomials, level ell-1), relinearised at
// level ell-1, rescaled again (level ell-2) and handed to the rotation tree.
//
// ct x pt (reading R9's products): the weight plaintexts B[k, j] e_{a_slot}
// of a group's matches are summed per A chunk, each sum multiplies its chunk,
// the products are added, rescaled once (level L-1) and handed to the tree.
// With the library's own weights, a sub-group's summed plaintext is encoded
// in one pass (coefficient-domain sum of the permuted one-hot encodings, one
// transform) instead of one encoding and transform per match.
//
// Rotation tree: merge_digits rotates each group by the lowest base-b digit
// of r, sums the results per (chunk, remaining amount) and rotates each sum
// by its next digit, digit by digit, until nothing remains; otherwise every
// group is rotated by the whole of r.  What remains is added into the result
// chunks.  Relinearisation and rotation are linear, so the products decrypt
// like Alg. 2's, with fewer key switches; the ciphertext bits differ.
//
// Alignment rotations (ct x ct) are computed per source ciphertext digit by
// digit from the highest base-b digit down: at each digit position, the
// ciphertexts that share the higher digits are rotated by every needed digit
// with one hoisted ModUp (rotate_hoisted), so a source needs one key switch
// per distinct (higher digits, nonzero digit) and one ModUp per stage input.
//
// Groups arrive at the tree in ascending (chunk, r) order, so a sum of the
// tree is complete as soon as the stream has passed its range of amounts and
// no sum at a lower level within that range is still pending; sums are
// rotated in batches as they complete, which bounds the tree's memory for
// any base.  The ct x ct variant keeps every distinct alignment rotation of
// the call in device memory when they fit in the free memory; otherwise it
// streams them: each batch of groups computes the alignment rotations its
// matches use (digit by digit as above, restricted to those amounts) and
// frees them before the next batch, so memory stays bounded at the cost of
// recomputing rotations that several batches use.  Both give the same bits.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <set>

#include "engine.h"

namespace spfhe {

namespace {

using Key = std::pair<int, long long>;   // (result chunk, amount)

void need_memory(size_t bytes, const char *what)
{
    size_t free_b = 0, total_b = 0;
    SPFHE_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t margin = (size_t)4 << 30;
    if (bytes + margin > free_b)
        throw Error(SPFHE_ENOMEM, std::string(what) + " needs " + std::to_string(bytes >> 20) + " MiB, " +
                                      std::to_string(free_b >> 20) + " MiB free");
}

// tgt[i] (+)= sum of srcs[i]; fresh targets start at zero
void sum_into(Ctx &ctx, int polys, int ell, const std::vector<u64 *> &tgt,
              const std::vector<std::vector<const u64 *>> &srcs, const std::vector<char> &fresh)
{
    Runtime &rt = *ctx.rt;
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<u64 *> t;
        std::vector<const u64 *> s;
        std::vector<int> seg{0};
        for (size_t i = 0; i < tgt.size(); ++i) {
            if ((fresh[i] != 0) != (pass == 0)) continue;
            t.push_back(tgt[i]);
            for (const u64 *p : srcs[i]) s.push_back(p);
            seg.push_back((int)s.size());
        }
        if (t.empty()) continue;
        accumulate_seg(ctx, polys, ell, (int)t.size(), rt.upload_vec(t), rt.upload_vec(s), rt.upload_vec(seg),
                       (int)s.size(), pass == 1);
    }
}

// Streaming rotation tree over ciphertexts at level lv (see the file comment).
class DigitTree {
  public:
    DigitTree(Ctx &ctx, const Keys &keys, int lv, bool merge, const std::vector<Ct *> &res)
        : ctx_(ctx), keys_(keys), lv_(lv), merge_(merge), res_(res), b_(ctx.rot_base), S_(ctx.S),
          cs_(2LL * lv * ctx.n), bm_(match_batch_size(ctx))
    {
        digits_ = 0;
        for (long long w = 1; w < S_; w *= b_) ++digits_;
        levels_.resize(std::max(digits_, 1));
    }
    ~DigitTree()
    {
        for (u64 *p : all_) dev_free(ctx_, p);
    }
    // every key the tree will use for an item of amount r
    static void check_keys(const Ctx &ctx, const Keys &keys, long long r, bool merge)
    {
        if (!merge) {
            for (int s : rotation_plan(ctx, r)) rotation_key(keys, s);
            return;
        }
        for (long long w = 1; w < ctx.S; w *= ctx.rot_base) {
            const int d = (int)((r / w) % ctx.rot_base);
            if (d) rotation_key(keys, (int)(d * w));
        }
    }
    // items in ascending (chunk, r) order; `next` = the key of the first item
    // not pushed yet ({INT_MAX, 0} when none follows)
    void push(const std::vector<Key> &key, const std::vector<const u64 *> &ct, Key next)
    {
        const int k = (int)key.size();
        if (!k) return;
        Runtime &rt = *ctx_.rt;
        u64 *out = rt.workspace(WS_TREE_ROT, (size_t)k * cs_);
        std::vector<const u64 *> src(ct);
        if (!merge_) {
            std::vector<int> amt(k);
            for (int i = 0; i < k; ++i) amt[i] = (int)key[i].second;
            if (rotate_accumulate_supported(ctx_)) {
                std::vector<u64 *> tg(k);
                for (int i = 0; i < k; ++i) tg[i] = res_[key[i].first]->d;
                rotate_accumulate_batch(ctx_, std::vector<const Keys *>(k, &keys_), lv_, ct, amt, tg, &ks);
                return;
            }
            rotate_batch(ctx_, keys_, lv_, ct, amt, out, &ks);
            for (int i = 0; i < k; ++i) src[i] = out + (long long)i * cs_;
            add_to_results(key, src);
            return;
        }
        if (rotate_accumulate_supported(ctx_)) {
            rotate_route(key, src, 1, 1);
        } else {
            rotate_digit(key, src, 1, out);
            route(key, src, 1, 1);
        }
        flush(next, false);
    }
    void finish()
    {
        if (merge_) flush(Key{INT_MAX, 0}, true);
    }
    uint64_t ks = 0;

  private:
    Ctx &ctx_;
    const Keys &keys_;
    int lv_;
    bool merge_;
    const std::vector<Ct *> &res_;
    long long b_, S_, cs_;
    int bm_, digits_;
    // levels_[t]: sums whose amounts have their t lowest digits removed
    std::vector<std::map<Key, u64 *>> levels_;
    std::vector<u64 *> pool_, all_;

    u64 *get()
    {
        if (!pool_.empty()) {
            u64 *p = pool_.back();
            pool_.pop_back();
            return p;
        }
        u64 *p = static_cast<u64 *>(dev_alloc(ctx_, (size_t)cs_ * sizeof(u64)));
        all_.push_back(p);
        return p;
    }
    long long weight(int t) const
    {
        long long w = 1;
        for (int i = 0; i < t; ++i) w *= b_;
        return w;
    }
    int digit(long long r, long long w) const { return (int)((r / w) % b_); }
    // rotate src[i] by its key's digit at weight w (those with a nonzero
    // digit); the rotated ciphertexts go to out and replace src[i]
    void rotate_digit(const std::vector<Key> &key, std::vector<const u64 *> &src, long long w, u64 *out)
    {
        std::vector<int> rid;
        for (size_t i = 0; i < key.size(); ++i)
            if (digit(key[i].second, w)) rid.push_back((int)i);
        if (rid.empty()) return;
        // equal keys next to each other for the inner product
        std::stable_sort(rid.begin(), rid.end(),
                         [&](int x, int y) { return digit(key[x].second, w) < digit(key[y].second, w); });
        std::vector<const u64 *> sin, skey;
        std::vector<int> sg;
        for (int i : rid) {
            const int d = digit(key[i].second, w);
            sin.push_back(src[i]);
            sg.push_back(galois_element(ctx_, (int)(d * w)));
            skey.push_back(rotation_key(keys_, (int)(d * w)));
        }
        rotate_step_batch(ctx_, lv_, sin, sg, skey, out);
        ks += sin.size();
        for (size_t j = 0; j < rid.size(); ++j) src[rid[j]] = out + (long long)j * cs_;
    }
    // add each (rotated) item into its sum at level t (amount minus its digit
    // at weight w), or into its result chunk when nothing remains
    void route(const std::vector<Key> &key, const std::vector<const u64 *> &src, int t, long long w)
    {
        std::map<Key, std::vector<const u64 *>> to_level;
        std::map<int, std::vector<const u64 *>> to_res;
        for (size_t i = 0; i < key.size(); ++i) {
            const long long rem = key[i].second - digit(key[i].second, w) * w;
            if (rem == 0) to_res[key[i].first].push_back(src[i]);
            else to_level[{key[i].first, rem}].push_back(src[i]);
        }
        std::vector<u64 *> tgt;
        std::vector<std::vector<const u64 *>> srcs;
        std::vector<char> fresh;
        for (auto &kv : to_level) {
            auto it = levels_[t].find(kv.first);
            const bool f = it == levels_[t].end();
            u64 *p = f ? (levels_[t][kv.first] = get()) : it->second;
            tgt.push_back(p);
            srcs.push_back(kv.second);
            fresh.push_back(f ? 1 : 0);
        }
        for (auto &kv : to_res) {
            tgt.push_back(res_[kv.first]->d);
            srcs.push_back(kv.second);
            fresh.push_back(0);
        }
        sum_into(ctx_, 2, lv_, tgt, srcs, fresh);
    }
    // rotate_digit followed by route with the rotated items' ModDown
    // transforms taken once per destination sum (rotate_step_accumulate):
    // items with a zero digit at weight w are summed as they are (starting
    // fresh sums), fresh sums that receive only rotated items start at zero,
    // then every rotated item is added into its sum
    void rotate_route(const std::vector<Key> &key, const std::vector<const u64 *> &src, long long w, int t)
    {
        const size_t k = key.size();
        std::vector<u64 *> dst(k);
        std::map<u64 *, char> fresh;   // destination -> 1 while it holds nothing yet
        for (size_t i = 0; i < k; ++i) {
            const long long rem = key[i].second - digit(key[i].second, w) * w;
            if (rem == 0) {
                dst[i] = res_[key[i].first]->d;
                fresh.emplace(dst[i], 0);
                continue;
            }
            const Key tk{key[i].first, rem};
            auto it = levels_[t].find(tk);
            if (it == levels_[t].end()) {
                dst[i] = levels_[t][tk] = get();
                fresh[dst[i]] = 1;
            } else {
                dst[i] = it->second;
                fresh.emplace(dst[i], 0);
            }
        }
        // items with a zero digit: plain sums (a fresh sum starts from them)
        std::map<u64 *, std::vector<const u64 *>> plain;
        for (size_t i = 0; i < k; ++i)
            if (!digit(key[i].second, w)) plain[dst[i]].push_back(src[i]);
        {
            std::vector<u64 *> tgt;
            std::vector<std::vector<const u64 *>> srcs;
            std::vector<char> fr;
            for (auto &kv : plain) {
                tgt.push_back(kv.first);
                srcs.push_back(kv.second);
                fr.push_back(fresh[kv.first]);
                fresh[kv.first] = 0;
            }
            if (!tgt.empty()) sum_into(ctx_, 2, lv_, tgt, srcs, fr);
        }
        for (auto &kv : fresh)
            if (kv.second)
                SPFHE_CHECK_CUDA(cudaMemsetAsync(kv.first, 0, (size_t)cs_ * sizeof(u64), ctx_.stream));
        std::vector<int> rid;
        for (size_t i = 0; i < k; ++i)
            if (digit(key[i].second, w)) rid.push_back((int)i);
        if (rid.empty()) return;
        // equal keys next to each other for the inner product
        std::stable_sort(rid.begin(), rid.end(),
                         [&](int x, int y) { return digit(key[x].second, w) < digit(key[y].second, w); });
        std::vector<const u64 *> sin, skey;
        std::vector<int> sg;
        std::vector<u64 *> st;
        for (int i : rid) {
            const int d = digit(key[i].second, w);
            sin.push_back(src[i]);
            sg.push_back(galois_element(ctx_, (int)(d * w)));
            skey.push_back(rotation_key(keys_, (int)(d * w)));
            st.push_back(dst[i]);
        }
        rotate_step_accumulate(ctx_, lv_, sin, sg, skey, st);
        ks += sin.size();
    }
    void add_to_results(const std::vector<Key> &key, const std::vector<const u64 *> &src)
    {
        std::map<int, std::vector<const u64 *>> by;
        for (size_t i = 0; i < key.size(); ++i) by[key[i].first].push_back(src[i]);
        std::vector<u64 *> tgt;
        std::vector<std::vector<const u64 *>> srcs;
        for (auto &kv : by) {
            tgt.push_back(res_[kv.first]->d);
            srcs.push_back(kv.second);
        }
        sum_into(ctx_, 2, lv_, tgt, srcs, std::vector<char>(tgt.size(), 0));
    }
    // rotate every complete sum by its next digit and pass it on (at least
    // bm_ sums of a level at a time unless forced)
    void flush(Key next, bool force)
    {
        for (int t = 1; t < digits_; ++t) {
            const long long w = weight(t);
            std::vector<Key> done;
            for (auto &kv : levels_[t]) {
                const Key &k = kv.first;
                // every group of amounts [k.second, k.second + w) has been pushed ...
                const Key end{k.first, k.second + w};
                if (!force && next < end) break;
                // ... and no sum at any lower level is still on its way to it
                bool fed = false;
                for (int u = 1; u < t && !fed; ++u) {
                    auto lo = levels_[u].lower_bound(k);
                    fed = lo != levels_[u].end() && lo->first < end;
                }
                if (fed) break;
                done.push_back(k);
            }
            if (done.empty() || (!force && (int)done.size() < bm_)) continue;
            for (size_t d0 = 0; d0 < done.size(); d0 += bm_) {
                const size_t d1 = std::min(done.size(), d0 + bm_);
                std::vector<Key> key(done.begin() + d0, done.begin() + d1);
                std::vector<const u64 *> src;
                std::vector<u64 *> owned;
                for (const Key &k : key) {
                    owned.push_back(levels_[t][k]);
                    src.push_back(levels_[t][k]);
                    levels_[t].erase(k);
                }
                if (rotate_accumulate_supported(ctx_)) {
                    rotate_route(key, src, w, t + 1 < digits_ ? t + 1 : t);
                } else {
                    u64 *out = ctx_.rt->workspace(WS_TREE_ROT, key.size() * (size_t)cs_);
                    rotate_digit(key, src, w, out);
                    route(key, src, t + 1 < digits_ ? t + 1 : t, w);
                }
                for (u64 *p : owned) pool_.push_back(p);
            }
        }
    }
};

struct PlanMatch {
    int src_a, src_b;   // >= 0 alignment store slot, < 0: -(chunk + 1)
    int slot;           // min_slot
};

void fill_stats(spfhe_stats *st, uint64_t matches, uint64_t relin, uint64_t align, uint64_t fin, uint64_t resc,
                uint64_t launches)
{
    if (!st) return;
    st->matches = matches;
    st->ks_relin = relin;
    st->ks_align = align;
    st->ks_final = fin;
    st->rescales = resc;
    st->launches = launches;
}

void free_results(Ctx &ctx, std::vector<Ct *> &res)
{
    for (Ct *&c : res)
        if (c) {
            dev_free(ctx, c->d);
            delete c;
            c = nullptr;
        }
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
    for (size_t c = 0; c < nC; ++c) C[c] = nullptr;
    std::vector<Ct *> av(Ach, Ach + nA), bv(Bch, Bch + nB);
    double rscale = 0;
    const int ell = check_ct_ct(ctx, A, av, B, bv, nC, &rscale);
    if (mask0 && mask0->level != ell) throw Error(SPFHE_ELEVEL, "the grouped product's mask is at the operands' level");
    const long long csL = 2LL * ell * n, cs1 = 2LL * (ell - 1) * n, cs2 = 2LL * (ell - 2) * n;
    const long long t3L = 3LL * ell * n, t31 = 3LL * (ell - 1) * n;

    // ---- plan: alignments, matches, groups in (chunk, amount) order ----
    const std::vector<MatchRec> ms = plan_alg1(A, B);
    if (!ms.empty() && !keys.relin) throw Error(SPFHE_EKEY, "no relinearisation key");
    std::map<std::tuple<int, int, int>, int> align_id;
    std::vector<std::tuple<int, int, int>> aligns;
    std::vector<PlanMatch> pm(ms.size());
    std::map<Key, std::vector<int>> groups;
    for (size_t x = 0; x < ms.size(); ++x) {
        const MatchRec &mt = ms[x];
        const int ca = mt.a_pos / S, sa = mt.a_pos % S, cb = mt.b_pos / S, sb = mt.b_pos % S;
        PlanMatch g{-(ca + 1), -(cb + 1), std::min(sa, sb)};
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
        pm[x] = g;
        const long long t = (long long)mt.i * B.cols + mt.j;
        groups[{(int)(t / S), ((g.slot - t % S) % S + S) % S}].push_back((int)x);
    }
    // alignment plan: per source ciphertext, its amounts digit by digit from
    // the top; one hoisted rotation batch per (source, higher digits)
    const long long b = ctx.rot_base;
    long long top = 1;
    while (top * b < S) top *= b;
    std::map<std::pair<int, int>, std::vector<int>> by_src;   // (operand, chunk) -> alignment ids
    for (size_t a = 0; a < aligns.size(); ++a)
        by_src[{std::get<0>(aligns[a]), std::get<1>(aligns[a])}].push_back((int)a);
    size_t n_rot = 0;
    for (auto &kv : by_src)
        for (long long w = top; w >= 1; w /= b) {
            std::set<std::pair<long long, int>> st;
            for (int a : kv.second) {
                const long long amt = std::get<2>(aligns[a]);
                const int d = (int)((amt / w) % b);
                if (d) {
                    st.insert({amt - amt % (w * b), d});
                    rotation_key(keys, (int)(d * w));   // every key, before anything is launched
                }
            }
            n_rot += st.size();
        }
    for (auto &kv : groups) DigitTree::check_keys(ctx, keys, kv.first.second, merge);
    // every distinct alignment rotation kept for the whole call when it fits;
    // otherwise (streaming) each batch of groups computes the rotations its
    // matches use and frees them before the next batch
    const size_t align_bytes = n_rot * (size_t)csL * sizeof(u64);
    bool streaming = align_bytes > ctx.align_budget;
    if (!streaming) {
        try {
            need_memory(align_bytes, "the alignment rotations");
        } catch (const Error &) {
            streaming = true;
        }
    }

    uint64_t st_align = 0, st_relin = 0, st_rescales = 0, st_final = 0;
    std::vector<Ct *> res(nC, nullptr);
    try {
        Scratch sc(ctx);
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

            // ---- alignment rotations: per source, digit by digit from the
            // top, the ciphertexts sharing the higher digits rotated by every
            // needed digit with one hoisted ModUp ----
            const int Bm = match_batch_size(ctx);
            std::vector<const u64 *> aligned(aligns.size(), nullptr);
            auto compute_aligns = [&](const std::map<std::pair<int, int>, std::vector<int>> &srcs, Scratch &mem) {
                for (auto &kv : srcs) {
                    const u64 *src = (kv.first.first == 0 ? Ach[kv.first.second] : Bch[kv.first.second])->d;
                    std::map<long long, const u64 *> cur{{0, src}};
                    for (long long w = top; w >= 1; w /= b) {
                        std::map<long long, const u64 *> nxt;
                        for (auto &ck : cur) {
                            std::set<int> digs;
                            for (int a : kv.second) {
                                const long long amt = std::get<2>(aligns[a]);
                                if (amt - amt % (w * b) == ck.first) digs.insert((int)((amt / w) % b));
                            }
                            std::vector<int> amts;
                            for (int d : digs)
                                if (d) amts.push_back((int)(d * w));
                            u64 *o = amts.empty() ? nullptr : mem.words(amts.size() * (size_t)csL);
                            rotate_hoisted(ctx, keys, ell, ck.second, amts, o);
                            st_align += amts.size();
                            size_t r = 0;
                            for (int d : digs) nxt[ck.first + d * w] = d ? o + (long long)(r++) * csL : ck.second;
                        }
                        cur.swap(nxt);
                    }
                    for (int a : kv.second) aligned[a] = cur.at(std::get<2>(aligns[a]));
                }
            };
            if (!streaming) compute_aligns(by_src, sc);
            auto operand = [&](int src, bool a_side) -> const u64 * {
                if (src < 0) return (a_side ? Ach[-src - 1] : Bch[-src - 1])->d;
                return aligned[src];
            };

            DigitTree tree(ctx, keys, ell - 2, merge, res);
            std::vector<const std::pair<const Key, std::vector<int>> *> gl;
            for (auto &kv : groups) gl.push_back(&kv);
            const size_t max_matches = (size_t)2 * Bm;
            // batches of at most Bm groups; streaming: also at most as many
            // as keep the batch's alignment rotations (every ciphertext the
            // digit-by-digit process creates for them) within half the free
            // memory left after a margin
            std::vector<size_t> ends;
            if (!streaming) {
                for (size_t gi = 0; gi < gl.size(); gi += Bm) ends.push_back(std::min(gl.size(), gi + Bm));
            } else {
                size_t free_b = 0, total_b = 0;
                SPFHE_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
                const size_t margin = (size_t)8 << 30;
                const size_t limit_cts =
                    std::max<size_t>(1, (free_b > margin ? (free_b - margin) / 2 : 0) / ((size_t)csL * sizeof(u64)));
                std::set<std::tuple<int, int, long long, long long>> nodes;   // (operand, chunk, stage, prefix + digit)
                std::set<int> seen;
                size_t gi = 0;
                for (size_t g = 0; g < gl.size(); ++g) {
                    std::vector<std::tuple<int, int, long long, long long>> add;
                    for (int x : gl[g]->second)
                        for (int a : {pm[x].src_a, pm[x].src_b}) {
                            if (a < 0 || seen.count(a)) continue;
                            const long long amt = std::get<2>(aligns[a]);
                            for (long long w = top; w >= 1; w /= b)
                                if ((amt / w) % b)
                                    add.emplace_back(std::get<0>(aligns[a]), std::get<1>(aligns[a]), w,
                                                     amt - amt % w);
                        }
                    size_t extra = 0;
                    for (auto &t : add) extra += nodes.count(t) ? 0 : 1;
                    if (g > gi && (g - gi >= (size_t)Bm || nodes.size() + extra > limit_cts)) {
                        ends.push_back(g);
                        gi = g;
                        nodes.clear();
                        seen.clear();
                    }
                    for (auto &t : add) nodes.insert(t);
                    for (int x : gl[g]->second)
                        for (int a : {pm[x].src_a, pm[x].src_b})
                            if (a >= 0) seen.insert(a);
                }
                ends.push_back(gl.size());
            }
            for (size_t bi = 0, gi = 0; bi < ends.size(); gi = ends[bi++]) {
                const size_t ge = ends[bi];
                const int k = (int)(ge - gi);
                // streaming: this batch's alignment rotations, freed at its end
                Scratch batch_mem(ctx);
                if (streaming) {
                    std::map<std::pair<int, int>, std::vector<int>> need;
                    std::set<int> seen;
                    for (size_t g = gi; g < ge; ++g)
                        for (int x : gl[g]->second)
                            for (int a : {pm[x].src_a, pm[x].src_b})
                                if (a >= 0 && seen.insert(a).second)
                                    need[{std::get<0>(aligns[a]), std::get<1>(aligns[a])}].push_back(a);
                    compute_aligns(need, batch_mem);
                }
                u64 *G = rt.workspace(WS_GRP_SUM, (size_t)k * t3L);
                u64 *R1 = rt.workspace(WS_LEVEL1, (size_t)k * t31);
                u64 *R2 = rt.workspace(WS_LEVEL2, (size_t)k * cs1);
                u64 *T = rt.workspace(WS_RS_TMP, (size_t)k * t3L);
                u64 *X = rt.workspace(WS_RELIN_OUT, (size_t)k * cs2);
                // tensor products and masks of the batch's matches, at most
                // max_matches at a time, summed into their groups
                std::vector<std::pair<int, int>> flat;   // (group in batch, match)
                for (int g = 0; g < k; ++g)
                    for (int x : gl[gi + g]->second) flat.push_back({g, x});
                std::vector<char> started(k, 0);
                for (size_t f0 = 0; f0 < flat.size(); f0 += max_matches) {
                    const size_t f1 = std::min(flat.size(), f0 + max_matches);
                    const int m = (int)(f1 - f0);
                    u64 *D = rt.workspace(WS_TENSOR, (size_t)m * t3L);
                    std::vector<const u64 *> pa, pb, mk;
                    std::vector<int> gal;
                    for (size_t f = f0; f < f1; ++f) {
                        const PlanMatch &x = pm[flat[f].second];
                        pa.push_back(operand(x.src_a, true));
                        pb.push_back(operand(x.src_b, false));
                        mk.push_back(mask);
                        // the mask for slot p is sigma_h of the slot-0 mask, h = 5^-p
                        gal.push_back(galois_element(ctx, -x.slot));
                    }
                    tensor(ctx, m, ell, rt.upload_vec(pa), rt.upload_vec(pb), D);
                    mul_plain_perm(ctx, m, ell, D, t3L, rt.upload_vec(mk), rt.upload_vec(gal), 3);
                    std::vector<u64 *> tgt;
                    std::vector<std::vector<const u64 *>> srcs;
                    std::vector<char> fresh;
                    for (size_t f = f0; f < f1;) {
                        const int g = flat[f].first;
                        size_t e = f;
                        while (e < f1 && flat[e].first == g) ++e;
                        tgt.push_back(G + (long long)g * t3L);
                        srcs.emplace_back();
                        for (size_t q = f; q < e; ++q) srcs.back().push_back(D + (long long)(q - f0) * t3L);
                        fresh.push_back(started[g] ? 0 : 1);
                        started[g] = 1;
                        f = e;
                    }
                    sum_into(ctx, 3, ell, tgt, srcs, fresh);
                }
                // rescale of the three polynomials, relinearisation at level
                // ell-1 (key switch of the s^2 part, added to the first two),
                // rescale of the ciphertext
                std::vector<const u64 *> g0(k), d2(k), base(k), x1(k), x2(k);
                std::vector<Key> key(k);
                for (int g = 0; g < k; ++g) {
                    g0[g] = G + (long long)g * t3L;
                    base[g] = R1 + (long long)g * t31;
                    d2[g] = base[g] + 2LL * (ell - 1) * n;
                    x1[g] = R2 + (long long)g * cs1;
                    x2[g] = X + (long long)g * cs2;
                    key[g] = gl[gi + g]->first;
                }
                rescale(ctx, k, ell, rt.upload_vec(g0), T, R1, t31, 3);
                std::vector<KeyGroup> kg;
                for (int g = 0; g < k; g += kRelinShare)
                    kg.push_back(KeyGroup{keys.relin, g, std::min(kRelinShare, k - g)});
                if (relin_rescale_supported(ctx, ell - 1)) {
                    relin_rescale_batch(ctx, k, ell - 1, rt.upload_vec(d2), kg, rt.upload_vec(base), T, X, cs2);
                } else {
                    keyswitch_batch(ctx, k, ell - 1, rt.upload_vec(d2), kg, rt.upload_vec(base), nullptr, true, R2,
                                    cs1);
                    rescale(ctx, k, ell - 1, rt.upload_vec(x1), T, X, cs2, 2);
                }
                st_relin += k;
                st_rescales += 2ull * k;
                tree.push(key, x2, ge < gl.size() ? gl[ge]->first : Key{INT_MAX, 0});
            }
            tree.finish();
            st_final = tree.ks;
        }
        ctx_sync(ctx);
    } catch (...) {
        free_results(ctx, res);
        throw;
    }
    for (size_t c = 0; c < nC; ++c) C[c] = res[c];
    fill_stats(out_stats, ms.size(), st_relin, st_align, st_final, st_rescales, ctx.launches - launches0);
}

void spmspm_ct_pt_grouped(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                          const spfhe_sparse_meta &B, const double *Bvals, Pt *const *Bpts, bool merge, Ct **C,
                          size_t nC, spfhe_stats *out_stats)
{
    const uint64_t launches0 = ctx.launches;
    Runtime &rt = *ctx.rt;
    validate_pair(A, B);
    const int S = ctx.S, L = ctx.L;
    const size_t n = ctx.n;
    if (L < 2) throw Error(SPFHE_ELEVEL, "ct x pt needs L >= 2");
    if (nA != chunks_for(A.nnz, S)) throw Error(SPFHE_EINVAL, "operand chunk count != ceil(nnz / S)");
    if (nC != chunks_for((long long)A.rows * B.cols, S))
        throw Error(SPFHE_EINVAL, "result chunk count != ceil(rows*cols / S)");
    if (!Bvals && !Bpts && B.nnz > 0) throw Error(SPFHE_EINVAL, "B values missing");
    for (size_t c = 0; c < nA; ++c)
        if (!Ach[c] || !Ach[c]->d || Ach[c]->level != L) throw Error(SPFHE_ELEVEL, "A chunks must be at level L");
    const double sa0 = Ach[0]->scale;
    for (size_t c = 0; c < nA; ++c)
        if (std::fabs(Ach[c]->scale - sa0) > 1e-9 * sa0) throw Error(SPFHE_ESCALE, "A chunk scales differ");
    for (size_t c = 0; c < nC; ++c) C[c] = nullptr;
    const double wscale = (double)ctx.mods[L - 1];
    const double rscale = sa0 * wscale / (double)ctx.mods[L - 1];
    const long long csL = 2LL * L * n, cs1 = 2LL * (L - 1) * n, plimb = (long long)L * n;

    const std::vector<MatchRec> ms = plan_alg1(A, B);
    // groups -> sub-groups per A chunk -> matches, all in key order
    std::map<Key, std::map<int, std::vector<int>>> groups;
    for (size_t x = 0; x < ms.size(); ++x) {
        const MatchRec &mt = ms[x];
        const int ca = mt.a_pos / S, sa = mt.a_pos % S;
        const long long t = (long long)mt.i * B.cols + mt.j;
        groups[{(int)(t / S), ((sa - t % S) % S + S) % S}][ca].push_back((int)x);
    }
    for (auto &kv : groups) DigitTree::check_keys(ctx, keys, kv.first.second, merge);
    if (Bpts)
        for (auto &mt : ms)
            if (!Bpts[mt.b_pos] || Bpts[mt.b_pos]->level != L)
                throw Error(SPFHE_ELEVEL, "B plaintexts must be at level L");

    uint64_t st_rescales = 0, st_final = 0;
    std::vector<Ct *> res(nC, nullptr);
    std::vector<int> mi(L);
    for (int i = 0; i < L; ++i) mi[i] = i;
    try {
        for (size_t c = 0; c < nC; ++c) {
            res[c] = ct_new(ctx, L - 1, rscale);
            SPFHE_CHECK_CUDA(cudaMemsetAsync(res[c]->d, 0, (size_t)cs1 * sizeof(u64), ctx.stream));
        }
        if (!ms.empty()) {
            const int Bm = match_batch_size(ctx);
            const size_t max_matches = (size_t)2 * Bm;
            DigitTree tree(ctx, keys, L - 1, merge, res);
            std::vector<const std::pair<const Key, std::map<int, std::vector<int>>> *> gl;
            for (auto &kv : groups) gl.push_back(&kv);
            for (size_t gi = 0; gi < gl.size(); gi += Bm) {
                const size_t ge = std::min(gl.size(), gi + Bm);
                const int k = (int)(ge - gi);
                // sub-groups of the batch
                std::vector<std::pair<int, int>> subs;   // (group in batch, A chunk)
                std::vector<std::pair<int, int>> flat;   // (sub-group, match)
                for (int g = 0; g < k; ++g)
                    for (auto &sg : gl[gi + g]->second) {
                        for (int x : sg.second) flat.push_back({(int)subs.size(), x});
                        subs.push_back({g, sg.first});
                    }
                const int nsub = (int)subs.size();
                u64 *PS = rt.workspace(WS_PTS, (size_t)nsub * plimb);        // summed weight plaintexts
                u64 *X = rt.workspace(WS_GRP_SUM, (size_t)nsub * csL);       // chunk x plaintext products
                u64 *G = rt.workspace(WS_RELIN_OUT, (size_t)k * csL);        // group sums
                u64 *Y = rt.workspace(WS_LEVEL1, (size_t)k * cs1);           // rescaled
                u64 *T = rt.workspace(WS_RS_TMP, (size_t)k * 2 * L * n);
                std::vector<char> started(nsub, 0);
                if (!Bpts) {
                    // the library's own weights: each sub-group's plaintext is
                    // encoded at once as its sum of permuted one-hot encodings
                    std::vector<int> seg{0}, ginv;
                    std::vector<double> vals;
                    for (size_t f = 0; f < flat.size(); ++f) {
                        const MatchRec &mt = ms[flat[f].second];
                        vals.push_back(Bvals[mt.b_pos]);
                        ginv.push_back(galois_element(ctx, mt.a_pos % S));
                        if (f + 1 == flat.size() || flat[f + 1].first != flat[f].first) seg.push_back((int)vals.size());
                    }
                    encode_onehot_sums(ctx, nsub, rt.upload_vec(seg), rt.upload_vec(vals), rt.upload_vec(ginv), L,
                                       wscale, PS);
                    to_montgomery(ctx, PS, L, mi.data(), nsub);
                }
                for (size_t f0 = 0; Bpts && f0 < flat.size(); f0 += max_matches) {
                    const size_t f1 = std::min(flat.size(), f0 + max_matches);
                    const int m = (int)(f1 - f0);
                    // weight plaintexts at slot 0 (Montgomery form), permuted to the match's slot
                    u64 *W0 = rt.workspace(WS_MASK, (size_t)m * plimb);
                    u64 *W = rt.workspace(WS_TENSOR, (size_t)m * plimb);
                    for (size_t f = f0; f < f1; ++f)
                        copy_words(ctx, W0 + (long long)(f - f0) * plimb, Bpts[ms[flat[f].second].b_pos]->d,
                                   (size_t)plimb);
                    to_montgomery(ctx, W0, L, mi.data(), m);
                    std::vector<const u64 *> win(m);
                    std::vector<int> gal(m);
                    for (size_t f = f0; f < f1; ++f) {
                        win[f - f0] = W0 + (long long)(f - f0) * plimb;
                        // B[k, j] e_p is sigma_h of B[k, j] e_0, h = 5^-p
                        gal[f - f0] = galois_element(ctx, -(ms[flat[f].second].a_pos % S));
                    }
                    automorph(ctx, m, 1, L, rt.upload_vec(win), 0, W, plimb, rt.upload_vec(gal));
                    std::vector<u64 *> tgt;
                    std::vector<std::vector<const u64 *>> srcs;
                    std::vector<char> fresh;
                    for (size_t f = f0; f < f1;) {
                        const int sgi = flat[f].first;
                        size_t e = f;
                        while (e < f1 && flat[e].first == sgi) ++e;
                        tgt.push_back(PS + (long long)sgi * plimb);
                        srcs.emplace_back();
                        for (size_t q = f; q < e; ++q) srcs.back().push_back(W + (long long)(q - f0) * plimb);
                        fresh.push_back(started[sgi] ? 0 : 1);
                        started[sgi] = 1;
                        f = e;
                    }
                    sum_into(ctx, 1, L, tgt, srcs, fresh);
                }
                // chunk x summed plaintext, then the sum over a group's chunks
                std::vector<const u64 *> ach(nsub), pts(nsub);
                std::vector<int> ident(nsub, 1);
                for (int i = 0; i < nsub; ++i) {
                    ach[i] = Ach[subs[i].second]->d;
                    pts[i] = PS + (long long)i * plimb;
                }
                gather_items(ctx, nsub, (size_t)csL, rt.upload_vec(ach), X, csL);
                mul_plain_perm(ctx, nsub, L, X, csL, rt.upload_vec(pts), rt.upload_vec(ident), 2);
                std::vector<u64 *> gt(k);
                std::vector<std::vector<const u64 *>> gs(k);
                for (int g = 0; g < k; ++g) gt[g] = G + (long long)g * csL;
                for (int i = 0; i < nsub; ++i) gs[subs[i].first].push_back(X + (long long)i * csL);
                sum_into(ctx, 2, L, gt, gs, std::vector<char>(k, 1));
                std::vector<const u64 *> gp(k), yp(k);
                std::vector<Key> key(k);
                for (int g = 0; g < k; ++g) {
                    gp[g] = G + (long long)g * csL;
                    yp[g] = Y + (long long)g * cs1;
                    key[g] = gl[gi + g]->first;
                }
                rescale(ctx, k, L, rt.upload_vec(gp), T, Y, cs1, 2);
                st_rescales += k;
                tree.push(key, yp, ge < gl.size() ? gl[ge]->first : Key{INT_MAX, 0});
            }
            tree.finish();
            st_final = tree.ks;
        }
        ctx_sync(ctx);
    } catch (...) {
        free_results(ctx, res);
        throw;
    }
    for (size_t c = 0; c < nC; ++c) C[c] = res[c];
    fill_stats(out_stats, ms.size(), 0, 0, st_final, st_rescales, ctx.launches - launches0);
}

}  // namespace spfhe
