// Task engine for encrypted sparse products (Alg. 1 + Alg. 2), shared by the
// single-product call, the many-product batch call and the serving loop.
//
// Each product ("job") is planned on the host into
//   - alignment tasks: one per distinct (operand, chunk, rotation amount);
//   - match tasks: one per Alg. 1 match, naming its two sources (a plain
//     operand chunk or an alignment task's output), its mask slot, final
//     rotation amount and result chunk.
// Work runs in waves per ciphertext level: up to G alignment tasks (from any
// job at that level) are rotated as one batch, then every match that depends
// on them (plus rotation-free matches) runs Alg. 2 in batches of Bm matches
// that may mix jobs.  Products of different jobs only meet in launches, never
// in arithmetic, and modular accumulation is order-free, so every job's result
// is bit-identical whether it runs alone or mixed with others.
#pragma once
#include <deque>
#include <map>
#include <memory>

#include "runtime.h"

namespace spfhe {

struct Job {
    const Keys *keys = nullptr;
    // metadata copies (the job may outlive the caller's arrays)
    std::vector<int32_t> aip, aix, bip, bix;
    spfhe_sparse_meta A{}, B{};
    std::vector<Ct *> Ach, Bch;
    const Pt *mask0 = nullptr;       // caller's slot-0 mask (nullptr: the library's own)
    u64 *own_mask = nullptr;         // Montgomery-form copy of mask0 (owned)
    const u64 *mask = nullptr;       // Montgomery-form mask used by the kernels
    int ell = 0;                     // operand level
    double rscale = 0;
    std::vector<Ct *> C;             // result chunks (allocated by the engine)
    size_t n_c = 0;
    uint64_t tasks_left = 0;
    uint64_t id = 0;
    uint64_t st_matches = 0, st_relin = 0, st_align = 0, st_final = 0, st_rescales = 0, st_launches = 0;
    cudaEvent_t done_ev = nullptr;
    bool finished = false;
    // element-wise baselines (Sec. 4): -1 = Alg. 1 over CSR x CSC packing;
    // otherwise SPFHE_NAIVE_* over row-major dense packing, with the zero
    // patterns (plaintext structure) of A (rows x inner) and B (inner x cols)
    int naive = -1;
    int rows = 0, inner = 0, cols = 0;
    std::vector<uint8_t> a_nz, b_nz;
    // host-side fault injection (tests of the serving loop's error
    // isolation): any wave that would run this job's tasks throws SPFHE_ECUDA
    // before launching anything
    bool inject_fault = false;
};

class Engine {
  public:
    explicit Engine(Ctx &ctx);
    ~Engine();
    // validate and plan a job; result chunks are allocated and zeroed here
    void add(Job *job);
    // run one wave of the level whose oldest pending job is oldest; false if idle
    bool step();
    void run_all()
    {
        while (step()) {
        }
    }
    bool idle() const;
    // jobs whose last task was enqueued (their done event is recorded)
    std::vector<Job *> take_finished();

  private:
    struct RotTask {
        Job *job;
        int op, chunk, amount;
        std::vector<int> deps;   // match task ids
        int partner = -1;        // the other operand's rotation of the same product (element-wise baselines)
    };
    struct MatchTask {
        Job *job;
        int src_a, src_b;        // >= 0 rotated-task id, < 0: -(chunk + 1)
        int min_slot, rf, rc;
    };
    struct LevelQueue {
        std::deque<int> rots;        // pending alignment tasks
        std::deque<int> free_matches;  // pending matches needing no alignment
    };
    Ctx &ctx_;
    std::vector<RotTask> rots_;
    std::vector<MatchTask> matches_;
    std::map<int, LevelQueue> levels_;
    std::deque<Job *> order_;        // jobs in arrival order (for level choice)
    std::vector<Job *> finished_;
    uint64_t next_id_ = 1;

    void run_wave(int ell, LevelQueue &q);
    void run_matches(int ell, const std::vector<int> &ids, const u64 *align, int r0,
                     const std::map<int, int> &slot_of);
    void task_done(Job *job, uint64_t count);
    const u64 *level_mask(int ell);
};

int match_batch_size(const Ctx &ctx);
// matches of one batch that share a relinearisation key read in the inner
// product (one CTA loads the key values once and serves them all; a whole
// default batch: measured 1 474 against 1 500 ms of inner products per
// 128x128 step with 8)
constexpr int kRelinShare = 64;
// fill a job from a single-product call (metadata is copied)
void fill_job(Job &job, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
              const spfhe_sparse_meta &B, Ct *const *Bch, size_t nB, const Pt *mask0, size_t nC);
// element-wise baselines (Sec. 4) through the engine (spmspm.cpp)
void naive_ct_ct(Ctx &ctx, const Keys &keys, int mode, int rows, int inner, int cols, const uint8_t *a_nz,
                 const uint8_t *b_nz, Ct *const *Ach, size_t nA, Ct *const *Bch, size_t nB, const Pt *mask0, Ct **C,
                 size_t nC, spfhe_stats *out_stats);
// free a job's private mask copy (and its results when free_results)
void release_job(Ctx &ctx, Job &job, bool free_results);
// after release_job(.., true): clear what Engine::add and the waves filled
// in, so the job can be added to an engine again
void reset_job(Job &job);
// Device memory an engine's waves at operand level ell may hold in the
// context's workspace cache (every batch buffer at its largest), bytes.
uint64_t engine_workspace_bound(const Ctx &ctx, int ell);
// Device memory Engine::add allocates for a job beyond its result chunks: the
// Montgomery copy of a caller's mask, or the library's own level mask when
// the context has none yet (bytes).
uint64_t job_mask_bytes(const Ctx &ctx, const Job &job);
size_t chunks_for(long long count, int S);
// checks shared by the ct x ct products (metadata, chunk counts, levels,
// scales); returns the operands' level and their product's result scale
int check_ct_ct(const Ctx &ctx, const spfhe_sparse_meta &A, const std::vector<Ct *> &Ach,
                const spfhe_sparse_meta &B, const std::vector<Ct *> &Bch, size_t n_c, double *rscale);
// lazy-accumulation variants of the products (grouped.cpp)
void spmspm_ct_ct_grouped(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                          const spfhe_sparse_meta &B, Ct *const *Bch, size_t nB, const Pt *mask0, bool merge_digits,
                          Ct **C, size_t nC, spfhe_stats *out_stats);
void spmspm_ct_pt_grouped(Ctx &ctx, const Keys &keys, const spfhe_sparse_meta &A, Ct *const *Ach, size_t nA,
                          const spfhe_sparse_meta &B, const double *Bvals, Pt *const *Bpts, bool merge_digits,
                          Ct **C, size_t nC, spfhe_stats *out_stats);
size_t result_chunks(const Ctx &ctx, const spfhe_matmul_req &r);
// many ct x ct products through one task engine (serve.cpp); C receives
// every request's chunks, request after request
void sparse_matmul_batch(Ctx &ctx, size_t n_req, const spfhe_matmul_req *reqs, Ct **C, size_t n_c_total,
                         spfhe_stats *stats);

}  // namespace spfhe
