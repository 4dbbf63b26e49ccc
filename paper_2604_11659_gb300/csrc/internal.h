// Internal host-side structures of libspfhe (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/spfhe.h"
#include "modarith.cuh"

namespace spfhe {

constexpr int kMaxMods = 96;      // L + K
constexpr int kMaxLimbSlots = 256; // limb slots one batched launch can address

// Error carrying an ABI status; converted at the boundary.
struct Error : std::runtime_error {
    spfhe_status code;
    Error(spfhe_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define SPFHE_CHECK_CUDA(expr)                                                             \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::spfhe::Error(SPFHE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Which limbs of a batch of items one launch touches: limb slot s addresses
// the n residues at item_base + off[s] * n, modulus index mi[s].
struct LimbMap {
    int nl;
    int off[kMaxLimbSlots];
    int mi[kMaxLimbSlots];
};

// Device-resident tables of one parameter set.
struct DevTables {
    ModConst *mc = nullptr;          // [M]
    u64 *tw = nullptr, *twp = nullptr;     // [M][n]  psi^brv(k) and Shoup companions
    u64 *itw = nullptr, *itwp = nullptr;   // [M][n]  psi^-brv(k)
    ulonglong2 *tw2 = nullptr, *itw2 = nullptr;   // [M][n] (twiddle, Shoup companion) pairs
    // ModUp basis conversion, one table per digit source set (indexed by the
    // digit's last limb + 1 = hi, 1..L): for source limb i of the digit
    // hat_inv[(hi-1)*alpha + i] (Shoup pair) and for every target modulus t
    // hat_split[((hi-1)*alpha + i) * M + t] = (D/q_i mod m_t) * 2^64 mod m_t,
    // split into 30-bit halves (low half in the low word).
    u64 *mu_hat_inv = nullptr, *mu_hat_inv_p = nullptr, *mu_hat_split = nullptr;
    // the same hat_inv times n^{-1} mod q_i (Shoup pairs): the conversion's
    // inputs come from inverse transforms that leave out the n^{-1}
    u64 *mu_hat_inv_n = nullptr, *mu_hat_inv_n_p = nullptr;
    // -D mod m_t in Montgomery form, split, with D = prod_{i in [lo, hi)} q_i: [(hi-1) * M + t]
    u64 *mu_negd_split = nullptr;
    double *inv_q = nullptr;                       // [M] 1 / m (correctly rounded double)
    // ModDown P -> Q: hat_inv over p_k, hat_split[k * M + i] (as above), and
    // P^{-1} mod q_i.
    u64 *md_hat_inv = nullptr, *md_hat_inv_p = nullptr, *md_hat_split = nullptr;
    u64 *md_hat_inv_n = nullptr, *md_hat_inv_n_p = nullptr;   // times n^{-1} mod p_k
    u64 *md_pinv = nullptr, *md_pinv_p = nullptr;   // [L]
    u64 *md_negp_split = nullptr;                   // [L] -P mod q_i in Montgomery form, split
    // Rescale dropping q_t: rs_inv[t * L + i] = q_t^{-1} mod q_i (Shoup pair),
    // rs_qt[t * L + i] = q_t mod q_i.
    u64 *rs_inv = nullptr, *rs_inv_p = nullptr, *rs_qt = nullptr;
};

// Kernel classes for launch accounting and the profiler.
enum KClass {
    K_NTT_FWD = 0, K_NTT_INV, K_MODUP, K_IP, K_MODDOWN_BCONV, K_MODDOWN_FINAL, K_TENSOR, K_RESCALE,
    K_AUTOMORPH, K_MASK, K_ACCUM, K_OTHER, K_KS_NTT_FWD, K_KS_NTT_INV, K_NCLASS
};

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> recs;
    uint64_t launches[K_NCLASS] = {};
    uint64_t timed[K_NCLASS] = {};
    double bytes[K_NCLASS] = {}, work[K_NCLASS] = {}, ms[K_NCLASS] = {};
    // transform classes: limbs by pass kind (0 = first pass, 1 = second
    // pass, 2 = second pass with a fused epilogue)
    double limbs[K_NCLASS][3] = {};
    // key switching as a whole: calls and algorithmic bytes (input poly,
    // output pair, and each key stream once per item group sharing it)
    uint64_t ks_calls = 0;
    double ks_bytes = 0;
};

struct Ctx {
    int log_n = 0, n = 0, L = 0, K = 0, M = 0, dnum = 0, alpha = 0, S = 0;
    double scale = 0;
    int rot_base = 2;
    std::vector<u64> mods, psis;
    std::vector<ModConst> mc;
    cudaStream_t stream = nullptr;
    int device = 0;
    DevTables dt;
    // the library's own one-hot slot-0 masks (Montgomery form) per operand
    // level ell: [ell-1][n] at scale q_{ell-2}, built on first use
    std::map<int, u64 *> masks;
    uint64_t launches = 0;
    struct Runtime *rt = nullptr;    // workspace cache + metadata ring
    double *cos_tab = nullptr;       // cos(pi j / n), j < n (device), for one-hot encodings
    Prof prof;
    int in_keyswitch = 0;            // NTT launches inside key switching are classed separately
    int match_batch = 0;             // matches per batch (0: default for the ring size)
    int ntt_chunk = 0;               // limbs per pass-A/pass-B launch pair (0: whole batch)
    int ntt_pa = 0;                  // stages in NTT pass A for n >= 2^12 (0: log_n / 2)
    int ntt_variant = 6;             // radix-16 kernel variant (0 to 6)
    bool fuse_epilogues = true;      // ModDown / rescale epilogues inside the forward transform
    // device memory the grouped ct x ct product may hold in alignment
    // rotations for the whole call; above it they are streamed per batch
    size_t align_budget = SIZE_MAX;
    // while a CUDA graph is being captured: its own buffers (graph.cpp)
    struct Capture *cap = nullptr;
};

// Resources of a graph under capture: every device buffer allocated while
// capturing (freed with the graph, never earlier: the graph's nodes use them
// at every launch), the workspaces of the capture, and an append-only
// pinned/device pair for the metadata uploads (the captured copies read the
// pinned bytes at every launch).
struct Capture {
    std::vector<void *> device;      // allocated while capturing (cudaMalloc)
    std::vector<void *> deferred;    // pool buffers released while capturing
    std::vector<void *> host;
    std::vector<u64 *> ws;           // workspace slot -> buffer
    std::vector<size_t> ws_words;
    char *up_host = nullptr, *up_dev = nullptr;
    size_t up_off = 0, up_cap = 0;
};

// host-side wait for the context stream; a no-op while a graph is captured
void ctx_sync(Ctx &ctx);

struct Keys {
    Ctx *ctx = nullptr;
    u64 *s = nullptr;                // secret, evaluation rep. over all M moduli, Montgomery form
    u64 *relin = nullptr;            // [dnum][2][M][n], Montgomery form
    std::map<int, u64 *> rot;        // amount -> [dnum][2][M][n], Montgomery form
    std::vector<long long> s_coef;   // host copy of the ternary secret (coefficients), for export
    size_t key_words() const;
};

struct Ct {
    Ctx *ctx = nullptr;
    int level = 0;
    double scale = 0;
    u64 *d = nullptr;                // [2][level][n] evaluation representation
};

struct Pt {
    Ctx *ctx = nullptr;
    int level = 0;
    double scale = 0;
    u64 *d = nullptr;                // [level][n]
};

// ---- host helpers (params.cpp) ----
u64 mulmod_host(u64 a, u64 b, u64 q);
u64 powmod_host(u64 a, u64 e, u64 q);
u64 invmod_host(u64 a, u64 q);
u64 shoup_pre(u64 w, u64 q);
void build_params(Ctx &ctx, const spfhe_params &p);
void upload_tables(Ctx &ctx);
void free_tables(Ctx &ctx);

// message returned by spfhe_last_error() for the calling thread (abi.cpp)
void set_last_error(const std::string &m);

// ---- memory (memory.cpp) ----
void *dev_alloc(Ctx &ctx, size_t bytes);
void dev_free(Ctx &ctx, void *p);

// Scratch buffers that live for one call (freed stream-ordered on destruction).
struct Scratch {
    Ctx &ctx;
    std::vector<void *> ptrs;
    explicit Scratch(Ctx &c) : ctx(c) {}
    u64 *words(size_t n) {
        void *p = dev_alloc(ctx, n * sizeof(u64));
        ptrs.push_back(p);
        return static_cast<u64 *>(p);
    }
    template <typename T> T *typed(size_t n) {
        void *p = dev_alloc(ctx, n * sizeof(T));
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~Scratch() {
        for (void *p : ptrs) dev_free(ctx, p);
    }
};

}  // namespace spfhe
