// common.cuh — internal definitions shared by the library's translation units.
//
// The feature space of §2.1 (Eq. 2) is never materialised.  It is described by a small
// plan: per level, one section per enabled operator with its first id and size, and for
// binary sections the pair rule.  Ids map to (operator, operand pair) by closed-form
// unranking (triangle rows by a square root and an integer fix-up), so any thread can
// decode any id in O(1) and rebuild the feature as a postfix program over the primaries.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/sisso.h"

namespace sg {

constexpr int kMaxRung = SISSO_MAX_RUNG;
constexpr int kNumOps = 12;
constexpr int kMaxSec = kMaxRung * kNumOps;
constexpr int kMaxDim = SISSO_MAX_DIM;
constexpr int kProgLen = 16;   // postfix nodes of a rung-3 tree: at most 15
constexpr double kValueCap = 1e12;     // |v| above this makes a feature invalid
constexpr double kConstRel = 1e-6;     // std <= 1e-6 max|v|: near-constant, invalid
constexpr double kScoreTie = 1e-9;     // |rho| within this of the current maximum: tie
constexpr double kDupTol = 1e-8;       // standardised vectors this close: duplicates
constexpr double kPivotMin = 1e-12;    // FP64 Cholesky pivot: singular at or below
constexpr float kPivotMin32 = 1e-5f;   // FP32 pivot at or below: refit in FP64
constexpr double kRssTie = 1e-12;      // RSS within this * SST of the minimum: tie
constexpr double kStopRel = 1e-10;     // RMSE <= this * std(y): exact fit, stop
constexpr double kScoreErr32 = 2e-4;   // bound on |FP32 kernel score - FP64 score|
constexpr double kScoreErr64 = 1e-6;   // ... FP64 kernel (FP32 score buffer)

enum Op : int { ADD = 0, SUB, MUL, DIV, EXP, LOG, SQRT, SQ, INV, SIN, CUBE, EXPNEG };
// kinds of sections: unary on new_{l-1}; symmetric or ordered pairs under either rule
enum Kind : int { K_UNARY = 0, K_SYM_EQ2, K_DIV_EQ2, K_SYM_NXP, K_DIV_NXP };

struct Section {
    int64_t base, count;   // first id, number of ids
    int64_t P, Q;          // |phi_{l-1}|, |phi_{l-2}| (Q = 0 at level 1)
    int level, op, kind, pad;
};

struct Space {
    int d, rung, grammar, nsec;
    int64_t phi[kMaxRung + 1];   // cumulative sizes |phi_l|
    Section sec[kMaxSec];
};

// Largest u with u*m - u(u-1)/2 <= r: the row of rank r in a triangle whose rows have
// m, m-1, ..., 1 entries.
__host__ __device__ inline int64_t tri_row(int64_t r, int64_t m) {
    double b = 2.0 * (double)m + 1.0;
    double disc = b * b - 8.0 * (double)r;
    int64_t u = (int64_t)((b - sqrt(disc > 0 ? disc : 0.0)) * 0.5);
    if (u < 0) u = 0;
    auto S = [m](int64_t x) { return x * m - x * (x - 1) / 2; };
    while (u > 0 && S(u) > r) --u;
    while (S(u + 1) <= r) ++u;
    return u;
}

__host__ __device__ inline int64_t tri_start(int64_t u, int64_t m) { return u * m - u * (u - 1) / 2; }

// rank within a section -> operand pair (binary) or operand (unary, b = -1)
__host__ __device__ inline void unrank(const Section& s, int64_t r, int64_t& a, int64_t& b) {
    const int64_t P = s.P, Q = s.Q;
    switch (s.kind) {
        case K_UNARY: a = Q + r; b = -1; return;
        case K_SYM_EQ2: {
            const int64_t A = Q > 0 ? Q - 1 : 0, L0 = P - Q;
            if (r < A * L0) { a = r / L0; b = Q + r % L0; return; }
            r -= A * L0;
            const int64_t m = P - 1 - A;
            const int64_t u = tri_row(r, m);
            a = A + u;
            b = a + 1 + (r - tri_start(u, m));
            return;
        }
        case K_DIV_EQ2: {
            const int64_t B1 = Q * (P - Q);
            if (r < B1) { a = r / (P - Q); b = Q + r % (P - Q); return; }
            r -= B1;
            a = Q + r / (P - 1);
            const int64_t jj = r % (P - 1);
            b = jj < a ? jj : jj + 1;
            return;
        }
        case K_SYM_NXP: a = r / (P - Q); b = Q + r % (P - Q); return;
        default: {  // K_DIV_NXP
            const int64_t B1 = Q * (P - Q);
            if (r < B1) { a = r / (P - Q); b = Q + r % (P - Q); return; }
            r -= B1;
            a = Q + r / Q;
            b = r % Q;
            return;
        }
    }
}

// operand pair -> rank within a binary section (inverse of unrank)
__host__ __device__ inline int64_t rank_of(const Section& s, int64_t i, int64_t j) {
    const int64_t P = s.P, Q = s.Q;
    switch (s.kind) {
        case K_SYM_EQ2: {
            const int64_t A = Q > 0 ? Q - 1 : 0, L0 = P - Q;
            if (i < A) return i * L0 + (j - Q);
            const int64_t m = P - 1 - A;
            return A * L0 + tri_start(i - A, m) + (j - i - 1);
        }
        case K_DIV_EQ2:
            if (i < Q) return i * (P - Q) + (j - Q);
            return Q * (P - Q) + (i - Q) * (P - 1) + (j < i ? j : j - 1);
        case K_SYM_NXP: return i * (P - Q) + (j - Q);
        case K_DIV_NXP:
            if (i < Q) return i * (P - Q) + (j - Q);
            return Q * (P - Q) + (i - Q) * Q + j;
        default: return -1;
    }
}

// id -> (level, op, a, b); op = -1 for a primary.  Returns false for an id out of range.
__host__ __device__ inline bool decode(const Space& sp, int64_t id, int& level, int& op,
                                       int64_t& a, int64_t& b) {
    if (id < 0 || id >= sp.phi[sp.rung]) return false;
    if (id < sp.d) { level = 0; op = -1; a = id; b = -1; return true; }
    for (int k = 0; k < sp.nsec; ++k) {
        const Section& s = sp.sec[k];
        if (id >= s.base && id < s.base + s.count) {
            level = s.level; op = s.op;
            unrank(s, id - s.base, a, b);
            return true;
        }
    }
    return false;
}

// A feature as a postfix program over the primaries: code >= 0 pushes column `code`,
// code < 0 applies operator (-code - 1).
struct Prog {
    int n;
    int16_t code[kProgLen];
};

// Postfix program of feature id: children first (a, then b), then the operator.
// Iterative depth-first walk with an explicit stack (a rung-3 tree has at most 7
// pending entries); no recursion, so the per-thread stack stays small and static.
__host__ __device__ inline bool build_prog(const Space& sp, int64_t id, Prog& p) {
    p.n = 0;
    int64_t st_id[12];
    int st_op[12];            // >= 0: emit operator; -1: expand st_id
    int top = 0;
    st_id[top] = id; st_op[top] = -1; ++top;
    while (top > 0) {
        --top;
        if (st_op[top] >= 0) {
            if (p.n >= kProgLen) return false;
            p.code[p.n++] = (int16_t)(-st_op[top] - 1);
            continue;
        }
        int level, op; int64_t a, b;
        if (!decode(sp, st_id[top], level, op, a, b)) return false;
        if (level == 0) {
            if (p.n >= kProgLen) return false;
            p.code[p.n++] = (int16_t)a;
            continue;
        }
        if (top + 3 > 12) return false;
        st_op[top] = op; st_id[top] = 0; ++top;                    // operator after children
        if (b >= 0) { st_id[top] = b; st_op[top] = -1; ++top; }   // b after a
        st_id[top] = a; st_op[top] = -1; ++top;                    // a first
    }
    return true;
}

template <typename T> __device__ __forceinline__ T op_unary(int op, T z);
template <> __device__ __forceinline__ float op_unary<float>(int op, float z) {
    switch (op) {
        case EXP: return expf(z);
        case LOG: return logf(z);
        case SQRT: return sqrtf(z);
        case SQ: return z * z;
        case INV: return __frcp_rn(z);
        case SIN: return sinf(z);
        case CUBE: return z * z * z;
        default: return expf(-z);
    }
}
template <> __device__ __forceinline__ double op_unary<double>(int op, double z) {
    switch (op) {
        case EXP: return exp(z);
        case LOG: return log(z);
        case SQRT: return sqrt(z);
        case SQ: return z * z;
        case INV: return 1.0 / z;
        case SIN: return sin(z);
        case CUBE: return z * z * z;
        default: return exp(-z);
    }
}

template <typename T> __device__ __forceinline__ T op_binary(int op, T x, T y) {
    switch (op) {
        case ADD: return x + y;
        case SUB: return x - y;
        case MUL: return x * y;
        default: return x / y;
    }
}

// value of program p at one sample, and in mag the magnitude |a| + |b| of the root's
// operands when the root is + or - (|v| otherwise)
template <typename T, typename F>
__device__ __forceinline__ T eval_prog_mag(const Prog& p, F x, T& mag) {
    T st[kMaxRung + 2];
    int top = 0;
    mag = T(0);
    for (int k = 0; k < p.n; ++k) {
        const int c = p.code[k];
        if (c >= 0) {
            st[top++] = x(c);
        } else {
            const int op = -c - 1;
            if (op >= EXP) {
                st[top - 1] = op_unary<T>(op, st[top - 1]);
            } else {
                const T rhs = st[--top];
                if (k == p.n - 1 && (op == ADD || op == SUB)) mag = fabs(st[top - 1]) + fabs(rhs);
                st[top - 1] = op_binary<T>(op, st[top - 1], rhs);
            }
        }
    }
    return st[0];
}

__host__ __device__ inline bool root_is_addsub(const Prog& p) {
    if (p.n == 0) return false;
    const int c = p.code[p.n - 1];
    return c < 0 && (-c - 1 == ADD || -c - 1 == SUB);
}

constexpr double kCancelRel = 1e-9;    // root +/- with max|v| <= this * max(|a|+|b|): zero

// A feature written over the FP64 operand values V (feature-major rows of N samples, one
// row per id of phi_{L-1}): ids below P are rows; top-level ids are one operator on one
// or two rows.
struct OpRef {
    int64_t a, b;   // rows (b = -1: unary or direct)
    int op;         // -1: row a itself
    const double* inv = nullptr;   // optional rows of 1/x (same layout as V): a / b as a * (1/b)
};

__host__ __device__ inline bool make_opref(const Space& sp, int64_t id, OpRef& r) {
    const int64_t P = sp.phi[sp.rung - 1];
    if (id >= 0 && id < P) { r.a = id; r.b = -1; r.op = -1; return true; }
    int level, op; int64_t a, b;
    if (!decode(sp, id, level, op, a, b)) return false;
    r.a = a; r.b = b; r.op = op;
    return true;
}

// value at sample s; mag = |a| + |b| for a root + or -, |v| otherwise
__device__ __forceinline__ double opref_val(const OpRef& r, const double* __restrict__ V, int N, int s,
                                            double& mag) {
    const double x = V[(size_t)r.a * N + s];
    if (r.op < 0) { mag = fabs(x); return x; }
    if (r.b < 0) { const double v = op_unary<double>(r.op, x); mag = fabs(v); return v; }
    if (r.op == DIV && r.inv) {       // one rounding more than x / y (relative 1.1e-16); x / y where 1/y overflows
        const double q = r.inv[(size_t)r.b * N + s];
        const double v = isfinite(q) ? x * q : x / V[(size_t)r.b * N + s];
        mag = fabs(v);
        return v;
    }
    const double y = V[(size_t)r.b * N + s];
    const double v = op_binary<double>(r.op, x, y);
    mag = (r.op == ADD || r.op == SUB) ? fabs(x) + fabs(y) : fabs(v);
    return v;
}
constexpr int kProbes = 8;             // standardised values kept per candidate for dedup
constexpr int kDupSlots = 16;          // partner candidates kept per screened candidate

// value of program p at one sample; x(c) returns primary c at that sample
template <typename T, typename F>
__device__ __forceinline__ T eval_prog(const Prog& p, F x) {
    T st[kMaxRung + 2];
    int top = 0;
    for (int k = 0; k < p.n; ++k) {
        const int c = p.code[k];
        if (c >= 0) {
            st[top++] = x(c);
        } else {
            const int op = -c - 1;
            if (op >= EXP) {
                st[top - 1] = op_unary<T>(op, st[top - 1]);
            } else {
                const T rhs = st[--top];
                st[top - 1] = op_binary<T>(op, st[top - 1], rhs);
            }
        }
    }
    return st[0];
}

// ------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// moments of the current screening target, computed on the device
struct TargetStats {
    double mean, sd;        // FP64 mean and population std of the target
    double tsum;            // FP64 sum of the centred target (rounding-level, kept exact)
    double sum32, srr32;    // sum and centred sum of squares of the FP32 copy
    float sd32, pad;
};

// small result block of one SIS walk, copied back to the host
struct WalkResult {
    int n_acc;              // accepted ids
    int exhausted;          // ran out of survivors before k were accepted
    int visited;            // survivors visited
    int dup_checks;         // vector comparisons made
    double last_score;      // FP64 score of the last visited candidate
    int thr_stop;           // ended at the SIS threshold (best remaining score <= threshold)
    int64_t acc[SISSO_MAX_SIS];
};

struct Winner {
    int found, pad;
    int pos[kMaxDim];
    double rss_gram, rss, rmse, r2;
    double gamma[kMaxDim];
    double coef[kMaxDim + 1];
    int64_t ids[kMaxDim];
    unsigned long long min_key;   // ordered key of the band minimum (FP32 or FP64 RSS)
    double thr;                   // band threshold
    int64_t examined;             // subsets enumerated
};

}  // namespace sg

struct sisso_ctx {
    int N, d, rung, k, max_dim;
    uint32_t ops;
    sisso_opts opts;
    sg::Space space;
    sg::Space* space_dev = nullptr;   // the same plan in device memory (kernels read it there)
    int64_t n_feat;
    cudaStream_t stream;
    bool own_stream;
    std::string err;

    // inputs
    double* Xc64 = nullptr;    // d x N (column-major: feature c at Xc[c*N + s])
    float* Xc32 = nullptr;     // d x N
    double* y64 = nullptr;     // N
    double* yc64 = nullptr;    // y - mean(y)
    double ybar = 0, syy = 0;  // mean(y), y~^T y~ / N (computed on the device)

    // screening
    float* scores = nullptr;           // |phi| FP32 scores
    double* target64 = nullptr;        // current screening target (N)
    double* tc64 = nullptr;            // centred target FP64
    float* tc32 = nullptr;             // centred target FP32
    sg::TargetStats* tstats = nullptr;
    unsigned int* hist = nullptr;      // radix-select histograms (3 x 4096)
    unsigned int* sel_state = nullptr; // radix-select state
    int64_t surv_cap = 0;              // capacity of the survivor buffers
    int64_t* surv_ids = nullptr;
    unsigned int* surv_count = nullptr;
    double* surv_score = nullptr;      // FP64 re-score
    double* surv_mean = nullptr;
    double* surv_sd = nullptr;
    int* surv_valid = nullptr;
    double* surv_probe = nullptr;      // kProbes standardised values per entry
    double* zcache = nullptr;          // standardised FP64 vectors of the window (zcap x N)
    int64_t zcap = 0;
    unsigned char* subvalid = nullptr; // FP64 validity (recursive) of every id of phi_{L-1}
    float* opcache32 = nullptr;        // values of phi_{L-1}, sample-major (N x id), or null
    double* opcache64 = nullptr;       // ... FP64 copy (FP64 screening only)
    double* opsum = nullptr;           // per operand: sum (x - x0), sum (x - x0) r, sum (x - x0)^2 (3 x |phi_{L-1}|)
    int opsum_prec = -1;               // cache the first half was computed from (0 FP64, 1 FP32)
    std::unordered_set<const void*> pooled;  // buffers from the library's device pool (api.cu)
    double* Wm = nullptr;              // whitening matrix W (N x N), or null (§2.4)
    double* w_raw = nullptr;           // whitened path: raw rows, whitened rows (w_chunk x N each),
    double* w_u = nullptr;             //   per-row scratch (3 w_chunk), probes, raw validity
    double* w_scr = nullptr;
    double* w_probe = nullptr;
    int* w_ok = nullptr;
    int w_chunk = 0;
    unsigned long long* fix_ids = nullptr;  // FP32 pair kernel: + / - candidates left to the direct sums
    unsigned* fix_count = nullptr;
    int fix_cap = 0;
    double* opval64 = nullptr;         // FP64 values of phi_{L-1}, feature-major (id x N), or null
    int* dup_list = nullptr;           // per sorted entry: partner candidates (kDupSlots)
    unsigned char* dup_ok = nullptr;   // ... confirmed duplicates
    int* dup_cnt = nullptr;            // ... number of partner candidates (-1: overflow)
    unsigned char* accepted = nullptr; // per window entry: accepted by the walk
    int64_t sort_cap = 0;
    double* sort_score = nullptr;      // sort buffers (power of two)
    int64_t* sort_id = nullptr;
    int* sort_src = nullptr;           // index into the survivor arrays
    unsigned char* removed = nullptr;  // walk: visited flags (sort_cap)
    sg::WalkResult* walk = nullptr;    // device
    sg::WalkResult* walk_h = nullptr;  // pinned host
    int64_t* S_dev = nullptr;          // S ids (device, acceptance order)
    int64_t* S_sorted = nullptr;       // S ids ascending (device)

    // subspace
    int n_cap = 0;                     // max |S| = max_dim * k
    double* Z = nullptr;               // standardised S features, n_cap x N
    double* Zmean = nullptr;
    double* Zsd = nullptr;
    double* G64 = nullptr;             // n_cap x n_cap
    double* b64 = nullptr;
    float* G32 = nullptr;
    float* b32 = nullptr;
    double* resid = nullptr;           // residual of the best model (N)
    double* ymom = nullptr;            // [mean(y), syy, sst] on device

    // l0
    int64_t band_cap = 0;
    uint64_t* band = nullptr;          // packed positions
    double* band_rss = nullptr;
    unsigned int* band_count = nullptr;
    float* band_r32 = nullptr;         // mixed precision: FP32 RSS of each band entry
    unsigned char* band_sel = nullptr; // mixed precision: entries refit in FP64
    uint64_t* prefixes = nullptr;
    int64_t prefix_cap = 0;
    int* work = nullptr;               // work counters
    sg::Winner* win = nullptr;         // device
    sg::Winner* win_h = nullptr;       // pinned host
    unsigned long long* blk_best = nullptr;  // per-block tie-break winners
    int blk_cap = 0;
    // dimensional analysis: unit labels of the primaries, the units rule of every id of
    // phi_{L-1} (recursive, one byte each) and of every id of phi_L (one bit each)
    std::vector<int> units;
    std::vector<int> primaries;        // original indices of the primaries (pre-screening)
    unsigned char* unit_ok = nullptr;
    unsigned* unit_mask = nullptr;
    // tiled FP32 enumeration: padded FP32 Gram, moments and diagonal (rows x tile_ld), tile list
    float* tile_G = nullptr;
    float* tile_b = nullptr;
    float* tile_diag = nullptr;
    int tile_rows = 0, tile_ld = 0;
    void* tile_info = nullptr;
    int tile_info_cap = 0;

    // results
    std::vector<int64_t> S;                       // acceptance order
    std::vector<int> n_sis;                       // accepted per step
    int n_dims = 0;
    std::vector<std::vector<int64_t>> res_ids;
    std::vector<std::vector<double>> res_coef;
    std::vector<double> res_rmse, res_r2;
    bool fitted = false;
    sisso_stats stats{};
    int sms = 0;

    // learned proposal for the D = 5 step (not owned)
    sisso_mlp* proposal = nullptr;
    double prune_frac = 0.01;
    int64_t learned_prefixes = 0;
    int64_t certified_prefixes = 0;    // 3-prefixes the certificate left to enumerate
    bool certify_proposal = true;      // the learned D = 5 step is followed by its certificate

    // tensor-core screening of the top level's pairs (mixed forms): 16-bit parts of the
    // operand rows, exponents, moments, chunk partials and the FP64 products
    bool tc_on = false, tc_ready = false;
    int tc_P = 0, tc_Pp = 0, tc_Kpad = 0;
    size_t tc_part_cap = 0;
    void* tc_L = nullptr;
    void* tc_R = nullptr;
    int* tc_eL = nullptr;
    int* tc_eR = nullptr;
    double* tc_mom = nullptr;
    double* tc_tgt = nullptr;
    int* tc_mex = nullptr;
    float* tc_part = nullptr;
    double* tc_C1 = nullptr;
    double* tc_C2 = nullptr;
    double* tc_recip = nullptr;
    double* opinv64 = nullptr;         // 1/x of every FP64 operand value (division in the FP64 re-score)
    int* tc_err = nullptr;
    unsigned long long* tc_raised = nullptr;
};

namespace sg {

// host-side helpers implemented in the .cu files
bool plan_space(int d, uint32_t ops, int rung, int grammar, Space& sp);
std::string feature_expr(const Space& sp, int64_t id);
sisso_status fail(sisso_ctx* c, sisso_status st, const std::string& msg);
sisso_status check_cuda(sisso_ctx* c, cudaError_t e, const char* what);

// screening (sis.cu)
sisso_status compute_subvalid(sisso_ctx* c);
sisso_status fill_opcache(sisso_ctx* c);
sisso_status fill_val64(sisso_ctx* c);
sisso_status prepare_target(sisso_ctx* c, const double* target_dev);
sisso_status score_all(sisso_ctx* c, int precision);
void apply_unit_mask(sisso_ctx* c);
// whitened data (whiten.cu)
sisso_status whiten_setup(sisso_ctx* c, const double* W);
void whiten_free(sisso_ctx* c);
sisso_status whiten_score_all(sisso_ctx* c);
sisso_status whiten_rescore(sisso_ctx* c, const int64_t* ids, int n, double* score, double* mean, double* sd,
                            int* valid, double* probe, double* zc);
sisso_status whiten_standardise(sisso_ctx* c, const int64_t* ids, int n, double* Z, double* Zmean, double* Zsd);
sisso_status sis_select(sisso_ctx* c, int k, const int64_t* S_prev_host, int n_prev,
                        std::vector<int64_t>& acc);
sisso_status eval_features(sisso_ctx* c, const int64_t* ids_dev, int64_t n, int precision,
                           double* out_dev);
// 32 x 32 operand-pair tiles of the top level's binary sections (upper left corners)
void pair_tiles(int64_t P, int64_t Q, bool nxp, std::vector<int2>& tiles);

// subspace and l0 (l0.cu)
sisso_status append_subspace(sisso_ctx* c, int n_old, int n_new, bool gram64);
sisso_status l0_solve_mixed(sisso_ctx* c, int n, int D, Winner& w);
sisso_status ensure_tile_buffers(sisso_ctx* c, int n);
sisso_status build_units(sisso_ctx* c);
sisso_status l0_certify(sisso_ctx* c, const double* G, const double* b, int ld, double syy, int n,
                        const int64_t* gid_dev, double bound0, Winner& w, int64_t* prefixes_kept);
int prescreen_keep(const double* score, int d, double q, int* keep);
sisso_status prescreen_scores(const double* X, const double* y, int N, int d, int method, double* scores,
                              std::string& why);
sisso_status winner_model_z(sisso_ctx* c, int n, int D, Winner& w);
sisso_status l0_solve(sisso_ctx* c, const double* G, const double* b, const float* G32, const float* b32,
                      int ld, double syy, int n, int D, const int64_t* gid_dev, int precision, Winner& w,
                      const int* prefix_list = nullptr, int64_t n_prefixes = 0);
sisso_status winner_model(sisso_ctx* c, int n, int D, Winner& w);

// learned proposal (learn.cu)
sisso_status l0_learned(sisso_ctx* c, sisso_mlp* mlp, const double* G, const double* b, const float* G32,
                        const float* b32, int ld, double syy, int n, const int64_t* gid_dev, double frac, Winner& w,
                        int64_t* n_selected);

// tensor-core screening of the top level's pairs (screen_tc.cu)
bool tc_screen_possible(const sisso_ctx* c, int screen);
sisso_status tc_screen_alloc(sisso_ctx* c);
sisso_status tc_screen_pairs(sisso_ctx* c, const int sec[4]);
sisso_status tc_screen_status(sisso_ctx* c);
void tc_screen_free(sisso_ctx* c);

// tensor-core Gram (gram_tc.cu)
sisso_status gram_tc(sisso_ctx* c, const double* Z, const double* yc, double sdy, int n, int N, int kind,
                     float* G32, int ldg, float* b32);

// timing
struct PhaseTimer {
    cudaEvent_t a, b;
};
double event_ms(cudaEvent_t a, cudaEvent_t b);

}  // namespace sg
