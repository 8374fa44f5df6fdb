/*
 * sisso.h — C ABI of the GB300 (sm_103a) SISSO hot path.
 *
 * SISSO (arXiv 2410.01752) fits y ~ c0 + sum_j c_j phi_j(x) where the phi_j are chosen
 * from an operator-generated feature space (§2.1, Eq. 2) by sure independence screening
 * (§2.2, Eqs. 5-6) and an exhaustive l0 search over the screened subspace (§2.3, Eqs. 7-8).
 * This library runs that path on one GPU: a fused generate-and-score kernel screens
 * every candidate without materialising the feature space, a device-wide selection and
 * an FP64 re-score pick the subspace, and a persistent enumerator solves every D-subset
 * by register Cholesky.
 *
 * Conventions for every entry point:
 *  - Status codes, never aborts, traps or prints.  After an error on a context,
 *    sisso_last_error(ctx) describes it (the string is owned by the context).
 *  - Pointers passed in may be host or device memory unless stated otherwise; the
 *    library copies what it keeps (unified addressing, cudaMemcpyDefault).
 *    Output buffers are owned by the caller and are HOST memory.
 *  - X is N x d, row-major (sample-major), FP64.  Feature ids are the canonical ids of
 *    the expanded space: level, then operator in the order of the table below, then the
 *    operand pair (i, j) in lexicographic order (see sisso_feature_expr for the meaning).
 *  - A context owns all device memory it allocates and one CUDA stream (or the caller's,
 *    see sisso_opts.cuda_stream).  Contexts are independent; one context must not be used
 *    from two host threads at once.
 */
#ifndef SISSO_H
#define SISSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sisso_ctx sisso_ctx;

typedef enum {
    SISSO_OK = 0,
    SISSO_ERR_ARG = -1,        /* invalid argument (sizes, op mask, rung, non-finite input) */
    SISSO_ERR_OOM = -2,        /* device allocation failed */
    SISSO_ERR_CUDA = -3,       /* a CUDA call failed (message in sisso_last_error) */
    SISSO_ERR_NUMERIC = -4,    /* no valid feature / every subset singular */
    SISSO_ERR_TIMEOUT = -5,    /* a bounded device wait ran out */
    SISSO_ERR_STATE = -6,      /* call out of order (e.g. get_descriptor before fit) */
    SISSO_ERR_CAPACITY = -7    /* a fixed-capacity buffer would overflow */
} sisso_status;

/* Operator table, in canonical order (§2.1; the paper's operators plus those its
 * examples use, §3.3 and Table 1).  Binary first: + and * are symmetric (i < j), - is
 * taken for i < j only (a-b = -(b-a) scores and fits the same), / takes both orders. */
enum {
    SISSO_OP_ADD = 1u << 0,    /* z_i + z_j      */
    SISSO_OP_SUB = 1u << 1,    /* z_i - z_j      */
    SISSO_OP_MUL = 1u << 2,    /* z_i * z_j      */
    SISSO_OP_DIV = 1u << 3,    /* z_i / z_j      */
    SISSO_OP_EXP = 1u << 4,    /* exp(z)         */
    SISSO_OP_LOG = 1u << 5,    /* log(z)         */
    SISSO_OP_SQRT = 1u << 6,   /* sqrt(z)        */
    SISSO_OP_SQ = 1u << 7,     /* z^2            */
    SISSO_OP_INV = 1u << 8,    /* z^-1           */
    SISSO_OP_SIN = 1u << 9,    /* sin(z)         */
    SISSO_OP_CUBE = 1u << 10,  /* z^3            */
    SISSO_OP_EXPNEG = 1u << 11 /* exp(-z)        */
};
#define SISSO_OP_ALL 0xFFFu

/* Arithmetic of the screening and l0 kernels.  FP64 and FP32 give the exact FP64 result
 * (FP32 work is error-bounded and whatever it cannot decide is re-scored or refit in
 * FP64).  The
 * mixed forms compute the subspace Gram on the tensor cores from BF16 or FP16 operands
 * (FP32 accumulation) and refit in FP64 the 100 best subsets and every subset whose
 * condition estimate exceeds 1e6. */
enum { SISSO_PREC_FP64 = 0, SISSO_PREC_FP32 = 1, SISSO_PREC_MIXED_BF16 = 2, SISSO_PREC_MIXED_FP16 = 3 };

/* Mixed forms: where the top level's binary candidates are scored (sisso_opts.screen). */
enum { SISSO_SCREEN_AUTO = 0, SISSO_SCREEN_CORES = 1, SISSO_SCREEN_TENSOR = 2 };

/* FP32 precision: how the subspace Gram of §2.3 Eq. 7 is formed (sisso_opts.gram). */
enum { SISSO_GRAM_AUTO = 0, SISSO_GRAM_FP64 = 1, SISSO_GRAM_TF32X3 = 2 };

/* Expansion grammar (§2.1 Eq. 2).  EQ2: every pair of phi_{l-1} except pairs already
 * in phi_{l-2}.  NEW_X_PREV: identical up to level 2; from level 3 one operand is new at
 * level l-1 and the other comes from phi_{l-2}.  Unary operators always act on the
 * features new at level l-1. */
enum { SISSO_GRAMMAR_EQ2 = 0, SISSO_GRAMMAR_NEW_X_PREV = 1 };

/* Pre-screening of the primaries (§3.1): mutual information with the target, estimated
 * with Gaussian kernel density estimates, or the Spearman rank correlation. */
enum { SISSO_PRESCREEN_NONE = 0, SISSO_PRESCREEN_MI = 1, SISSO_PRESCREEN_SPEARMAN = 2 };

#define SISSO_MAX_RUNG 3
#define SISSO_MAX_DIM 5
#define SISSO_MAX_SIS 1024

typedef struct {
    int precision;          /* SISSO_PREC_*: arithmetic of the screening and l0 kernels;
                               selection and refits are always FP64 (default FP32) */
    int grammar;            /* SISSO_GRAMMAR_* (default EQ2) */
    int survivors;          /* FP32 screening window: candidates re-scored in FP64 per
                               step (0 = max(5 k, min(max(4096, 32 k), 2^26 / N))); grown
                               x4 automatically when it cannot prove the selection exact */
    double band_rel;        /* l0: FP32 RSS band, relative to SST, refit in FP64
                               (0 = 1e-4) */
    int64_t max_band;       /* l0: capacity of the FP64 refit list (0 = 1<<22) */
    void* cuda_stream;      /* cudaStream_t to run on; NULL = a stream the context owns */
    int device;             /* CUDA device ordinal (default 0) */
    double sis_threshold;   /* threshold variant of SIS (§2.2, last paragraph: keep the
                               features whose correlation exceeds a threshold): in [0, 1),
                               on the Pearson |rho| the walk ranks by; a step ends when the
                               best remaining score is at or below it, or at sis_size
                               accepted ids (0 = top sis_size only, the default).  A fit
                               whose first step accepts nothing ends with no descriptor. */
    double stop_rmse;       /* "low enough error" stop of the iteration (§2.3): after a step
                               whose RMSE is at or below this (in units of y), no further
                               step runs (0 = only the exact-fit stop, the default) */
    int prescreen;          /* pre-screening of the primaries (§3.1; §3.3 initial_screening):
                               SISSO_PRESCREEN_NONE (default), _MI or _SPEARMAN; the context
                               is then built on the kept primaries only (renumbered x1..;
                               sisso_get_primaries maps them back) */
    double prescreen_quantile; /* fraction q in (0, 1] of the primaries kept: those scoring
                               strictly above the (1 - q)-quantile of the scores */
    int64_t wait_limit_ns;  /* batched form: the persistent kernel gives up (SISSO_ERR_TIMEOUT,
                               every CTA returns) after this long without progress anywhere
                               on its work queue (0 = 10 s, the default) */
    const int* units;       /* dimensional analysis (§2.1, closing paragraph; §3.3
                               dimensionality): d unit labels, HOST memory, copied by
                               sisso_create; primaries with equal labels share units, -1
                               is dimensionless (NULL = no units, the default).  Units are
                               exponent vectors over the labels: + and - need equal units,
                               exp, log, sin and exp(-.) a dimensionless operand, the other
                               operators combine units.  A feature that breaks the rule, or
                               is built from one that does, is invalid (scores -1, never
                               selected); ids are those of the space without units. */
    int screen;             /* mixed forms' scoring of the top level's binary candidates:
                               SISSO_SCREEN_AUTO (default) from split 16-bit tensor-core
                               products (§2.2 Eq. 5 as a contraction; each key carries its
                               error bound, see sisso_bilinear_tc) when the pairs lie within
                               phi_{L-1} (EQ2 grammar, or rung <= 2) and |phi_{L-1}| <= 4096,
                               else the FP32 CUDA-core kernel; SISSO_SCREEN_CORES always the
                               CUDA-core kernel; SISSO_SCREEN_TENSOR the tensor cores also for
                               the NEW_X_PREV pairs phi_{L-2} x new_{L-1} at rung >= 3 (when
                               |phi_{L-2}| <= 4096 and the products fit 48 GB) */
    int gram;               /* FP32 precision's subspace Gram (§2.3 Eq. 7):
                               SISSO_GRAM_AUTO (default) and SISSO_GRAM_FP64 build it from
                               FP64 rows on the CUDA cores, and the l0 result is the FP64
                               search's; SISSO_GRAM_TF32X3 forms it on the tensor cores from
                               3xTF32 split products (tcgen05.mma kind::tf32, FP32
                               accumulation over runs of 512 samples, runs added in FP64;
                               entries within 2.4e-5 of the FP64 Gram; the partial sums
                               are capped at 512 MB, which lengthens the runs, and the bound
                               with them, above about 1000 features at 65 536 samples), and
                               the l0 step then refits in FP64, from the standardised rows,
                               its 100 best subsets and every subset with a small pivot, as
                               the mixed forms do (a learned proposal set on the context is
                               not used).
                               Other precisions accept AUTO or FP64 only. */
    const double* whiten;   /* whitening (§2.4): W = Sigma^-1/2 (N x N, row-major FP64, host
                               or device, copied by sisso_create) for noise with a known
                               covariance Sigma; SISSO then runs on W y and W Phi: every
                               candidate valid on the samples is mapped to W v (which must
                               pass the same value rules), the intercept stays a constant
                               column in the transformed space, and coefficients, RMSE and
                               R^2 are those of the transformed fit.  Needs SISSO_PREC_FP64
                               and no pre-screening (else SISSO_ERR_ARG); candidates are
                               scored row by row (an N x N FP64 product per candidate), and
                               the FP64 operand values and the window's vectors must fit
                               (else SISSO_ERR_CAPACITY).  Targets passed to
                               sisso_score_all / sisso_sis_step on such a context are taken
                               as already whitened.  NULL = none (the default). */
} sisso_opts;

/* Per-context counters and device timings (CUDA events on the context's stream). */
typedef struct {
    int64_t candidates_scored;   /* ids scored by the screening kernels, all steps */
    int64_t subsets_fit;         /* l0 subsets solved in FP32/FP64, all steps */
    int64_t subsets_refit;       /* subsets re-solved in FP64 */
    int64_t survivors_rescored;  /* candidates re-scored in FP64 */
    int window_grown;            /* times the screening window was enlarged */
    int window_saturated;        /* 1 if the window hit its cap without proof */
    int launches;                /* kernels launched by the last sisso_fit */
    double ms_screen;            /* fused generate+score kernels */
    double ms_screen_pair;       /* ... of which the top-level pair kernel */
    int screen_pair_launches;    /* launches of the top-level pair kernel */
    double ms_select;            /* device-wide selection, FP64 re-score, walk */
    double ms_radix;             /* ... radix select and compaction */
    double ms_rescore;           /* ... FP64 re-score of the window */
    double ms_sort;              /* ... sort of the window */
    double ms_walk;              /* ... tie/duplicate walk */
    int64_t walk_visited;        /* candidates visited by the walks */
    int64_t walk_dup_checks;     /* duplicate checks (vector comparisons) made */
    double ms_gram;              /* subspace Gram */
    double ms_l0;                /* l0 enumeration (FP32 or FP64) */
    double ms_refit;             /* FP64 refit, winner, residual */
    double ms_fit;               /* whole sisso_fit, device time */
    double ms_l0_enum;           /* ... of ms_l0: the tiled FP32 enumeration kernel alone */
    int l0_enum_launches;        /* launches of the tiled FP32 enumeration kernel */
    int64_t l0_candidates;       /* subsets its filter sent to the exact FP32/FP64 test */
    int64_t certified_prefixes;  /* learned D = 5 step: 3-prefixes its certificate left to enumerate */
    int screen_tc;               /* 1 if the top level's pairs were scored on the tensor cores */
    int64_t tc_keys_raised;      /* ... keys raised to their error bound (bound above the FP32
                                    screening margin, or the variance not resolved) */
    int64_t pm_keys_direct;      /* FP32 top-level + / - candidates whose cross-sum key was left
                                    open (operands that nearly cancel) and scored from the
                                    direct sums instead, all steps */
} sisso_stats;

void sisso_default_opts(sisso_opts* opts);

/* Create a context: copies X (N x d row-major FP64) and y (N) to the device, plans the
 * feature space phi_rung (§2.1) for the operator mask and grammar, and allocates every
 * buffer sisso_fit needs.  sis_size is k of §2.2 (features added per step), max_dim the
 * number of terms T of §2.3.  Errors: SISSO_ERR_ARG for N < max_dim+1, d < 1, rung not
 * in 1..SISSO_MAX_RUNG, max_dim not in 1..SISSO_MAX_DIM, sis_size not in
 * 1..SISSO_MAX_SIS, an empty op mask, sis_threshold outside [0, 1), stop_rmse < 0, a unit
 * label outside -1..d-1, or non-finite X/y; SISSO_ERR_OOM; SISSO_ERR_CUDA.
 * On error *out is NULL. */
sisso_status sisso_create(const double* X, const double* y, int N, int d, uint32_t op_set,
                          int rung, int sis_size, int max_dim, const sisso_opts* opts,
                          sisso_ctx** out);

/* Run SISSO (§2.3 Eq. 8): for t = 1..max_dim, screen phi against y (t = 1) or the best
 * (t-1)-term residual, append the k accepted ids to S, solve every t-subset of S and
 * keep the lowest-RSS model.  Stops early when a model is exact to FP64 rounding
 * (RMSE <= 1e-10 std(y)) or S has fewer than t features.  Synchronous: returns when
 * the results are on the host. */
sisso_status sisso_fit(sisso_ctx* ctx);

/* Original indices (0-based) of the primaries the context was built on, in the order of
 * its x1, x2, ...: all d without pre-screening.  idx: HOST, cap entries; *n = count. */
sisso_status sisso_get_primaries(const sisso_ctx* ctx, int* idx, int cap, int* n);

/* Pre-screening scores of the d primaries of X (N x d row-major FP64, host or device)
 * against y (§3.1; §3.3): method SISSO_PRESCREEN_MI, MI(y; x_i) = mean over the samples of
 * log(p(x, y) / (p(x) p(y))) with Gaussian kernel density estimates at the samples (Scott's
 * rule: kernel covariance N^(-2/(k+4)) times the sample covariance of the k-dimensional
 * variable, the full 2 x 2 covariance for the joint density; kernel values in FP32,
 * sums in FP64), or SISSO_PRESCREEN_SPEARMAN, |Spearman rank correlation| (average ranks
 * for ties).  keep: flags of the primaries in the top quantile q (strictly above the
 * (1 - q)-quantile of the scores, linear interpolation); scores, keep (may be NULL) and
 * n_keep (may be NULL) HOST.  Runs on the current device with its own buffers.  Errors:
 * SISSO_ERR_ARG (sizes, method, q outside (0, 1], a constant primary or target for MI),
 * SISSO_ERR_OOM, SISSO_ERR_CUDA. */
sisso_status sisso_prescreen(const double* X, const double* y, int N, int d, int method, double quantile,
                             double* scores, int* keep, int* n_keep);

/* Number of descriptors produced by the last fit (<= max_dim). */
sisso_status sisso_get_n_dims(const sisso_ctx* ctx, int* n_dims);

/* Descriptor of dimension dim (1-based), the best dim-term model of §2.3 (Eq. 7: the
 * least-squares coefficients c_t of the chosen columns, with the constant feature as the
 * intercept) reported as §3.3's fit outputs (equation, RMSE, R^2): ids[dim] ascending,
 * coef[dim+1] with coef[0] the intercept and coef[j+1] the coefficient of ids[j] in the
 * original units, rmse = sqrt(RSS/N), r2 = 1 - RSS/SST.  Any output pointer may be NULL.
 * Errors: SISSO_ERR_STATE before a fit, SISSO_ERR_ARG for dim outside 1..n_dims. */
sisso_status sisso_get_descriptor(const sisso_ctx* ctx, int dim, int64_t* ids, double* coef,
                                  double* rmse, double* r2);

/* Ids accepted by SIS at step `step` (1-based), in acceptance order; *n = count. */
sisso_status sisso_get_sis(const sisso_ctx* ctx, int step, int64_t* ids, int cap, int* n);

/* |phi_rung| and |phi_l| for l = 0..rung (sizes[rung+1]; may be NULL). */
sisso_status sisso_feature_count(const sisso_ctx* ctx, int64_t* n_features, int64_t* sizes);

/* Expression of feature id of the expanded space (§2.1, Eq. 2: the operator tree that
 * generated it), e.g. "(x1*(x2/x3))": primaries are x1..xd; binary
 * "(a+b)", "(a-b)", "(a*b)", "(a/b)"; unary "exp(a)", "log(a)", "sqrt(a)", "(a)^2",
 * "(a)^-1", "sin(a)", "(a)^3", "exp(-a)". */
sisso_status sisso_feature_expr(const sisso_ctx* ctx, int64_t id, char* buf, size_t len);

sisso_status sisso_get_stats(const sisso_ctx* ctx, sisso_stats* out);
const char* sisso_last_error(const sisso_ctx* ctx);
/* Destroy a context: its device buffers go back to a memory pool per device that the library
 * keeps (up to 32 GB of freed memory) for the next context, so that creating contexts one
 * after another does not map and unmap gigabytes each time; sisso_release_memory returns
 * that memory to the device. */
void sisso_destroy(sisso_ctx* ctx);

/* Release the device memory the library's pool keeps for device `device` after its contexts
 * were destroyed (memory of live contexts stays).  Synchronises the device.  Errors:
 * SISSO_ERR_ARG (no such device), SISSO_ERR_CUDA. */
sisso_status sisso_release_memory(int device);

/* ---- feature space without a context (host only, no GPU needed) ------------------- */

/* Sizes |phi_l|, l = 0..rung, of the space planned for (d, op_set, rung, grammar)
 * (§2.1 Eq. 2 with the rule above).  sizes: HOST, rung+1 entries. */
sisso_status sisso_space_sizes(int d, uint32_t op_set, int rung, int grammar, int64_t* sizes);

/* Expression string of feature id in that space (same format as sisso_feature_expr). */
sisso_status sisso_space_expr(int d, uint32_t op_set, int rung, int grammar, int64_t id, char* buf,
                              size_t len);

/* ---- kernel-level entry points (parity tests, benchmark) -------------------------- */

/* Values of features ids[0..n) at every sample, evaluated on the device in `precision`
 * from the primaries (§2.1).  out: HOST, n x N row-major, double (FP32 results are
 * widened). */
sisso_status sisso_eval_features(sisso_ctx* ctx, const int64_t* ids, int64_t n, int precision,
                                 double* out);

/* Screening scores of every id of phi_rung against `target` (N values; §2.2 Eqs. 5-6:
 * Pearson |rho|) from the fused generate-and-score kernels in `precision`.  Invalid
 * features score -1.  scores: HOST, |phi_rung| floats. */
sisso_status sisso_score_all(sisso_ctx* ctx, const double* target, int precision, float* scores);

/* One SIS step (§2.2) with the device-wide selection, FP64 re-score and walk: accepts up
 * to k ids not in S_prev (n_prev ids) and not duplicates of S_prev or of each other.
 * acc: HOST, k entries; *n_acc = number accepted. */
sisso_status sisso_sis_step(sisso_ctx* ctx, const double* target, const int64_t* S_prev,
                            int n_prev, int k, int64_t* acc, int* n_acc);

/* Exhaustive l0 (§2.3) over every D-subset of n standardised features given their
 * FP64 Gram G (n x n, Z^T Z / N), moments b (n, Z^T y~ / N) and syy = y~^T y~ / N:
 * FP32 (or FP64) enumeration, FP64 refit of the band, tie rule on gid (n global ids).
 * best_pos: HOST, D positions ascending; best_rss: RSS of the winner.  *examined: C(n,D).
 * n <= 65535 for D <= 4, n <= 4095 for D = 5. */
sisso_status sisso_l0_search(sisso_ctx* ctx, const double* G, const double* b, double syy,
                             int n, int D, const int64_t* gid, int precision, int* best_pos,
                             double* best_rss, int64_t* examined);

/* FP64 subspace Gram of the n features ids (n <= max_dim x sis_size of the context): the
 * features evaluated and standardised on the device (§2.3), G = Z Z^T / N (n x n) and
 * b = Z y~ / N (n), HOST; *syy (may be NULL) = y~^T y~ / N. */
sisso_status sisso_subspace_gram(sisso_ctx* ctx, const int64_t* ids, int n, double* G, double* b, double* syy);

/* Subspace Gram on the tcgen05 tensor cores (§2.3 Eq. 7): with Z n standardised rows of N
 * samples (FP64, row-major) and yc the centred target with population std sdy, returns
 * G = Z Z^T / N (n x n) and b = Z yc / N (n), computed from BF16 (kind =
 * SISSO_PREC_MIXED_BF16) or FP16 (SISSO_PREC_MIXED_FP16) operands with FP32 accumulation
 * (the mixed forms' Gram), or (kind = SISSO_PREC_FP32) from 3xTF32 split products: each
 * value is h + l with h = tf32(z), l = tf32(z - h), and z_i z_j is taken as h_i h_j + h_i l_j
 * + l_i h_j, accumulated in FP32 over runs of 512 samples and the runs added in FP64 (the
 * FP32 precision's tensor-core Gram, sisso_opts.gram; entries within 3 2^-22 + 192 2^-23 =
 * 2.4e-5 of the exact Gram, the second term the tensor cores' FP32 accumulation).  Inputs
 * host or device; G and b HOST.  Uses the current device and the legacy default stream.  Errors: SISSO_ERR_ARG, SISSO_ERR_CUDA, SISSO_ERR_TIMEOUT. */
sisso_status sisso_gram_tc(const double* Z, const double* yc, double sdy, int n, int N, int kind, float* G,
                           float* b);

/* Split-precision tensor-core product (the mixed forms' screening sums, §2.2 Eq. 5 written
 * as a contraction over the samples): out[i][j] = sum_s L[i][s] R[j][s] for the m rows of L
 * and n rows of R (N samples each, FP64, row-major, HOST; out m x n FP64 HOST).  Every row
 * is scaled by a power of two and split into 16-bit parts (FP16: two, BF16: three); the
 * part products of tcgen05.mma kind::f16 accumulate in FP32 over chunks of 1024 samples,
 * the chunks in FP64.  |out - exact| stays within about 2^-21 of the Cauchy-Schwarz scale
 * sqrt(sum L_i^2 sum R_j^2) (the screening bounds each key with 2^-17).  kind:
 * SISSO_PREC_MIXED_BF16 or _FP16.  m, n <= 65536.  Current device, default stream.
 * Errors: SISSO_ERR_ARG, SISSO_ERR_CUDA, SISSO_ERR_TIMEOUT (a bounded wait ran out). */
sisso_status sisso_bilinear_tc(const double* L, const double* R, int m, int n, int N, int kind, double* out);

/* Measured FMA throughput of the current device in TFLOP/s, the denominator of the ALU-bound
 * kernels' roofline: kind 0 FP32 (fma.rn.f32, 2 flop), 1 paired FP32 (fma.rn.f32x2, 4 flop),
 * 2 FP64.  Every SM busy with independent chains; best of five timed launches of about
 * 16 ms each (80 ms FP64), after one (the burst rate; legacy default stream).  Errors: SISSO_ERR_ARG, SISSO_ERR_CUDA. */
sisso_status sisso_measure_alu_peak(int kind, double* tflops);

/* ---- batched multi-task form ----------------------------------------------------------
 *
 * Many independent SISSO problems (each §2.1-2.3: feature space Eq. 2, SIS Eqs. 5-6, l0
 * Eqs. 7-8), possibly of different sizes, solved by one persistent kernel launch captured
 * in a CUDA graph.  Every task shares the operator set, rung, grammar, sis_size and
 * max_dim; each has its own N and d.  Each task computes what sisso_create + sisso_fit
 * with precision SISSO_PREC_FP32 computes (FP32 screening and l0 enumeration, FP64
 * re-score, refit and model), so its descriptors equal the per-problem path's.
 *
 * The paper solves one problem at a time; this form serves many small ones at once.
 */
typedef struct sisso_batch sisso_batch;

typedef struct {
    const double* X;    /* N x d row-major, HOST memory */
    const double* y;    /* N, HOST memory */
    int N, d;
} sisso_task;

/* One task's result.  status: SISSO_OK or the task's own error (SISSO_ERR_NUMERIC: no
 * valid feature or every subset singular; SISSO_ERR_CAPACITY: a window or band
 * overflowed).  Dimension t = 1..n_dims is row t-1: ids ascending, coef[0] the intercept
 * and coef[j] the coefficient of ids[j-1], in original units. */
typedef struct {
    int status;
    int n_dims;
    int64_t ids[SISSO_MAX_DIM][SISSO_MAX_DIM];
    double coef[SISSO_MAX_DIM][SISSO_MAX_DIM + 1];
    double rmse[SISSO_MAX_DIM];
    double r2[SISSO_MAX_DIM];
} sisso_task_result;

/* Launch shape of the persistent kernel (0 = keep the current value). */
typedef struct {
    int score_units;    /* screening units (32 x 32 pair tiles, 32-operand unary blocks,
                           256-id blocks) per work item */
    int enum_items;     /* l0 work units (a (D-2)-prefix x 16 rows of subsets) per work item */
    int gram_rows;      /* new subspace rows per Gram work item */
    int ctas_per_sm;    /* resident CTAs per SM: 1 or 2 */
    int window;         /* first screening window (candidates re-scored in FP64) */
} sisso_batch_tune;

/* Per-batch counters of the last run. */
typedef struct {
    double ms_run;              /* device time of the last sisso_batch_run (CUDA events) */
    int64_t candidates_scored;  /* all tasks, all steps */
    int64_t subsets_fit;        /* l0 subsets enumerated, all tasks and steps */
    int64_t subsets_refit;      /* band entries re-solved in FP64 */
    int windows_grown;
    int windows_saturated;      /* tasks whose window hit its cap without proof */
    int tasks_failed;           /* tasks with status != SISSO_OK */
    int grid;                   /* CTAs launched */
    int64_t walk_visits;        /* screening walks: candidates visited, all tasks and steps */
    int64_t walk_checks;        /* ... full duplicate comparisons */
    /* device-clock profile of the last run, per stage: 0 unused, 1 start, 2 level, 3 score,
       4 gram, 5 bound, 6 band, 7 validity flattening, 8 select, 9 refit, 10 waiting for
       work, 11 per-operand sums, and the parts of select: 12 radix select, 13 FP64 re-score, 14 sort,
       15 walk.  stage_ms sums the CTAs' time, stage_max_ms is the longest single
       occurrence, stage_count the occurrences. */
    double stage_ms[16];
    double stage_max_ms[16];
    int64_t stage_count[16];
} sisso_batch_stats;

/* Plan every task (feature space, work units, memory), copy the inputs to pinned host
 * and device memory, and allocate all device memory the runs need (one arena).  opts:
 * grammar, max_band (band capacity per task and step, default 16384), cuda_stream and
 * device are used; precision must be SISSO_PREC_FP32 (or default), sis_threshold and
 * stop_rmse 0 (top-k screening, exact-fit stop), units NULL.  Limits: n_tasks <=
 * 2^20, max_dim <= 4, max_dim * sis_size <= 512, every task N >= max_dim + 1 and d >= 1, finite inputs,
 * non-constant y, and at most 2^18 screening units per task.  Errors: SISSO_ERR_ARG
 * (message names the task), SISSO_ERR_OOM, SISSO_ERR_CUDA.  On error *out is NULL and
 * the message is in sisso_batch_create_error(). */
sisso_status sisso_batch_create(const sisso_task* tasks, int n_tasks, uint32_t op_set, int rung, int sis_size,
                                int max_dim, const sisso_opts* opts, sisso_batch** out);
const char* sisso_batch_create_error(void);

/* Replace the launch shape (fields 0 keep their value); the graphs are re-captured. */
sisso_status sisso_batch_set_tune(sisso_batch* b, const sisso_batch_tune* tune);
sisso_status sisso_batch_get_tune(const sisso_batch* b, sisso_batch_tune* tune);

/* Replace the no-progress limit of the work-queue wait (ns; 0 = 10 s); the graphs are
 * re-captured.  A run whose wait runs out returns SISSO_ERR_TIMEOUT after every CTA has
 * returned; the next run starts from a clean state. */
sisso_status sisso_batch_set_wait_limit(sisso_batch* b, int64_t ns);

/* Autotuner: times candidate launch shapes on this batch (each a full run, reps times,
 * CUDA events) one parameter at a time and keeps the fastest.  cache_path (may be NULL):
 * a text file of earlier choices keyed by the batch's shape signature; a hit skips the
 * timing, a miss appends the choice.  chosen (may be NULL) receives it. */
sisso_status sisso_batch_autotune(sisso_batch* b, int reps, const char* cache_path, sisso_batch_tune* chosen);

/* Replace task inputs with new values of the same shapes (HOST memory, copied to the
 * pinned staging buffer; the device copy happens in the next run with copies = 1). */
sisso_status sisso_batch_load(sisso_batch* b, const sisso_task* tasks, int n_tasks);

/* One run of every task: a CUDA graph launch on the batch's stream, waited for.  copies =
 * 1: the graph also copies the inputs host -> device before the kernel and the results
 * device -> host after it; copies = 0: inputs already on the device (from an earlier
 * copying run or create), results fetched by sisso_batch_results.  Errors:
 * SISSO_ERR_TIMEOUT (a bounded device wait ran out), SISSO_ERR_CAPACITY (work queue),
 * SISSO_ERR_CUDA.  Per-task errors are in the results, not here. */
sisso_status sisso_batch_run(sisso_batch* b, int copies);

/* Results of the last run for tasks [0, n): out HOST, n entries. */
sisso_status sisso_batch_results(sisso_batch* b, sisso_task_result* out, int n);

/* Per-task device timestamps of the last run, in ms from the launch's first CTA start:
 * start[i] when task i began, end[i] when its last result was written.  HOST, n each
 * (either may be NULL). */
sisso_status sisso_batch_timing(sisso_batch* b, double* start, double* end, int n);

sisso_status sisso_batch_get_stats(sisso_batch* b, sisso_batch_stats* out);
const char* sisso_batch_last_error(const sisso_batch* b);
void sisso_batch_destroy(sisso_batch* b);

/* Convenience: create, one copying run, results, destroy.  results: HOST, n_tasks. */
sisso_status sisso_fit_batch(const sisso_task* tasks, int n_tasks, uint32_t op_set, int rung, int sis_size,
                             int max_dim, const sisso_opts* opts, sisso_task_result* results);

/* ---- learned subset proposal ----------------------------------------------------------
 *
 * For the l0 search at D = 5 (§2.3, Eq. 7) a small network ranks the search's 3-prefixes
 * {p0 < p1 < p2} (p = positions in the screened subspace) by its prediction of the lowest
 * RSS/SST (log10) among the 5-subsets that extend them with higher positions; the best
 * prefixes are taken until their extensions make up a fraction of C(n, 5), and only those
 * are solved, exactly.  The network: SISSO_MLP_IN inputs describing a candidate 5-subset
 * (the upper triangle of its 5 x 5 standardised sub-Gram in row order, then its 5
 * correlations with the target); a prefix is described by its greedy completion (the
 * feature above p2 that lowers its RSS most, then the next such feature; slots of features
 * that do not exist are 0).  Two hidden layers of SISSO_MLP_HIDDEN with ReLU, one output; BF16 weights, activations and gradients with FP32 accumulation on the tensor
 * cores, FP32 master weights, MSE loss, Adam.  The paper has no counterpart; exhaustive
 * search (sisso_l0_search) remains the fallback and the judge.
 *
 * Parameter layout (FP32, SISSO_MLP_PARAMS values): W1 [256 x 20] row-major (output x input),
 * b1 [256], W2 [256 x 256], b2 [256], w3 [256], b3 [1].
 *
 * Ownership: the caller owns every buffer it passes and the sisso_mlp it creates (destroy it
 * after the last context that uses it as a proposal).  Errors, for every entry point below:
 * SISSO_ERR_ARG for a NULL required pointer or an out-of-range size (n, M, B, batch, frac in
 * (0, 1], lr > 0), checked before the device is touched; SISSO_ERR_OOM / SISSO_ERR_CUDA for
 * device failures; SISSO_ERR_TIMEOUT when a bounded wait in the network's tensor-core
 * kernels ran out (the network is then in an undefined state: destroy it).
 */
#define SISSO_MLP_IN 20
#define SISSO_MLP_HIDDEN 256
#define SISSO_MLP_PARAMS (256 * 20 + 256 + 256 * 256 + 256 + 256 + 1)

typedef struct sisso_mlp sisso_mlp;

/* A network on the current device, He-uniform weights from the seed, zero biases. */
sisso_status sisso_mlp_create(uint64_t seed, sisso_mlp** out);
void sisso_mlp_destroy(sisso_mlp* mlp);
/* params: HOST (get) / host or device (set), SISSO_MLP_PARAMS floats in the layout above. */
sisso_status sisso_mlp_get_params(sisso_mlp* mlp, float* params);
sisso_status sisso_mlp_set_params(sisso_mlp* mlp, const float* params);
/* out[i] = network(X[i]) for M rows X (M x SISSO_MLP_IN, host or device); out HOST. */
sisso_status sisso_mlp_forward(sisso_mlp* mlp, const float* X, int64_t M, float* out);
/* Mean squared error of one batch (B a multiple of 128) and its gradient (HOST,
 * SISSO_MLP_PARAMS floats, the parameter layout); loss may be NULL. */
sisso_status sisso_mlp_gradients(sisso_mlp* mlp, const float* X, const float* t, int B, float* loss, float* grad);
/* Adam (lr, betas 0.9 / 0.999) on the MSE over M examples for `epochs` epochs of batches of
 * `batch` rows (a multiple of 128) in a seeded order; *final_loss: the last epoch's mean. */
sisso_status sisso_mlp_train(sisso_mlp* mlp, const float* X, const float* t, int64_t M, int epochs, int batch,
                             float lr, uint64_t seed, float* final_loss);

/* Network inputs of every 3-prefix of n standardised features (G n x n, b, syy as for
 * sisso_l0_search), prefixes in colex order (rank C(p2,3) + C(p1,2) + p0), each described by
 * its greedy completion (computed in FP32): out HOST, C(n,3) x SISSO_MLP_IN floats;
 * prefixes (may be NULL) HOST, C(n,3) x 3 positions; base (may be NULL) HOST, C(n,3)
 * values log10(RSS/SST) of the completions (0 for a prefix without one). */
sisso_status sisso_prefix_features(const double* G, const double* b, double syy, int n, float* out, int* prefixes,
                                   float* base);
/* Training labels: per 3-prefix (same order), the lowest FP32 RSS / SST over the 5-subsets
 * extending it with higher positions (exhaustive; +inf when it has none).  n in 5..1400.
 * out HOST. */
sisso_status sisso_prefix_labels(const double* G, const double* b, double syy, int N, int n, float* out);

/* Training examples of every 3-prefix (same order as above), computed on the device:
 * inputs (C(n,3) x SISSO_MLP_IN), labels (as sisso_prefix_labels) and the network's
 * training target, log10(max(label, 1e-12)) minus the base score log10(RSS/SST) of the
 * prefix's greedy completion (NaN for a prefix without extensions).  n in 5..1400; all
 * outputs HOST. */
sisso_status sisso_prefix_training(const double* G, const double* b, double syy, int N, int n, float* inputs,
                                   float* labels, float* targets);

/* The learned l0 search at D = 5 on the context's device: network scores of every 3-prefix,
 * prefixes best first up to frac x C(n,5) subsets, their extensions solved exactly (same
 * FP32 enumeration, FP64 confirmation and tie rule as sisso_l0_search).  Outputs as
 * sisso_l0_search; *examined the subsets solved, *n_prefixes (may be NULL) those taken.
 * n in 5..1400. */
sisso_status sisso_l0_learned(sisso_ctx* ctx, const double* G, const double* b, double syy, int n,
                              const int64_t* gid, sisso_mlp* mlp, double frac, int* best_pos, double* best_rss,
                              int64_t* examined, int64_t* n_prefixes);

/* The learned search followed by its certificate, so that the result is the exhaustive
 * search's: every 5-subset extending a 3-prefix P = {p0 < p1 < p2} with two higher features
 * lies in the superset {p0, p1} U [p2, n) and has at least its RSS (least squares on a
 * superset fits at least as well).  Those superset RSS values, for every prefix at once,
 * come from one reversed-order FP64 Cholesky of G and running sums per pair {p0, p1}; a
 * prefix whose bound exceeds the learned winner's FP64 RSS (plus the tie window, 1e-9 SST
 * and 1e-7 relative) is skipped, and the others are enumerated exactly by the tiled FP32
 * search with FP64 confirmation, started from the learned winner.  Suffix sets whose
 * Cholesky pivot falls to 1e-6 or below are never pruned.  Outputs as sisso_l0_learned;
 * *examined: the subsets of both searches; *prefixes_kept (may be NULL): the prefixes the
 * certificate left to enumerate.  n in 5..1400. */
sisso_status sisso_l0_learned_certified(sisso_ctx* ctx, const double* G, const double* b, double syy, int n,
                                        const int64_t* gid, sisso_mlp* mlp, double frac, int* best_pos,
                                        double* best_rss, int64_t* examined, int64_t* n_prefixes,
                                        int64_t* prefixes_kept);

/* Make sisso_fit use the learned search for its D = 5 step (mlp NULL: exhaustive again),
 * with the certificate above, so that the fit's descriptors are those of the exhaustive
 * search.  The context does not own the network. */
sisso_status sisso_set_proposal(sisso_ctx* ctx, sisso_mlp* mlp, double frac);

/* The same with the certificate on (certify != 0) or off: off, the D = 5 step returns the
 * best of the proposed subsets only, which is the exhaustive search's winner when the
 * proposal contains it (the recall the tests and the benchmark report). */
sisso_status sisso_set_proposal_ex(sisso_ctx* ctx, sisso_mlp* mlp, double frac, int certify);

/* ---- allocation-free l0 search --------------------------------------------------------
 *
 * sisso_l0_search_noalloc: the same search as sisso_l0_search, for callers that cannot
 * allocate device memory — for example a plug-in that may only use the memory its host
 * hands to it, a framework that routes every device allocation through its own pool and
 * forbids raw cudaMalloc, or a latency-critical loop that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree.  It needs no context and allocates nothing:
 * its working memory (about 1.8 MB) is one array inside the library, reserved on every
 * device that loads the library until the process exits.  The paper has no counterpart;
 * this is an interface convenience.
 *
 * G (n x n, row-major, FP64), b (n) and gid (n) may be host or device memory; N is the
 * number of samples behind G and b (RSS = N (syy - b_E^T G_E^-1 b_E)).  precision is
 * SISSO_PREC_FP32 (error-bounded FP32 enumeration and FP64 refit) or SISSO_PREC_FP64.
 * stream: a cudaStream_t, or NULL for the legacy default stream.  Outputs are HOST memory:
 * best_pos (D positions, ascending), *best_rss, *examined (C(n, D)); the call returns
 * once they are written.
 *
 * Limits: n <= SISSO_NOALLOC_MAX_N; the FP64 refit band holds at most
 * SISSO_NOALLOC_MAX_BAND subsets.  Larger problems return SISSO_ERR_CAPACITY (use
 * sisso_l0_search).  Other errors: SISSO_ERR_ARG (bad sizes, NULL pointers),
 * SISSO_ERR_NUMERIC (every subset singular), SISSO_ERR_CUDA.
 *
 * The first call on each device looks up the device address of the working array
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  Every call on a device shares the one array, which keeps the last
 * call's contents (the call clears what must start at zero): calls that overlap on the
 * GPU — from two host threads or two streams — race and must be serialised by the caller.
 */
#define SISSO_NOALLOC_MAX_N 256
#define SISSO_NOALLOC_MAX_BAND 65536

sisso_status sisso_l0_search_noalloc(const double* G, const double* b, double syy, int N, int n, int D,
                                     const int64_t* gid, int precision, void* stream, int* best_pos,
                                     double* best_rss, int64_t* examined);

#ifdef __cplusplus
}
#endif
#endif /* SISSO_H */
