/*
 * sisso_oracle.h — interface of the plain FP64 CPU SISSO oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct statement of
 * what the GPU library computes; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * Paper passages followed (arXiv 2410.01752):
 *   §2.1 Eq. 2   recursive feature expansion phi_l = { O[z_i, z_j] : z_i, z_j in phi_{l-1} }
 *   §2.1 Eq. 3   the count bound d_l <= m_u d_{l-1} + (m_bs/2 + m_bns) d_{l-1}(d_{l-1}-1)
 *   §2.1 (text after Eq. 3) pairs regenerated from phi_{l-2} are not new
 *   §2.2 Eqs. 5-6  SIS: standardised columns, w = Phi^T y, keep the k largest |w|
 *   §2.3 Eq. 7   least-squares residual of a t-term model (the printed transpose on the
 *                Gram factor is read as an inverse)
 *   §2.3 Eq. 8   S_{t+1} = S_t U SIS(r*_t, Phi), S_1 = SIS(y, Phi); exhaustive l0 over
 *                all t-subsets of S_t; the constant feature (intercept) is always included
 */
#ifndef SISSO_ORACLE_H
#define SISSO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* operator bits (same meaning as the library's public op mask) */
enum {
    ORC_ADD = 0, ORC_SUB, ORC_MUL, ORC_DIV,                 /* binary */
    ORC_EXP, ORC_LOG, ORC_SQRT, ORC_SQ, ORC_INV, ORC_SIN,  /* unary  */
    ORC_CUBE, ORC_EXPNEG,
    ORC_NOPS
};
enum { ORC_GRAMMAR_EQ2 = 0, ORC_GRAMMAR_NEW_X_PREV = 1 };
#define ORC_MAX_RUNG 4
#define ORC_MAX_DIM 8

/* sizes |phi_0| .. |phi_rung| (cumulative); returns 0 on success */
int oracle_space_sizes(int d, uint32_t ops, int rung, int grammar, int64_t* sizes_out);
/* number of features new at `level` made by operator `op` (0 if op disabled) */
int64_t oracle_section_count(int d, uint32_t ops, int rung, int grammar, int level, int op);
/* id -> (level, op, child a, child b); op = -1 for a primary (a = column index). b = -1 for unary */
int oracle_decode(int d, uint32_t ops, int rung, int grammar, int64_t id,
                  int* level, int* op, int64_t* a, int64_t* b);
/* Eq. 2 pair rule as a predicate (used by the pins to check the enumerator) */
int oracle_pair_allowed(int grammar, int level, int op, int64_t i, int64_t j, int64_t P, int64_t Q);
/* expression string of a feature; returns length or -1 */
int oracle_expr(int d, uint32_t ops, int rung, int grammar, int64_t id, char* buf, int len);
/* FP64 values of feature `id` on X (N x d row-major) */
int oracle_eval(int d, uint32_t ops, int rung, int grammar, const double* X, int N, int64_t id, double* out);
/* validity (1/0) and Pearson |rho| against target t for a list of ids */
int oracle_scores(int d, uint32_t ops, int rung, int grammar, const double* X, int N,
                  const double* target, const int64_t* ids, int64_t n_ids,
                  double* score_out, int* valid_out, int nthreads);
/* the same for every id of phi_rung, evaluated level by level (bit-identical results) */
int oracle_scores_all(int d, uint32_t ops, int rung, int grammar, const int* units, const double* X, int N,
                      const double* target, double* score_out, int* valid_out, int nthreads);
/* dimensional analysis: units (d labels, -1 dimensionless; NULL: none) of feature id as
   exponents over the labels in sixteenths (exps_out: d ints); returns 1 if consistent */
int oracle_units(int d, uint32_t ops, int rung, int grammar, const int* units, int64_t id, int* exps_out);
/* one SIS step: accept up to k ids (written to acc_out); returns number accepted or <0 */
int oracle_sis(int d, uint32_t ops, int rung, int grammar, const double* X, int N,
               const double* target, const int64_t* S_prev, int n_prev, int k,
               int64_t* acc_out, int nthreads);
/* the same with the threshold variant of §2.2: the walk ends when the best remaining
   score is at or below thr (thr = 0: top k only) */
int oracle_sis_ex(int d, uint32_t ops, int rung, int grammar, const int* units, const double* X, int N,
                  const double* target, const int64_t* S_prev, int n_prev, int k, double thr,
                  int64_t* acc_out, int nthreads);
/* exhaustive l0 over all D-subsets of n standardised features.
 * G (n x n), b (n) are Z^T Z / N and Z^T y~ / N; syy = y~^T y~ / N; gid[n] = global ids used
 * for the tie rule.  Writes the winning positions (ascending) and its RSS; returns the
 * number of subsets examined, or <0 if every subset is singular. */
int64_t oracle_l0(const double* G, const double* b, double syy, int N, int n, int D,
                  const int64_t* gid, int* best_pos, double* best_rss, int nthreads);

/* pre-screening of the primaries (§3.1; §3.3): MI(y; x_i) by Gaussian kernel density
   estimates (Scott's rule, resubstitution), Spearman rank correlation, and the top-quantile
   rule; X N x d row-major */
int oracle_mi_kde(const double* X, int N, int d, const double* y, double* mi_out);
int oracle_spearman(const double* X, int N, int d, const double* y, double* rho_out);
int oracle_prescreen_keep(const double* score, int d, double q, int* keep_out);

typedef struct {
    int n_dims;                         /* descriptors produced (<= max_dim) */
    int n_sis[ORC_MAX_DIM];             /* ids accepted by SIS at step t */
    int64_t sis_ids[ORC_MAX_DIM * 1024];/* S in order: all accepted ids, step by step */
    int64_t ids[ORC_MAX_DIM][ORC_MAX_DIM];   /* descriptor of dimension t (ascending ids) */
    double coef[ORC_MAX_DIM][ORC_MAX_DIM + 1];/* [0] intercept, then per id */
    double rmse[ORC_MAX_DIM];
    double r2[ORC_MAX_DIM];
    double rss_gram[ORC_MAX_DIM];       /* RSS of the winner from the Gram/Cholesky form */
    int64_t subsets[ORC_MAX_DIM];       /* subsets examined at step t */
} oracle_result;

int oracle_fit(const double* X, const double* y, int N, int d, uint32_t ops, int rung,
               int grammar, int k, int max_dim, int nthreads, oracle_result* out);
/* the same with the SIS threshold (0: top k only) and the "low enough error" stop: after a
   step whose RMSE <= stop_rmse (0: only the exact-fit stop) */
int oracle_fit_ex(const double* X, const double* y, int N, int d, uint32_t ops, int rung,
                  int grammar, const int* units, int k, int max_dim, double sis_threshold, double stop_rmse,
                  int nthreads, oracle_result* out);
/* the same on whitened data (§2.4): W (N x N, row-major; NULL = none) maps the target and
   every candidate column, SISSO then runs on W y and W Phi (the intercept a constant column
   in the transformed space); coefficients, RMSE and R^2 are those of the transformed fit */
int oracle_fit_w(const double* X, const double* y, int N, int d, uint32_t ops, int rung,
                 int grammar, const int* units, const double* W, int k, int max_dim, double sis_threshold,
                 double stop_rmse, int nthreads, oracle_result* out);

#ifdef __cplusplus
}
#endif
#endif
