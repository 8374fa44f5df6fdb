/*
 * sisso_oracle.c — plain, slow FP64 CPU implementation of SISSO (arXiv 2410.01752).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA library is checked against.  It is
 * called by the tests, by the smoke check and by the benchmark's CPU-baseline leg, never
 * by the library.  It shares no code with the CUDA path.  Everything is FP64; threads
 * only split independent loops (candidate ids, first subset index) and the results are
 * merged with the same rule a single thread would apply.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous on these):
 *  - Expansion (§2.1 Eq. 2 and the worked example after it): phi_l = phi_{l-1} U new_l,
 *    new_l = { u(z) : z in new_{l-1} } U { b(z_i, z_j) : z_i, z_j in phi_{l-1}, i != j,
 *    not both in phi_{l-2} }.  +, x and - take i < j (a-b = -(b-a) has the same |rho| and
 *    RSS); / takes both orders.  Grammar NEW_X_PREV replaces, for l >= 3 only, the binary
 *    partner set by one operand in new_{l-1} and the other in phi_{l-2}.
 *  - Canonical id order: level, then operator in table order, then (i, j) lexicographic.
 *  - Validity: a feature is invalid if any value is non-finite or |v| > 1e12, or if its
 *    population std <= 1e-6 * max|v| (near-constant), or if it is identically zero: its
 *    root operator is + or - and max|v| <= 1e-9 * max(|a| + |b|) over the samples (the
 *    operands cancel to rounding noise, e.g. x1 - (x3 + (x1 - x3))).  Validity is
 *    recursive: a feature built from an invalid feature is invalid (§2.1 builds level l
 *    from the features of level l-1; log(x2 * x2^-1), the log of a constant, is not a
 *    feature).  Ids do not depend on validity: the enumeration stays data independent.
 *  - SIS score (§2.2 Eqs. 5-6): Pearson |rho| with population moments; this ranks the
 *    same as |Phi^T y| on standardised columns.  Walk: repeatedly take, among the
 *    remaining candidates whose score is within 1e-9 of the current maximum, the lowest
 *    id.  Skip members of S_{t-1} and duplicates: a candidate whose standardised vector
 *    equals, up to sign, that of an S_{t-1} member or of an id accepted earlier in the
 *    step (max-norm difference <= 1e-8).  Stop after k accepted.
 *  - l0 (§2.3 Eqs. 7-8): intercept always present; centred target y~ = y - mean(y);
 *    standardised features Z; G = Z^T Z / N, b = Z^T y~ / N; per subset a Cholesky of
 *    G_E (pivot <= 1e-12: singular, skipped), RSS = N (y~^T y~/N - |L^-1 b_E|^2).  Winner:
 *    lowest RSS; subsets within 1e-12 * SST of the lowest are tied and the one whose
 *    ascending global-id tuple is lexicographically smallest wins.
 *  - Winner refit: Householder QR on the raw N x (t+1) matrix [1, Phi_E]; coefficients,
 *    RMSE = |y - yhat| / sqrt(N), R^2 = 1 - RSS/SST come from that fit.
 *  - Stop (§2.3, "low enough error"): after a step whose RMSE <= 1e-10 * std(y) (the fit
 *    is exact to FP64 rounding), after a step whose RMSE is at or below the caller's
 *    tolerance (stop_rmse > 0), or when S holds fewer than t features.
 *  - Whitening (§2.4: W = Sigma^-1/2, y~ = W y, Phi~ = W Phi, then SISSO in the transformed
 *    space): every candidate is evaluated on the samples and checked by the rules above
 *    on those raw values; its column is then mapped to W v, and that column must pass the
 *    same finite / cap / near-constant rules.  Scores, standardised vectors, the Gram and
 *    the refit use the whitened columns and the whitened target W y; the intercept stays
 *    a constant column in the transformed space (the paper fits SISSO, intercept included,
 *    to the transformed data), and coefficients, residuals and RMSE are those of that fit.
 *  - Dimensional analysis (§2.1, closing paragraph; §3.3 dimensionality, one unit label per
 *    primary): units are exponent vectors over the labels; + and - need equal units,
 *    exp, log, sin and exp(-.) a dimensionless operand, the other operators combine
 *    units.  A feature that breaks the rule, or is built from one that does, is invalid
 *    (the enumeration and the ids stay those of the space without units).
 *  - Threshold SIS (§2.2, last paragraph: keep the features whose correlation exceeds a
 *    threshold): the score is the same Pearson |rho| as the ranking; the walk runs as
 *    above and ends when the best remaining score is at or below the threshold, or at k
 *    accepted ids (k stays the per-step capacity).
 */
#include "sisso_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define VALUE_CAP 1e12
#define CONST_REL 1e-6
#define SCORE_TIE 1e-9
#define DUP_TOL 1e-8
#define PIVOT_MIN 1e-12
#define RSS_TIE 1e-12
#define STOP_REL 1e-10
#define CANCEL_REL 1e-9

/* ------------------------------------------------------------------------------------ */
/* feature space (§2.1)                                                                  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int d, rung, grammar;
    uint32_t ops;
    int64_t phi[ORC_MAX_RUNG + 1];                 /* |phi_l|, cumulative */
    int64_t sec[ORC_MAX_RUNG + 1][ORC_NOPS];       /* features new at level l by op */
    const int* units;                              /* unit label per primary (-1: none), or NULL */
    const double* W;                               /* whitening matrix (N x N, row-major), or NULL */
} space_t;

/* v <- W v (§2.4); a no-op without whitening */
static void whiten(const space_t* s, int N, double* v) {
    if (!s->W) return;
    double* t = (double*)malloc(sizeof(double) * (size_t)N);
    for (int i = 0; i < N; i++) {
        double acc = 0.0;
        for (int k = 0; k < N; k++) acc += s->W[(size_t)i * N + k] * v[k];
        t[i] = acc;
    }
    memcpy(v, t, sizeof(double) * (size_t)N);
    free(t);
}

static int op_is_binary(int op) { return op <= ORC_DIV; }
static int op_enabled(const space_t* s, int op) { return (s->ops >> op) & 1u; }

/* |phi_{l-1}| and |phi_{l-2}| (the latter 0 for l == 1) */
static int64_t sz_P(const space_t* s, int l) { return s->phi[l - 1]; }
static int64_t sz_Q(const space_t* s, int l) { return l >= 2 ? s->phi[l - 2] : 0; }

int oracle_pair_allowed(int grammar, int level, int op, int64_t i, int64_t j, int64_t P, int64_t Q) {
    if (i < 0 || j < 0 || i >= P || j >= P || i == j) return 0;
    if (op != ORC_DIV && !(i < j)) return 0;
    if (grammar == ORC_GRAMMAR_NEW_X_PREV && level >= 3)
        return (i < Q) != (j < Q);      /* one operand from phi_{l-2}, the other new at l-1 */
    return !(i < Q && j < Q);           /* not both from phi_{l-2}: those pairs already exist */
}

/* the allowed partners j of row i, as up to two half-open ranges */
static int row_ranges(const space_t* s, int l, int op, int64_t i, int64_t lo[2], int64_t hi[2]) {
    int64_t P = sz_P(s, l), Q = sz_Q(s, l);
    int sym = (op != ORC_DIV);
    int n = 0;
    if (s->grammar == ORC_GRAMMAR_NEW_X_PREV && l >= 3) {
        if (i < Q) { lo[0] = Q; hi[0] = P; return P > Q ? 1 : 0; }
        if (sym) return 0;
        lo[0] = 0; hi[0] = Q; return Q > 0 ? 1 : 0;
    }
    if (sym) {
        int64_t a = (i + 1 > Q) ? i + 1 : Q;
        if (a >= P) return 0;
        lo[0] = a; hi[0] = P; return 1;
    }
    if (i < Q) { lo[0] = Q; hi[0] = P; return P > Q ? 1 : 0; }
    if (i > 0) { lo[n] = 0; hi[n] = i; n++; }
    if (i + 1 < P) { lo[n] = i + 1; hi[n] = P; n++; }
    return n;
}

static int64_t row_count(const space_t* s, int l, int op, int64_t i) {
    int64_t lo[2], hi[2], c = 0;
    int n = row_ranges(s, l, op, i, lo, hi);
    for (int r = 0; r < n; r++) c += hi[r] - lo[r];
    return c;
}

static int space_init(space_t* s, int d, uint32_t ops, int rung, int grammar) {
    s->W = NULL;
    if (d < 1 || rung < 0 || rung > ORC_MAX_RUNG) return -1;
    memset(s, 0, sizeof(*s));
    s->d = d; s->ops = ops; s->rung = rung; s->grammar = grammar;
    s->phi[0] = d;
    for (int l = 1; l <= rung; l++) {
        int64_t P = sz_P(s, l), Q = sz_Q(s, l), total = 0;
        for (int op = 0; op < ORC_NOPS; op++) {
            int64_t c = 0;
            if (op_enabled(s, op)) {
                if (op_is_binary(op)) {
                    for (int64_t i = 0; i < P; i++) c += row_count(s, l, op, i);
                } else {
                    c = P - Q;                  /* unary on the features new at l-1 */
                }
            }
            s->sec[l][op] = c;
            total += c;
        }
        s->phi[l] = P + total;
    }
    return 0;
}

int oracle_space_sizes(int d, uint32_t ops, int rung, int grammar, int64_t* sizes_out) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar)) return -1;
    for (int l = 0; l <= rung; l++) sizes_out[l] = s.phi[l];
    return 0;
}

int64_t oracle_section_count(int d, uint32_t ops, int rung, int grammar, int level, int op) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar) || level < 1 || level > rung) return -1;
    return s.sec[level][op];
}

static int decode(const space_t* s, int64_t id, int* level, int* op, int64_t* a, int64_t* b) {
    if (id < 0 || id >= s->phi[s->rung]) return -1;
    if (id < s->d) { *level = 0; *op = -1; *a = id; *b = -1; return 0; }
    int l = 1;
    while (id >= s->phi[l]) l++;
    int64_t r = id - s->phi[l - 1];
    for (int o = 0; o < ORC_NOPS; o++) {
        if (r >= s->sec[l][o]) { r -= s->sec[l][o]; continue; }
        *level = l; *op = o;
        if (!op_is_binary(o)) { *a = sz_Q(s, l) + r; *b = -1; return 0; }
        for (int64_t i = 0; i < sz_P(s, l); i++) {
            int64_t lo[2], hi[2];
            int n = row_ranges(s, l, o, i, lo, hi);
            for (int q = 0; q < n; q++) {
                int64_t w = hi[q] - lo[q];
                if (r < w) { *a = i; *b = lo[q] + r; return 0; }
                r -= w;
            }
        }
        return -2;
    }
    return -3;
}

int oracle_decode(int d, uint32_t ops, int rung, int grammar, int64_t id,
                  int* level, int* op, int64_t* a, int64_t* b) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar)) return -1;
    return decode(&s, id, level, op, a, b);
}

/* ------------------------------------------------------------------------------------ */
/* expression strings and FP64 evaluation                                                */
/* ------------------------------------------------------------------------------------ */

static int expr_rec(const space_t* s, int64_t id, char* buf, int len) {
    int level, op; int64_t a, b;
    if (decode(s, id, &level, &op, &a, &b)) return -1;
    if (level == 0) return snprintf(buf, (size_t)len, "x%lld", (long long)(a + 1));
    char* ea = (char*)malloc(8192);
    char* eb = (char*)malloc(8192);
    int r = -1;
    if (expr_rec(s, a, ea, 8192) >= 0 && (b < 0 || expr_rec(s, b, eb, 8192) >= 0)) {
        switch (op) {
            case ORC_ADD: r = snprintf(buf, (size_t)len, "(%s+%s)", ea, eb); break;
            case ORC_SUB: r = snprintf(buf, (size_t)len, "(%s-%s)", ea, eb); break;
            case ORC_MUL: r = snprintf(buf, (size_t)len, "(%s*%s)", ea, eb); break;
            case ORC_DIV: r = snprintf(buf, (size_t)len, "(%s/%s)", ea, eb); break;
            case ORC_EXP: r = snprintf(buf, (size_t)len, "exp(%s)", ea); break;
            case ORC_LOG: r = snprintf(buf, (size_t)len, "log(%s)", ea); break;
            case ORC_SQRT: r = snprintf(buf, (size_t)len, "sqrt(%s)", ea); break;
            case ORC_SQ: r = snprintf(buf, (size_t)len, "(%s)^2", ea); break;
            case ORC_INV: r = snprintf(buf, (size_t)len, "(%s)^-1", ea); break;
            case ORC_SIN: r = snprintf(buf, (size_t)len, "sin(%s)", ea); break;
            case ORC_CUBE: r = snprintf(buf, (size_t)len, "(%s)^3", ea); break;
            case ORC_EXPNEG: r = snprintf(buf, (size_t)len, "exp(-%s)", ea); break;
        }
    }
    free(ea); free(eb);
    return r;
}

int oracle_expr(int d, uint32_t ops, int rung, int grammar, int64_t id, char* buf, int len) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar)) return -1;
    return expr_rec(&s, id, buf, len);
}

static double apply_unary(int op, double z) {
    switch (op) {
        case ORC_EXP: return exp(z);
        case ORC_LOG: return log(z);
        case ORC_SQRT: return sqrt(z);
        case ORC_SQ: return z * z;
        case ORC_INV: return 1.0 / z;
        case ORC_SIN: return sin(z);
        case ORC_CUBE: return z * z * z;
        case ORC_EXPNEG: return exp(-z);
    }
    return NAN;
}

static double apply_binary(int op, double x, double y) {
    switch (op) {
        case ORC_ADD: return x + y;
        case ORC_SUB: return x - y;
        case ORC_MUL: return x * y;
        case ORC_DIV: return x / y;
    }
    return NAN;
}

/* ------------------------------------------------------------------------------------ */
/* dimensional analysis (§2.1, closing paragraph; §3.3 dimensionality)                   */
/* ------------------------------------------------------------------------------------ */

/* Units of feature id as exponents over the primaries' unit labels (label j is base unit
   j; -1 is dimensionless), in sixteenths so that up to four nested square roots stay
   exact.  Returns 1 if the feature and every operand is dimensionally consistent: + and -
   need operands of equal units, exp, log, sin and exp(-.) a dimensionless operand; the
   other operators combine units (x adds, / subtracts, ^2 ^3 ^-1 sqrt scale the exponents). */
#define UNIT_SCALE 16
static int units_rec(const space_t* s, int64_t id, int* e) {
    int level, op; int64_t a, b;
    if (decode(s, id, &level, &op, &a, &b)) return 0;
    int d = s->d;
    if (level == 0) {
        for (int j = 0; j < d; j++) e[j] = 0;
        int lab = s->units[a];
        if (lab >= 0) e[lab] = UNIT_SCALE;
        return 1;
    }
    int* ea = (int*)malloc(sizeof(int) * (size_t)d);
    int ok = units_rec(s, a, ea);
    if (ok && b >= 0) {
        int* eb = (int*)malloc(sizeof(int) * (size_t)d);
        ok = units_rec(s, b, eb);
        for (int j = 0; ok && j < d; j++) {
            switch (op) {
                case ORC_ADD: case ORC_SUB:
                    if (ea[j] != eb[j]) ok = 0;
                    e[j] = ea[j];
                    break;
                case ORC_MUL: e[j] = ea[j] + eb[j]; break;
                case ORC_DIV: e[j] = ea[j] - eb[j]; break;
            }
        }
        free(eb);
    } else if (ok) {
        for (int j = 0; ok && j < d; j++) {
            switch (op) {
                case ORC_EXP: case ORC_LOG: case ORC_SIN: case ORC_EXPNEG:
                    if (ea[j] != 0) ok = 0;
                    e[j] = 0;
                    break;
                case ORC_SQRT:
                    if (ea[j] % 2) ok = 0;
                    e[j] = ea[j] / 2;
                    break;
                case ORC_SQ: e[j] = 2 * ea[j]; break;
                case ORC_CUBE: e[j] = 3 * ea[j]; break;
                case ORC_INV: e[j] = -ea[j]; break;
            }
        }
    }
    free(ea);
    return ok;
}

static int units_ok(const space_t* s, int64_t id) {
    if (!s->units) return 1;
    int* e = (int*)malloc(sizeof(int) * (size_t)s->d);
    int ok = units_rec(s, id, e);
    free(e);
    return ok;
}

int oracle_units(int d, uint32_t ops, int rung, int grammar, const int* units, int64_t id, int* exps_out) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar) || !units) return -1;
    s.units = units;
    return units_rec(&s, id, exps_out);
}

/* values of feature id at all N samples, recursively from the primaries */
static int eval_rec(const space_t* s, const double* X, int N, int64_t id, double* out) {
    int level, op; int64_t a, b;
    if (decode(s, id, &level, &op, &a, &b)) return -1;
    if (level == 0) {
        for (int i = 0; i < N; i++) out[i] = X[(int64_t)i * s->d + a];
        return 0;
    }
    double* va = (double*)malloc(sizeof(double) * (size_t)N);
    if (eval_rec(s, X, N, a, va)) { free(va); return -1; }
    if (b < 0) {
        for (int i = 0; i < N; i++) out[i] = apply_unary(op, va[i]);
    } else {
        double* vb = (double*)malloc(sizeof(double) * (size_t)N);
        if (eval_rec(s, X, N, b, vb)) { free(va); free(vb); return -1; }
        for (int i = 0; i < N; i++) out[i] = apply_binary(op, va[i], vb[i]);
        free(vb);
    }
    free(va);
    return 0;
}

/* values of feature id and, when its root operator is + or -, whether the operands cancel
   to rounding noise at every sample (an identically zero feature) */
static int eval_checked(const space_t* s, const double* X, int N, int64_t id, double* out, int* cancelled) {
    int level, op; int64_t a, b;
    *cancelled = 0;
    if (decode(s, id, &level, &op, &a, &b)) return -1;
    if (level == 0 || (op != ORC_ADD && op != ORC_SUB)) return eval_rec(s, X, N, id, out);
    double* va = (double*)malloc(sizeof(double) * (size_t)N);
    double* vb = (double*)malloc(sizeof(double) * (size_t)N);
    int rc = eval_rec(s, X, N, a, va) || eval_rec(s, X, N, b, vb);
    double mv = 0.0, mo = 0.0;
    for (int i = 0; i < N && !rc; i++) {
        out[i] = apply_binary(op, va[i], vb[i]);
        if (fabs(out[i]) > mv) mv = fabs(out[i]);
        if (fabs(va[i]) + fabs(vb[i]) > mo) mo = fabs(va[i]) + fabs(vb[i]);
    }
    *cancelled = !rc && mv <= CANCEL_REL * mo;
    free(va); free(vb);
    return rc ? -1 : 0;
}

int oracle_eval(int d, uint32_t ops, int rung, int grammar, const double* X, int N, int64_t id, double* out) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar)) return -1;
    return eval_rec(&s, X, N, id, out);
}

/* ------------------------------------------------------------------------------------ */
/* validity, standardisation, Pearson score (§2.2)                                       */
/* ------------------------------------------------------------------------------------ */

/* mean and population std of v; returns 1 if the feature is valid */
static int moments(const double* v, int N, double* mean, double* sd) {
    double s = 0.0, mx = 0.0;
    for (int i = 0; i < N; i++) {
        if (!isfinite(v[i]) || fabs(v[i]) > VALUE_CAP) return 0;
        s += v[i];
        if (fabs(v[i]) > mx) mx = fabs(v[i]);
    }
    double m = s / N, ss = 0.0;
    for (int i = 0; i < N; i++) ss += (v[i] - m) * (v[i] - m);
    double sdev = sqrt(ss / N);
    *mean = m; *sd = sdev;
    return sdev > CONST_REL * mx;
}

/* |rho(v, t)| with population moments; tc = t - mean(t), tsd = std(t) */
static double pearson(const double* v, int N, double mean, double sd, const double* tc, double tsd) {
    double c = 0.0;
    for (int i = 0; i < N; i++) c += (v[i] - mean) * tc[i];
    return fabs(c) / ((double)N * sd * tsd);
}

/* own rules on the values of feature id (finite, |v| <= 1e12, not identically zero, not
   near-constant), then recursively the same for its operands */
static int valid_rec(const space_t* s, const double* X, int N, int64_t id) {
    int level, op; int64_t a, b;
    if (decode(s, id, &level, &op, &a, &b)) return 0;
    if (!units_ok(s, id)) return 0;
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    double m, sd;
    int cancelled;
    int ok = eval_checked(s, X, N, id, v, &cancelled) == 0 && !cancelled && moments(v, N, &m, &sd);
    free(v);
    if (!ok) return 0;
    if (level == 0) return 1;
    return valid_rec(s, X, N, a) && (b < 0 || valid_rec(s, X, N, b));
}

typedef struct {
    const space_t* s; const double* X; int N;
    const double* tc; double tsd;
    const int64_t* ids; int64_t n_ids;
    double* score; int* valid;
    int64_t begin, end;
} score_job;

static void* score_worker(void* p) {
    score_job* j = (score_job*)p;
    double* v = (double*)malloc(sizeof(double) * (size_t)j->N);
    for (int64_t q = j->begin; q < j->end; q++) {
        int64_t id = j->ids ? j->ids[q] : q;
        double m, sd;
        int cancelled, level, op;
        int64_t a, b;
        int ok = (eval_checked(j->s, j->X, j->N, id, v, &cancelled) == 0) && !cancelled &&
                 moments(v, j->N, &m, &sd) && units_ok(j->s, id);
        if (ok && decode(j->s, id, &level, &op, &a, &b) == 0 && level > 0)
            ok = valid_rec(j->s, j->X, j->N, a) && (b < 0 || valid_rec(j->s, j->X, j->N, b));
        if (ok && j->s->W) {             /* the whitened column passes the same rules */
            whiten(j->s, j->N, v);
            ok = moments(v, j->N, &m, &sd);
        }
        j->valid[q] = ok;
        j->score[q] = ok ? pearson(v, j->N, m, sd, j->tc, j->tsd) : 0.0;
    }
    free(v);
    return NULL;
}

static int default_threads(int nthreads) {
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* centred target and its population std */
static double centre(const double* t, int N, double* tc) {
    double m = 0.0, ss = 0.0;
    for (int i = 0; i < N; i++) m += t[i];
    m /= N;
    for (int i = 0; i < N; i++) { tc[i] = t[i] - m; ss += tc[i] * tc[i]; }
    return sqrt(ss / N);
}

static void scores_threaded(const space_t* s, const double* X, int N, const double* tc, double tsd,
                            const int64_t* ids, int64_t n_ids, double* score, int* valid, int nthreads) {
    nthreads = default_threads(nthreads);
    if (nthreads > n_ids) nthreads = (int)(n_ids > 0 ? n_ids : 1);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    score_job* jobs = (score_job*)malloc(sizeof(score_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) {
        score_job j = { s, X, N, tc, tsd, ids, n_ids, score, valid,
                        n_ids * t / nthreads, n_ids * (t + 1) / nthreads };
        jobs[t] = j;
        pthread_create(&th[t], NULL, score_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th); free(jobs);
}

/* ---- every id at once, level by level ------------------------------------------------
 *
 * Scoring the whole of phi_rung one id at a time re-derives each operand from the
 * primaries.  Here the features of phi_{rung-1} are evaluated once (eval_rec) with their
 * recursive validity (valid_rec) and kept; each feature new at level `rung` is then built
 * from its operands' stored values, walking the sections in canonical id order (operator
 * in table order, then row i, then partner j), the way §2.1 builds level l from level
 * l-1.  Every FP64 operation is the one eval_checked, moments and pearson perform, so the
 * scores and validity flags equal those of the per-id path bit for bit. */

#define LEVEL_TABLE_MAX_BYTES ((size_t)24 << 30)

typedef struct {
    const space_t* s; int N;
    const double* X;
    const double* vals;   /* phi_{rung-1} values, id-major (P x N) */
    int* vok;             /* recursive validity of phi_{rung-1} */
    int* uexp;            /* units of phi_{rung-1} (P x d), when the space has units */
    const double* tc; double tsd;
    double* score; int* valid;
    int tid, nthreads;
} level_job;

/* values and recursive validity of the ids tid, tid + nthreads, ... of phi_{rung-1} */
static void* level_table_worker(void* p) {
    level_job* j = (level_job*)p;
    int64_t P = j->s->phi[j->s->rung - 1];
    for (int64_t id = j->tid; id < P; id += j->nthreads) {
        double* v = (double*)j->vals + (size_t)id * (size_t)j->N;
        j->vok[id] = eval_rec(j->s, j->X, j->N, id, v) == 0 && valid_rec(j->s, j->X, j->N, id);
        if (j->uexp) units_rec(j->s, id, j->uexp + (size_t)id * (size_t)j->s->d);
    }
    return NULL;
}

/* the units rule of a feature new at the top level, from its operands' stored units */
static int binary_units_ok(const level_job* j, int op, int64_t a, int64_t b) {
    if (!j->uexp || (op != ORC_ADD && op != ORC_SUB)) return 1;
    const int d = j->s->d;
    return memcmp(j->uexp + (size_t)a * d, j->uexp + (size_t)b * d, sizeof(int) * (size_t)d) == 0;
}
static int unary_units_ok(const level_job* j, int op, int64_t a) {
    if (!j->uexp || !(op == ORC_EXP || op == ORC_LOG || op == ORC_SIN || op == ORC_EXPNEG)) return 1;
    const int d = j->s->d;
    for (int q = 0; q < d; q++) if (j->uexp[(size_t)a * d + q]) return 0;
    return 1;
}

/* score of the stored feature v (valid flag ok) */
static void score_values(const level_job* j, const double* v, int ok, int64_t id) {
    double m, sd;
    ok = ok && moments(v, j->N, &m, &sd);
    j->valid[id] = ok;
    j->score[id] = ok ? pearson(v, j->N, m, sd, j->tc, j->tsd) : 0.0;
}

static void* level_score_worker(void* p) {
    level_job* j = (level_job*)p;
    const space_t* s = j->s;
    int l = s->rung, N = j->N;
    int64_t P = sz_P(s, l), Q = sz_Q(s, l);
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    /* features of phi_{rung-1}: their stored values */
    for (int64_t id = j->tid; id < P; id += j->nthreads)
        score_values(j, j->vals + (size_t)id * (size_t)N, j->vok[id], id);
    /* features new at level rung: rows (op, i) of binary sections, one row per feature
       of new_{rung-1} for unary sections; row r of the whole level goes to thread r mod n */
    int64_t id0 = P, row = 0;
    for (int op = 0; op < ORC_NOPS; op++) {
        if (s->sec[l][op] == 0) continue;
        if (!op_is_binary(op)) {
            for (int64_t r = 0; r < P - Q; r++, row++) {
                int64_t id = id0 + r, a = Q + r;
                if (row % j->nthreads != j->tid) continue;
                const double* va = j->vals + (size_t)a * (size_t)N;
                for (int q = 0; q < N; q++) v[q] = apply_unary(op, va[q]);
                score_values(j, v, j->vok[a] && unary_units_ok(j, op, a), id);
            }
            id0 += P - Q;
            continue;
        }
        for (int64_t i = 0; i < P; i++, row++) {
            int64_t lo[2], hi[2];
            int nr = row_ranges(s, l, op, i, lo, hi);
            int64_t w = 0;
            for (int q = 0; q < nr; q++) w += hi[q] - lo[q];
            if (row % j->nthreads == j->tid) {
                int64_t id = id0;
                const double* va = j->vals + (size_t)i * (size_t)N;
                for (int q = 0; q < nr; q++) {
                    for (int64_t b = lo[q]; b < hi[q]; b++, id++) {
                        const double* vb = j->vals + (size_t)b * (size_t)N;
                        double mv = 0.0, mo = 0.0;
                        for (int e = 0; e < N; e++) {
                            v[e] = apply_binary(op, va[e], vb[e]);
                            if (fabs(v[e]) > mv) mv = fabs(v[e]);
                            if (fabs(va[e]) + fabs(vb[e]) > mo) mo = fabs(va[e]) + fabs(vb[e]);
                        }
                        int cancelled = (op == ORC_ADD || op == ORC_SUB) && mv <= CANCEL_REL * mo;
                        score_values(j, v, !cancelled && j->vok[i] && j->vok[b] && binary_units_ok(j, op, i, b), id);
                    }
                }
            }
            id0 += w;
        }
    }
    free(v);
    return NULL;
}

/* scores and validity of every id of phi_rung by the level table; returns -1 (nothing
   written) when the table would not fit in LEVEL_TABLE_MAX_BYTES or rung < 1 */
static int scores_all_levelwise(const space_t* s, const double* X, int N, const double* tc, double tsd,
                                double* score, int* valid, int nthreads) {
    if (s->rung < 1 || s->W) return -1;            /* whitened columns: the per-id path */
    int64_t P = s->phi[s->rung - 1];
    if ((size_t)P * (size_t)N > LEVEL_TABLE_MAX_BYTES / sizeof(double)) return -1;
    double* vals = (double*)malloc(sizeof(double) * (size_t)P * (size_t)N);
    int* vok = (int*)malloc(sizeof(int) * (size_t)P);
    int* uexp = s->units ? (int*)calloc((size_t)P * (size_t)s->d, sizeof(int)) : NULL;
    if (!vals || !vok || (s->units && !uexp)) { free(vals); free(vok); free(uexp); return -1; }
    nthreads = default_threads(nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    level_job* jobs = (level_job*)malloc(sizeof(level_job) * (size_t)nthreads);
    for (int phase = 0; phase < 2; phase++) {
        for (int t = 0; t < nthreads; t++) {
            level_job jb = { s, N, X, vals, vok, uexp, tc, tsd, score, valid, t, nthreads };
            jobs[t] = jb;
            pthread_create(&th[t], NULL, phase == 0 ? level_table_worker : level_score_worker, &jobs[t]);
        }
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    }
    free(th); free(jobs); free(vals); free(vok); free(uexp);
    return 0;
}

int oracle_scores_all(int d, uint32_t ops, int rung, int grammar, const int* units, const double* X, int N,
                      const double* target, double* score_out, int* valid_out, int nthreads) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar) || N < 2) return -1;
    s.units = units;
    double* tc = (double*)malloc(sizeof(double) * (size_t)N);
    double tsd = centre(target, N, tc);
    if (!(tsd > 0.0)) { free(tc); return -2; }
    if (scores_all_levelwise(&s, X, N, tc, tsd, score_out, valid_out, nthreads))
        scores_threaded(&s, X, N, tc, tsd, NULL, s.phi[rung], score_out, valid_out, nthreads);
    free(tc);
    return 0;
}

int oracle_scores(int d, uint32_t ops, int rung, int grammar, const double* X, int N,
                  const double* target, const int64_t* ids, int64_t n_ids,
                  double* score_out, int* valid_out, int nthreads) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar) || N < 2) return -1;
    double* tc = (double*)malloc(sizeof(double) * (size_t)N);
    double tsd = centre(target, N, tc);
    if (!(tsd > 0.0)) { free(tc); return -2; }
    scores_threaded(&s, X, N, tc, tsd, ids, n_ids, score_out, valid_out, nthreads);
    free(tc);
    return 0;
}

/* standardised vector z = (v - mean)/sd of a valid feature; returns 0 if valid */
static int standardised(const space_t* s, const double* X, int N, int64_t id, double* z) {
    double m, sd;
    int cancelled;
    if (eval_checked(s, X, N, id, z, &cancelled) || cancelled || !moments(z, N, &m, &sd)) return -1;
    if (s->W) {
        whiten(s, N, z);
        if (!moments(z, N, &m, &sd)) return -1;
    }
    for (int i = 0; i < N; i++) z[i] = (z[i] - m) / sd;
    return 0;
}

static int is_duplicate(const double* za, const double* zb, int N) {
    double dm = 0.0, dp = 0.0;
    for (int i = 0; i < N; i++) {
        double e1 = fabs(za[i] - zb[i]), e2 = fabs(za[i] + zb[i]);
        if (e1 > dm) dm = e1;
        if (e2 > dp) dp = e2;
    }
    return dm <= DUP_TOL || dp <= DUP_TOL;
}

typedef struct { double score; int64_t id; } cand_t;

static int cand_cmp(const void* x, const void* y) {
    const cand_t* a = (const cand_t*)x;
    const cand_t* b = (const cand_t*)y;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    return (a->id < b->id) ? -1 : (a->id > b->id);
}

static int sis_step(const space_t* s, const double* X, int N, const double* target,
                    const int64_t* S_prev, int n_prev, int k, double thr, int64_t* acc, int nthreads) {
    int64_t n_all = s->phi[s->rung];
    double* tc = (double*)malloc(sizeof(double) * (size_t)N);
    double tsd = centre(target, N, tc);
    if (!(tsd > 0.0)) { free(tc); return -2; }
    double* score = (double*)malloc(sizeof(double) * (size_t)n_all);
    int* valid = (int*)malloc(sizeof(int) * (size_t)n_all);
    if (scores_all_levelwise(s, X, N, tc, tsd, score, valid, nthreads))
        scores_threaded(s, X, N, tc, tsd, NULL, n_all, score, valid, nthreads);

    /* candidates: valid and not already in S */
    cand_t* c = (cand_t*)malloc(sizeof(cand_t) * (size_t)n_all);
    int64_t nc = 0;
    for (int64_t id = 0; id < n_all; id++) {
        if (!valid[id]) continue;
        int in_s = 0;
        for (int q = 0; q < n_prev; q++) if (S_prev[q] == id) { in_s = 1; break; }
        if (in_s) continue;
        c[nc].score = score[id]; c[nc].id = id; nc++;
    }
    qsort(c, (size_t)nc, sizeof(cand_t), cand_cmp);

    /* standardised vectors of the S members and of accepted ids, for the duplicate rule */
    double* zref = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(n_prev + k));
    int nref = 0;
    for (int q = 0; q < n_prev; q++) {
        if (standardised(s, X, N, S_prev[q], zref + (size_t)nref * N) == 0) nref++;
    }
    double* zc = (double*)malloc(sizeof(double) * (size_t)N);
    char* removed = (char*)calloc((size_t)(nc > 0 ? nc : 1), 1);
    int n_acc = 0;
    int64_t p = 0;
    while (n_acc < k) {
        while (p < nc && removed[p]) p++;
        if (p >= nc) break;
        double m = c[p].score;
        /* threshold variant (§2.2, last paragraph): only features whose correlation
           exceeds thr; the walk ends when the best remaining score is at or below it */
        if (thr > 0.0 && m <= thr) break;
        int64_t best = p;
        for (int64_t q = p; q < nc && c[q].score >= m - SCORE_TIE; q++)
            if (!removed[q] && c[q].id < c[best].id) best = q;
        removed[best] = 1;
        if (standardised(s, X, N, c[best].id, zc)) continue;
        int dup = 0;
        for (int r = 0; r < nref && !dup; r++) dup = is_duplicate(zc, zref + (size_t)r * N, N);
        if (dup) continue;
        memcpy(zref + (size_t)nref * N, zc, sizeof(double) * (size_t)N);
        nref++;
        acc[n_acc++] = c[best].id;
    }
    free(tc); free(score); free(valid); free(c); free(zref); free(zc); free(removed);
    return n_acc;
}

int oracle_sis_ex(int d, uint32_t ops, int rung, int grammar, const int* units, const double* X, int N,
                  const double* target, const int64_t* S_prev, int n_prev, int k, double thr,
                  int64_t* acc_out, int nthreads) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar) || N < 2 || k < 1 || thr < 0.0) return -1;
    s.units = units;
    return sis_step(&s, X, N, target, S_prev, n_prev, k, thr, acc_out, nthreads);
}

int oracle_sis(int d, uint32_t ops, int rung, int grammar, const double* X, int N,
               const double* target, const int64_t* S_prev, int n_prev, int k,
               int64_t* acc_out, int nthreads) {
    return oracle_sis_ex(d, ops, rung, grammar, NULL, X, N, target, S_prev, n_prev, k, 0.0, acc_out, nthreads);
}

/* ------------------------------------------------------------------------------------ */
/* exhaustive l0 (§2.3)                                                                   */
/* ------------------------------------------------------------------------------------ */

/* RSS of subset pos[0..D-1] by Cholesky of G_E; returns 0 and sets *rss, or -1 if singular */
static int subset_rss(const double* G, const double* b, double syy, int N, int n, int D,
                      const int* pos, double* rss) {
    double L[ORC_MAX_DIM][ORC_MAX_DIM], w[ORC_MAX_DIM];
    for (int j = 0; j < D; j++) {
        double dj = G[(size_t)pos[j] * n + pos[j]];
        for (int m = 0; m < j; m++) dj -= L[j][m] * L[j][m];
        if (dj <= PIVOT_MIN) return -1;
        L[j][j] = sqrt(dj);
        for (int i = j + 1; i < D; i++) {
            double v = G[(size_t)pos[i] * n + pos[j]];
            for (int m = 0; m < j; m++) v -= L[i][m] * L[j][m];
            L[i][j] = v / L[j][j];
        }
    }
    double q = 0.0;
    for (int j = 0; j < D; j++) {
        double v = b[pos[j]];
        for (int m = 0; m < j; m++) v -= L[j][m] * w[m];
        w[j] = v / L[j][j];
        q += w[j] * w[j];
    }
    *rss = (double)N * (syy - q);
    return 0;
}

/* next combination in lexicographic order; returns 0 when exhausted */
static int next_comb(int* pos, int D, int n) {
    int j = D - 1;
    while (j >= 0 && pos[j] == n - D + j) j--;
    if (j < 0) return 0;
    pos[j]++;
    for (int m = j + 1; m < D; m++) pos[m] = pos[m - 1] + 1;
    return 1;
}

/* ascending global-id tuple of a subset */
static void gid_tuple(const int64_t* gid, const int* pos, int D, int64_t* out) {
    for (int j = 0; j < D; j++) out[j] = gid[pos[j]];
    for (int a = 1; a < D; a++)
        for (int c = a; c > 0 && out[c - 1] > out[c]; c--) { int64_t t = out[c]; out[c] = out[c - 1]; out[c - 1] = t; }
}

static int tuple_less(const int64_t* a, const int64_t* b, int D) {
    for (int j = 0; j < D; j++) if (a[j] != b[j]) return a[j] < b[j];
    return 0;
}

typedef struct {
    const double* G; const double* b; double syy; int N, n, D;
    const int64_t* gid;
    int pass;                        /* 1: minimum RSS, 2: tie-broken winner */
    double min_rss, tol;
    int tid, nthreads;               /* this thread takes first positions f = tid mod nthreads */
    /* per-first-position results, indexed by f */
    double* f_rss; int* f_have; int* f_pos; int64_t* f_tuple; int64_t* f_examined;
} l0_job;

static void* l0_worker(void* p) {
    l0_job* j = (l0_job*)p;
    int D = j->D, nf = j->n - D + 1;
    int pos[ORC_MAX_DIM];
    for (int f = j->tid; f < nf; f += j->nthreads) {
        double best = INFINITY;
        int have = 0;
        int64_t examined = 0, tup_best[ORC_MAX_DIM];
        int pos_best[ORC_MAX_DIM];
        for (int m = 0; m < D; m++) pos[m] = f + m;
        do {
            if (pos[0] != f) break;
            examined++;
            double rss;
            if (subset_rss(j->G, j->b, j->syy, j->N, j->n, D, pos, &rss)) continue;
            if (j->pass == 1) {
                if (rss < best) { best = rss; have = 1; }
            } else if (rss <= j->min_rss + j->tol) {
                int64_t tup[ORC_MAX_DIM];
                gid_tuple(j->gid, pos, D, tup);
                if (!have || tuple_less(tup, tup_best, D)) {
                    have = 1; best = rss;
                    memcpy(tup_best, tup, sizeof(int64_t) * (size_t)D);
                    memcpy(pos_best, pos, sizeof(int) * (size_t)D);
                }
            }
        } while (next_comb(pos, D, j->n));
        j->f_rss[f] = best;
        j->f_have[f] = have;
        j->f_examined[f] = examined;
        if (j->pass == 2 && have) {
            memcpy(j->f_pos + (size_t)f * ORC_MAX_DIM, pos_best, sizeof(int) * (size_t)D);
            memcpy(j->f_tuple + (size_t)f * ORC_MAX_DIM, tup_best, sizeof(int64_t) * (size_t)D);
        }
    }
    return NULL;
}

int64_t oracle_l0(const double* G, const double* b, double syy, int N, int n, int D,
                  const int64_t* gid, int* best_pos, double* best_rss, int nthreads) {
    if (D < 1 || D > ORC_MAX_DIM || n < D) return -1;
    int nf = n - D + 1;
    nthreads = default_threads(nthreads);
    if (nthreads > nf) nthreads = nf;
    double* f_rss = (double*)malloc(sizeof(double) * (size_t)nf);
    int* f_have = (int*)calloc((size_t)nf, sizeof(int));
    int* f_pos = (int*)malloc(sizeof(int) * (size_t)nf * ORC_MAX_DIM);
    int64_t* f_tuple = (int64_t*)malloc(sizeof(int64_t) * (size_t)nf * ORC_MAX_DIM);
    int64_t* f_examined = (int64_t*)calloc((size_t)nf, sizeof(int64_t));
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    l0_job* jobs = (l0_job*)malloc(sizeof(l0_job) * (size_t)nthreads);
    double min_rss = INFINITY;
    int64_t examined = 0;
    /* pass 1: the lowest RSS over all subsets; pass 2: among subsets within the tie
       tolerance of it, the smallest ascending global-id tuple */
    for (int pass = 1; pass <= 2; pass++) {
        for (int t = 0; t < nthreads; t++) {
            l0_job jb = { G, b, syy, N, n, D, gid, pass, min_rss, RSS_TIE * (double)N * syy,
                          t, nthreads, f_rss, f_have, f_pos, f_tuple, f_examined };
            jobs[t] = jb;
            pthread_create(&th[t], NULL, l0_worker, &jobs[t]);
        }
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
        if (pass == 1) {
            for (int f = 0; f < nf; f++) {
                examined += f_examined[f];
                if (f_have[f] && f_rss[f] < min_rss) min_rss = f_rss[f];
            }
            if (!isfinite(min_rss)) break;
        }
    }
    int w = -1;
    if (isfinite(min_rss)) {
        for (int f = 0; f < nf; f++) {
            if (!f_have[f]) continue;
            if (w < 0 || tuple_less(f_tuple + (size_t)f * ORC_MAX_DIM, f_tuple + (size_t)w * ORC_MAX_DIM, D)) w = f;
        }
    }
    if (w >= 0) {
        memcpy(best_pos, f_pos + (size_t)w * ORC_MAX_DIM, sizeof(int) * (size_t)D);
        *best_rss = f_rss[w];
    }
    free(f_rss); free(f_have); free(f_pos); free(f_tuple); free(f_examined); free(th); free(jobs);
    return w >= 0 ? examined : -2;
}

/* ------------------------------------------------------------------------------------ */
/* winner refit by Householder QR on [1, Phi_E] and the SISSO iteration (§2.3 Eq. 8)     */
/* ------------------------------------------------------------------------------------ */

/* least squares min |y - A c| for A (N x p, column-major copy), by Householder QR */
static int lstsq_qr(const double* A_in, const double* y_in, int N, int p, double* c) {
    double* A = (double*)malloc(sizeof(double) * (size_t)N * (size_t)p);
    double* y = (double*)malloc(sizeof(double) * (size_t)N);
    memcpy(A, A_in, sizeof(double) * (size_t)N * (size_t)p);
    memcpy(y, y_in, sizeof(double) * (size_t)N);
    int ok = 0;
    for (int j = 0; j < p; j++) {
        double* a = A + (size_t)j * N;
        double nrm = 0.0;
        for (int i = j; i < N; i++) nrm += a[i] * a[i];
        nrm = sqrt(nrm);
        if (nrm == 0.0) { ok = -1; break; }
        double alpha = a[j] > 0 ? -nrm : nrm;        /* v = a - alpha e_j */
        double v0 = a[j] - alpha;
        double vv = v0 * v0;
        for (int i = j + 1; i < N; i++) vv += a[i] * a[i];
        /* apply H = I - 2 v v^T / (v^T v) to the remaining columns and to y */
        for (int k = j + 1; k < p; k++) {
            double* ak = A + (size_t)k * N;
            double s = v0 * ak[j];
            for (int i = j + 1; i < N; i++) s += a[i] * ak[i];
            s = 2.0 * s / vv;
            ak[j] -= s * v0;
            for (int i = j + 1; i < N; i++) ak[i] -= s * a[i];
        }
        double s = v0 * y[j];
        for (int i = j + 1; i < N; i++) s += a[i] * y[i];
        s = 2.0 * s / vv;
        y[j] -= s * v0;
        for (int i = j + 1; i < N; i++) y[i] -= s * a[i];
        a[j] = alpha;                                  /* R(j,j) */
    }
    if (ok == 0) {
        for (int j = p - 1; j >= 0; j--) {             /* back substitution R c = (Q^T y)[0:p] */
            double v = y[j];
            for (int k = j + 1; k < p; k++) v -= A[(size_t)k * N + j] * c[k];
            c[j] = v / A[(size_t)j * N + j];
        }
    }
    free(A); free(y);
    return ok;
}

int oracle_fit(const double* X, const double* y, int N, int d, uint32_t ops, int rung,
               int grammar, int k, int max_dim, int nthreads, oracle_result* out) {
    return oracle_fit_ex(X, y, N, d, ops, rung, grammar, NULL, k, max_dim, 0.0, 0.0, nthreads, out);
}

int oracle_fit_ex(const double* X, const double* y, int N, int d, uint32_t ops, int rung,
                  int grammar, const int* units, int k, int max_dim, double sis_threshold, double stop_rmse,
                  int nthreads, oracle_result* out) {
    return oracle_fit_w(X, y, N, d, ops, rung, grammar, units, NULL, k, max_dim, sis_threshold, stop_rmse,
                        nthreads, out);
}

int oracle_fit_w(const double* X, const double* y_in, int N, int d, uint32_t ops, int rung,
                 int grammar, const int* units, const double* W, int k, int max_dim, double sis_threshold,
                 double stop_rmse, int nthreads, oracle_result* out) {
    space_t s;
    if (space_init(&s, d, ops, rung, grammar) || N < 2 || k < 1 || k > 1024 ||
        max_dim < 1 || max_dim > ORC_MAX_DIM || N < max_dim + 1 || sis_threshold < 0.0 ||
        stop_rmse < 0.0) return -1;
    s.units = units;
    s.W = W;
    /* whitening (§2.4): SISSO on W y and W Phi */
    double* yw = (double*)malloc(sizeof(double) * (size_t)N);
    memcpy(yw, y_in, sizeof(double) * (size_t)N);
    whiten(&s, N, yw);
    const double* y = yw;
    memset(out, 0, sizeof(*out));
    double ybar = 0.0, sst = 0.0;
    for (int i = 0; i < N; i++) ybar += y[i];
    ybar /= N;
    double* yc = (double*)malloc(sizeof(double) * (size_t)N);
    for (int i = 0; i < N; i++) { yc[i] = y[i] - ybar; sst += yc[i] * yc[i]; }
    double syy = sst / N, ysd = sqrt(syy);
    double* target = (double*)malloc(sizeof(double) * (size_t)N);
    memcpy(target, y, sizeof(double) * (size_t)N);
    int64_t* S = out->sis_ids;
    int nS = 0;
    int rc = 0;
    for (int t = 1; t <= max_dim; t++) {
        /* SIS on y (t = 1) or on the best residual of step t-1 */
        int na = sis_step(&s, X, N, target, S, nS, k, sis_threshold, S + nS, nthreads);
        if (na < 0) { rc = (t == 1) ? -3 : 0; break; }
        out->n_sis[t - 1] = na;
        nS += na;
        if (nS < t) break;
        /* standardised S features, Gram and moment vector */
        double* Z = (double*)malloc(sizeof(double) * (size_t)nS * (size_t)N);
        for (int q = 0; q < nS; q++) standardised(&s, X, N, S[q], Z + (size_t)q * N);
        double* G = (double*)malloc(sizeof(double) * (size_t)nS * (size_t)nS);
        double* b = (double*)malloc(sizeof(double) * (size_t)nS);
        for (int p = 0; p < nS; p++) {
            double v = 0.0;
            for (int i = 0; i < N; i++) v += Z[(size_t)p * N + i] * yc[i];
            b[p] = v / N;
            for (int q = 0; q < nS; q++) {
                double g = 0.0;
                for (int i = 0; i < N; i++) g += Z[(size_t)p * N + i] * Z[(size_t)q * N + i];
                G[(size_t)p * nS + q] = g / N;
            }
        }
        int pos[ORC_MAX_DIM];
        double rss_g;
        int64_t ex = oracle_l0(G, b, syy, N, nS, t, S, pos, &rss_g, nthreads);
        free(Z); free(G); free(b);
        if (ex < 0) break;
        /* winner ids in ascending order; refit on the raw features with an intercept */
        int64_t ids[ORC_MAX_DIM];
        for (int j = 0; j < t; j++) ids[j] = S[pos[j]];
        for (int a = 1; a < t; a++)
            for (int c = a; c > 0 && ids[c - 1] > ids[c]; c--) { int64_t tmp = ids[c]; ids[c] = ids[c - 1]; ids[c - 1] = tmp; }
        double* A = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(t + 1));
        for (int i = 0; i < N; i++) A[i] = 1.0;
        for (int j = 0; j < t; j++) {
            eval_rec(&s, X, N, ids[j], A + (size_t)(j + 1) * N);
            whiten(&s, N, A + (size_t)(j + 1) * N);
        }
        double coef[ORC_MAX_DIM + 1];
        if (lstsq_qr(A, y, N, t + 1, coef)) { free(A); rc = -4; break; }
        double rss = 0.0;
        for (int i = 0; i < N; i++) {
            double f = coef[0];
            for (int j = 0; j < t; j++) f += coef[j + 1] * A[(size_t)(j + 1) * N + i];
            target[i] = y[i] - f;                      /* r*_t, the next SIS target */
            rss += target[i] * target[i];
        }
        free(A);
        int di = t - 1;
        memcpy(out->ids[di], ids, sizeof(int64_t) * (size_t)t);
        memcpy(out->coef[di], coef, sizeof(double) * (size_t)(t + 1));
        out->rmse[di] = sqrt(rss / N);
        out->r2[di] = sst > 0 ? 1.0 - rss / sst : 0.0;
        out->rss_gram[di] = rss_g;
        out->subsets[di] = ex;
        out->n_dims = t;
        if (out->rmse[di] <= STOP_REL * ysd) break;    /* exact fit: nothing left to screen */
        /* "low enough error" (§2.3): the caller's RMSE tolerance */
        if (stop_rmse > 0.0 && out->rmse[di] <= stop_rmse) break;
    }
    free(yc); free(target); free(yw);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* pre-screening of the primaries (§3.1; §3.3 initial_screening)                          */
/* ------------------------------------------------------------------------------------ */

#define ORC_PI 3.14159265358979323846

static void mean_var(const double* v, int N, int stride, double* m, double* var) {
    double s = 0.0;
    for (int i = 0; i < N; i++) s += v[(size_t)i * stride];
    double mu = s / N, ss = 0.0;
    for (int i = 0; i < N; i++) { double e = v[(size_t)i * stride] - mu; ss += e * e; }
    *m = mu;
    *var = ss / (N - 1);              /* unbiased, as the KDE bandwidth rule takes it */
}

/* MI(y; x_i) of Eq. (MI) estimated by resubstitution with Gaussian kernel density
   estimates: MI = mean_s log( p(x_s, y_s) / (p(x_s) p(y_s)) ).  Reading: the bandwidths
   follow Scott's rule, the kernel covariance of a d-dimensional estimate being
   N^(-2/(d+4)) times the sample covariance (the joint density uses the full 2 x 2
   covariance of (x_i, y)).  X is N x d row-major; mi_out: d values. */
int oracle_mi_kde(const double* X, int N, int d, const double* y, double* mi_out) {
    if (N < 3 || d < 1) return -1;
    double my, vy;
    mean_var(y, N, 1, &my, &vy);
    double f1 = pow((double)N, -2.0 / 5.0), f2 = pow((double)N, -2.0 / 6.0);
    double hy2 = f1 * vy;
    /* p(y_s) */
    double* py = (double*)malloc(sizeof(double) * (size_t)N);
    for (int s = 0; s < N; s++) {
        double acc = 0.0;
        for (int t = 0; t < N; t++) { double u = y[s] - y[t]; acc += exp(-0.5 * u * u / hy2); }
        py[s] = acc / (N * sqrt(2.0 * ORC_PI * hy2));
    }
    for (int i = 0; i < d; i++) {
        double mx, vx;
        mean_var(X + i, N, d, &mx, &vx);
        double cxy = 0.0;
        for (int s = 0; s < N; s++) cxy += (X[(size_t)s * d + i] - mx) * (y[s] - my);
        cxy /= (N - 1);
        double hx2 = f1 * vx;
        /* joint kernel covariance H = f2 * [[vx, cxy], [cxy, vy]] and its inverse */
        double a = f2 * vx, b = f2 * cxy, c = f2 * vy;
        double det = a * c - b * b;
        if (!(vx > 0.0) || !(det > 0.0)) { free(py); return -2; }
        double ia = c / det, ib = -b / det, ic = a / det;
        double sum = 0.0;
        for (int s = 0; s < N; s++) {
            double xs = X[(size_t)s * d + i], kx = 0.0, kxy = 0.0;
            for (int t = 0; t < N; t++) {
                double u = xs - X[(size_t)t * d + i], v = y[s] - y[t];
                kx += exp(-0.5 * u * u / hx2);
                kxy += exp(-0.5 * (ia * u * u + 2.0 * ib * u * v + ic * v * v));
            }
            double px = kx / (N * sqrt(2.0 * ORC_PI * hx2));
            double pxy = kxy / (N * 2.0 * ORC_PI * sqrt(det));
            sum += log(pxy / (px * py[s]));
        }
        mi_out[i] = sum / N;
    }
    free(py);
    return 0;
}

/* average ranks (1-based; ties share the mean of their positions) of v (stride) */
static void ranks(const double* v, int N, int stride, double* r) {
    for (int s = 0; s < N; s++) {
        int less = 0, equal = 0;
        for (int t = 0; t < N; t++) {
            double a = v[(size_t)s * stride], b = v[(size_t)t * stride];
            if (b < a) less++;
            else if (b == a) equal++;
        }
        r[s] = less + (equal + 1) / 2.0;
    }
}

/* Spearman rank correlation of x_i and y (the Pearson correlation of average ranks) */
int oracle_spearman(const double* X, int N, int d, const double* y, double* rho_out) {
    if (N < 2 || d < 1) return -1;
    double* ry = (double*)malloc(sizeof(double) * (size_t)N);
    double* rx = (double*)malloc(sizeof(double) * (size_t)N);
    ranks(y, N, 1, ry);
    for (int i = 0; i < d; i++) {
        ranks(X + i, N, d, rx);
        double mx = 0.0, my = 0.0;
        for (int s = 0; s < N; s++) { mx += rx[s]; my += ry[s]; }
        mx /= N; my /= N;
        double sxy = 0.0, sxx = 0.0, syy = 0.0;
        for (int s = 0; s < N; s++) {
            sxy += (rx[s] - mx) * (ry[s] - my);
            sxx += (rx[s] - mx) * (rx[s] - mx);
            syy += (ry[s] - my) * (ry[s] - my);
        }
        rho_out[i] = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
    }
    free(rx); free(ry);
    return 0;
}

static int dbl_cmp(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Keep the primaries whose score lies in the top quantile q (0 < q <= 1): score strictly
   above the (1 - q)-quantile of the d scores (linear interpolation between order
   statistics, position (d - 1)(1 - q)); with q = 1 every primary is kept.  Reading of
   §3.3 ("only features with MI inside of this quantile range").  keep_out: d flags;
   returns the number kept. */
int oracle_prescreen_keep(const double* score, int d, double q, int* keep_out) {
    if (d < 1 || !(q > 0.0 && q <= 1.0)) return -1;
    if (q >= 1.0) { for (int i = 0; i < d; i++) keep_out[i] = 1; return d; }
    double* s = (double*)malloc(sizeof(double) * (size_t)d);
    memcpy(s, score, sizeof(double) * (size_t)d);
    qsort(s, (size_t)d, sizeof(double), dbl_cmp);
    double pos = (d - 1) * (1.0 - q);
    int lo = (int)floor(pos);
    double fr = pos - lo;
    double cut = lo + 1 < d ? s[lo] + fr * (s[lo + 1] - s[lo]) : s[lo];
    int n = 0;
    for (int i = 0; i < d; i++) { keep_out[i] = score[i] > cut; n += keep_out[i]; }
    free(s);
    return n;
}
