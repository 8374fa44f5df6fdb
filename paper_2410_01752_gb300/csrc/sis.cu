// sis.cu — sure independence screening (§2.2, Eqs. 5-6) on the device.
//
//  1. k_score_pairs: the fused generate-and-score kernel for the top level's binary
//     sections (almost all of phi_L).  A CTA owns a 32 x 32 tile of operand pairs; for
//     each 32-sample chunk it rebuilds the 64 operand features from the primaries
//     (postfix programs, one warp per feature, lanes over samples) into shared memory,
//     then every thread accumulates, for 4 pairs x 5 operators (+, -, *, a/b, b/a), the
//     shifted sums S1 = sum v', S2 = sum v'^2, SR = sum v' r~ with v' = v - v(sample 0).
//     Nothing but one FP32 score per candidate leaves the CTA.
//  2. k_score_generic: every other id (lower levels, unary sections), thread per id.
//  3. Selection: a 3-pass radix select finds the score of the M-th best candidate, the
//     ids at or above it are compacted, re-scored in FP64 (k_rescore), sorted by
//     (score desc, id asc) and walked by one CTA (k_walk) with the tie and duplicate
//     rules.  The host checks that the k-th accepted FP64 score clears the FP32 cut-off
//     by the FP32 error margin; if not, the window grows and selection repeats.
#include "sis_device.cuh"

#include <algorithm>
#include <map>
#include <cfloat>
#include <cstring>

namespace sg {
namespace {

// ---------------------------------------------------------------------------------
// target moments: one block
// ---------------------------------------------------------------------------------
__global__ void k_prepare_target(const double* __restrict__ t, int N, double* __restrict__ tc64,
                                 float* __restrict__ tc32, TargetStats* st) {
    __shared__ double red[32];
    prepare_target_block(t, N, tc64, tc32, st, red);
}

// FP64 validity of ids [lo, hi) (one level), one warp per id: the value rules (finite,
// |v| <= 1e12, not identically zero, std > 1e-6 max|v|) and the operands' validity
// (lower levels, already computed)
// FP64 values of every id of phi_{L-1}, feature-major (one warp per id, lanes over samples)
__global__ void k_fill_val64(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, int64_t n_ids,
                             double* __restrict__ V) {
    const int64_t id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (id >= n_ids) return;
    Prog p;
    const bool ok = build_prog(*sp, id, p);
    for (int s = lane; s < N; s += 32)
        V[(size_t)id * N + s] = ok ? eval_prog<double>(p, [&](int c) { return Xc[(size_t)c * N + s]; }) : NAN;
}

// the FP64 values of the ids [lo, hi) of one level >= 2 from the stored values of the levels
// below: one operation per sample on the operands' rows, the operation eval_prog applies last
// (a op b, or op(a)), on the values its sub-programs produce, so the values are bitwise those
// of the full programs (one warp per id, lanes over samples)
__global__ void k_fill_val64_level(const Space* __restrict__ sp, int N, int64_t lo, int64_t hi,
                                   double* __restrict__ V) {
    const int64_t id = lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (id >= hi) return;
    int level, op;
    int64_t a, b;
    const bool ok = decode(*sp, id, level, op, a, b) && a >= 0 && a < lo && b < lo;
    double* out = V + (size_t)id * N;
    const double* va = V + (size_t)(ok ? a : 0) * N;
    const double* vb = V + (size_t)(ok && b >= 0 ? b : 0) * N;
    for (int s = lane; s < N; s += 32)
        out[s] = !ok ? NAN : b >= 0 ? op_binary<double>(op, va[s], vb[s]) : op_unary<double>(op, va[s]);
}

// 1/x of every FP64 operand value (the re-score's divisions become products)
__global__ void k_fill_inv64(const double* __restrict__ V, int64_t total, double* __restrict__ inv) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        inv[e] = 1.0 / V[e];
}

__global__ void k_subvalid(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, int64_t lo,
                           int64_t hi, const double* __restrict__ V, const unsigned char* __restrict__ unit_ok,
                           unsigned char* __restrict__ valid) {
    const int64_t id = lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (id >= hi) return;
    int level, op; int64_t a, b;
    Prog p;
    if (!decode(*sp, id, level, op, a, b) || !build_prog(*sp, id, p)) { if (lane == 0) valid[id] = 0; return; }
    if (level > 0 && (!valid[a] || (b >= 0 && !valid[b]))) { if (lane == 0) valid[id] = 0; return; }
    double s = 0.0, mx = 0.0, mo = 0.0;
    int bad = 0;
    const bool addsub = level > 0 && (op == ADD || op == SUB);
    for (int i = lane; i < N; i += 32) {
        double mag;
        double v;
        if (V) {
            v = V[(size_t)id * N + i];
            mag = addsub ? fabs(V[(size_t)a * N + i]) + fabs(V[(size_t)b * N + i]) : fabs(v);
        } else {
            v = eval_prog_mag<double>(p, [&](int c) { return Xc[(size_t)c * N + i]; }, mag);
        }
        if (!isfinite(v) || fabs(v) > kValueCap) bad = 1;
        s += v;
        mx = fmax(mx, fabs(v));
        mo = fmax(mo, mag);
    }
    bad = warp_or(bad);
    s = warp_sum(s);
    mx = warp_max(mx);
    mo = warp_max(mo);
    const double mean = s / N;
    double ss = 0.0;
    if (!bad)
        for (int i = lane; i < N; i += 32) {
            const double v = (V ? V[(size_t)id * N + i] : eval_prog<double>(p, [&](int c) { return Xc[(size_t)c * N + i]; })) - mean;
            ss += v * v;
        }
    ss = warp_sum(ss);
    if (lane == 0) {
        const bool cancelled = root_is_addsub(p) && mx <= kCancelRel * mo;
        valid[id] = !bad && !cancelled && sqrt(ss / N) > kConstRel * mx && (!unit_ok || unit_ok[id]);
    }
}

// ---------------------------------------------------------------------------------
// generic scoring: one thread per id
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void k_score_generic(const Space* __restrict__ sp, const T* __restrict__ Xc, int N, const float* tc32,
                                const double* tc64, const TargetStats* st, int64_t id_lo,
                                int64_t id_hi, const unsigned char* __restrict__ subvalid,
                                float* __restrict__ scores) {
    const int64_t id = id_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= id_hi) return;
    Prog p;
    int level, op; int64_t a, b;
    if (!decode(*sp, id, level, op, a, b) || !build_prog(*sp, id, p)) { scores[id] = -1.f; return; }
    // invalid for certain: ids below the top level carry their exact validity; top-level
    // ids are invalid when an operand is
    const int64_t top0 = sp->phi[sp->rung - 1];
    if (id < top0 ? !subvalid[id] : (!subvalid[a] || (b >= 0 && !subvalid[b]))) { scores[id] = -1.f; return; }
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const T v0 = eval_prog<T>(p, [&](int c) { return Xc[(size_t)c * N]; });
    T s1 = 0, s2 = 0, sr = 0;
    for (int s = 0; s < N; ++s) {
        const T v = eval_prog<T>(p, [&](int c) { return Xc[(size_t)c * N + s]; }) - v0;
        s1 += v;
        s2 = fma(v, v, s2);
        sr = fma(v, tc[s], sr);
    }
    scores[id] = finalize<T>(s1, s2, sr, v0, N, TgtView<T>::sum(st), TgtView<T>::sd(st));
}

// ---------------------------------------------------------------------------------
// operand cache: values of every feature of phi_{L-1} (they do not depend on the target),
// feature-major rows of N samples.  With it, lower-level ids and the top level's unary
// sections score from cached rows, and the pair kernel stages operands by plain loads.
// ---------------------------------------------------------------------------------
// sample-major layout: cache[s * P + id], so that a warp reads 32 consecutive features of
// one sample with one coalesced access.  Values are evaluated in FP64 from the FP64
// primaries and rounded once to T: an operand built by cancellation (x_i - x_j of nearly
// equal columns) keeps its full relative precision, and so does every candidate the top
// level builds from it (1/(x_i - x_j) is then within a few FP32 roundings at every sample).
template <typename T>
__global__ void k_fill_cache_w(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, int64_t n_ids,
                               T* __restrict__ cache) {
    const int64_t id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (id >= n_ids) return;
    Prog p;
    const bool ok = build_prog(*sp, id, p);
    for (int s = lane; s < N; s += 32)
        cache[(size_t)s * n_ids + id] =
            ok ? (T)eval_prog<double>(p, [&](int c) { return Xc[(size_t)c * N + s]; }) : T(NAN);
}

template <typename T>
__global__ void k_fill_cache(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, int64_t n_ids,
                             T* __restrict__ cache) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_ids) return;
    Prog p;
    const bool ok = build_prog(*sp, id, p);
    for (int s = 0; s < N; ++s)
        cache[(size_t)s * n_ids + id] =
            ok ? (T)eval_prog<double>(p, [&](int c) { return Xc[(size_t)c * N + s]; }) : T(NAN);
}

// the same cache as the transpose of the feature-major FP64 values (the same evaluation,
// rounded once to T): 32 x 32 tiles through shared memory, both sides coalesced
template <typename T>
__global__ void k_cache_from_val64(const double* __restrict__ V, int N, int64_t n_ids, T* __restrict__ cache) {
    __shared__ double t[32][33];
    const int64_t id0 = (int64_t)blockIdx.y * 32;
    const int s0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int64_t id = id0 + r;
        const int s = s0 + tx;
        t[r][tx] = id < n_ids && s < N ? V[(size_t)id * N + s] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int s = s0 + r;
        const int64_t id = id0 + tx;
        if (id < n_ids && s < N) cache[(size_t)s * n_ids + id] = (T)t[tx][r];
    }
}

// ids [lo, hi) below the top level (P = |phi_{L-1}| of them) scored from the cache: one
// thread per id, coalesced across the warp for each sample

template <typename T>
__global__ void k_score_cached(const T* __restrict__ cache, int N, int64_t P, const float* tc32,
                               const double* tc64, const TargetStats* st, int64_t lo, int64_t hi,
                               const unsigned char* __restrict__ subvalid, float* __restrict__ scores) {
    const int64_t id = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= hi) return;
    score_cached_id<T>(cache, N, P, tc32, tc64, st, id, subvalid, scores);
}


// the same with one warp per id (few ids, many samples): lanes split the samples
template <typename T>
__global__ void k_score_cached_w(const T* __restrict__ cache, int N, int64_t P, const float* tc32,
                                 const double* tc64, const TargetStats* st, int64_t lo, int64_t hi,
                                 const unsigned char* __restrict__ subvalid, float* __restrict__ scores) {
    const int64_t id = lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (id >= hi) return;
    if (!subvalid[id]) { if (lane == 0) scores[id] = -1.f; return; }
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const T v0 = cache[id];
    T s1 = 0, s2 = 0, sr = 0;
    for (int s = lane; s < N; s += 32) {
        const T v = cache[(size_t)s * P + id] - v0;
        s1 += v;
        s2 = fma(v, v, s2);
        sr = fma(v, tc[s], sr);
    }
    s1 = warp_sum(s1); s2 = warp_sum(s2); sr = warp_sum(sr);
    if (lane == 0) scores[id] = finalize<T>(s1, s2, sr, v0, N, TgtView<T>::sum(st), TgtView<T>::sd(st));
}

// per operand f of phi_{L-1}: A1[f] = sum_s (x_fs - x_f0) and A2[f] = sum_s (x_fs - x_f0)^2
// (when A1ON) and AR[f] = sum_s (x_fs - x_f0) r_s, with r the centred target the pair kernel
// uses.  For + and - the pair kernel's sums of v' = (a - a0) +/- (b - b0), of v'^2 and of v' r
// follow from these and the pair's cross sum sum a' b'.  Products and runs of 32 samples of
// A1 and AR are summed in T (FP32 for the FP32 screening: the FP32 pipe, not the 64x slower
// FP64 one), the runs in FP64; A2 is summed in FP64 from the T values the pair kernel sees
// (the square of an FP32 value is exact in FP64).  A1 and A2 do not depend on the target:
// computed once.
template <typename T, bool A1ON>
__global__ void k_opsums(const T* __restrict__ cache, int N, int64_t P, const float* tc32, const double* tc64,
                         double* __restrict__ A1, double* __restrict__ AR, double* __restrict__ A2) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= P) return;
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const T x0 = cache[f];
    double a = 0.0, ar = 0.0, a2 = 0.0;
    for (int s0 = 0; s0 < N; s0 += 32) {
        const int e = s0 + 32 < N ? s0 + 32 : N;
        T pa = T(0), pr = T(0);
        for (int s = s0; s < e; ++s) {
            const T v = cache[(size_t)s * P + f] - x0;
            if (A1ON) { pa += v; a2 = fma((double)v, (double)v, a2); }
            pr = fma(v, tc[s], pr);
        }
        a += (double)pa;
        ar += (double)pr;
    }
    if (A1ON) { A1[f] = a; A2[f] = a2; }
    AR[f] = ar;
}

// the same with one warp per operand
template <typename T, bool A1ON>
__global__ void k_opsums_w(const T* __restrict__ cache, int N, int64_t P, const float* tc32, const double* tc64,
                           double* __restrict__ A1, double* __restrict__ AR, double* __restrict__ A2) {
    const int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (f >= P) return;
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const T x0 = cache[f];
    T pa = T(0), pr = T(0);
    double a2 = 0.0;
    for (int s = lane; s < N; s += 32) {
        const T v = cache[(size_t)s * P + f] - x0;
        if (A1ON) { pa += v; a2 = fma((double)v, (double)v, a2); }
        pr = fma(v, tc[s], pr);
    }
    const double a = warp_sum((double)pa), ar = warp_sum((double)pr);
    if (A1ON) a2 = warp_sum(a2);
    if (lane == 0) { if (A1ON) { A1[f] = a; A2[f] = a2; } AR[f] = ar; }
}

// the top level's unary sections when operands are few and samples many: one warp per
// (operand, run of samples) computes every enabled operator from the operand's feature-major
// FP64 row (coalesced; rounded to T as the cache is) and leaves its shifted sums (shift: the
// value at sample 0) in part[run][op][operand][3]; k_unary_finish adds the runs in FP64
template <typename T>
__global__ void k_score_unary_runs(UnaryArgs U, const double* __restrict__ val, const float* tc32, const double* tc64,
                                   const unsigned char* __restrict__ subvalid, int runs, double* __restrict__ part) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nz = U.P - U.Q;
    if (w >= nz * runs) return;
    const int run = (int)(w / nz);
    const int64_t z = U.Q + w % nz;
    const int N = U.N;
    const int lo = (int)((int64_t)N * run / runs), hi = (int)((int64_t)N * (run + 1) / runs);
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const double* row = val + (size_t)z * N;
    const bool ok = subvalid[z];
    T v0[kUnaryMax], s1[kUnaryMax], s2[kUnaryMax], sr[kUnaryMax];
    const T x0 = (T)row[0];
#pragma unroll
    for (int k = 0; k < kUnaryMax; ++k) {
        v0[k] = k < U.n_ops ? op_unary<T>(U.op[k], x0) : T(0);
        s1[k] = s2[k] = sr[k] = T(0);
    }
    if (ok)
        for (int s = lo + lane; s < hi; s += 32) {
            const T x = (T)row[s], r = tc[s];
#pragma unroll
            for (int k = 0; k < kUnaryMax; ++k) {
                if (k >= U.n_ops) break;
                const T v = op_unary<T>(U.op[k], x) - v0[k];
                s1[k] += v;
                s2[k] = fma(v, v, s2[k]);
                sr[k] = fma(v, r, sr[k]);
            }
        }
#pragma unroll
    for (int k = 0; k < kUnaryMax; ++k) {
        if (k >= U.n_ops) break;
        const double a = warp_sum((double)s1[k]), b = warp_sum((double)s2[k]), c = warp_sum((double)sr[k]);
        if (lane == 0) {
            double* o = part + (((size_t)run * U.n_ops + k) * nz + (z - U.Q)) * 3;
            o[0] = a; o[1] = b; o[2] = c;
        }
    }
}

template <typename T>
__global__ void k_unary_finish(UnaryArgs U, const double* __restrict__ val, const TargetStats* st,
                               const unsigned char* __restrict__ subvalid, int runs, const double* __restrict__ part,
                               float* __restrict__ scores) {
    const int64_t nz = U.P - U.Q;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nz * U.n_ops) return;
    const int k = (int)(e / nz);
    const int64_t z = U.Q + e % nz;
    if (!subvalid[z]) { scores[U.base[k] + (z - U.Q)] = -1.f; return; }
    double a = 0.0, b = 0.0, c = 0.0;
    for (int run = 0; run < runs; ++run) {
        const double* o = part + (((size_t)run * U.n_ops + k) * nz + (z - U.Q)) * 3;
        a += o[0]; b += o[1]; c += o[2];
    }
    const T v0 = op_unary<T>(U.op[k], (T)val[(size_t)z * U.N]);
    scores[U.base[k] + (z - U.Q)] = finalize<T>((T)a, (T)b, (T)c, v0, U.N, TgtView<T>::sum(st), TgtView<T>::sd(st));
}

// the top level's unary sections from cached operand rows: a CTA takes 32 operands and
// every enabled unary operator (warp w = operator w, lane = operand), 32-sample chunks
// staged in shared memory



// the top level's unary sections: one warp per 32 operands (lane = operand) and every
// enabled operator, reading the sample-major cache directly (coalesced, no staging, no block
// barrier: no warp waits for the slowest operator of another).  Each (operand, operator)
// accumulates its shifted sums over the samples in order, the arithmetic of unary_block.
// STD5: the operators are exp, log, sqrt, ^2, ^-1 in that order, unrolled at compile time.
template <typename T, bool STD5>
__global__ void __launch_bounds__(256)
k_score_unary_w(UnaryArgs U, const T* __restrict__ cache, const float* tc32, const double* tc64,
                const TargetStats* st, const unsigned char* __restrict__ subvalid, float* __restrict__ scores) {
    const int lane = threadIdx.x & 31;
    const int64_t z0 = U.Q + ((((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5);
    if (z0 >= U.P) return;
    const int64_t z = z0 + lane;
    const bool active = z < U.P;
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const int N = U.N;
    constexpr int K = STD5 ? 5 : kUnaryMax;
    constexpr int kStd[5] = {EXP, LOG, SQRT, SQ, INV};
    T v0[K], s1[K], s2[K], sr[K];
    const T x0 = active ? cache[z] : T(1);
#pragma unroll
    for (int o = 0; o < K; ++o) {
        const int op = STD5 ? kStd[o] : (o < U.n_ops ? U.op[o] : EXP);
        v0[o] = op_unary<T>(op, x0);
        s1[o] = s2[o] = sr[o] = T(0);
    }
#pragma unroll 4
    for (int s = 0; s < N; ++s) {
        const T x = active ? cache[(size_t)s * U.P + z] : T(1);
        const T r = tc[s];
#pragma unroll
        for (int o = 0; o < K; ++o) {
            if (!STD5 && o >= U.n_ops) continue;
            const T v = op_unary<T>(STD5 ? kStd[o] : U.op[o], x) - v0[o];
            s1[o] += v;
            s2[o] = fma(v, v, s2[o]);
            sr[o] = fma(v, r, sr[o]);
        }
    }
    if (!active) return;
    const bool ok = subvalid[z];
#pragma unroll
    for (int o = 0; o < K; ++o) {
        if (!STD5 && o >= U.n_ops) continue;
        scores[U.base[o] + (z - U.Q)] = ok ? finalize<T>(s1[o], s2[o], sr[o], v0[o], N, TgtView<T>::sum(st), TgtView<T>::sd(st))
                                           : -1.f;
    }
}

// ---------------------------------------------------------------------------------
// fused generate-and-score for the top level's binary sections
// ---------------------------------------------------------------------------------
constexpr int kCrossMaxN = 4096;      // samples up to which + and - use the cross sum

template <typename T, bool LIN, bool XS = false>
__global__ void __launch_bounds__(NG * 32, sizeof(T) == 4 ? 2 : 1)
k_score_pairs(PairArgs A, const T* __restrict__ Xc, const float* __restrict__ tc32,
              const double* __restrict__ tc64, const TargetStats* __restrict__ st,
              const unsigned char* __restrict__ subvalid, const T* __restrict__ cache,
              const double* __restrict__ A1, const double* __restrict__ AR) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PairSmem<T>& S = *reinterpret_cast<PairSmem<T>*>(smem_raw);
    for (int tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x)
        pair_tile<T, LIN, XS>(A, Xc, tc32, tc64, st, subvalid, cache, A1, AR, S, A.tiles[tile].x, A.tiles[tile].y);
}

// + and - candidates whose key the cross-sum form left open (the pair nearly cancels): the
// direct shifted sum of ((a - a0) +/- (b - b0))^2 over the values the pair kernel stages
// (the FP32 operand cache is the FP64 operand rows rounded once, so the rows are read
// feature-major and rounded here: coalesced), one warp per candidate, lanes over samples
__global__ void k_fix_pm(PairArgs A, const double* __restrict__ V, const TargetStats* __restrict__ st,
                         const double* __restrict__ A1, const double* __restrict__ AR) {
    const unsigned n = min(*A.fix_count, (unsigned)A.fix_cap);
    const int lane = threadIdx.x & 31;
    const float sum_t = TgtView<float>::sum(st), sd_t = TgtView<float>::sd(st);
    for (unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n; e += (gridDim.x * blockDim.x) >> 5) {
        const unsigned long long w = A.fix[e];
        const int o = (int)(w >> 62);
        const int64_t i = (int64_t)((w >> 31) & 0x7FFFFFFFull), j = (int64_t)(w & 0x7FFFFFFFull);
        const double* vi = V + (size_t)i * A.N;
        const double* vj = V + (size_t)j * A.N;
        const float a0 = (float)vi[0], b0 = (float)vj[0];
        float q = 0.f;
        for (int s = lane; s < A.N; s += 32) {
            const float at = (float)vi[s] - a0, bt = (float)vj[s] - b0;
            const float v = o == 0 ? at + bt : at - bt;
            q = fmaf(v, v, q);
        }
        q = warp_sum(q);
        if (lane == 0) {
            const Section& sc = A.sp->sec[A.sec[o]];
            A.scores[sc.base + rank_of(sc, i, j)] =
                o == 0 ? finalize_lin<float>(A1[i] + A1[j], q, AR[i] + AR[j], a0 + b0, A.N, sum_t, sd_t)
                       : finalize_lin<float>(A1[i] - A1[j], q, AR[i] - AR[j], a0 - b0, A.N, sum_t, sd_t);
        }
    }
}

// ---------------------------------------------------------------------------------
// radix select of the M-th largest score, then compaction
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned key_of(float s) { return s > 0.f ? __float_as_uint(s) : 0u; }

// state: [0] prefix bits, [1] remaining count, [2] threshold key, [3] 1 if every
// nonzero key is selected
__global__ void k_hist(const float* __restrict__ scores, int64_t n, int pass,
                       const unsigned* __restrict__ state, unsigned* __restrict__ hist) {
    __shared__ unsigned h[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned prefix = pass ? state[0] : 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = key_of(scores[i]);
        if (k == 0u) continue;
        if (pass == 0) atomicAdd(&h[k >> 20], 1u);
        else if (pass == 1) { if ((k >> 20) == prefix) atomicAdd(&h[(k >> 8) & 0xFFFu], 1u); }
        else { if ((k >> 8) == prefix) atomicAdd(&h[k & 0xFFu], 1u); }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[pass * 4096 + i], h[i]);
}

// the bin, counted from the top, where the running count of keys first reaches the number
// still needed: one CTA of 1024 threads, four bins each, a block-wide prefix sum
constexpr int kFindThreads = 1024;
__global__ void __launch_bounds__(kFindThreads) k_find(const unsigned* __restrict__ hist, int pass, unsigned* state,
                                                       unsigned M) {
    __shared__ unsigned wsum[kFindThreads / 32];
    __shared__ unsigned total;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nb = pass == 2 ? 256 : 4096;
    if (pass > 0 && state[3]) return;                  // uniform: every thread returns
    const unsigned need = pass == 0 ? M : state[1];
    // positions p = 4 t .. 4 t + 3 from the top: bin nb - 1 - p
    unsigned c[4], local = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int p = 4 * t + q;
        c[q] = p < nb ? hist[pass * 4096 + (nb - 1 - p)] : 0u;
        local += c[q];
    }
    // exclusive prefix of local over the threads
    unsigned incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned x = wsum[lane], y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += v;
        }
        wsum[lane] = y - x;                             // exclusive prefix of the warps
        if (lane == 31) total = y;
    }
    __syncthreads();
    unsigned cum = wsum[w] + incl - local;             // keys above this thread's first position
    if (cum < need && cum + local >= need) {           // exactly one thread
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (cum + c[q] >= need) {
                const unsigned b = (unsigned)(nb - 1 - (4 * t + q));
                const unsigned prefix = pass == 0 ? b : pass == 1 ? ((state[0] << 12) | b) : ((state[0] << 8) | b);
                state[0] = prefix;
                state[1] = need - cum;
                if (pass == 2) state[2] = prefix;
                return;
            }
            cum += c[q];
        }
    }
    if (t == 0 && total < need) {                      // fewer than M nonzero keys: take them all
        state[3] = 1u;
        state[2] = 1u;
    }
}

__global__ void k_compact(const float* __restrict__ scores, int64_t n, const unsigned* __restrict__ state,
                          int64_t* __restrict__ out, unsigned* count, int64_t cap) {
    const unsigned thr = state[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = key_of(scores[i]);
        if (k != 0u && k >= thr) {
            const unsigned slot = atomicAdd(count, 1u);
            if (slot < cap) out[slot] = i;
        }
    }
}

// ---------------------------------------------------------------------------------
// FP64 re-score: one warp per id, lanes over samples.  Applies the exact validity rules
// (every |v| <= 1e12 and finite, not identically zero, std > 1e-6 max|v|), computes the
// Pearson score with two passes as the definition does, and keeps the standardised
// vector (zc, when given) and kProbes of its values for the duplicate rule.
// ---------------------------------------------------------------------------------

__global__ void k_rescore(const Space* __restrict__ sp, const double* __restrict__ Xc, int N,
                          const double* __restrict__ tc, const TargetStats* __restrict__ st,
                          const int64_t* __restrict__ ids, int n, const unsigned char* __restrict__ subvalid,
                          const double* __restrict__ V, double* score, double* mean_out, double* sd_out,
                          int* valid_out, double* __restrict__ probe, double* __restrict__ zc,
                          const double* __restrict__ Vinv) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    rescore_one(sp, Xc, N, N, tc, st, ids[w], w, subvalid, V, score, mean_out, sd_out, valid_out, probe, zc, false,
                Vinv);
}

// The same re-score with one CTA of kRescoreThreads per id (many samples): the warp form
// keeps too few independent FP64 chains per SM to cover the pipe's latency.  Sums are
// combined warp by warp in a fixed order.
constexpr int kRescoreThreads = 256;
__global__ void __launch_bounds__(kRescoreThreads)
k_rescore_cta(const Space* __restrict__ sp, int N, const double* __restrict__ tc, const TargetStats* __restrict__ st,
              const int64_t* __restrict__ ids, const unsigned char* __restrict__ subvalid, const double* __restrict__ V,
              const double* __restrict__ Vinv, double* score, double* mean_out, double* sd_out, int* valid_out,
              double* __restrict__ probe, double* __restrict__ zc) {
    constexpr int W = kRescoreThreads / 32;
    __shared__ double red[W][5];
    __shared__ int red_bad[W];
    const int w = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int64_t id = ids[w];
    int level, op; int64_t a, b;
    const int64_t Pbot = sp->phi[sp->rung - 1];
    OpRef ref{};
    bool built = decode(*sp, id, level, op, a, b) && make_opref(*sp, id, ref);
    ref.inv = Vinv;
    if (built && id < Pbot && !subvalid[id]) built = false;
    if (built && id >= Pbot && (!subvalid[a] || (b >= 0 && !subvalid[b]))) built = false;
    if (!built) {
        if (t == 0) { score[w] = -1.0; valid_out[w] = 0; mean_out[w] = 0; sd_out[w] = 0; }
        if (t < kProbes) probe[(size_t)w * kProbes + t] = 0.0;
        return;
    }
    double* z = zc ? zc + (size_t)w * N : nullptr;
    double mag0;
    const double v0 = opref_val(ref, V, N, 0, mag0);
    double s1 = 0.0, s2 = 0.0, sc = 0.0, mx = 0.0, mo = 0.0;
    int bad = 0;
    // one comparison per sample catches non-finite values and the cap; the operands'
    // magnitude (the cancellation rule) only for a top-level + or -
    const bool need_mag = id >= Pbot && (op == ADD || op == SUB);
    auto body = [&](int i, double v, double mag, bool with_mag) {
        const double av = fabs(v);
        if (!(av <= kValueCap)) bad = 1;
        const double u = v - v0;
        s1 += u;
        s2 = fma(u, u, s2);
        sc = fma(u, tc[i], sc);
        mx = fmax(mx, av);
        if (with_mag) mo = fmax(mo, mag);
        if (z) z[i] = v;
    };
    if (need_mag)
        for (int i = t; i < N; i += kRescoreThreads) {
            double mag;
            const double v = opref_val(ref, V, N, i, mag);
            body(i, v, mag, true);
        }
    else
        for (int i = t; i < N; i += kRescoreThreads) {
            double mag;
            const double v = opref_val(ref, V, N, i, mag);
            body(i, v, 0.0, false);
        }
    bad = warp_or(bad);
    s1 = warp_sum(s1); s2 = warp_sum(s2); sc = warp_sum(sc); mx = warp_max(mx); mo = warp_max(mo);
    if (lane == 0) { red[wp][0] = s1; red[wp][1] = s2; red[wp][2] = sc; red[wp][3] = mx; red[wp][4] = mo; red_bad[wp] = bad; }
    __syncthreads();
    s1 = red[0][0]; s2 = red[0][1]; sc = red[0][2]; mx = red[0][3]; mo = red[0][4]; bad = red_bad[0];
    for (int q = 1; q < W; ++q) {
        s1 += red[q][0]; s2 += red[q][1]; sc += red[q][2];
        mx = fmax(mx, red[q][3]); mo = fmax(mo, red[q][4]); bad |= red_bad[q];
    }
    const bool cancelled = need_mag && mx <= kCancelRel * mo;
    const double mean = v0 + s1 / N;
    const double var = s2 / N - (s1 / N) * (s1 / N);
    const double sd = bad || !(var > 0.0) ? 0.0 : sqrt(var);
    const int ok = !bad && !cancelled && sd > kConstRel * mx;
    const double inv = ok ? 1.0 / sd : 0.0;
    if (z) {
        for (int i = t; i < N; i += kRescoreThreads) z[i] = (z[i] - mean) * inv;
        __syncthreads();
    }
    if (t < kProbes) {
        const int i = (int)(((int64_t)t * N) / kProbes);
        double mag;
        probe[(size_t)w * kProbes + t] = z ? z[i] : (opref_val(ref, V, N, i, mag) - mean) * inv;
    }
    if (t == 0) {
        valid_out[w] = ok;
        mean_out[w] = mean;
        sd_out[w] = sd;
        score[w] = ok ? fabs(sc - (s1 / N) * st->tsum) / ((double)N * sd * st->sd) : -1.0;
    }
}

// sort keys: valid survivors not in S (and, with units, dimensionally consistent) get
// their FP64 score, others -1; padding -2
__global__ void k_sort_keys(const int64_t* __restrict__ ids, const double* __restrict__ score,
                            const int* __restrict__ valid, int n, const int64_t* __restrict__ S_sorted,
                            int nS, int n_pad, const unsigned* __restrict__ unit_mask, double* sk, int64_t* sid,
                            int* ssrc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    if (i >= n) { sk[i] = -2.0; sid[i] = INT64_MAX; ssrc[i] = -1; return; }
    const int64_t id = ids[i];
    int lo = 0, hi = nS;            // binary search in S (ascending)
    while (lo < hi) { const int m = (lo + hi) >> 1; if (S_sorted[m] < id) lo = m + 1; else hi = m; }
    const bool inS = lo < nS && S_sorted[lo] == id;
    const bool units = !unit_mask || ((unit_mask[id >> 5] >> (id & 31)) & 1u);
    sk[i] = (valid[i] && !inS && units) ? score[i] : -1.0;
    sid[i] = id;
    ssrc[i] = i;
}

__device__ __forceinline__ bool before(double sa, int64_t ia, double sb, int64_t ib) {
    return sa > sb || (sa == sb && ia < ib);
}

__global__ void k_bitonic(double* sk, int64_t* sid, int* ssrc, int n, int k, int j) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = i ^ j;
    if (l <= i) return;
    const bool up = (i & k) == 0;
    const double si = sk[i], sl = sk[l];
    const int64_t ii = sid[i], il = sid[l];
    const bool swap = up ? before(sl, il, si, ii) : before(si, ii, sl, il);
    if (swap) {
        sk[i] = sl; sk[l] = si;
        sid[i] = il; sid[l] = ii;
        const int t = ssrc[i]; ssrc[i] = ssrc[l]; ssrc[l] = t;
    }
}

// the same network in one CTA's shared memory (windows of up to kSortBlock entries):
// one launch instead of one per stage
constexpr int kSortBlock = 8192;
constexpr size_t kSortSmem = (size_t)kSortBlock * (sizeof(double) + sizeof(int64_t) + sizeof(int));

__global__ void __launch_bounds__(1024) k_sort_block(double* sk, int64_t* sid, int* ssrc, int n) {
    extern __shared__ __align__(16) unsigned char ssm[];
    double* k_ = reinterpret_cast<double*>(ssm);
    int64_t* id_ = reinterpret_cast<int64_t*>(k_ + n);
    int* src_ = reinterpret_cast<int*>(id_ + n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) { k_[i] = sk[i]; id_[i] = sid[i]; src_[i] = ssrc[i]; }
    __syncthreads();
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int l = i ^ j;
                if (l <= i) continue;
                const bool up = (i & k) == 0;
                const double si = k_[i], sl = k_[l];
                const int64_t ii = id_[i], il = id_[l];
                if (up ? before(sl, il, si, ii) : before(si, ii, sl, il)) {
                    k_[i] = sl; k_[l] = si;
                    id_[i] = il; id_[l] = ii;
                    const int t = src_[i]; src_[i] = src_[l]; src_[l] = t;
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) { sk[i] = k_[i]; sid[i] = id_[i]; ssrc[i] = src_[i]; }
}

// ---------------------------------------------------------------------------------
// duplicate rule.  Two features are duplicates when their standardised vectors agree up
// to sign within kDupTol (max norm).  Necessary conditions, checked first: their scores
// differ by at most kDupScore (|rho_a - rho_b| <= |z_a -/+ z_b|_inf) and their kProbes
// probe values agree.  k_dup_find lists, per screened entry, the window entries and S
// members passing both; k_dup_confirm checks every listed pair on all samples; the walk
// then only reads the confirmed pairs.
// ---------------------------------------------------------------------------------
constexpr double kDupScore = 2e-8;
// partner slots confirmed ahead of the walk: a cluster's accepted representative is its
// smallest id, so later members find it in the first slots; with few samples a full check
// costs little and more slots spare the walk its CTA-wide path, with many samples fewer
__host__ __device__ __forceinline__ int n_confirm(int N) { return N <= 8192 ? 8 : 2; }
constexpr int kMaxRefs = 2048;          // slow path: S members / accepted ids gathered per round

__device__ __forceinline__ bool probes_match(const double* a, const double* b) {
    bool same = true, flip = true;
#pragma unroll
    for (int r = 0; r < kProbes; ++r) {
        same = same && fabs(a[r] - b[r]) <= kDupTol;
        flip = flip && fabs(a[r] + b[r]) <= kDupTol;
    }
    return same || flip;
}

// one warp per sorted entry: the lanes test 32 candidates at a time; matches enter the
// partner list in the order the serial rule takes them (S members by position, then window
// entries, whose keys are distinct ids), so the list is the same whatever the lane count
__global__ void k_dup_find(const double* __restrict__ sk, const int* __restrict__ ssrc,
                           const int64_t* __restrict__ sid, int n_sorted,
                           const double* __restrict__ sv_score, const double* __restrict__ sv_sd,
                           const double* __restrict__ probe, int s_off, int nS, int* __restrict__ dup_list,
                           int* __restrict__ dup_cnt) {
    __shared__ int64_t s_key[8][kDupSlots];
    __shared__ int s_val[8][kDupSlots];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= n_sorted) return;
    const double s = sk[i];
    if (s < 0.0) { if (lane == 0) dup_cnt[i] = 0; return; }
    const int src = ssrc[i];
    double pc[kProbes];
#pragma unroll
    for (int r = 0; r < kProbes; ++r) pc[r] = probe[(size_t)src * kProbes + r];
    int64_t* key = s_key[wb];
    int* val = s_val[wb];
    // keep the kDupSlots partners with the smallest keys: S members first (key -1), then
    // window entries by id (a cluster's earliest-visited member is its smallest id)
    int n = 0, total = 0;
    int64_t last = 0;                                    // key[n - 1] once the list is full
    auto offer = [&](bool match, int m, int64_t k) {
        const unsigned all = __ballot_sync(0xffffffffu, match);
        total += __popc(all);
        unsigned b = __ballot_sync(0xffffffffu, match && (n < kDupSlots || k < last));
        while (b) {
            const int l = __ffs(b) - 1;
            b &= b - 1;
            const int64_t kk = __shfl_sync(0xffffffffu, k, l);
            const int mm = __shfl_sync(0xffffffffu, m, l);
            if (n == kDupSlots && kk >= last) continue;
            if (lane == 0) {
                int q = n < kDupSlots ? n : n - 1;
                while (q > 0 && key[q - 1] > kk) { key[q] = key[q - 1]; val[q] = val[q - 1]; --q; }
                key[q] = kk;
                val[q] = mm;
            }
            __syncwarp();
            if (n < kDupSlots) ++n;
            last = key[n - 1];
            __syncwarp();
        }
    };
    for (int q0 = 0; q0 < nS; q0 += 32) {
        const int q = q0 + lane, m = s_off + q;
        const bool c = q < nS && sv_sd[m] > 0.0 && fabs(sv_score[m] - s) <= kDupScore &&
                       probes_match(pc, probe + (size_t)m * kProbes);
        offer(c, m, -1);
    }
    for (int b0 = 0;; b0 += 32) {                        // higher scores (sorted descending)
        const int j = i - 1 - b0 - lane;
        const bool in = j >= 0 && sk[j] - s <= kDupScore;
        const int mj = in ? ssrc[j] : 0;
        offer(in && probes_match(pc, probe + (size_t)mj * kProbes), mj, in ? sid[j] : 0);
        if (__ballot_sync(0xffffffffu, in) != 0xffffffffu) break;
    }
    for (int b0 = 0;; b0 += 32) {                        // lower scores
        const int j = i + 1 + b0 + lane;
        const bool in = j < n_sorted && sk[j] >= 0.0 && s - sk[j] <= kDupScore;
        const int mj = in ? ssrc[j] : 0;
        offer(in && probes_match(pc, probe + (size_t)mj * kProbes), mj, in ? sid[j] : 0);
        if (__ballot_sync(0xffffffffu, in) != 0xffffffffu) break;
    }
    if (lane < n) dup_list[(size_t)i * kDupSlots + lane] = val[lane];
    // overflow: n partners kept, more exist (the walk falls back to a full check)
    if (lane == 0) dup_cnt[i] = total > kDupSlots ? -n - 1 : n;
}

// one warp per sorted entry: every listed partner compared on all samples
__global__ void k_dup_confirm(const Space* __restrict__ sp, const double* __restrict__ Xc, int N,
                              const int* __restrict__ ssrc, const int64_t* __restrict__ sid, int n_sorted,
                              const int64_t* __restrict__ sv_ids, const double* __restrict__ sv_mean,
                              const double* __restrict__ sv_sd, const double* __restrict__ zc,
                              const double* __restrict__ V, const int* __restrict__ dup_list,
                              const int* __restrict__ dup_cnt, unsigned char* __restrict__ dup_ok,
                              const double* __restrict__ Vinv) {
    const int lane = threadIdx.x & 31;
    // one warp per (sorted entry, listed partner)
    for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < (int64_t)n_sorted * kDupSlots;
         wi += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int i = (int)(wi / kDupSlots), q = (int)(wi % kDupSlots);
        const int raw = dup_cnt[i];
        const int cnt = min(raw < 0 ? -raw - 1 : raw, n_confirm(N));
        if (q >= cnt) continue;
        const int src = ssrc[i];
        Prog pc;
        OpRef rc{};
        if (!zc) { if (V) make_opref(*sp, sid[i], rc); else build_prog(*sp, sid[i], pc); }
        rc.inv = Vinv;
        const double mc = sv_mean[src], dc = sv_sd[src];
        {
            const int m = dup_list[(size_t)i * kDupSlots + q];
            Prog pm;
            OpRef rm{};
            if (!zc) { if (V) make_opref(*sp, sv_ids[m], rm); else build_prog(*sp, sv_ids[m], pm); }
            rm.inv = Vinv;
            const double mm = sv_mean[m], dm = sv_sd[m];
            double e1 = 0.0, e2 = 0.0;
            // the pair is a duplicate iff max|za - zb| or max|za + zb| stays within kDupTol:
            // the warp stops as soon as both have exceeded it somewhere (the common case).
            // Cached vectors: four samples per lane per round, so that eight loads are in flight.
            if (zc) {
                const double* pa = zc + (size_t)src * N;
                const double* pb = zc + (size_t)m * N;
                for (int t0 = 0; t0 < N; t0 += 128) {
                    double a4[4], b4[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int t = t0 + 32 * u + lane;
                        a4[u] = t < N ? pa[t] : 0.0;
                        b4[u] = t < N ? pb[t] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        e1 = fmax(e1, fabs(a4[u] - b4[u]));
                        e2 = fmax(e2, fabs(a4[u] + b4[u]));
                    }
                    if (__any_sync(0xffffffffu, e1 > kDupTol) && __any_sync(0xffffffffu, e2 > kDupTol)) break;
                }
            } else
            for (int t0 = 0; t0 < N; t0 += 32) {
                const int t = t0 + lane;
                if (t < N) {
                    double za, zb, mg;
                    if (zc) {
                        za = zc[(size_t)src * N + t];
                        zb = zc[(size_t)m * N + t];
                    } else if (V) {
                        za = (opref_val(rc, V, N, t, mg) - mc) / dc;
                        zb = (opref_val(rm, V, N, t, mg) - mm) / dm;
                    } else {
                        za = (eval_prog<double>(pc, [&](int col) { return Xc[(size_t)col * N + t]; }) - mc) / dc;
                        zb = (eval_prog<double>(pm, [&](int col) { return Xc[(size_t)col * N + t]; }) - mm) / dm;
                    }
                    e1 = fmax(e1, fabs(za - zb));
                    e2 = fmax(e2, fabs(za + zb));
                }
                if (__any_sync(0xffffffffu, e1 > kDupTol) && __any_sync(0xffffffffu, e2 > kDupTol)) break;
            }
            e1 = warp_max(e1);
            e2 = warp_max(e2);
            if (lane == 0) dup_ok[(size_t)i * kDupSlots + q] = (e1 <= kDupTol || e2 <= kDupTol);
        }
    }
}

// ---------------------------------------------------------------------------------
// the walk: one CTA.  Lane 0 of warp 0 picks, among the remaining candidates whose score
// is within kScoreTie of the current maximum, the lowest id; warp 0 then checks the pick's
// listed partners in parallel and accepts it unless a confirmed duplicate of it is an S
// member or an id accepted before it.  Entries whose partner list overflowed are checked by
// the whole CTA against every S member and accepted id.  When the sorted window fits
// (kWalkStage entries), its scores, ids, partner counts and the walk's flags are held in
// shared memory for the walk's dependent reads.
// ---------------------------------------------------------------------------------
constexpr int kWalkThreads = 1024;
constexpr int kHeapCap = 2048;          // tie-window entries held in the shared-memory heap
constexpr int kWalkStage = 4096;        // sorted entries staged in shared memory
constexpr size_t kWalkSmem = (size_t)kWalkStage * (sizeof(double) + sizeof(int64_t) + 2 * sizeof(int) + 2);

__global__ void __launch_bounds__(kWalkThreads)
k_walk(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, const double* __restrict__ sk_g,
       const int64_t* __restrict__ sid_g, const int* __restrict__ ssrc_g, int n_sorted,
       const int64_t* __restrict__ sv_ids, const double* __restrict__ sv_score,
       const double* __restrict__ sv_mean, const double* __restrict__ sv_sd,
       const double* __restrict__ probe, const double* __restrict__ zc, const double* __restrict__ V,
       const int* __restrict__ dup_list, const int* __restrict__ cnt_g, const unsigned char* __restrict__ dup_ok,
       int s_off, int nS, int k, double thr, unsigned char* __restrict__ removed_g,
       unsigned char* __restrict__ accepted_g, WalkResult* out) {
    extern __shared__ __align__(16) unsigned char wsm[];
    __shared__ int acc_src[SISSO_MAX_SIS];
    __shared__ int64_t heap_id[kHeapCap];
    __shared__ int heap_ix[kHeapCap];
    __shared__ int refs[kMaxRefs];
    __shared__ int cur, n_acc, done, exhausted, visited, checks, n_refs, dup_found;
    __shared__ double cur_score, last_score;
    const int tid = threadIdx.x;
    // staged copies (the flags start cleared) or the global arrays
    const bool staged = n_sorted <= kWalkStage && s_off <= kWalkStage;
    const double* sk = sk_g;
    const int64_t* sid = sid_g;
    const int* dup_cnt = cnt_g;
    const int* ssrc = ssrc_g;
    unsigned char* removed = removed_g;
    unsigned char* accepted = accepted_g;
    if (staged) {
        double* s_sk = reinterpret_cast<double*>(wsm);
        int64_t* s_sid = reinterpret_cast<int64_t*>(s_sk + kWalkStage);
        int* s_cnt = reinterpret_cast<int*>(s_sid + kWalkStage);
        int* s_src = s_cnt + kWalkStage;
        unsigned char* s_rem = reinterpret_cast<unsigned char*>(s_src + kWalkStage);
        unsigned char* s_acc = s_rem + kWalkStage;
        for (int q = tid; q < n_sorted; q += blockDim.x) {
            s_sk[q] = sk_g[q];
            s_sid[q] = sid_g[q];
            s_cnt[q] = cnt_g[q];
            s_src[q] = ssrc_g[q];
            s_rem[q] = 0;
        }
        for (int q = tid; q < s_off; q += blockDim.x) s_acc[q] = 0;
        sk = s_sk; sid = s_sid; dup_cnt = s_cnt; ssrc = s_src; removed = s_rem; accepted = s_acc;
    }
    if (tid == 0) {
        n_acc = 0; done = 0; exhausted = 0; visited = 0; checks = 0; last_score = -1.0;
        out->thr_stop = 0;
    }
    // lane 0's state: first remaining entry p, window end e, heap of the window's
    // remaining entries keyed by id (the window only grows as the maximum falls)
    int p = 0, e = 0, hn = 0;
    __syncthreads();
    while (true) {
        if (tid < 32) {
            const int lane = tid;
            while (true) {
                int best = -1, stop = 0;
                if (lane == 0) {
                    while (p < n_sorted && removed[p]) ++p;
                    if (n_acc >= k || p >= n_sorted || sk[p] < 0.0 || (thr > 0.0 && sk[p] <= thr)) {
                        // threshold variant (§2.2): the best remaining score is at or below it
                        if (n_acc < k && p < n_sorted && sk[p] >= 0.0) out->thr_stop = 1;
                        done = 1;
                        exhausted = n_acc < k;
                        stop = 1;
                    } else {
                        const double m = sk[p];
                        if (e < p) e = p;
                        while (e < n_sorted && sk[e] >= 0.0 && sk[e] >= m - kScoreTie) {
                            if (hn == kHeapCap) break;
                            int q = hn++;                          // push (sift up)
                            const int64_t xid = sid[e];
                            while (q > 0 && heap_id[(q - 1) >> 1] > xid) {
                                heap_id[q] = heap_id[(q - 1) >> 1];
                                heap_ix[q] = heap_ix[(q - 1) >> 1];
                                q = (q - 1) >> 1;
                            }
                            heap_id[q] = xid;
                            heap_ix[q] = e;
                            ++e;
                        }
                        if (hn == kHeapCap && e < n_sorted && sk[e] >= 0.0 && sk[e] >= m - kScoreTie) {
                            // window larger than the heap: plain scan (still exact)
                            best = p;
                            for (int q = p; q < n_sorted && sk[q] >= m - kScoreTie; ++q)
                                if (!removed[q] && sid[q] < sid[best]) best = q;
                            // the heap may hold best: drop it lazily (skipped when popped)
                        } else {
                            while (hn > 0) {                       // pop min id (lazy deletion)
                                const int top = heap_ix[0];
                                const int64_t last_id = heap_id[hn - 1];
                                const int last_ix = heap_ix[hn - 1];
                                --hn;
                                int q = 0;
                                while (true) {
                                    int ch = 2 * q + 1;
                                    if (ch >= hn) break;
                                    if (ch + 1 < hn && heap_id[ch + 1] < heap_id[ch]) ++ch;
                                    if (heap_id[ch] >= last_id) break;
                                    heap_id[q] = heap_id[ch];
                                    heap_ix[q] = heap_ix[ch];
                                    q = ch;
                                }
                                if (hn > 0) { heap_id[q] = last_id; heap_ix[q] = last_ix; }
                                if (!removed[top]) { best = top; break; }
                            }
                        }
                        if (best < 0) best = p;
                        removed[best] = 1;
                        cur = best;
                        cur_score = sk[best];
                        last_score = sk[best];
                        ++visited;
                    }
                }
                stop = __shfl_sync(0xffffffffu, stop, 0);
                if (stop) break;
                best = __shfl_sync(0xffffffffu, best, 0);
                __syncwarp();
                // the first reference among the listed partners decides: a confirmed
                // duplicate rejects; a reference beyond the confirmed slots, or partners
                // beyond the list, leave the pick to the full check
                const int raw = dup_cnt[best];
                const int cnt = raw < 0 ? -raw - 1 : raw;
                bool ref = false, okq = false;
                if (lane < cnt) {                          // both reads issued together
                    const int mm = dup_list[(size_t)best * kDupSlots + lane];
                    okq = lane < n_confirm(N) && dup_ok[(size_t)best * kDupSlots + lane] != 0;
                    ref = mm >= s_off || accepted[mm];
                }
                const bool dup = __ballot_sync(0xffffffffu, ref && okq) != 0;
                const bool unknown = raw < 0 || __ballot_sync(0xffffffffu, ref && lane >= n_confirm(N)) != 0;
                if (lane == 0) {
                    checks += cnt;
                    if (!dup && !unknown) {
                        const int src = ssrc[best];
                        accepted[src] = 1;
                        acc_src[n_acc] = src;
                        out->acc[n_acc] = sid[best];
                        ++n_acc;
                    }
                }
                __syncwarp();
                if (!dup && unknown) break;
            }
            if (lane == 0) n_refs = 0;
        }
        __syncthreads();
        if (done) break;
        // slow path: every S member and accepted id that passes the score and probe tests
        // (gathered in parallel), compared on all samples, one warp per reference
        const int c = cur;
        const int csrc = ssrc[c];
        const int64_t cid = sid[c];
        Prog pc;
        OpRef rc{};
        if (!zc) { if (V) make_opref(*sp, cid, rc); else build_prog(*sp, cid, pc); }
        const double mc = sv_mean[csrc], dc = sv_sd[csrc];
        int dupf = 0;
        const int nall = nS + n_acc;
        for (int r0 = 0; r0 < nall && !dupf; r0 += kMaxRefs) {
        if (tid == 0) n_refs = 0;
        __syncthreads();
        for (int q = r0 + tid; q < nall && q < r0 + kMaxRefs; q += blockDim.x) {
            const int src = q < nS ? s_off + q : acc_src[q - nS];
            if (sv_sd[src] > 0.0 && fabs(sv_score[src] - cur_score) <= kDupScore &&
                probes_match(probe + (size_t)csrc * kProbes, probe + (size_t)src * kProbes)) {
                const int slot = atomicAdd(&n_refs, 1);
                refs[slot] = src;
            }
        }
        __syncthreads();
        // one warp per gathered reference, all of them at once; a warp stops at the first
        // sample that rules its pair out both ways, and every warp stops once one has found
        // a duplicate (the outcome is whether any reference is one)
        const int nr = n_refs;
        if (tid == 0) dup_found = 0;
        __syncthreads();
        const int wq = tid >> 5, lq = tid & 31;
        for (int q = wq; q < nr; q += (int)(blockDim.x >> 5)) {
            if (__any_sync(0xffffffffu, *(volatile int*)&dup_found)) break;
            const int src = refs[q];
            Prog pm;
            OpRef rm{};
            if (!zc) { if (V) make_opref(*sp, sv_ids[src], rm); else build_prog(*sp, sv_ids[src], pm); }
            const double mm = sv_mean[src], dm = sv_sd[src];
            double e1 = 0.0, e2 = 0.0;
            for (int t0 = 0; t0 < N; t0 += 32) {
                const int t = t0 + lq;
                if (t < N) {
                    double za, zb, mg;
                    if (zc) {
                        za = zc[(size_t)csrc * N + t];
                        zb = zc[(size_t)src * N + t];
                    } else if (V) {
                        za = (opref_val(rc, V, N, t, mg) - mc) / dc;
                        zb = (opref_val(rm, V, N, t, mg) - mm) / dm;
                    } else {
                        za = (eval_prog<double>(pc, [&](int col) { return Xc[(size_t)col * N + t]; }) - mc) / dc;
                        zb = (eval_prog<double>(pm, [&](int col) { return Xc[(size_t)col * N + t]; }) - mm) / dm;
                    }
                    e1 = fmax(e1, fabs(za - zb));
                    e2 = fmax(e2, fabs(za + zb));
                }
                if (__any_sync(0xffffffffu, e1 > kDupTol) && __any_sync(0xffffffffu, e2 > kDupTol)) break;
            }
            e1 = warp_max(e1);
            e2 = warp_max(e2);
            if (lq == 0) {
                atomicAdd(&checks, 1);
                if (e1 <= kDupTol || e2 <= kDupTol) atomicExch(&dup_found, 1);
            }
        }
        __syncthreads();
        dupf = dup_found;
        __syncthreads();
        }
        if (tid == 0 && !dupf) {
            accepted[csrc] = 1;
            acc_src[n_acc] = csrc;
            out->acc[n_acc] = cid;
            ++n_acc;
        }
        __syncthreads();
    }
    if (tid == 0) {
        out->n_acc = n_acc;
        out->exhausted = exhausted;
        out->visited = visited;
        out->dup_checks = checks;
        out->last_score = last_score;
    }
}

// features' values (n ids) in FP32 or FP64, one warp per id; out is n x N (FP64)
template <typename T>
__global__ void k_eval(const Space* __restrict__ sp, const T* __restrict__ Xc, int N, const int64_t* __restrict__ ids,
                       int64_t n, double* __restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    Prog p;
    const bool ok = build_prog(*sp, ids[w], p);
    for (int s = lane; s < N; s += 32)
        out[w * N + s] = ok ? (double)eval_prog<T>(p, [&](int c) { return Xc[(size_t)c * N + s]; }) : NAN;
}

}  // namespace

// ===================================================================================
// host side
// ===================================================================================

// validity of every id of phi_{L-1}, level by level (operands before their features)
// ---------------------------------------------------------------------------------
// dimensional analysis (§2.1, closing paragraph; §3.3 dimensionality)
// ---------------------------------------------------------------------------------
__global__ void k_apply_unit_mask(const unsigned* __restrict__ mask, int64_t n, float* __restrict__ scores) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!((mask[i >> 5] >> (i & 31)) & 1u)) scores[i] = -1.0f;
}

// one bit per id of phi_L: ids of phi_{L-1} carry their own (recursive) rule; a top-level
// id is consistent when its operands are and its operator's rule holds on their classes
// (+ and -: equal units; exp, log, sin, exp(-.): dimensionless operand)
__global__ void k_unit_mask_build(const Space* __restrict__ sp, int64_t P, int64_t n,
                                  const unsigned char* __restrict__ unit_ok, const int* __restrict__ cls,
                                  int dimless, unsigned* __restrict__ mask) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;     // word
    if (w * 32 >= n) return;
    unsigned bits = 0;
    for (int q = 0; q < 32; ++q) {
        const int64_t id = w * 32 + q;
        if (id >= n) break;
        bool ok;
        if (id < P) {
            ok = unit_ok[id] != 0;
        } else {
            int level, op;
            int64_t a, b;
            ok = decode(*sp, id, level, op, a, b) && unit_ok[a] && (b < 0 || unit_ok[b]);
            if (ok && (op == ADD || op == SUB)) ok = cls[a] == cls[b];
            if (ok && (op == EXP || op == LOG || op == SIN || op == EXPNEG)) ok = cls[a] == dimless;
        }
        bits |= ok ? (1u << q) : 0u;
    }
    mask[w] = bits;
}

// Units of every id of phi_{L-1} on the host (exponent vectors over the labels, in
// sixteenths, interned as classes; a few hundred thousand ids at most), then the bitmask
// of phi_L on the device.  No units: nothing to do.
sisso_status build_units(sisso_ctx* c) {
    if (c->units.empty()) return SISSO_OK;
    const Space& sp = c->space;
    const int64_t P = sp.phi[c->rung - 1], n = c->n_feat;
    const int d = c->d;
    std::map<std::vector<int>, int> classes;
    std::vector<std::vector<int>> vec_of;
    auto intern = [&](const std::vector<int>& e) {
        auto it = classes.find(e);
        if (it != classes.end()) return it->second;
        const int k = (int)vec_of.size();
        classes.emplace(e, k);
        vec_of.push_back(e);
        return k;
    };
    const int dimless = intern(std::vector<int>(d, 0));
    std::vector<int> cls((size_t)P);
    std::vector<unsigned char> ok((size_t)P);
    for (int64_t id = 0; id < P; ++id) {
        int level, op;
        int64_t a, b;
        decode(sp, id, level, op, a, b);
        std::vector<int> e(d, 0);
        bool good = true;
        if (level == 0) {
            if (c->units[a] >= 0) e[c->units[a]] = 16;
        } else {
            const std::vector<int>& ea = vec_of[cls[a]];
            good = ok[a] && (b < 0 || ok[b]);
            for (int j = 0; j < d; ++j) {
                const int x = ea[j], y = b >= 0 ? vec_of[cls[b]][j] : 0;
                switch (op) {
                    case ADD: case SUB: if (x != y) good = false; e[j] = x; break;
                    case MUL: e[j] = x + y; break;
                    case DIV: e[j] = x - y; break;
                    case EXP: case LOG: case SIN: case EXPNEG: if (x != 0) good = false; e[j] = 0; break;
                    case SQRT: if (x % 2) good = false; e[j] = x / 2; break;
                    case SQ: e[j] = 2 * x; break;
                    case CUBE: e[j] = 3 * x; break;
                    default: e[j] = -x; break;      // INV
                }
            }
        }
        cls[(size_t)id] = intern(e);
        ok[(size_t)id] = good ? 1 : 0;
    }
    int* d_cls = nullptr;
    sisso_status st;
    const int64_t words = (n + 31) / 32;
    if ((st = check_cuda(c, cudaMalloc(&c->unit_ok, (size_t)P), "unit_ok")) ||
        (st = check_cuda(c, cudaMalloc(&c->unit_mask, sizeof(unsigned) * (size_t)words), "unit_mask")) ||
        (st = check_cuda(c, cudaMallocAsync(&d_cls, sizeof(int) * (size_t)P, c->stream), "unit classes")))
        return st;
    cudaMemcpyAsync(c->unit_ok, ok.data(), (size_t)P, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_cls, cls.data(), sizeof(int) * (size_t)P, cudaMemcpyHostToDevice, c->stream);
    k_unit_mask_build<<<(int)((words + 255) / 256), 256, 0, c->stream>>>(c->space_dev, P, n, c->unit_ok, d_cls,
                                                                        dimless, c->unit_mask);
    c->stats.launches++;
    cudaFreeAsync(d_cls, c->stream);
    // the host vectors are freed on return: the copies must have left them
    return check_cuda(c, cudaStreamSynchronize(c->stream), "build_units");
}

sisso_status compute_subvalid(sisso_ctx* c) {
    const Space& sp = c->space;
    for (int l = 0; l < sp.rung; ++l) {
        const int64_t lo = l == 0 ? 0 : sp.phi[l - 1], hi = sp.phi[l];
        const int64_t n = hi - lo;
        if (n <= 0) continue;
        k_subvalid<<<(int)((n * 32 + 255) / 256), 256, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, lo, hi,
                                                                       c->opval64, c->unit_ok, c->subvalid);
        c->stats.launches++;
    }
    return check_cuda(c, cudaGetLastError(), "subvalid");
}

sisso_status fill_val64(sisso_ctx* c) {
    if (!c->opval64) return SISSO_OK;
    const int64_t n = c->space.phi[c->rung - 1];
    // levels 0 and 1 from the primaries, every higher level from the one below
    const int64_t n01 = c->rung - 1 >= 1 ? c->space.phi[1] : n;
    k_fill_val64<<<(int)((n01 * 32 + 255) / 256), 256, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, n01, c->opval64);
    c->stats.launches++;
    for (int l = 2; l <= c->rung - 1; ++l) {
        const int64_t lo = c->space.phi[l - 1], hi = c->space.phi[l];
        if (hi <= lo) continue;
        k_fill_val64_level<<<(int)(((hi - lo) * 32 + 255) / 256), 256, 0, c->stream>>>(c->space_dev, c->N, lo, hi,
                                                                                         c->opval64);
        c->stats.launches++;
    }
    if (c->opinv64) {
        const int64_t total = n * (int64_t)c->N;
        k_fill_inv64<<<(int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->sms * 16, (total + 255) / 256)), 256, 0,
                       c->stream>>>(c->opval64, total, c->opinv64);
        c->stats.launches++;
    }
    return check_cuda(c, cudaGetLastError(), "fill_val64");
}

sisso_status fill_opcache(sisso_ctx* c) {
    const int64_t n = c->space.phi[c->rung - 1];
    const bool few = n < 65536;     // few features: a warp per feature splits the samples
    const int grid = few ? (int)((n * 32 + 255) / 256) : (int)((n + 127) / 128);
    const int block = few ? 256 : 128;
    if (c->opval64 && (c->opcache32 || c->opcache64) && (n + 31) / 32 <= 65535) {   // fill_val64 ran first
        const dim3 grid2((unsigned)((c->N + 31) / 32), (unsigned)((n + 31) / 32));
        if (c->opcache32) k_cache_from_val64<float><<<grid2, 256, 0, c->stream>>>(c->opval64, c->N, n, c->opcache32);
        if (c->opcache64) k_cache_from_val64<double><<<grid2, 256, 0, c->stream>>>(c->opval64, c->N, n, c->opcache64);
        c->stats.launches++;
        return check_cuda(c, cudaGetLastError(), "fill_opcache");
    }
    if (c->opcache32) {
        if (few) k_fill_cache_w<float><<<grid, block, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, n, c->opcache32);
        else k_fill_cache<float><<<grid, block, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, n, c->opcache32);
        c->stats.launches++;
    }
    if (c->opcache64) {
        if (few) k_fill_cache_w<double><<<grid, block, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, n, c->opcache64);
        else k_fill_cache<double><<<grid, block, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, n, c->opcache64);
        c->stats.launches++;
    }
    return check_cuda(c, cudaGetLastError(), "fill_opcache");
}

sisso_status prepare_target(sisso_ctx* c, const double* target_dev) {
    k_prepare_target<<<1, 1024, 0, c->stream>>>(target_dev, c->N, c->tc64, c->tc32, c->tstats);
    c->stats.launches++;
    return check_cuda(c, cudaGetLastError(), "prepare_target");
}

// tiles of the top level's pair set (i tile origin, j tile origin), listed j-major: the
// CTAs that run at the same time share j tiles, so each j tile of the operand cache is
// read from DRAM about once (listed i-major, every row of i tiles re-read the whole cache)
void pair_tiles(int64_t P, int64_t Q, bool nxp, std::vector<int2>& tiles) {
    tiles.clear();
    for (int64_t i0 = 0; i0 < P; i0 += TI) {
        if (nxp && i0 >= Q) break;
        int64_t jstart = nxp ? (Q / TJ) * TJ : (i0 / TJ) * TJ;
        if (!nxp && Q > 0) jstart = std::max<int64_t>(jstart, (Q / TJ) * TJ);
        for (int64_t j0 = jstart; j0 < P; j0 += TJ) {
            if (j0 + TJ - 1 <= i0) continue;         // no i < j in the tile
            if (j0 + TJ <= Q) continue;              // no j >= Q
            tiles.push_back(make_int2((int)i0, (int)j0));
        }
    }
    std::stable_sort(tiles.begin(), tiles.end(), [](const int2& a, const int2& b) { return a.y < b.y; });
}

// dimensional analysis: non-physical candidates score -1
void apply_unit_mask(sisso_ctx* c) {
    if (!c->unit_mask) return;
    k_apply_unit_mask<<<std::max(1, std::min(c->sms * 8, (int)((c->n_feat + 255) / 256))), 256, 0, c->stream>>>(
        c->unit_mask, c->n_feat, c->scores);
    c->stats.launches++;
}

sisso_status score_all(sisso_ctx* c, int precision) {
    if (c->Wm) return whiten_score_all(c);       // whitened data (§2.4): scored row by row
    const Space& sp = c->space;
    const int L = sp.rung;
    const bool fp64 = precision == SISSO_PREC_FP64;
    PairArgs A{};
    A.sp = c->space_dev;
    for (int o = 0; o < 4; ++o) A.sec[o] = -1;
    A.P = sp.phi[L - 1];
    A.Q = L >= 2 ? sp.phi[L - 2] : 0;
    A.nxp = sp.grammar == SISSO_GRAMMAR_NEW_X_PREV && L >= 3;
    A.N = c->N;
    A.scores = c->scores;
    // id ranges outside the top level's binary sections go to the generic kernel
    std::vector<std::pair<int64_t, int64_t>> ranges;
    ranges.push_back({0, sp.phi[L - 1]});
    for (int s = 0; s < sp.nsec; ++s) {
        const Section& sc = sp.sec[s];
        if (sc.level == L && sc.op <= DIV) A.sec[sc.op] = s;
        else if (sc.level == L) ranges.push_back({sc.base, sc.base + sc.count});
    }
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
    cudaEventRecord(e0, c->stream);
    const bool cached = fp64 ? c->opcache64 != nullptr : c->opcache32 != nullptr;
    if (cached) {
        // lower levels from cached rows; the top level's unary sections from cached operands
        const int64_t nlow = sp.phi[L - 1];
        const bool few = nlow < 65536;      // few ids: a warp per id splits the samples
        const int gl = few ? (int)((nlow * 32 + 255) / 256) : (int)((nlow + 255) / 256);
        if (fp64) {
            if (few) k_score_cached_w<double><<<gl, 256, 0, c->stream>>>(c->opcache64, c->N, nlow, c->tc32, c->tc64, c->tstats, 0, nlow, c->subvalid, c->scores);
            else k_score_cached<double><<<gl, 256, 0, c->stream>>>(c->opcache64, c->N, nlow, c->tc32, c->tc64, c->tstats, 0, nlow, c->subvalid, c->scores);
        } else {
            if (few) k_score_cached_w<float><<<gl, 256, 0, c->stream>>>(c->opcache32, c->N, nlow, c->tc32, c->tc64, c->tstats, 0, nlow, c->subvalid, c->scores);
            else k_score_cached<float><<<gl, 256, 0, c->stream>>>(c->opcache32, c->N, nlow, c->tc32, c->tc64, c->tstats, 0, nlow, c->subvalid, c->scores);
        }
        c->stats.launches++;
        UnaryArgs U{};
        U.Q = A.Q; U.P = A.P; U.N = c->N;
        for (int q = 0; q < sp.nsec; ++q)
            if (sp.sec[q].level == L && sp.sec[q].op > DIV) { U.op[U.n_ops] = sp.sec[q].op; U.base[U.n_ops] = sp.sec[q].base; ++U.n_ops; }
        if (U.n_ops > 0) {
            const int gu = (int)((A.P - A.Q + 31) / 32);
            if (gu >= 2 * c->sms || !c->opval64) {
                const bool std5 = U.n_ops == 5 && U.op[0] == EXP && U.op[1] == LOG && U.op[2] == SQRT &&
                                  U.op[3] == SQ && U.op[4] == INV;
                const int gb = (gu + 7) / 8;           // eight warps per block, a warp per 32 operands
                if (fp64) {
                    if (std5) k_score_unary_w<double, true><<<gb, 256, 0, c->stream>>>(U, c->opcache64, c->tc32, c->tc64, c->tstats, c->subvalid, c->scores);
                    else k_score_unary_w<double, false><<<gb, 256, 0, c->stream>>>(U, c->opcache64, c->tc32, c->tc64, c->tstats, c->subvalid, c->scores);
                } else {
                    if (std5) k_score_unary_w<float, true><<<gb, 256, 0, c->stream>>>(U, c->opcache32, c->tc32, c->tc64, c->tstats, c->subvalid, c->scores);
                    else k_score_unary_w<float, false><<<gb, 256, 0, c->stream>>>(U, c->opcache32, c->tc32, c->tc64, c->tstats, c->subvalid, c->scores);
                }
            } else {      // few operands: warps over (operand, run of samples)
                const int64_t nz = A.P - A.Q;
                const int runs = (int)std::max<int64_t>(1, std::min<int64_t>((c->N + 1023) / 1024,
                                                                             ((int64_t)c->sms * 32 + nz - 1) / nz));
                double* part = nullptr;
                const sisso_status su = check_cuda(
                    c, cudaMallocAsync((void**)&part, sizeof(double) * 3 * (size_t)runs * U.n_ops * nz, c->stream),
                    "unary partials");
                if (su) return su;
                const int gw = (int)((nz * runs * 32 + 255) / 256), gf = (int)((nz * U.n_ops + 255) / 256);
                if (fp64) {
                    k_score_unary_runs<double><<<gw, 256, 0, c->stream>>>(U, c->opval64, c->tc32, c->tc64, c->subvalid, runs, part);
                    k_unary_finish<double><<<gf, 256, 0, c->stream>>>(U, c->opval64, c->tstats, c->subvalid, runs, part, c->scores);
                } else {
                    k_score_unary_runs<float><<<gw, 256, 0, c->stream>>>(U, c->opval64, c->tc32, c->tc64, c->subvalid, runs, part);
                    k_unary_finish<float><<<gf, 256, 0, c->stream>>>(U, c->opval64, c->tstats, c->subvalid, runs, part, c->scores);
                }
                cudaFreeAsync(part, c->stream);
                c->stats.launches++;
            }
            c->stats.launches++;
        }
    } else {
        for (auto& r : ranges) {
            const int64_t n = r.second - r.first;
            if (n <= 0) continue;
            const int grid = (int)((n + 127) / 128);
            if (fp64)
                k_score_generic<double><<<grid, 128, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, c->tc32, c->tc64, c->tstats, r.first, r.second, c->subvalid, c->scores);
            else
                k_score_generic<float><<<grid, 128, 0, c->stream>>>(c->space_dev, c->Xc32, c->N, c->tc32, c->tc64, c->tstats, r.first, r.second, c->subvalid, c->scores);
            c->stats.launches++;
        }
    }
    sisso_status st = check_cuda(c, cudaGetLastError(), "score_generic");
    if (st) return st;
    cudaEventRecord(e1, c->stream);
    bool any = false;
    for (int o = 0; o < 4; ++o) any |= A.sec[o] >= 0;
    const bool tc = any && c->tc_on && (precision == SISSO_PREC_MIXED_BF16 || precision == SISSO_PREC_MIXED_FP16);
    if (tc) {
        cudaEventRecord(e1, c->stream);
        if ((st = tc_screen_pairs(c, A.sec))) return st;
        c->stats.screen_pair_launches++;
        c->stats.screen_tc = 1;
    } else if (any) {
        std::vector<int2> tiles;
        pair_tiles(A.P, A.Q, A.nxp, tiles);
        int2* d_tiles = nullptr;
        st = check_cuda(c, cudaMallocAsync(&d_tiles, sizeof(int2) * tiles.size(), c->stream), "tiles");
        if (st) return st;
        cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, c->stream);
        A.tiles = d_tiles;
        A.n_tiles = (int)tiles.size();
        const double* A1 = nullptr;
        const double* AR = nullptr;
        if (cached) {
            const bool few = A.P < 65536;
            const int go = few ? (int)((A.P * 32 + 255) / 256) : (int)((A.P + 255) / 256);
            const bool a1 = c->opsum_prec != (fp64 ? 0 : 1);   // A1 of this cache not yet computed
#define SG_OPSUMS(TT, CACHE)                                                                                   \
    do {                                                                                                       \
        if (few) {                                                                                             \
            if (a1) k_opsums_w<TT, true><<<go, 256, 0, c->stream>>>(CACHE, c->N, A.P, c->tc32, c->tc64, c->opsum, c->opsum + A.P, c->opsum + 2 * A.P); \
            else k_opsums_w<TT, false><<<go, 256, 0, c->stream>>>(CACHE, c->N, A.P, c->tc32, c->tc64, c->opsum, c->opsum + A.P, c->opsum + 2 * A.P); \
        } else {                                                                                               \
            if (a1) k_opsums<TT, true><<<go, 256, 0, c->stream>>>(CACHE, c->N, A.P, c->tc32, c->tc64, c->opsum, c->opsum + A.P, c->opsum + 2 * A.P); \
            else k_opsums<TT, false><<<go, 256, 0, c->stream>>>(CACHE, c->N, A.P, c->tc32, c->tc64, c->opsum, c->opsum + A.P, c->opsum + 2 * A.P); \
        }                                                                                                      \
    } while (0)
            if (fp64) SG_OPSUMS(double, c->opcache64);
            else SG_OPSUMS(float, c->opcache32);
#undef SG_OPSUMS
            c->opsum_prec = fp64 ? 0 : 1;
            c->stats.launches++;
            A1 = c->opsum;
            AR = c->opsum + A.P;
        }
        cudaEventRecord(e1, c->stream);
        const int grid = std::min<int>(A.n_tiles, c->sms * 16);
#define SG_PAIRS(TT, LINV, XSV, XC, CACHE)                                                             \
    do {                                                                                                \
        const size_t sm = sizeof(PairSmem<TT>);                                                         \
        cudaFuncSetAttribute(k_score_pairs<TT, LINV, XSV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        k_score_pairs<TT, LINV, XSV><<<grid, NG * 32, sm, c->stream>>>(A, XC, c->tc32, c->tc64, c->tstats,  \
                                                                       c->subvalid, CACHE, A1, AR);     \
    } while (0)
        // FP32 with the operand cache: + and - from the cross sum, the open keys from the
        // direct sums (k_fix_pm); if the open list overflows, the direct kernel again.  The
        // cross sum's rounding bound grows with the number of 32-sample runs: up to 4096
        // samples (128 runs) it leaves open only pairs that nearly cancel, beyond that most
        // keys, so longer problems keep the direct sums
        const bool cross = !fp64 && cached && c->fix_ids && c->opval64 && c->N <= kCrossMaxN;
        if (cross) {
            A.A2 = c->opsum + 2 * A.P;
            A.fix = c->fix_ids; A.fix_count = c->fix_count; A.fix_cap = c->fix_cap;
            cudaMemsetAsync(c->fix_count, 0, sizeof(unsigned), c->stream);
        }
        if (fp64) { if (cached) SG_PAIRS(double, true, false, c->Xc64, c->opcache64); else SG_PAIRS(double, false, false, c->Xc64, c->opcache64); }
        else if (cross) SG_PAIRS(float, true, true, c->Xc32, c->opcache32);
        else { if (cached) SG_PAIRS(float, true, false, c->Xc32, c->opcache32); else SG_PAIRS(float, false, false, c->Xc32, c->opcache32); }
        c->stats.launches++;
        c->stats.screen_pair_launches++;
        if (cross) {
            k_fix_pm<<<c->sms * 4, 256, 0, c->stream>>>(A, c->opval64, c->tstats, A1, AR);
            c->stats.launches++;
            unsigned h_fix = 0;
            cudaMemcpyAsync(&h_fix, c->fix_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
            if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "score_pairs cross"))) {
                cudaFreeAsync(d_tiles, c->stream);
                return st;
            }
            c->stats.pm_keys_direct += (int64_t)h_fix;
            if (h_fix > (unsigned)c->fix_cap) {
                SG_PAIRS(float, true, false, c->Xc32, c->opcache32);
                c->stats.launches++;
                c->stats.screen_pair_launches++;
            }
        }
#undef SG_PAIRS
        st = check_cuda(c, cudaGetLastError(), "score_pairs");
        cudaFreeAsync(d_tiles, c->stream);
        if (st) return st;
    }
    cudaEventRecord(e2, c->stream);
    apply_unit_mask(c);
    cudaEvent_t e3;
    cudaEventCreate(&e3);
    cudaEventRecord(e3, c->stream);
    cudaEventSynchronize(e3);
    if (tc && (st = tc_screen_status(c))) return st;
    c->stats.ms_screen += event_ms(e0, e3);
    c->stats.ms_screen_pair += event_ms(e1, e2);
    cudaEventDestroy(e3);
    c->stats.candidates_scored += c->n_feat;
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
    return SISSO_OK;
}

sisso_status eval_features(sisso_ctx* c, const int64_t* ids_dev, int64_t n, int precision, double* out_dev) {
    const int grid = (int)((n * 32 + 255) / 256);
    if (precision == SISSO_PREC_FP64)
        k_eval<double><<<grid, 256, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, ids_dev, n, out_dev);
    else
        k_eval<float><<<grid, 256, 0, c->stream>>>(c->space_dev, c->Xc32, c->N, ids_dev, n, out_dev);
    c->stats.launches++;
    return check_cuda(c, cudaGetLastError(), "eval_features");
}

// One SIS step on the scores already in c->scores (against the target prepared by
// prepare_target).  S_prev_host: S_{t-1} in acceptance order.
sisso_status sis_select(sisso_ctx* c, int k, const int64_t* S_prev_host, int n_prev,
                        std::vector<int64_t>& acc) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    sisso_status st = SISSO_OK;
    // S, ascending, for membership tests; S in order after the survivors for re-scoring
    std::vector<int64_t> Ss(S_prev_host, S_prev_host + n_prev);
    std::sort(Ss.begin(), Ss.end());
    if (n_prev > 0)
        cudaMemcpyAsync(c->S_sorted, Ss.data(), sizeof(int64_t) * n_prev, cudaMemcpyHostToDevice, c->stream);
    const bool fp_kernel64 = c->opts.precision == SISSO_PREC_FP64;
    const double eps = fp_kernel64 ? kScoreErr64 : kScoreErr32;   // bound on |score_kernel - score_FP64|
    // default window: max(4096, 32 k) candidates, but at most about 2^26 sample evaluations of
    // FP64 re-scoring (the re-score costs M x N) and never below 5 k
    int64_t M = c->opts.survivors > 0
                    ? c->opts.survivors
                    : std::max<int64_t>(5LL * k, std::min<int64_t>(std::max<int64_t>(4096, 32LL * k), (1LL << 26) / c->N));
    const int64_t n = c->n_feat;
    const int gridS = std::max(1, c->sms * 8);
    cudaEvent_t q[5];
    for (auto& e : q) cudaEventCreate(&e);
    while (true) {
        M = std::min<int64_t>(M, c->surv_cap - n_prev);
        cudaEventRecord(q[0], c->stream);
        cudaMemsetAsync(c->hist, 0, sizeof(unsigned) * 3 * 4096, c->stream);
        cudaMemsetAsync(c->sel_state, 0, sizeof(unsigned) * 4, c->stream);
        cudaMemsetAsync(c->surv_count, 0, sizeof(unsigned), c->stream);
        for (int pass = 0; pass < 3; ++pass) {
            k_hist<<<gridS, kBlock, 0, c->stream>>>(c->scores, n, pass, c->sel_state, c->hist);
            k_find<<<1, kFindThreads, 0, c->stream>>>(c->hist, pass, c->sel_state, (unsigned)M);
            c->stats.launches += 2;
        }
        k_compact<<<gridS, kBlock, 0, c->stream>>>(c->scores, n, c->sel_state, c->surv_ids, c->surv_count,
                                                   c->surv_cap - n_prev);
        c->stats.launches++;
        unsigned h_state[4], h_count = 0;
        cudaMemcpyAsync(h_state, c->sel_state, sizeof(h_state), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(&h_count, c->surv_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
        if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "select"))) break;
        if ((int64_t)h_count > c->surv_cap - n_prev) {
            st = fail(c, SISSO_ERR_CAPACITY, "screening window overflow (tied scores)");
            break;
        }
        const int ns = (int)h_count;
        const bool all = h_state[3] != 0;
        float t32 = 0.f;
        if (!all) std::memcpy(&t32, &h_state[2], sizeof(float));
        // re-score survivors and S members in FP64
        if (n_prev > 0)
            cudaMemcpyAsync(c->surv_ids + ns, S_prev_host, sizeof(int64_t) * n_prev, cudaMemcpyHostToDevice, c->stream);
        const int nr = ns + n_prev;
        cudaEventRecord(q[1], c->stream);
        double* zc = (int64_t)nr <= c->zcap ? c->zcache : nullptr;   // cache the vectors if they fit
        if (c->Wm) {            // whitened data: every window vector cached (checked at creation)
            if (!zc) { st = fail(c, SISSO_ERR_CAPACITY, "whitened window exceeds the vector cache"); break; }
            if ((st = whiten_rescore(c, c->surv_ids, nr, c->surv_score, c->surv_mean, c->surv_sd, c->surv_valid,
                                     c->surv_probe, zc)))
                break;
        } else if (c->opval64 && c->N >= 4096 && nr > 0)
            k_rescore_cta<<<nr, kRescoreThreads, 0, c->stream>>>(c->space_dev, c->N, c->tc64, c->tstats, c->surv_ids,
                                                                 c->subvalid, c->opval64, c->opinv64, c->surv_score,
                                                                 c->surv_mean, c->surv_sd, c->surv_valid,
                                                                 c->surv_probe, zc);
        else
            k_rescore<<<(nr * 32 + 255) / 256, 256, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, c->tc64, c->tstats,
                                                                     c->surv_ids, nr, c->subvalid, c->opval64,
                                                                     c->surv_score, c->surv_mean, c->surv_sd,
                                                                     c->surv_valid, c->surv_probe, zc, c->opinv64);
        int n_pad = 1;
        while (n_pad < std::max(ns, 1)) n_pad <<= 1;
        k_sort_keys<<<(n_pad + 255) / 256, 256, 0, c->stream>>>(c->surv_ids, c->surv_score, c->surv_valid, ns,
                                                                 c->S_sorted, n_prev, n_pad, c->unit_mask,
                                                                 c->sort_score, c->sort_id, c->sort_src);
        c->stats.launches += 2;
        cudaEventRecord(q[2], c->stream);
        if (n_pad <= kSortBlock) {
            const size_t sm = (size_t)n_pad * (sizeof(double) + sizeof(int64_t) + sizeof(int));
            cudaFuncSetAttribute(k_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
            k_sort_block<<<1, 1024, sm, c->stream>>>(c->sort_score, c->sort_id, c->sort_src, n_pad);
            c->stats.launches++;
        } else {
            for (int kk = 2; kk <= n_pad; kk <<= 1)
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    k_bitonic<<<(n_pad + 255) / 256, 256, 0, c->stream>>>(c->sort_score, c->sort_id, c->sort_src, n_pad, kk,
                                                                          j);
                    c->stats.launches++;
                }
        }
        cudaEventRecord(q[3], c->stream);
        cudaMemsetAsync(c->removed, 0, (size_t)n_pad, c->stream);
        cudaMemsetAsync(c->accepted, 0, (size_t)ns, c->stream);
        k_dup_find<<<(int)(((int64_t)n_pad * 32 + 255) / 256), 256, 0, c->stream>>>(c->sort_score, c->sort_src, c->sort_id, n_pad, c->surv_score,
                                                               c->surv_sd, c->surv_probe, ns, n_prev, c->dup_list,
                                                               c->dup_cnt);
        k_dup_confirm<<<(int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->sms * 32, ((int64_t)n_pad * kDupSlots * 32 + 255) / 256)), 256, 0, c->stream>>>(
            c->space_dev, c->Xc64, c->N, c->sort_src, c->sort_id, n_pad, c->surv_ids, c->surv_mean, c->surv_sd, zc,
            c->opval64, c->dup_list, c->dup_cnt, c->dup_ok, c->opinv64);
        cudaFuncSetAttribute(k_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWalkSmem);
        const size_t wsm = n_pad <= kWalkStage && ns <= kWalkStage ? kWalkSmem : 0;
        k_walk<<<1, kWalkThreads, wsm, c->stream>>>(c->space_dev, c->Xc64, c->N, c->sort_score, c->sort_id, c->sort_src,
                                                  n_pad, c->surv_ids, c->surv_score, c->surv_mean, c->surv_sd,
                                                  c->surv_probe, zc, c->opval64, c->dup_list, c->dup_cnt, c->dup_ok,
                                                  ns, n_prev, k, c->opts.sis_threshold, c->removed, c->accepted,
                                                  c->walk);
        c->stats.launches += 3;
        cudaEventRecord(q[4], c->stream);
        cudaMemcpyAsync(c->walk_h, c->walk, sizeof(WalkResult), cudaMemcpyDeviceToHost, c->stream);
        if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "walk"))) break;
        c->stats.ms_radix += event_ms(q[0], q[1]);
        c->stats.ms_rescore += event_ms(q[1], q[2]);
        c->stats.ms_sort += event_ms(q[2], q[3]);
        c->stats.ms_walk += event_ms(q[3], q[4]);
        c->stats.walk_visited += c->walk_h->visited;
        c->stats.walk_dup_checks += c->walk_h->dup_checks;
        c->stats.survivors_rescored += nr;
        const WalkResult& w = *c->walk_h;
        // exact iff every candidate outside the window scores (FP64) below the last
        // accepted one by more than the tie tolerance, or, when the walk ended at the SIS
        // threshold, below the threshold by more than the tie tolerance (no outside
        // candidate could be picked above it, nor tie with a pick)
        const double thr = c->opts.sis_threshold;
        const bool safe = all || (w.n_acc == k && w.last_score - kScoreTie > (double)t32 + eps) ||
                          (w.thr_stop && (double)t32 + eps < thr - kScoreTie);
        const bool can_grow = M < c->surv_cap - n_prev;
        if (safe || !can_grow) {
            if (!safe) c->stats.window_saturated = 1;
            acc.assign(w.acc, w.acc + w.n_acc);
            break;
        }
        M *= 4;
        c->stats.window_grown++;
    }
    for (auto& e : q) cudaEventDestroy(e);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    c->stats.ms_select += event_ms(e0, e1);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    return st;
}

}  // namespace sg
