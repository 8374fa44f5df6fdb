// sis_device.cuh — device building blocks of the screening kernels, shared by the
// per-problem kernels (sis.cu) and the persistent multi-task kernel (batch.cu).
#pragma once

#include "common.cuh"

#include <type_traits>

namespace sg {
namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_or(int v) { return __any_sync(0xffffffffu, v); }

// sum over a block of blockDim.x threads (multiple of 32); result valid in all threads
template <typename T> __device__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T r = 0;
    for (int i = 0; i < nw; ++i) r += red[i];
    __syncthreads();
    return r;
}
template <typename T> __device__ T block_max(T v, T* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T r = red[0];
    for (int i = 1; i < nw; ++i) r = max(r, red[i]);
    __syncthreads();
    return r;
}

// score from shifted sums (v' = v - v0): Pearson |rho| with population moments, or -1
// when the feature is certainly invalid.  The exact validity rule (every |v| <= 1e12,
// std > 1e-6 max|v|) is applied by the FP64 re-score; here a feature is rejected only
// if it must fail it (non-finite sums, |v0| > 1e12, std <= 1e-6 max(|v0|, |mean|)).
template <typename T>
__device__ __forceinline__ float finalize(T s1, T s2, T sr, T v0, int N, T sum_t, T sd_t) {
    const T inv_n = T(1) / T(N);
    const T ms = s1 * inv_n;
    const T var = s2 * inv_n - ms * ms;
    const T cov = sr * inv_n - ms * (sum_t * inv_n);
    const T mean = v0 + ms;
    const bool finite = isfinite(s1) && isfinite(s2) && isfinite(sr) && isfinite(v0);
    if (!finite || !(fabs(v0) <= T(kValueCap)) || !(var > T(0))) return -1.f;
    const T sd = sqrt(var);
    const T mx = fabs(v0) > fabs(mean) ? fabs(v0) : fabs(mean);
    if (!(sd > T(kConstRel) * mx)) return -1.f;
    return (float)(fabs(cov) / (sd * sd_t));
}

// the same, for + and -: the sums of v' and v' r come from per-operand FP64 sums; only
// their combination is done in FP64 (where a and b nearly cancel), the rest in T (FP64
// throughput is a small fraction of FP32 on this part)
template <typename T>
__device__ __forceinline__ float finalize_lin(double s1, T s2, double sr, T v0, int N, T sum_t, T sd_t) {
    return finalize<T>((T)s1, s2, (T)sr, v0, N, sum_t, sd_t);
}

// + and - from the cross sum (FP32 form): the sum of v'^2 is q2 = A2[a] + A2[b] +/- 2 X with
// X = sum a'b' accumulated in FP32 and |q2 - the exact sum| <= dq.  Where dq cannot change
// the key by more than a small share of the FP32 screening margin (dq / N <= kCrossTol var,
// a relative score change <= 5e-5) the score is final; where it could (a and b nearly
// cancel) or where it decides the validity tests, kCrossOpen asks for the direct sums.
constexpr float kCrossTol = 1e-4f;
constexpr float kCrossOpen = -2.f;
__device__ __forceinline__ float finalize_x(double s1d, double q2d, float dq, double srd, float v0, int N, float sum_t,
                                            float sd_t) {
    const float s1 = (float)s1d, s2 = (float)q2d, sr = (float)srd;
    const float inv_n = 1.f / (float)N;
    const float ms = s1 * inv_n;
    const float var = s2 * inv_n - ms * ms;
    const float cov = sr * inv_n - ms * (sum_t * inv_n);
    const float mean = v0 + ms;
    const bool finite = isfinite(s1) && isfinite(s2) && isfinite(sr) && isfinite(v0) && isfinite(dq);
    if (!finite || !(fabsf(v0) <= (float)kValueCap)) return -1.f;
    const float dv = dq * inv_n;
    const float lim = (float)kConstRel * fmaxf(fabsf(v0), fabsf(mean));
    if (!(var + dv > 0.f) || !(sqrtf(var + dv) > lim)) return -1.f;       // rejected at either end
    if (!(dv <= kCrossTol * var) || !(sqrtf(var - dv) > lim)) return kCrossOpen;
    return fabsf(cov) / (sqrtf(var) * sd_t);
}

template <typename T> struct TgtView;
template <> struct TgtView<float> {
    __device__ static const float* tc(const float* t32, const double*) { return t32; }
    __device__ static float sum(const TargetStats* st) { return (float)st->sum32; }
    __device__ static float sd(const TargetStats* st) { return st->sd32; }
};
template <> struct TgtView<double> {
    __device__ static const double* tc(const float*, const double* t64) { return t64; }
    __device__ static double sum(const TargetStats*) { return 0.0; }
    __device__ static double sd(const TargetStats* st) { return st->sd; }
};

constexpr int TJ = 32;          // j operands per tile (= lanes)
constexpr int NG = 8;           // warps per CTA, one group of i operands each
constexpr int RI = 4;           // i operands per thread
constexpr int TI = NG * RI;     // i operands per tile
constexpr int TS = 32;          // samples per chunk

struct PairArgs {
    const Space* sp;            // plan in device memory
    int sec[4];                 // section index of +, -, *, / at the top level (-1: off)
    int64_t P, Q;
    int nxp;
    int N;
    const int2* tiles;
    int n_tiles;
    float* scores;
    // cross-sum form of + and - (FP32 with the operand cache): per-operand sums of squared
    // shifted values, and the list of candidates whose key the cross sum leaves open
    const double* A2;
    unsigned long long* fix;
    unsigned* fix_count;
    int fix_cap;
};

// four consecutive values from shared memory (16-byte aligned)
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

template <typename T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }

// one j operand at one sample: shifted value, raw value, reciprocal, and the target's
// value at that sample, read with one vector load
template <typename T> struct Quad;
template <> struct __align__(16) Quad<float> { float t, v, r, y; };
template <> struct __align__(32) Quad<double> { double t, v, r, y; };

template <typename T>
struct __align__(32) PairBuf {
    T at[TS][TI], av[TS][TI], ar[TS][TI];   // i operands: shifted, raw, reciprocal
    Quad<T> bq[TS][TJ];                     // j operands and the target
};

template <typename T>
struct __align__(32) PairSmem {
    PairBuf<T> buf[2];                      // double buffer: stage chunk c+1 while computing c
    T a0[TI], b0[TJ];                       // sample-0 values
    unsigned char ok[TI + TJ];              // operand validity (FP64, recursive)
    Prog prog[TI + TJ];                     // operand programs (on-the-fly staging only)
};

__device__ __forceinline__ bool pair_ok(int64_t i, int64_t j, int64_t P, int64_t Q, int nxp) {
    if (!(i < j && j < P)) return false;
    return nxp ? (i < Q && j >= Q) : (j >= Q);
}

// Staging: warp g owns samples g, g+8, g+16, g+24 of a chunk for both operand sides; lane
// = operand.  With the operand cache (sample-major) every access is one coalesced load
// and a conflict-free row of shared memory; without it the lane evaluates its operand's
// program from the primaries.
constexpr int kStageSlots = 2 * TS / NG;    // (sample, side) slots per warp and chunk

template <typename T>
__device__ __forceinline__ void stage_load(const PairArgs& A, const T* __restrict__ Xc, const T* __restrict__ cache,
                                           const T* __restrict__ tc, const PairSmem<T>& S, int64_t i0, int64_t j0,
                                           int s0, int g, int lane, T (&v)[kStageSlots], T (&y)[kStageSlots / 2]) {
    const int N = A.N;
#pragma unroll
    for (int q = 0; q < kStageSlots; ++q) {
        const int s = s0 + g + NG * (q >> 1);
        const int side = q & 1;
        const int64_t f = (side ? j0 : i0) + lane;
        T x = T(0);
        if (s < N && f < A.P) {
            if (cache) x = cache[(size_t)s * A.P + f];
            else {
                const Prog& p = S.prog[side ? TI + lane : lane];
                if (p.n) x = eval_prog<T>(p, [&](int c) { return Xc[(size_t)c * N + s]; });
            }
        }
        v[q] = x;
        if (side) y[q >> 1] = s < N ? tc[s] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void stage_store(PairSmem<T>& S, int b, const T (&v)[kStageSlots],
                                            const T (&y)[kStageSlots / 2], int g, int lane) {
    PairBuf<T>& B = S.buf[b];
#pragma unroll
    for (int q = 0; q < kStageSlots; ++q) {
        const int s = g + NG * (q >> 1);
        if (q & 1) {
            Quad<T> e;
            e.t = v[q] - S.b0[lane];
            e.v = v[q];
            e.r = rcp<T>(v[q]);
            e.y = y[q >> 1];
            B.bq[s][lane] = e;
        } else {
            B.at[s][lane] = v[q] - S.a0[lane];
            B.av[s][lane] = v[q];
            B.ar[s][lane] = rcp<T>(v[q]);
        }
    }
}


// moments of a screening target t (one block of any multiple of 32 threads): the centred
// copies in FP64 and FP32 and their sums
__device__ void prepare_target_block(const double* t, int N, double* tc64, float* tc32, TargetStats* st,
                                     double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += t[i];
    const double mean = block_sum(s, red) / N;
    double ss = 0.0, s32 = 0.0, ss32 = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double c = t[i] - mean;
        const float f = (float)c;
        tc64[i] = c;
        tc32[i] = f;
        ss += c * c;
        s32 += (double)f;
        ss32 += (double)f * (double)f;
    }
    ss = block_sum(ss, red);
    double tsum = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tsum += tc64[i];
    tsum = block_sum(tsum, red);
    s32 = block_sum(s32, red);
    ss32 = block_sum(ss32, red);
    if (threadIdx.x == 0) {
        st->mean = mean;
        st->sd = sqrt(ss / N);
        st->tsum = tsum;
        st->sum32 = s32;
        st->srr32 = ss32 - s32 * s32 / N;
        st->sd32 = (float)sqrt(st->srr32 / N);
    }
}

// one id below the top level scored from the sample-major cache (row stride P)
template <typename T>
__device__ __forceinline__ void score_cached_id(const T* cache, int N, int64_t P, const float* tc32, const double* tc64,
                                                const TargetStats* st, int64_t id, const unsigned char* subvalid,
                                                float* scores) {
    if (!subvalid[id]) { scores[id] = -1.f; return; }
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const T v0 = cache[id];
    T s1 = 0, s2 = 0, sr = 0;
    for (int s = 0; s < N; ++s) {
        const T v = cache[(size_t)s * P + id] - v0;
        s1 += v;
        s2 = fma(v, v, s2);
        sr = fma(v, tc[s], sr);
    }
    scores[id] = finalize<T>(s1, s2, sr, v0, N, TgtView<T>::sum(st), TgtView<T>::sd(st));
}

constexpr int kUnaryMax = 8;
struct UnaryArgs {
    int n_ops;
    int op[kUnaryMax];
    int64_t base[kUnaryMax];   // first id of each operator's section
    int64_t Q, P;              // operands: new_{L-1} = [Q, P)
    int N;
};

// the top level's unary sections from cached operand rows: a block of kUnaryMax warps takes
// 32 operands (from U.Q + 32 blk) and every enabled unary operator (warp w = operator w,
// lane = operand), 32-sample chunks staged in shared memory (xs, r)
template <typename T>
__device__ __forceinline__ void unary_block(const UnaryArgs& U, const T* cache, const float* tc32, const double* tc64,
                                            const TargetStats* st, const unsigned char* subvalid, float* scores,
                                            int64_t blk, T (*xs)[33], T* r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t z0 = U.Q + blk * 32;
    const int64_t z = z0 + lane;
    const int N = U.N;
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const bool active = w < U.n_ops && z < U.P;
    const int op = w < U.n_ops ? U.op[w] : EXP;
    const T v0 = active ? op_unary<T>(op, cache[z]) : T(0);
    T s1 = 0, s2 = 0, sr = 0;
    for (int s0 = 0; s0 < N; s0 += 32) {
        __syncthreads();
        // warp w stages samples w, w+8, ...: 32 consecutive operands each (coalesced)
        for (int q = w; q < 32; q += kUnaryMax)
            xs[q][lane] = (z < U.P && s0 + q < N) ? cache[(size_t)(s0 + q) * U.P + z] : T(1);
        if (w == 0) r[lane] = s0 + lane < N ? tc[s0 + lane] : T(0);
        __syncthreads();
        const int ns = min(32, N - s0);
        // the operator is fixed per warp: one loop per operator, no branch per sample
        auto run = [&](auto opc) {
            for (int s = 0; s < ns; ++s) {
                const T v = op_unary<T>(decltype(opc)::value, xs[s][lane]) - v0;
                s1 += v;
                s2 = fma(v, v, s2);
                sr = fma(v, r[s], sr);
            }
        };
        if (active) {
            switch (op) {
                case EXP: run(std::integral_constant<int, EXP>{}); break;
                case LOG: run(std::integral_constant<int, LOG>{}); break;
                case SQRT: run(std::integral_constant<int, SQRT>{}); break;
                case SQ: run(std::integral_constant<int, SQ>{}); break;
                case INV: run(std::integral_constant<int, INV>{}); break;
                case SIN: run(std::integral_constant<int, SIN>{}); break;
                case CUBE: run(std::integral_constant<int, CUBE>{}); break;
                default: run(std::integral_constant<int, EXPNEG>{}); break;
            }
        }
    }
    if (active)
        scores[U.base[w] + (z - U.Q)] = subvalid[z] ? finalize<T>(s1, s2, sr, v0, N, TgtView<T>::sum(st), TgtView<T>::sd(st)) : -1.f;
}

// FP64 re-score of one id by one warp (lanes over samples), written to entry w of the
// output arrays: the exact validity rules (every |v| <= 1e12 and finite, not identically
// zero, std > 1e-6 max|v|), the Pearson score, kProbes standardised values for the
// duplicate rule, and the standardised vector (zc, when given, row stride N; the raw
// values instead with zc_raw).  Operand
// values come from V (row stride ldv) when given, else from the primaries Xc.
__device__ __forceinline__ void rescore_one(const Space* sp, const double* Xc, int N, int ldv, const double* tc,
                                            const TargetStats* st, int64_t id, int w,
                                            const unsigned char* subvalid, const double* V, double* score,
                                            double* mean_out, double* sd_out, int* valid_out, double* probe,
                                            double* zc, bool zc_raw = false, const double* Vinv = nullptr) {
    const int lane = threadIdx.x & 31;
    Prog p;
    int level, op; int64_t a, b;
    const int64_t Pbot = sp->phi[sp->rung - 1];
    OpRef ref{};
    bool built = decode(*sp, id, level, op, a, b) && (V ? make_opref(*sp, id, ref) : build_prog(*sp, id, p));
    ref.inv = Vinv;
    if (built && id < Pbot && !subvalid[id]) built = false;                                  // exact, recursive
    if (built && id >= Pbot && (!subvalid[a] || (b >= 0 && !subvalid[b]))) built = false;   // invalid operand
    if (!built) {
        if (lane == 0) { score[w] = -1.0; valid_out[w] = 0; mean_out[w] = 0; sd_out[w] = 0; }
        if (lane < kProbes) probe[(size_t)w * kProbes + lane] = 0.0;
        return;
    }
    double* z = zc ? zc + (size_t)w * N : nullptr;
    auto value = [&](int i, double& mag) -> double {
        return V ? opref_val(ref, V, ldv, i, mag) : eval_prog_mag<double>(p, [&](int c) { return Xc[(size_t)c * N + i]; }, mag);
    };
    // one pass of sums shifted by the sample-0 value (FP64: relative error ~1e-14, far
    // inside the 1e-9 tie window of the walk)
    double mag0;
    const double v0 = value(0, mag0);
    double s1 = 0.0, s2 = 0.0, sc = 0.0, mx = 0.0, mo = 0.0;
    int bad = 0;
    for (int i = lane; i < N; i += 32) {
        double mag;
        const double v = value(i, mag);
        if (!isfinite(v) || fabs(v) > kValueCap) bad = 1;
        const double u = v - v0;
        s1 += u;
        s2 += u * u;
        sc += u * tc[i];
        mx = fmax(mx, fabs(v));
        mo = fmax(mo, mag);
        if (z) z[i] = v;
    }
    bad = warp_or(bad);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    sc = warp_sum(sc);
    mx = warp_max(mx);
    mo = warp_max(mo);
    // identically zero: a top-level + or - whose operands cancel (lower ids: in subvalid)
    const bool top_addsub = id >= Pbot && (op == ADD || op == SUB);
    const bool cancelled = top_addsub && mx <= kCancelRel * mo;
    const double mean = v0 + s1 / N;
    const double var = s2 / N - (s1 / N) * (s1 / N);
    const double sd = bad || !(var > 0.0) ? 0.0 : sqrt(var);
    const int ok = !bad && !cancelled && sd > kConstRel * mx;
    const double inv = ok ? 1.0 / sd : 0.0;
    if (z && !zc_raw)
        for (int i = lane; i < N; i += 32) z[i] = (z[i] - mean) * inv;
    if (lane < kProbes) {
        const int i = (int)(((int64_t)lane * N) / kProbes);
        double mag;
        const double v = z ? (zc_raw ? (z[i] - mean) * inv : z[i]) : (value(i, mag) - mean) * inv;
        probe[(size_t)w * kProbes + lane] = v;
    }
    if (lane == 0) {
        valid_out[w] = ok;
        mean_out[w] = mean;
        sd_out[w] = sd;
        score[w] = ok ? fabs(sc - (s1 / N) * st->tsum) / ((double)N * sd * st->sd) : -1.0;
    }
}


// paired FP32 arithmetic (two lanes of FP32 in one 64-bit register, one instruction for both)
using f2 = unsigned long long;
__device__ __forceinline__ f2 f2pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2up(f2 x, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x)); }
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// One 32 x 32 tile of operand pairs (i0.., j0..): stage operands chunk by chunk, accumulate
// the shifted sums of + - * a/b b/a for 4 pairs per thread, write the scores.  Called by
// every thread of an 8-warp CTA; S is that CTA's shared memory.
template <typename T, bool LIN, bool XS = false>
__device__ __forceinline__ void pair_tile(const PairArgs& A, const T* __restrict__ Xc, const float* __restrict__ tc32,
                                          const double* __restrict__ tc64, const TargetStats* __restrict__ st,
                                          const unsigned char* __restrict__ subvalid, const T* __restrict__ cache,
                                          const double* __restrict__ A1, const double* __restrict__ AR, PairSmem<T>& S,
                                          int64_t i0, int64_t j0) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int N = A.N;
    const T* tc = TgtView<T>::tc(tc32, tc64);
    const T sum_t = TgtView<T>::sum(st), sd_t = TgtView<T>::sd(st);
    __syncthreads();
    // operand programs (on-the-fly only), validity and sample-0 values
    if (tid < TI + TJ) {
        const int64_t f = tid < TI ? i0 + tid : j0 + (tid - TI);
        Prog& p = S.prog[tid];
        p.n = 0;
        if (f < A.P && !cache && !build_prog(*A.sp, f, p)) p.n = 0;
        S.ok[tid] = f < A.P && subvalid[f];
        T v = T(0);
        if (f < A.P) v = cache ? cache[f] : (p.n ? eval_prog<T>(p, [&](int c) { return Xc[(size_t)c * N]; }) : T(0));
        if (tid < TI) S.a0[tid] = v; else S.b0[tid - TI] = v;
    }
    __syncthreads();

    const int64_t j = j0 + lane;
    T Km[RI], Kd[RI], Ke[RI];
    const T b0 = S.b0[lane];
    const T rb0 = rcp<T>(b0);
#pragma unroll
    for (int q = 0; q < RI; ++q) {
        const T a0 = S.a0[g * RI + q];
        Km[q] = a0 * b0;
        Kd[q] = a0 * rb0;
        Ke[q] = b0 * rcp<T>(a0);
    }
    // + and -: only the sum of squares per pair (first sums from per-operand sums when
    // available); *, a/b, b/a: all three sums.  Without per-operand sums (no operand
    // cache) + and - accumulate all three as well.
    constexpr bool lin = LIN;
    T q2[2][RI], l1[2][RI], lr[2][RI];
    T s1[3][RI], s2[3][RI], sr[3][RI];
#pragma unroll
    for (int q = 0; q < RI; ++q) {
        q2[0][q] = q2[1][q] = l1[0][q] = l1[1][q] = lr[0][q] = lr[1][q] = T(0);
#pragma unroll
        for (int o = 0; o < 3; ++o) { s1[o][q] = T(0); s2[o][q] = T(0); sr[o][q] = T(0); }
    }

    // FP32 with per-operand sums: the same sums kept in pairs of i operands (q, q + 1), two FP32
    // lanes per register (fma/add/sub.f32x2: half the FP32 instructions to issue)
    constexpr bool kPair = std::is_same<T, float>::value && LIN;
    // cross-sum form (XS): + and - keep only X = sum a'b' per pair, in 32-sample runs (XC)
    // added into XT, so the rounding of X stays within (TS + runs + 2) u sum |a'b'|
    constexpr bool kX = kPair && XS;
    constexpr int RH = RI / 2;
    f2 Q2[2][RH], L1[2][RH], LR[2][RH], S1[3][RH], S2[3][RH], SR[3][RH], NKM[RH], NKD[RH], NKE[RH];
    f2 XT[RH], XC[RH];
    if constexpr (kPair) {
#pragma unroll
        for (int h = 0; h < RH; ++h) {
            const f2 z = f2pk(0.f, 0.f);
            Q2[0][h] = Q2[1][h] = L1[0][h] = L1[1][h] = LR[0][h] = LR[1][h] = z;
            XT[h] = XC[h] = z;
#pragma unroll
            for (int o = 0; o < 3; ++o) { S1[o][h] = z; S2[o][h] = z; SR[o][h] = z; }
            NKM[h] = f2pk(-(float)Km[2 * h], -(float)Km[2 * h + 1]);
            NKD[h] = f2pk(-(float)Kd[2 * h], -(float)Kd[2 * h + 1]);
            NKE[h] = f2pk(-(float)Ke[2 * h], -(float)Ke[2 * h + 1]);
        }
    }

    T pf[kStageSlots], py[kStageSlots / 2];
    stage_load<T>(A, Xc, cache, tc, S, i0, j0, 0, g, lane, pf, py);
    stage_store<T>(S, 0, pf, py, g, lane);
    __syncthreads();
    int b = 0;
    for (int s0 = 0; s0 < N; s0 += TS, b ^= 1) {
        const bool more = s0 + TS < N;
        if (more) stage_load<T>(A, Xc, cache, tc, S, i0, j0, s0 + TS, g, lane, pf, py);   // in flight during compute
        const PairBuf<T>& B = S.buf[b];
        const int ns = min(TS, N - s0);
        auto step = [&](int s) {
            if constexpr (kPair) {
                const Quad<T> bq = B.bq[s][lane];
                const f2 r2 = f2pk((float)bq.y, (float)bq.y), bt2 = f2pk((float)bq.t, (float)bq.t);
                const f2 bv2 = f2pk((float)bq.v, (float)bq.v), br2 = f2pk((float)bq.r, (float)bq.r);
                const ulonglong2 at = *reinterpret_cast<const ulonglong2*>(&B.at[s][g * RI]);
                const ulonglong2 av = *reinterpret_cast<const ulonglong2*>(&B.av[s][g * RI]);
                const ulonglong2 ar = *reinterpret_cast<const ulonglong2*>(&B.ar[s][g * RI]);
                const f2 atp[RH] = {at.x, at.y}, avp[RH] = {av.x, av.y}, arp[RH] = {ar.x, ar.y};
#pragma unroll
                for (int h = 0; h < RH; ++h) {
                    f2 v;
                    if constexpr (kX) {
                        XC[h] = f2fma(atp[h], bt2, XC[h]);
                    } else {
                    v = f2add(atp[h], bt2);           Q2[0][h] = f2fma(v, v, Q2[0][h]);
                    if constexpr (!LIN) { L1[0][h] = f2add(L1[0][h], v); LR[0][h] = f2fma(v, r2, LR[0][h]); }
                    v = f2sub(atp[h], bt2);           Q2[1][h] = f2fma(v, v, Q2[1][h]);
                    if constexpr (!LIN) { L1[1][h] = f2add(L1[1][h], v); LR[1][h] = f2fma(v, r2, LR[1][h]); }
                    }
                    v = f2fma(avp[h], bv2, NKM[h]);   S1[0][h] = f2add(S1[0][h], v); S2[0][h] = f2fma(v, v, S2[0][h]); SR[0][h] = f2fma(v, r2, SR[0][h]);
                    v = f2fma(avp[h], br2, NKD[h]);   S1[1][h] = f2add(S1[1][h], v); S2[1][h] = f2fma(v, v, S2[1][h]); SR[1][h] = f2fma(v, r2, SR[1][h]);
                    v = f2fma(bv2, arp[h], NKE[h]);   S1[2][h] = f2add(S1[2][h], v); S2[2][h] = f2fma(v, v, S2[2][h]); SR[2][h] = f2fma(v, r2, SR[2][h]);
                }
            } else {
            const Quad<T> bq = B.bq[s][lane];
            const T r = bq.y, bt = bq.t, bv = bq.v, br = bq.r;
            T at[RI], av[RI], ar[RI];
            load4(&B.at[s][g * RI], at);
            load4(&B.av[s][g * RI], av);
            load4(&B.ar[s][g * RI], ar);
#pragma unroll
            for (int q = 0; q < RI; ++q) {
                T v;
                v = at[q] + bt;             q2[0][q] = fma(v, v, q2[0][q]);
                if constexpr (!LIN) { l1[0][q] += v; lr[0][q] = fma(v, r, lr[0][q]); }
                v = at[q] - bt;             q2[1][q] = fma(v, v, q2[1][q]);
                if constexpr (!LIN) { l1[1][q] += v; lr[1][q] = fma(v, r, lr[1][q]); }
                v = fma(av[q], bv, -Km[q]); s1[0][q] += v; s2[0][q] = fma(v, v, s2[0][q]); sr[0][q] = fma(v, r, sr[0][q]);
                v = fma(av[q], br, -Kd[q]); s1[1][q] += v; s2[1][q] = fma(v, v, s2[1][q]); sr[1][q] = fma(v, r, sr[1][q]);
                v = fma(bv, ar[q], -Ke[q]); s1[2][q] += v; s2[2][q] = fma(v, v, s2[2][q]); sr[2][q] = fma(v, r, sr[2][q]);
            }
            }
        };
        if (ns == TS) {
#pragma unroll 4
            for (int s = 0; s < TS; ++s) step(s);
        } else {
            for (int s = 0; s < ns; ++s) step(s);
        }
        if constexpr (kX) {
#pragma unroll
            for (int h = 0; h < RH; ++h) { XT[h] = f2add(XT[h], XC[h]); XC[h] = f2pk(0.f, 0.f); }
        }
        if (more) stage_store<T>(S, b ^ 1, pf, py, g, lane);
        __syncthreads();
    }

    float xs[RI];     // cross sums (kX)
    if constexpr (kPair) {
#pragma unroll
        for (int h = 0; h < RH; ++h) {
            float a, b;
            if constexpr (kX) { f2up(XT[h], a, b); xs[2 * h] = a; xs[2 * h + 1] = b; }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                if constexpr (!kX) { f2up(Q2[o][h], a, b); q2[o][2 * h] = a; q2[o][2 * h + 1] = b; }
                f2up(L1[o][h], a, b); l1[o][2 * h] = a; l1[o][2 * h + 1] = b;
                f2up(LR[o][h], a, b); lr[o][2 * h] = a; lr[o][2 * h + 1] = b;
            }
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                f2up(S1[o][h], a, b); s1[o][2 * h] = a; s1[o][2 * h + 1] = b;
                f2up(S2[o][h], a, b); s2[o][2 * h] = a; s2[o][2 * h + 1] = b;
                f2up(SR[o][h], a, b); sr[o][2 * h] = a; sr[o][2 * h + 1] = b;
            }
        }
    }

    // scores of the (up to) 20 candidates of this thread
    const bool okj = S.ok[TI + lane];
    const double a1j = lin && j < A.P ? A1[j] : 0.0, arj = lin && j < A.P ? AR[j] : 0.0;
#pragma unroll
    for (int q = 0; q < RI; ++q) {
        // indices, validity and shifts recomputed here (same values): in the paired form they
        // are not live across the sample loop, which leaves the registers to the accumulators
        const int64_t i = i0 + g * RI + q;
        if (!pair_ok(i, j, A.P, A.Q, A.nxp)) continue;
        const T a0 = S.a0[g * RI + q];
        const T kmq = kPair ? a0 * b0 : Km[q];
        const T kdq = kPair ? a0 * rb0 : Kd[q];
        const T keq = kPair ? b0 * rcp<T>(a0) : Ke[q];
        const bool opv = okj && S.ok[g * RI + q];   // both operands valid
        const double a1i = lin ? A1[i] : 0.0, ari = lin ? AR[i] : 0.0;
        if constexpr (kX) {
            if (A.sec[0] >= 0 || A.sec[1] >= 0) {
                // rounding bound of X: (TS + runs + 2) u per unit of sum |a'b'| <= sqrt(A2[i] A2[j]),
                // twice in q2 (u = 2^-24; 0.1% for second-order terms)
                const double a2i = A.A2[i], a2j = A.A2[j];
                const double a2s = a2i + a2j, x2 = 2.0 * (double)xs[q];
                const float dq = 2.002f * (float)(TS + (N + TS - 1) / TS + 2) * 5.9604645e-8f *
                                 sqrtf((float)a2i) * sqrtf((float)a2j);
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    if (A.sec[o] < 0) continue;
                    const Section& sc = A.sp->sec[A.sec[o]];
                    float v = -1.f;
                    if (opv) {
                        v = o == 0 ? finalize_x(a1i + a1j, a2s + x2, dq, ari + arj, a0 + b0, N, sum_t, sd_t)
                                   : finalize_x(a1i - a1j, a2s - x2, dq, ari - arj, a0 - b0, N, sum_t, sd_t);
                        if (v == kCrossOpen) {      // scored by the direct sums afterwards
                            const unsigned slot = atomicAdd(A.fix_count, 1u);
                            if (slot < (unsigned)A.fix_cap)
                                A.fix[slot] = ((unsigned long long)o << 62) | ((unsigned long long)i << 31) |
                                              (unsigned long long)j;
                            v = -1.f;
                        }
                    }
                    A.scores[sc.base + rank_of(sc, i, j)] = v;
                }
            }
        } else {
        if (A.sec[0] >= 0) {
            const Section& sc = A.sp->sec[A.sec[0]];
            float v = -1.f;
            if (opv) v = lin ? finalize_lin<T>(a1i + a1j, q2[0][q], ari + arj, a0 + b0, N, sum_t, sd_t)
                             : finalize<T>(l1[0][q], q2[0][q], lr[0][q], a0 + b0, N, sum_t, sd_t);
            A.scores[sc.base + rank_of(sc, i, j)] = v;
        }
        if (A.sec[1] >= 0) {
            const Section& sc = A.sp->sec[A.sec[1]];
            float v = -1.f;
            if (opv) v = lin ? finalize_lin<T>(a1i - a1j, q2[1][q], ari - arj, a0 - b0, N, sum_t, sd_t)
                             : finalize<T>(l1[1][q], q2[1][q], lr[1][q], a0 - b0, N, sum_t, sd_t);
            A.scores[sc.base + rank_of(sc, i, j)] = v;
        }
        }
        if (A.sec[2] >= 0) {
            const Section& sc = A.sp->sec[A.sec[2]];
            A.scores[sc.base + rank_of(sc, i, j)] = opv ? finalize<T>(s1[0][q], s2[0][q], sr[0][q], kmq, N, sum_t, sd_t) : -1.f;
        }
        if (A.sec[3] >= 0) {
            const Section& sc = A.sp->sec[A.sec[3]];
            A.scores[sc.base + rank_of(sc, i, j)] = opv ? finalize<T>(s1[1][q], s2[1][q], sr[1][q], kdq, N, sum_t, sd_t) : -1.f;
            A.scores[sc.base + rank_of(sc, j, i)] = opv ? finalize<T>(s1[2][q], s2[2][q], sr[2][q], keq, N, sum_t, sd_t) : -1.f;
        }
    }
}

}  // namespace
}  // namespace sg
