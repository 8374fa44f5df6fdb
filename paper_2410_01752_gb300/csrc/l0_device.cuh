// l0_device.cuh — device building blocks of the l0 search (§2.3, Eqs. 7-8), shared by the
// per-problem kernels (l0.cu) and the persistent multi-task kernel (batch.cu).
#pragma once

#include "common.cuh"

namespace sg {
namespace {

constexpr int kWarps = 8;
constexpr int kRows = 16;                 // i1 rows per work item

template <typename T> __device__ __forceinline__ T l0_warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// order-preserving maps of floating values to unsigned integers (for atomicMin)
__device__ __forceinline__ unsigned long long okey(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_inv(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)u);
}

// ---------------------------------------------------------------------------------
// enumeration
// ---------------------------------------------------------------------------------
template <typename T>
struct EnumArgs {
    const T* G;                 // n x n (leading dimension ld)
    const T* b;
    int ld, n, N;
    T syy;                      // y~^T y~ / N
    double sst;                 // N * syy
    int cpp;                    // work items per prefix (chunks of kRows i1 rows)
    int64_t n_items;            // C(n - 2, D - 2) prefixes x cpp
    int* counter;               // work counter
    float tau;                  // pivots at or below: FP32 -> refit list; FP64 -> singular
    int fp32;                   // error-bounded FP32 mode
    unsigned long long* ub_key; // pass 1 output (ordered key of the bound)
    const Winner* win;          // pass 2 input: win->thr
    uint64_t* band;
    unsigned int* band_count;
    int64_t band_cap;
    unsigned long long* examined;
    double sqrt_syy;            // FP32 mode: sqrt(syy) for the a posteriori error bound
    float* band_r32;            // optional: the FP32 RSS of each band entry (NaN: flagged by a pivot)
    const double* G64;          // optional FP64 Gram (ld) and moments: a subset flagged by an FP32
    const double* b64;          //   pivot is solved in FP64 on the spot and kept in the band only
    double syy64;               //   when its RSS is within tie64 of the pass-2 threshold
    double tie64;
    const int* prefix_list;     // optional: the prefixes to enumerate (D-2 positions each, ascending),
                                //   item = list index x chunk; otherwise every prefix in colex order
};


// subset positions packed into 64 bits: 16 bits each for D <= 4 (n <= 65535), 12 bits each
// for D = 5 (n <= 4095)
__host__ __device__ constexpr int pos_bits(int D) { return D <= 4 ? 16 : 12; }

template <int DP> __device__ __forceinline__ uint64_t pack_subset(const int (&pre)[DP > 0 ? DP : 1], int i1, int i2) {
    constexpr int W = pos_bits(DP + 2);
    uint64_t k = 0;
    int s = 0;
#pragma unroll
    for (int m = 0; m < DP; ++m) { k |= (uint64_t)pre[m] << s; s += W; }
    k |= (uint64_t)i1 << s; s += W;
    k |= (uint64_t)i2 << s;
    return k;
}

// r-th DP-combination in colex order (largest element first): p[DP-1] is the largest m
// with C(m, DP) <= r, then the rest recursively
__device__ __forceinline__ int64_t binom2(int64_t m) { return m * (m - 1) / 2; }
__device__ __forceinline__ int64_t binom3(int64_t m) { return m * (m - 1) * (m - 2) / 6; }

__device__ __forceinline__ int64_t binom4(int64_t m) { return m * (m - 1) * (m - 2) * (m - 3) / 24; }

// largest m with C(m, 2) <= r
__device__ __forceinline__ int64_t colex_top2(int64_t r) {
    int64_t m = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)r)) * 0.5);
    while (m > 1 && binom2(m) > r) --m;
    while (binom2(m + 1) <= r) ++m;
    return m;
}
__device__ __forceinline__ int64_t colex_top3(int64_t r) {
    int64_t m = (int64_t)cbrt(6.0 * (double)r) + 1;
    while (m > 2 && binom3(m) > r) --m;
    while (binom3(m + 1) <= r) ++m;
    return m;
}
__device__ __forceinline__ int64_t colex_top4(int64_t r) {
    int64_t m = (int64_t)sqrt(sqrt(24.0 * (double)r)) + 2;
    while (m > 3 && binom4(m) > r) --m;
    while (binom4(m + 1) <= r) ++m;
    return m;
}

template <int DP> __device__ __forceinline__ void colex_unrank(int64_t r, int (&p)[DP > 0 ? DP : 1]) {
    if (DP == 0) return;
    if (DP == 1) { p[0] = (int)r; return; }
    int64_t m;
    if (DP >= 4) { m = colex_top4(r); p[DP > 3 ? 3 : 0] = (int)m; r -= binom4(m); }
    if (DP >= 3) { m = colex_top3(r); p[DP > 2 ? 2 : 0] = (int)m; r -= binom3(m); }
    m = colex_top2(r);
    p[1] = (int)m;
    p[0] = (int)(r - binom2(m));
}

// MODE 0: bound (min of RSS + err); MODE 1: band collection

__device__ double rss64(const double* G, const double* b, int ld, double syy, int N, int D, const int* pos,
                        double* gamma) {
    double L[kMaxDim][kMaxDim], w[kMaxDim];
    for (int j = 0; j < D; ++j) {
        double dj = G[(size_t)pos[j] * ld + pos[j]];
        for (int m = 0; m < j; ++m) dj -= L[j][m] * L[j][m];
        if (!(dj > kPivotMin)) return INFINITY;
        L[j][j] = sqrt(dj);
        for (int i = j + 1; i < D; ++i) {
            double v = G[(size_t)pos[i] * ld + pos[j]];
            for (int m = 0; m < j; ++m) v -= L[i][m] * L[j][m];
            L[i][j] = v / L[j][j];
        }
    }
    double q = 0.0;
    for (int j = 0; j < D; ++j) {
        double v = b[pos[j]];
        for (int m = 0; m < j; ++m) v -= L[j][m] * w[m];
        w[j] = v / L[j][j];
        q += w[j] * w[j];
    }
    if (gamma) {   // back substitution L^T gamma = w
        for (int j = D - 1; j >= 0; --j) {
            double v = w[j];
            for (int m = j + 1; m < D; ++m) v -= L[m][j] * gamma[m];
            gamma[j] = v / L[j][j];
        }
    }
    return (double)N * (syy - q);
}

__device__ __forceinline__ void unpack(uint64_t key, int D, int* pos) {
    const int W = pos_bits(D);
    const uint64_t mask = (1ull << W) - 1;
    for (int j = 0; j < D; ++j) pos[j] = (int)((key >> (W * j)) & mask);
}

// pass 2, a subset flagged by an FP32 pivot: keep it for the FP64 refit?  With the FP64
// Gram at hand, only if its FP64 RSS can reach the threshold (the band must hold every
// subset within the tie window of the minimum, and the minimum is at most the threshold)
template <typename T>
__device__ __forceinline__ bool keep_flagged(const EnumArgs<T>& A, const int* pos, int D, double thr) {
    if (!A.G64) return true;
    const double r = rss64(A.G64, A.b64, A.ld, A.syy64, A.N, D, pos, nullptr);
    return r <= thr + A.tie64;
}

// One enumeration item, a (D-2)-prefix in colex order and a run of kRows i1 rows, for one
// warp.  tab: this warp's tables ((DP + 2) x n values).  MODE 0 lowers the lane's bound
// best; MODE 1 collects the band below thr.
// D = 1, feature i: pass 1 puts its RSS into the bound (FP64 when the FP64 Gram is at hand
// in the FP32 mode, else in T); pass 2 keeps it when it may lie within the tie window of
// the minimum (thr: the bound, plus the tie window in the FP64 mode)
template <typename T, int MODE>
__device__ __forceinline__ void single_subset(const EnumArgs<T>& A, int i, double thr) {
    if (MODE == 0) atomicAdd(A.examined, 1ull);
    auto add = [&](float r32) {
        const unsigned slot = atomicAdd(A.band_count, 1u);
        if (slot < A.band_cap) {
            A.band[slot] = (uint64_t)i;
            if (A.band_r32) A.band_r32[slot] = r32;
        }
    };
    if (A.fp32 && A.G64) {
        const double r = rss64(A.G64, A.b64, A.ld, A.syy64, A.N, 1, &i, nullptr);
        if (!(r < INFINITY)) return;
        if (MODE == 0) atomicMin(A.ub_key, okey(r));
        else if (r <= thr + A.tie64) add((float)r);
        return;
    }
    const T d = A.G[(size_t)i * A.ld + i];
    const T bi = A.b[i];
    if (!(d > T(A.tau))) {
        if (MODE == 1 && A.fp32) add(__int_as_float(0x7fc00000));
        return;
    }
    const T rss = T(A.N) * (A.syy - bi * bi / d);
    if (MODE == 0) atomicMin(A.ub_key, okey((double)rss));
    else if ((double)rss <= thr) add((float)rss);
}

// A posteriori bound on |RSS_FP32 - RSS| of one subset in the FP32 mode with the FP64
// Gram at hand.  With L, w the computed FP32 Cholesky factor and forward solution and
// gamma = L^-T w the coefficients, backward error analysis of the factorisation and the
// solve gives q_FP32 = b'^T (G + E)^-1 b' with |E| <= (1 + 3.1 (D+1)) u (entries of |L||L^T|
// <= 1 for unit-diagonal G) and |b' - b| <= u |b| <= u sqrt(syy); to first order
// |q_FP32 - q| <= 2 u sqrt(syy) s + (1 + 3.1 (D+1)) u s^2 with s = sum |gamma_i|, plus the
// rounding of syy - q.  RSS = N (syy - q); the bound carries a factor 2 of safety.
template <typename T>
__device__ __forceinline__ T apost_err(const EnumArgs<T>& A, int D, T s, T rss) {
    const T u = T(5.9604644775390625e-8);              // 2^-24
    const T c1 = T(1) + T(3.1) * T(D + 1);
    return T(2) * u * (T(A.N) * (T(2) * T(A.sqrt_syy) * s + c1 * s * s) +
                       T(D + 3) * (T(2) * T(A.sst) + fabs(rss)));
}

// One enumeration item, a (D-2)-prefix in colex order and a run of kRows i1 rows, for one
// warp.  tab: this warp's tables ((DP + 2) x n values).  MODE 0 lowers the lane's best
// FP32 RSS (best, best_key); MODE 1 collects the band: every subset that may lie within
// the tie window of the minimum given thr, an upper bound of the minimum.  In the FP32
// mode with the FP64 Gram (A.G64) a subset enters the band only after an FP64 solve
// confirms it; without it (mixed precision) the FP32 RSS is compared directly.
template <typename T> __device__ __forceinline__ T round_up(double x);
template <> __device__ __forceinline__ float round_up<float>(double x) { return __double2float_ru(x); }
template <> __device__ __forceinline__ double round_up<double>(double x) { return x; }

template <typename T, int DP, int MODE>
__device__ __forceinline__ void enum_item(const EnumArgs<T>& A, T* tab, int64_t item, T& best,
                                          unsigned long long& best_key, double thr, unsigned long long& my_examined) {
    const int lane = threadIdx.x & 31;
    const int n = A.n;
    T* Rt = tab;
    T* dpart = tab + (size_t)DP * n;
    T* npart = dpart + n;
    const T N = T(A.N);
    const bool apost = A.fp32 && A.G64 != nullptr;
    // pass-2 threshold in T, rounded up so that no subset at the bound is lost
    const T thr_eff = MODE == 1 ? round_up<T>(thr + (apost ? A.tie64 : 0.0)) : T(0);
    // item -> (prefix in colex order, chunk): prefixes are the (D-2)-combinations of
    // [0, n-2) ordered by their largest element, so the longest sweeps come first
    int pre[DP > 0 ? DP : 1];
    const int64_t prank = item / A.cpp;
    const int chunk = (int)(item % A.cpp);
    if (A.prefix_list) {
#pragma unroll
        for (int m = 0; m < DP; ++m) pre[m] = A.prefix_list[prank * (DP > 0 ? DP : 1) + m];
    } else {
        colex_unrank<DP>(prank, pre);
    }
    const int i1s = (DP > 0 ? pre[DP - 1] + 1 : 0) + chunk * kRows;
    if (i1s >= n - 1) return;
    // prefix factor (warp-uniform, redundant in every lane)
    T L[DP > 0 ? DP : 1][DP > 0 ? DP : 1], invd[DP > 0 ? DP : 1], wv[DP > 0 ? DP : 1];
    T pw2 = T(0);
    bool pre_ok = true;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        T dj = A.G[(size_t)pre[j] * A.ld + pre[j]];
#pragma unroll
        for (int m = 0; m < j; ++m) dj -= L[j][m] * L[j][m];
        pre_ok = pre_ok && dj > T(A.tau);
        const T ljj = sqrt(dj > T(0) ? dj : T(1));
        L[j][j] = ljj;
        invd[j] = T(1) / ljj;
#pragma unroll
        for (int i = j + 1; i < DP; ++i) {
            T v = A.G[(size_t)pre[i] * A.ld + pre[j]];
#pragma unroll
            for (int m = 0; m < j; ++m) v -= L[i][m] * L[j][m];
            L[i][j] = v * invd[j];
        }
        T v = A.b[pre[j]];
#pragma unroll
        for (int m = 0; m < j; ++m) v -= L[j][m] * wv[m];
        wv[j] = v * invd[j];
        pw2 += wv[j] * wv[j];
    }
    const int i1e = min(i1s + kRows, n - 1);
    if (MODE == 0 && lane == 0)
        for (int i1 = i1s; i1 < i1e; ++i1) my_examined += (unsigned long long)(n - 1 - i1);
    if (!A.fp32 && !pre_ok) return;      // FP64: singular prefix, every extension skipped
    // tables for x in [i1s, n)
    for (int x = i1s + lane; x < n; x += 32) {
        T r[DP > 0 ? DP : 1];
        T dp = A.G[(size_t)x * A.ld + x], np = A.b[x];
#pragma unroll
        for (int m = 0; m < DP; ++m) {
            T v = A.G[(size_t)pre[m] * A.ld + x];        // G symmetric: row pre[m], lanes coalesced
#pragma unroll
            for (int q = 0; q < m; ++q) v -= r[q] * L[m][q];
            r[m] = v * invd[m];
            Rt[(size_t)m * n + x] = r[m];
            dp -= r[m] * r[m];
            np -= r[m] * wv[m];
        }
        dpart[x] = dp;
        npart[x] = np;
    }
    __syncwarp();
    // RB rows i1 per pass over i2: the i2 tables are read once for RB subsets and RB
    // independent loads of G are in flight
    constexpr int RB = 4;
    for (int i1b = i1s; i1b < i1e; i1b += RB) {
        T r1[RB][DP > 0 ? DP : 1], isd1[RB], w1[RB], base_c[RB], c_cmp[RB];
        bool ok1[RB], live[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const int i1 = i1b + k;
            live[k] = i1 < i1e;
            const int ic = live[k] ? i1 : i1s;
#pragma unroll
            for (int m = 0; m < DP; ++m) r1[k][m] = Rt[(size_t)m * n + ic];
            const T d1 = dpart[ic];
            ok1[k] = pre_ok && d1 > T(A.tau);
            if (!A.fp32 && !ok1[k]) live[k] = false;          // FP64: singular, every extension skipped
            isd1[k] = T(1) / sqrt(d1 > T(0) ? d1 : T(1));
            w1[k] = npart[ic] * isd1[k];
            base_c[k] = A.syy - (pw2 + w1[k] * w1[k]);
            // rss < best (MODE 0) or rss <= thr_eff (MODE 1)  <=>  num^2 - c d2 > 0 (>= 0)
            c_cmp[k] = MODE == 0 ? base_c[k] - best / N : base_c[k] - thr_eff / N;
        }
        for (int i2 = i1b + 1 + lane; i2 < n; i2 += 32) {
            T rt[DP > 0 ? DP : 1];
#pragma unroll
            for (int m = 0; m < DP; ++m) rt[m] = Rt[(size_t)m * n + i2];
            const T dp2 = dpart[i2], np2 = npart[i2];
            T gk[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k)
                gk[k] = (live[k] && i2 > i1b + k) ? A.G[(size_t)(i1b + k) * A.ld + i2] : T(0);
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                if (!live[k] || i2 <= i1b + k) continue;
                const int i1 = i1b + k;
                T g = gk[k];
#pragma unroll
                for (int m = 0; m < DP; ++m) g -= r1[k][m] * rt[m];
                const T rr = g * isd1[k];
                const T d2 = dp2 - rr * rr;
                const T num = np2 - rr * w1[k];
                if (!ok1[k] || !(d2 > T(A.tau))) {
                    // flagged by a pivot: the FP32 factor says nothing; FP64 decides (pass 2)
                    if (MODE == 1 && A.fp32) {
                        int pos[DP + 2];
#pragma unroll
                        for (int m = 0; m < DP; ++m) pos[m] = pre[m];
                        pos[DP] = i1;
                        pos[DP + 1] = i2;
                        if (!keep_flagged(A, pos, DP + 2, thr)) continue;
                        const unsigned slot = atomicAdd(A.band_count, 1u);
                        if (slot < A.band_cap) {
                            A.band[slot] = pack_subset<DP>(pre, i1, i2);
                            if (A.band_r32) A.band_r32[slot] = __int_as_float(0x7fc00000);
                        }
                    }
                    continue;
                }
                const T f = num * num - c_cmp[k] * d2;
                if (MODE == 0) {
                    if (!(f > T(0))) continue;
                    best = N * (base_c[k] - num * num / d2);
                    best_key = pack_subset<DP>(pre, i1, i2);
#pragma unroll
                    for (int kk = 0; kk < RB; ++kk) c_cmp[kk] = base_c[kk] - best / N;
                    continue;
                }
                const T rss = N * (base_c[k] - num * num / d2);
                if (!(f >= T(0))) {
                    if (!apost) continue;
                    // back substitution L^T gamma = w, then the a posteriori bound
                    const T g2 = num / d2;
                    const T g1 = (w1[k] - rr * g2) * isd1[k];
                    T sg = fabs(g2) + fabs(g1);
                    T gp[DP > 0 ? DP : 1];
#pragma unroll
                    for (int j = DP - 1; j >= 0; --j) {
                        T v = wv[j] - r1[k][j] * g1 - rt[j] * g2;
#pragma unroll
                        for (int m = j + 1; m < DP; ++m) v -= L[m][j] * gp[m];
                        gp[j] = v * invd[j];
                        sg += fabs(gp[j]);
                    }
                    if (!(rss - apost_err(A, DP + 2, sg, rss) <= thr_eff)) continue;
                }
                if (apost) {
                    int pos[DP + 2];
#pragma unroll
                    for (int m = 0; m < DP; ++m) pos[m] = pre[m];
                    pos[DP] = i1;
                    pos[DP + 1] = i2;
                    if (!keep_flagged(A, pos, DP + 2, thr)) continue;
                }
                const unsigned slot = atomicAdd(A.band_count, 1u);
                if (slot < A.band_cap) {
                    A.band[slot] = pack_subset<DP>(pre, i1, i2);
                    if (A.band_r32) A.band_r32[slot] = (float)rss;
                }
            }
        }
    }
    __syncwarp();
}

// pass 1: the warp's best subset into the global bound (with the FP64 Gram: that subset's
// FP64 RSS, an exact upper bound of the minimum; otherwise the FP32 or FP64 value), and
// the subsets examined
template <typename T>
__device__ __forceinline__ void enum_flush(const EnumArgs<T>& A, int D, T best, unsigned long long best_key,
                                           unsigned long long my_examined) {
    const int lane = threadIdx.x & 31;
    double bv = (double)best;
    int src = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int os = __shfl_xor_sync(0xffffffffu, src, o);
        if (ov < bv || (ov == bv && os < src)) { bv = ov; src = os; }
    }
    const unsigned long long key = __shfl_sync(0xffffffffu, best_key, src);
    if (lane == 0 && bv < INFINITY) {
        if (A.fp32 && A.G64) {
            int pos[kMaxDim];
            unpack(key, D, pos);
            const double r = rss64(A.G64, A.b64, A.ld, A.syy64, A.N, D, pos, nullptr);
            if (r < INFINITY) atomicMin(A.ub_key, okey(r));
        } else {
            atomicMin(A.ub_key, okey(bv));
        }
    }
    unsigned long long ex = l0_warp_sum(my_examined);
    if (lane == 0) atomicAdd(A.examined, ex);
}





__device__ __forceinline__ void gid_tuple(const int64_t* gid, const int* pos, int D, int64_t* t) {
    for (int j = 0; j < D; ++j) t[j] = gid[pos[j]];
    for (int a = 1; a < D; ++a)
        for (int c = a; c > 0 && t[c - 1] > t[c]; --c) { const int64_t x = t[c]; t[c] = t[c - 1]; t[c - 1] = x; }
}

__device__ __forceinline__ bool tuple_less(const int64_t* a, const int64_t* b, int D) {
    for (int j = 0; j < D; ++j) if (a[j] != b[j]) return a[j] < b[j];
    return false;
}


}  // namespace
}  // namespace sg
