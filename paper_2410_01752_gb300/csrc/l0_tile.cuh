// l0_tile.cuh — single-pass tiled enumeration of the exhaustive l0 search (§2.3, Eqs. 7-8)
// in FP32 with an FP64 Gram at hand: every D-subset {p_0 < .. < p_{D-3} < i1 < i2} is
// examined once, and the result is the exact FP64 optimum.
//
// Work decomposition.  The (i1, i2) plane is cut into tiles of kTR rows (i1) x kTC columns
// (i2), column tiles starting at their row block; a work unit is one tile and one
// (D-2)-prefix in colex order, taken by one warp from a global counter.  The warp factors
// the prefix block, tabulates the prefix-reduced values of the tile's rows (shared memory,
// per warp) and of the 8 columns each lane owns, cb + lane + 32 j (registers; the window
// [cb, cb + kTC) ends at n for the last tile), and sweeps the rows in segments of equal
// first live column group, so that no per-group bound is tested inside the sweep.  Per
// subset, with 1/d1 and w1/sqrt(d1) precomputed per row:
//     g = G[i1][i2] - sum_m R[m][i1] R[m][i2],   d2 = dp[i2] - g^2 / d1,
//     num = np[i2] - g w1 / sqrt(d1),   RSS = N (c - num^2 / d2),  c = syy - |w_prefix|^2 - w1^2
// as in the two-pass enumerator, but the decision is a division-free filter:
//     candidate  <=>  not ( num^2 - cB d2 < 0   and   S1 |num| - Rk d2 <= 0   and  d2 > tau )
// cB puts the FP32 RSS above B + tie + E1 (B the running bound, below), and the second
// test bounds the subset's coefficient 1-norm s = |gamma|_1 by Smax: with a = L_P^-T w_P,
// a1 = L_P^-T R[.][i1], a2 = L_P^-T R[.][i2] (prefix back substitutions),
//     s <= |a|_1 + (1 + |a1|_1) |w1| / sqrt(d1)
//            + ((1 + |a1|_1) |r| / sqrt(d1) + 1 + |a2|_1) |num| / d2,   |r| <= 1,
// i.e. s <= S0 + S1' |num| / d2, and s <= Smax keeps the a posteriori FP32 error below E1/2.
// So a subset that is not a candidate has RSS_FP32 - err > B + tie: it cannot be the
// minimum nor tie with it.  Candidates (a fraction of a percent on screened subspaces)
// go through a per-warp queue to the exact test of the two-pass form: the FP32 RSS and
// its a posteriori bound from the back-substituted coefficients, then an FP64 solve from
// the FP64 Gram; a subset whose FP64 RSS is within B + tie enters the band and lowers B.
//
// Running bound.  B starts at the FP64 RSS of a greedy forward selection (an upper bound
// of the minimum M) and only decreases, to FP64 RSS values of visited subsets, so B >= M
// at every moment.  The optimum E* has RSS_FP32 - err <= M <= B, and every tie E of it
// RSS_FP64(E) <= M + tie <= B + tie: both are candidates whenever visited and enter the
// band.  The band (records and ties) is then refit in FP64 and the tie rule picks the
// winner, exactly as after the two-pass form.
#pragma once

#include "l0_device.cuh"

namespace sg {
namespace {

// paired FP32 arithmetic (two columns per 64-bit register, one instruction for both)
using p2 = unsigned long long;
__device__ __forceinline__ p2 pk2(float a, float b) {
    p2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(p2 x, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x)); }
__device__ __forceinline__ p2 fma2(p2 a, p2 b, p2 c) {
    p2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ p2 mul2(p2 a, p2 b) {
    p2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

constexpr int kTR = 64;                  // i1 rows per tile
constexpr int kTC = 256;                 // i2 columns per tile: 8 per lane
constexpr int kTW = 8;                   // warps per CTA = prefixes per work item
constexpr int kTQ = kTC + 64;            // per-warp candidate queue (entries)
constexpr int kClaim = 4;                // work units a warp claims per atomic

struct TileInfo {
    int a, c;                            // first row, first column
    int64_t n_pre;                       // prefixes (colex ranks 0 .. n_pre-1)
    int64_t item0;                       // first work item of this tile
};

struct TileArgs {
    const float* G;                      // FP32 Gram, padded: row stride ldp (multiple of kTC), 16-byte rows
    const float* b;                      // FP32 moments, padded to ldp with zeros
    const float* diag;                   // G[x][x], padded to ldp with ones
    int ldp, n, N, D;
    float syy, tau;
    double sst, sqrt_syy;
    float E1, Smax;                      // filter window and coefficient bound (FP32 RSS units / sqrt(syy) units)
    const TileInfo* tiles;
    int n_tiles;
    int64_t n_items;
    int* counter;
    unsigned long long* ub_key;          // running bound B (ordered FP64 key)
    double tie64;
    const double* G64;                   // FP64 Gram (ld64) and moments for the confirmations
    const double* b64;
    int ld64;
    double syy64;
    uint64_t* band;
    unsigned* band_count;
    int64_t band_cap;
    float* band_r32;
    unsigned long long* examined;
    unsigned long long* candidates;      // subsets sent to the exact test
    const unsigned* prefix_mask;         // optional: one bit per (D-2)-prefix in colex order;
                                         //   prefixes whose bit is clear are skipped
};

// a posteriori bound on |RSS_FP32 - RSS| (the same formula as the two-pass form)
__device__ __forceinline__ float tile_apost_err(const TileArgs& A, float s, float rss) {
    const float u = 5.9604644775390625e-8f;
    const float c1 = 1.f + 3.1f * (float)(A.D + 1);
    return 2.f * u * ((float)A.N * (2.f * (float)A.sqrt_syy * s + c1 * s * s) +
                      (float)(A.D + 3) * (2.f * (float)A.sst + fabsf(rss)));
}

// r-th DP-combination in colex order, as colex_unrank but from FP32 estimates of the
// largest element (sqrt / cbrt of the rank) corrected by exact 64-bit integer steps: the
// GB300 FP64 pipe runs at a small fraction of the FP32 rate
__device__ __forceinline__ int64_t top2_fast(int64_t r) {
    int64_t m = (int64_t)((1.f + sqrtf(1.f + 8.f * (float)r)) * 0.5f);
    if (m < 1) m = 1;
    while (m > 1 && binom2(m) > r) --m;
    while (binom2(m + 1) <= r) ++m;
    return m;
}
__device__ __forceinline__ int64_t top3_fast(int64_t r) {
    int64_t m = (int64_t)cbrtf(6.f * (float)r) + 1;
    if (m < 2) m = 2;
    while (m > 2 && binom3(m) > r) --m;
    while (binom3(m + 1) <= r) ++m;
    return m;
}
template <int DP> __device__ __forceinline__ void colex_unrank_fast(int64_t r, int (&p)[DP > 0 ? DP : 1]) {
    if (DP == 0) return;
    if (DP == 1) { p[0] = (int)r; return; }
    int64_t m;
    if (DP >= 3) { m = top3_fast(r); p[DP > 2 ? 2 : 0] = (int)m; r -= binom3(m); }
    m = top2_fast(r);
    p[1] = (int)m;
    p[0] = (int)(r - binom2(m));
}

// prefix factor of one warp's current prefix, in shared memory (read by the exact test)
struct PrefixSm {
    int pre[4];
    float L[3][3], invd[3], wv[3];
};

// prefix-reduced values of feature x: R[m][x], dp = G[x][x] - sum R^2, np = b[x] - sum R w
template <int DP>
__device__ __forceinline__ void prefix_reduce(const TileArgs& A, const int (&pre)[DP > 0 ? DP : 1],
                                              const float (&L)[DP > 0 ? DP : 1][DP > 0 ? DP : 1],
                                              const float (&invd)[DP > 0 ? DP : 1], const float (&wv)[DP > 0 ? DP : 1],
                                              int x, float (&r)[DP > 0 ? DP : 1], float& dp, float& np) {
    dp = A.diag[x];
    np = A.b[x];
#pragma unroll
    for (int m = 0; m < DP; ++m) {
        float v = A.G[(size_t)pre[m] * A.ldp + x];
#pragma unroll
        for (int q = 0; q < m; ++q) v -= r[q] * L[m][q];
        r[m] = v * invd[m];
        dp -= r[m] * r[m];
        np -= r[m] * wv[m];
    }
}

// |L_P^-T v|_1
template <int DP>
__device__ __forceinline__ float back_l1(const float (&L)[DP > 0 ? DP : 1][DP > 0 ? DP : 1],
                                         const float (&invd)[DP > 0 ? DP : 1], const float (&v)[DP > 0 ? DP : 1]) {
    float g[DP > 0 ? DP : 1];
    float s = 0.f;
#pragma unroll
    for (int j = DP - 1; j >= 0; --j) {
        float t = v[j];
#pragma unroll
        for (int m = j + 1; m < DP; ++m) t -= L[m][j] * g[m];
        g[j] = t * invd[j];
        s += fabsf(g[j]);
    }
    return s;
}

// per-warp row record: R[.][i1], 1/sqrt(d1), w1, c, S1, Rk, flags (bit 1: pivots of the
// prefix and of i1 are above tau), padded to a multiple of 4 words
__host__ __device__ constexpr int row_words(int DP) { return ((DP + 6) + 3) & ~3; }

template <int DP>
__device__ __forceinline__ void add_band(const TileArgs& A, const int (&pos)[DP + 2], float r32) {
    const unsigned slot = atomicAdd(A.band_count, 1u);
    if (slot < A.band_cap) {
        uint64_t k = 0;
        int s = 0;
        const int W = pos_bits(DP + 2);
#pragma unroll
        for (int m = 0; m < DP + 2; ++m) { k |= (uint64_t)pos[m] << s; s += W; }
        A.band[slot] = k;
        if (A.band_r32) A.band_r32[slot] = r32;
    }
}

// the exact decision for one candidate (i1 = a + k, column x); returns the lane's new bound
template <int DP>
__device__ __noinline__ double tile_exact(const TileArgs& A, const PrefixSm* Ps, const float* rowrec, const float* colv,
                                          int a, int k, int off, int cb, float g, double B, double thr, float thr32) {
    const int i1 = a + k, x = cb + off;
    if (!(x > i1 && x < A.n)) return B;
    constexpr int RW = row_words(DP);
    int pre[DP > 0 ? DP : 1];
    float L[DP > 0 ? DP : 1][DP > 0 ? DP : 1], invd[DP > 0 ? DP : 1], wv[DP > 0 ? DP : 1];
#pragma unroll
    for (int m = 0; m < DP; ++m) {
        pre[m] = Ps->pre[m];
        invd[m] = Ps->invd[m];
        wv[m] = Ps->wv[m];
#pragma unroll
        for (int q = 0; q < DP; ++q) L[m][q] = Ps->L[m][q];
    }
    const float* rr_ = rowrec + k * RW;
    float r1[DP > 0 ? DP : 1];
#pragma unroll
    for (int m = 0; m < DP; ++m) r1[m] = rr_[m];
    const float isd1 = rr_[DP], w1 = rr_[DP + 1], base_c = rr_[DP + 2];
    const int flags = __float_as_int(rr_[DP + 5]);
    float rt[DP > 0 ? DP : 1];
#pragma unroll
    for (int m = 0; m < DP; ++m) rt[m] = colv[m * kTC + off];
    const float dp2 = colv[DP * kTC + off], np2 = colv[(DP + 1) * kTC + off];
    const float rr = g * isd1;
    const float d2 = dp2 - rr * rr;
    const float num = np2 - rr * w1;
    int pos[DP + 2];
#pragma unroll
    for (int m = 0; m < DP; ++m) pos[m] = pre[m];
    pos[DP] = i1;
    pos[DP + 1] = x;
    float r32 = __int_as_float(0x7fc00000);
    if ((flags & 2) && d2 > A.tau) {
        const float rss = (float)A.N * (base_c - num * num / d2);
        r32 = rss;
        if (!(rss <= thr32)) {
            // coefficients gamma = L^-T w and the a posteriori bound
            const float g2 = num / d2;
            const float g1 = (w1 - rr * g2) * isd1;
            float sg = fabsf(g2) + fabsf(g1);
            float gp[DP > 0 ? DP : 1];
#pragma unroll
            for (int j = DP - 1; j >= 0; --j) {
                float v = wv[j] - r1[j] * g1 - rt[j] * g2;
#pragma unroll
                for (int m = j + 1; m < DP; ++m) v -= L[m][j] * gp[m];
                gp[j] = v * invd[j];
                sg += fabsf(gp[j]);
            }
            if (!(rss - tile_apost_err(A, sg, rss) <= thr32)) return B;
        }
    }
    // FP64 confirmation from the FP64 Gram
    const double r64 = rss64(A.G64, A.b64, A.ld64, A.syy64, A.N, DP + 2, pos, nullptr);
    if (!(r64 <= thr)) return B;
    add_band<DP>(A, pos, r32);
    if (r64 < B) {
        atomicMin(A.ub_key, okey(r64));
        return r64;
    }
    return B;
}

// the warp's queued candidates (row k, column cb + offset) through the exact test;
// returns the warp's bound
template <int DP>
__device__ __forceinline__ double tile_flush(const TileArgs& A, const PrefixSm* Ps, const float* rowrec,
                                             const float* colv, const unsigned short* q, const float* qg, int qn,
                                             int a, int cb, int lane, double B) {
    // the threshold of the whole flush: B + tie (a lane's own B only decreases meanwhile,
    // so the flush keeps a superset of what the lane-current threshold would keep)
    const double thr = B + A.tie64;
    const float thr32 = __double2float_ru(thr);
    for (int e = lane; e < qn; e += 32) {
        const unsigned v = q[e];
        B = tile_exact<DP>(A, Ps, rowrec, colv, a, (int)(v >> 8), (int)(v & 255u), cb, qg[e], B, thr, thr32);
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) B = fmin(B, __shfl_xor_sync(0xffffffffu, B, o));
    return fmin(B, okey_inv(*(volatile unsigned long long*)A.ub_key));
}

template <int DP>
__global__ void __launch_bounds__(kTW * 32, 2) k_l0_tile(TileArgs A) {
    constexpr int DPa = DP > 0 ? DP : 1;
    constexpr int RW = row_words(DP);
    extern __shared__ __align__(16) unsigned char tile_smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per warp: row records, column table (DP + 2 rows of kTC values), candidate queue
    // (packed row / column and the candidate's g), prefix factor
    float* rowrec = reinterpret_cast<float*>(tile_smem) + (size_t)w * kTR * RW;
    float* colv = reinterpret_cast<float*>(tile_smem) + (size_t)kTW * kTR * RW + (size_t)w * (DP + 2) * kTC;
    float* qg = reinterpret_cast<float*>(tile_smem) + (size_t)kTW * (kTR * RW + (DP + 2) * kTC) + (size_t)w * kTQ;
    PrefixSm* Ps = reinterpret_cast<PrefixSm*>(reinterpret_cast<float*>(tile_smem) +
                                               (size_t)kTW * (kTR * RW + (DP + 2) * kTC + kTQ)) + w;
    unsigned short* q = reinterpret_cast<unsigned short*>(reinterpret_cast<PrefixSm*>(
                            reinterpret_cast<float*>(tile_smem) + (size_t)kTW * (kTR * RW + (DP + 2) * kTC + kTQ)) +
                        kTW) + (size_t)w * kTQ;
    const float N = (float)A.N;
    double B = INFINITY;                            // fmin ignores an unset (NaN) key
    B = fmin(B, okey_inv(*(volatile unsigned long long*)A.ub_key));
    unsigned long long my_examined = 0, my_cand = 0;

    // work units (tile, prefix) are claimed kClaim at a time from the global counter: one
    // same-address atomic per kClaim units instead of one per unit (about 3e5 units per
    // launch at C(400, 4)); the claim after the current one is requested when the current
    // one starts, so the atomic's round trip overlaps the current units (claims are handed
    // out in increasing order, so a warp that runs past the end holds no unit below it)
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(A.counter);
    int64_t ahead = 0;
    if (lane == 0) ahead = (int64_t)atomicAdd(ctr, (unsigned long long)kClaim);
    int64_t next = 0, end = 0;
    while (true) {
        if (next == end) {
            next = __shfl_sync(0xffffffffu, ahead, 0);
            end = next + kClaim;
            if (lane == 0) ahead = (int64_t)atomicAdd(ctr, (unsigned long long)kClaim);
        }
        const int64_t item = next++;
        if (item >= A.n_items) break;
        int lo = 0, hi = A.n_tiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.tiles[mid].item0 <= item) lo = mid; else hi = mid - 1;
        }
        const int a = A.tiles[lo].a, c = A.tiles[lo].c;
        const int64_t prank = item - A.tiles[lo].item0;
        if (A.prefix_mask && !((A.prefix_mask[prank >> 5] >> (prank & 31)) & 1u)) continue;

        // column groups j (columns c + 32 j + lane) and rows of this unit
        int pm = -1;
        int row_lo, row_hi, j_lo, jc, cb;
        float q2 = 0.f, pw2 = 0.f;
        float rt[8][DPa], dp2[8], np2[8];
        {
            // ---- prefix factor (warp-uniform, redundant in every lane) ---------------
            int pre[DPa];
            float L[DPa][DPa], invd[DPa], wv[DPa];
            colex_unrank_fast<DP>(prank, pre);
            bool ok = true;
#pragma unroll
            for (int j = 0; j < DP; ++j) {
                float dj = A.diag[pre[j]];
#pragma unroll
                for (int m = 0; m < j; ++m) dj -= L[j][m] * L[j][m];
                ok = ok && dj > A.tau;
                const float ljj = sqrtf(dj > 0.f ? dj : 1.f);
                L[j][j] = ljj;
                invd[j] = 1.f / ljj;
#pragma unroll
                for (int i = j + 1; i < DP; ++i) {
                    float v = A.G[(size_t)pre[i] * A.ldp + pre[j]];
#pragma unroll
                    for (int m = 0; m < j; ++m) v -= L[i][m] * L[j][m];
                    L[i][j] = v * invd[j];
                }
                float v = A.b[pre[j]];
#pragma unroll
                for (int m = 0; m < j; ++m) v -= L[j][m] * wv[m];
                wv[j] = v * invd[j];
                pw2 += wv[j] * wv[j];
            }
#pragma unroll
            for (int i = 0; i < DP; ++i)
#pragma unroll
                for (int j = i + 1; j < DP; ++j) L[i][j] = 0.f;
            if (lane == 0) {
#pragma unroll
                for (int m = 0; m < DP; ++m) {
                    Ps->pre[m] = pre[m];
                    Ps->invd[m] = invd[m];
                    Ps->wv[m] = wv[m];
#pragma unroll
                    for (int qq = 0; qq < DP; ++qq) Ps->L[m][qq] = L[m][qq];
                }
            }
            const float A0 = back_l1<DP>(L, invd, wv);
            if (DP > 0) pm = pre[DP > 0 ? DP - 1 : 0];
            row_lo = max(a, pm + 1);                                       // first row with subsets
            row_hi = min(a + kTR - 1, min(A.n - 2, c + kTC - 2));          // last
            // the lanes' columns cb + lane + 32 j: the window [cb, cb + kTC) holds the tile's
            // columns [c, min(c + kTC, n)) and ends at n for the last tile (cb may be < 0:
            // the padded copy has kTC zero columns on the left)
            cb = min(c, A.n - kTC);
            jc = (c - cb) >> 5;                                            // group of column c
            j_lo = max(jc, (row_lo + 1 - cb) >> 5);                        // first group right of row_lo

            // ---- columns: this lane's columns c + lane + 32 j in registers -----------
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int x = cb + lane + 32 * j;
                if (j >= j_lo && x >= c && x < A.n) {
                    prefix_reduce<DP>(A, pre, L, invd, wv, x, rt[j], dp2[j], np2[j]);
                    q2 = fmaxf(q2, back_l1<DP>(L, invd, rt[j]));
                } else {
#pragma unroll
                    for (int m = 0; m < DP; ++m) rt[j][m] = 0.f;
                    dp2[j] = 1.f;
                    np2[j] = 0.f;
                }
#pragma unroll
                for (int m = 0; m < DP; ++m) colv[m * kTC + lane + 32 * j] = rt[j][m];
                colv[DP * kTC + lane + 32 * j] = dp2[j];
                colv[(DP + 1) * kTC + lane + 32 * j] = np2[j];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q2 = fmaxf(q2, __shfl_xor_sync(0xffffffffu, q2, o));

            // ---- rows: record per row in shared memory --------------------------------
            for (int i1 = row_lo + lane; i1 <= row_hi; i1 += 32) {
                float* rr_ = rowrec + (i1 - a) * RW;
                float r1[DPa], d1, n1;
                prefix_reduce<DP>(A, pre, L, invd, wv, i1, r1, d1, n1);
                const bool piv = ok && d1 > A.tau;
                const float isd1 = 1.f / sqrtf(d1 > 0.f ? d1 : 1.f);
                const float w1 = n1 * isd1;
                const float a1 = back_l1<DP>(L, invd, r1);
                const float S0 = A0 + (1.f + a1) * fabsf(w1) * isd1;
                const float S1 = 1.02f * ((1.f + a1) * isd1 * 1.0001f + 1.f + q2);
#pragma unroll
                for (int m = 0; m < DP; ++m) rr_[m] = r1[m];
                rr_[DP] = isd1;
                rr_[DP + 1] = w1;
                rr_[DP + 2] = A.syy - (pw2 + w1 * w1);
                rr_[DP + 3] = S1;
                rr_[DP + 4] = piv ? A.Smax - 1.02f * S0 : -INFINITY;
                rr_[DP + 5] = __int_as_float(piv ? 2 : 0);
                const int lo_c = max(c, i1 + 1), hi_c = min(c + kTC, A.n);
                if (hi_c > lo_c) my_examined += (unsigned long long)(hi_c - lo_c);
            }
        }
        __syncwarp();

        // ---- sweep -------------------------------------------------------------------
        // the column values in pairs of groups (2 jp, 2 jp + 1): the per-subset arithmetic
        // runs as paired FP32 instructions, the same roundings as one column at a time
        p2 rtp[4][DPa], dpp[4], npp[4];
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
#pragma unroll
            for (int m = 0; m < DP; ++m) rtp[jp][m] = pk2(rt[2 * jp][m], rt[2 * jp + 1][m]);
            dpp[jp] = pk2(dp2[2 * jp], dp2[2 * jp + 1]);
            npp[jp] = pk2(np2[2 * jp], np2[2 * jp + 1]);
        }
        // this lane's columns that belong to the tile: bits j with c <= cb + lane + 32 j < n
        unsigned nmask = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int x = cb + lane + 32 * j;
            nmask |= (x >= c && x < A.n) ? (1u << j) : 0u;
        }
        int qn = 0;                                     // queue length (warp-uniform)
        float thrN = (float)((B + A.tie64) / (double)A.N) + A.E1 / N;
        int i1 = row_lo;
        // rows in segments of equal first live group J (the groups holding a column right
        // of i1 are J .. 7), so that every segment's group range is fixed at compile time
#pragma unroll
        for (int J = 0; J < 8; ++J) {
            const int seg_end = J < j_lo ? row_lo - 1 : (J == 7 ? row_hi : min(row_hi, cb + 32 * J + 30));
            for (; i1 <= seg_end; ++i1) {
                const int k = i1 - a;
                const float4* rv = reinterpret_cast<const float4*>(rowrec + k * RW);
                float rec[RW];
#pragma unroll
                for (int v4 = 0; v4 < RW / 4; ++v4) {
                    const float4 t = rv[v4];
                    rec[4 * v4] = t.x; rec[4 * v4 + 1] = t.y; rec[4 * v4 + 2] = t.z; rec[4 * v4 + 3] = t.w;
                }
                // per row: 1/d1 and w1/sqrt(d1), so that r = g/sqrt(d1) is never formed:
                // d2 = dp2 - g^2/d1, num = np2 - g w1/sqrt(d1)
                const float isd1 = rec[DP], w1 = rec[DP + 1];
                const float id1 = isd1 * isd1, w1s = w1 * isd1;
                const float S1 = rec[DP + 3], Rk = rec[DP + 4];
                const float cB = rec[DP + 2] - thrN;
                // columns right of i1: j >= js, js the smallest j with cb + lane + 32 j > i1
                const int dj = i1 - cb - lane;
                const int js = dj < 0 ? 0 : (dj >> 5) + 1;
                const unsigned vmask = nmask & (js >= 8 ? 0u : (0xFFu << js));
                const float* grow = A.G + (size_t)i1 * A.ldp + cb + lane;
                float gv[8];
#pragma unroll
                for (int j = J; j < 8; ++j) gv[j] = grow[32 * j];
                unsigned mask = 0;
                // per column: g = G - sum R R, d2 = dp2 - g^2 / d1, num = np2 - g w1 / sqrt(d1),
                // f = num^2 - cB d2, e = S1 |num| - Rk d2 (as fma(-a, b, c) and fma(a, a, -(c d)))
                // dismissed <=> f < 0 and e <= 0 and d2 > tau, evaluated without branches
                auto decide = [&](int j, float d2, float num, float f) {
                    const float e = fmaf(S1, fabsf(num), -(Rk * d2));
                    const bool dismiss = (f < 0.f) & (e <= 0.f) & (d2 > A.tau);
                    mask |= (unsigned)(!dismiss) << j;
                };
                if (J & 1) {           // a first group without its pair partner
                    float g = gv[J];
                    float rtJ[DPa], dJ, nJ, u;
#pragma unroll
                    for (int m = 0; m < DP; ++m) up2(rtp[J >> 1][m], u, rtJ[m]);
                    up2(dpp[J >> 1], u, dJ);
                    up2(npp[J >> 1], u, nJ);
#pragma unroll
                    for (int m = 0; m < DP; ++m) g = fmaf(-rec[m], rtJ[m], g);
                    gv[J] = g;
                    const float d2 = fmaf(-(g * g), id1, dJ);
                    const float num = fmaf(-g, w1s, nJ);
                    decide(J, d2, num, fmaf(num, num, -(cB * d2)));
                }
                {
                    p2 nrec[DPa];
#pragma unroll
                    for (int m = 0; m < DP; ++m) nrec[m] = pk2(-rec[m], -rec[m]);
                    const p2 nid1 = pk2(-id1, -id1), nw1s = pk2(-w1s, -w1s), ncB = pk2(-cB, -cB);
#pragma unroll
                    for (int jp = (J + 1) >> 1; jp < 4; ++jp) {
                        p2 g = pk2(gv[2 * jp], gv[2 * jp + 1]);
#pragma unroll
                        for (int m = 0; m < DP; ++m) g = fma2(nrec[m], rtp[jp][m], g);
                        const p2 d2 = fma2(mul2(g, g), nid1, dpp[jp]);
                        const p2 num = fma2(g, nw1s, npp[jp]);
                        const p2 f = fma2(num, num, mul2(ncB, d2));
                        float ga, gb, da, db, na, nb, fa, fb;
                        up2(g, ga, gb); up2(d2, da, db); up2(num, na, nb); up2(f, fa, fb);
                        gv[2 * jp] = ga; gv[2 * jp + 1] = gb;
                        decide(2 * jp, da, na, fa);
                        decide(2 * jp + 1, db, nb, fb);
                    }
                }
                mask &= vmask;
                if (__any_sync(0xffffffffu, mask != 0)) {
                    const int cnt = __popc(mask);
                    int off = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, off, o);
                        if (lane >= o) off += t;
                    }
                    const int total = __shfl_sync(0xffffffffu, off, 31);
                    off -= cnt;
#pragma unroll
                    for (int j = J; j < 8; ++j) {
                        if (!((mask >> j) & 1u)) continue;
                        q[qn + off] = (unsigned short)((k << 8) | (lane + 32 * j));
                        qg[qn + off] = gv[j];
                        ++off;
                    }
                    qn += total;
                    __syncwarp();
                    if (qn > kTQ - kTC) {
                        B = tile_flush<DP>(A, Ps, rowrec, colv, q, qg, qn, a, cb, lane, B);
                        my_cand += qn;
                        qn = 0;
                        thrN = (float)((B + A.tie64) / (double)A.N) + A.E1 / N;
                    }
                }
            }
        }
        if (qn > 0) {
            B = tile_flush<DP>(A, Ps, rowrec, colv, q, qg, qn, a, cb, lane, B);
            my_cand += qn;
        }
        __syncwarp();
    }
    my_examined = l0_warp_sum(my_examined);
    if (lane == 0) {
        atomicAdd(A.examined, my_examined);
        atomicAdd(A.candidates, my_cand);
    }
}

// dynamic shared memory of k_l0_tile<DP>
__host__ __device__ constexpr size_t tile_smem_bytes(int DP) {
    return sizeof(float) * (size_t)kTW * (kTR * row_words(DP) + (DP + 2) * kTC + kTQ) + sizeof(PrefixSm) * kTW +
           sizeof(unsigned short) * (size_t)kTW * kTQ;
}

// ---------------------------------------------------------------------------------
// certificate of a D = 5 incumbent by superset bounds
// ---------------------------------------------------------------------------------
// Every 5-subset extending the prefix P = {a < b < p2} with two features above p2 is a
// subset of T(P) = {a, b} U [p2, n), so its RSS is at least RSS(T(P)): least squares on a
// superset can only fit better.  With L the Cholesky factor of G in reversed feature order
// (row r <-> feature n-1-r), the leading m x m block of L factors the suffix [n-m, n), and
// row r of L (r >= m, first m entries) is L_m^-1 applied to the Gram column of feature
// n-1-r: the projections a pair {a, b} needs.  So for every prefix
//     RSS(T) = N (syy - |w_m|^2 - t^T S^-1 t),   m = n - p2,
// with w = L^-1 b (reversed), S_uv = G_uv - sum_{j<m} L[r_u][j] L[r_v][j] and
// t_u = b_u - sum_{j<m} L[r_u][j] w[j] (u, v in {a, b}) -- running sums over m.

// reversed-order FP64 Cholesky of G (n x n, ld) and w = L^-1 b (reversed); *m_ok: the
// number of leading columns with a pivot above tau (the suffixes that have a factor)
__global__ void __launch_bounds__(1024) k_rev_chol(const double* __restrict__ G, const double* __restrict__ b,
                                                  int ld, int n, double tau, double* __restrict__ L,
                                                  double* __restrict__ w, int* __restrict__ m_ok) {
    __shared__ double s_ljj, s_red[32];
    __shared__ int s_stop;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) { s_stop = 0; *m_ok = n; }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const int oj = n - 1 - j;
        // pivot: G_rev[j][j] - |L[j][0..j)|^2
        double p = 0.0;
        for (int k = threadIdx.x; k < j; k += blockDim.x) p += L[(size_t)j * n + k] * L[(size_t)j * n + k];
        p = l0_warp_sum(p);
        if (lane == 0) s_red[wid] = p;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < nw; ++q) t += s_red[q];
            const double dj = G[(size_t)oj * ld + oj] - t;
            if (!(dj > tau)) { s_stop = 1; *m_ok = j; }
            s_ljj = sqrt(dj > 0.0 ? dj : 1.0);
            L[(size_t)j * n + j] = s_ljj;
            // w[j] = (b_rev[j] - L[j][0..j) . w[0..j)) / L[j][j]
            double v = b[oj];
            for (int k = 0; k < j; ++k) v -= L[(size_t)j * n + k] * w[k];
            w[j] = v / s_ljj;
        }
        __syncthreads();
        if (s_stop) return;
        // rows i > j, one warp per row: L[i][j] = (G_rev[i][j] - L[i][0..j) . L[j][0..j)) / L[j][j]
        for (int i = j + 1 + wid; i < n; i += nw) {
            double v = 0.0;
            for (int k = lane; k < j; k += 32) v += L[(size_t)i * n + k] * L[(size_t)j * n + k];
            v = l0_warp_sum(v);
            if (lane == 0) L[(size_t)i * n + j] = (G[(size_t)(n - 1 - i) * ld + oj] - v) / s_ljj;
        }
        __syncthreads();
    }
}

// one thread per pair a < b: the superset bound of every prefix {a, b, p2}, p2 = n-m for
// m = 3 .. n-b-1; a prefix survives (bit set) unless the bound clears thr, or its suffix has
// no factor (m > m_ok) or the 2 x 2 Schur complement is not positive
__global__ void k_superset_mask(const double* __restrict__ G, const double* __restrict__ b, int ld, int n, int N,
                                double syy, const double* __restrict__ L, const double* __restrict__ w,
                                const double* __restrict__ q, const int* __restrict__ m_ok_p, double thr,
                                unsigned* __restrict__ mask, unsigned long long* __restrict__ survivors) {
    const int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npair = (int64_t)n * (n - 1) / 2;
    if (pr >= npair) return;
    // pair rank -> (a < b): b the largest with b (b-1) / 2 <= pr
    int bb = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) * 0.5);
    while (bb > 1 && (int64_t)bb * (bb - 1) / 2 > pr) --bb;
    while ((int64_t)(bb + 1) * bb / 2 <= pr) ++bb;
    const int aa = (int)(pr - (int64_t)bb * (bb - 1) / 2);
    if (bb > n - 3) return;
    const int m_ok = *m_ok_p;
    const int ra = n - 1 - aa, rb = n - 1 - bb;
    const double* La = L + (size_t)ra * n;
    const double* Lb = L + (size_t)rb * n;
    double saa = 0.0, sab = 0.0, sbb = 0.0, ta = 0.0, tb = 0.0;
    const double gaa = G[(size_t)aa * ld + aa], gab = G[(size_t)aa * ld + bb], gbb = G[(size_t)bb * ld + bb];
    const double pre2 = (double)bb * (bb - 1) / 2 + aa;          // C(b, 2) + a
    unsigned long long surv = 0;
    for (int m = 1; m <= n - bb - 1; ++m) {
        const int j = m - 1;
        if (m <= m_ok) {
            const double la = La[j], lb = Lb[j], wj = w[j];
            saa += la * la; sab += la * lb; sbb += lb * lb; ta += la * wj; tb += lb * wj;
        }
        if (m < 3) continue;
        const int p2 = n - m;
        bool keep = true;
        if (m <= m_ok) {
            const double Saa = gaa - saa, Sab = gab - sab, Sbb = gbb - sbb;
            const double Ta = b[aa] - ta, Tb = b[bb] - tb;
            const double det = Saa * Sbb - Sab * Sab;
            if (Saa > 0.0 && det > 1e-12 * Saa * Sbb) {
                const double extra = (Sbb * Ta * Ta - 2.0 * Sab * Ta * Tb + Saa * Tb * Tb) / det;
                const double lb_rss = (double)N * (syy - q[m] - extra);
                keep = !(lb_rss > thr);
            }
        }
        if (keep) {
            const int64_t rank = (int64_t)p2 * (p2 - 1) * (p2 - 2) / 6 + (int64_t)pre2;
            atomicOr(&mask[rank >> 5], 1u << (rank & 31));
            ++surv;
        }
    }
    if (surv) atomicAdd(survivors, surv);
}

// q[m] = |w[0..m)|^2, m = 0 .. n
__global__ void k_prefix_sq(const double* __restrict__ w, int n, const int* __restrict__ m_ok, double* __restrict__ q) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        q[0] = 0.0;
        for (int m = 1; m <= n; ++m) {
            if (m <= *m_ok) s += w[m - 1] * w[m - 1];
            q[m] = s;
        }
    }
}

// greedy forward selection in FP64: its D-subset's RSS is an upper bound of the minimum
__global__ void k_greedy_bound(const double* __restrict__ G, const double* __restrict__ b, int ld, double syy, int N,
                               int n, int D, unsigned long long* ub_key) {
    __shared__ double s_val[256];
    __shared__ int s_idx[256];
    __shared__ int sel[kMaxDim];
    int pos[kMaxDim];
    for (int t = 0; t < D; ++t) {
        double best = INFINITY;
        int bi = -1;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            bool used = false;
            for (int j = 0; j < t; ++j) used |= sel[j] == x;
            if (used) continue;
            for (int j = 0; j < t; ++j) pos[j] = sel[j];
            pos[t] = x;
            const double r = rss64(G, b, ld, syy, N, t + 1, pos, nullptr);
            if (r < best) { best = r; bi = x; }
        }
        s_val[threadIdx.x] = best;
        s_idx[threadIdx.x] = bi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double bv = INFINITY;
            int bx = -1;
            for (int q = 0; q < (int)blockDim.x; ++q)
                if (s_idx[q] >= 0 && s_val[q] < bv) { bv = s_val[q]; bx = s_idx[q]; }
            if (bx < 0) {                       // every extension singular: give up (bound stays)
                sel[t] = -1;
            } else {
                sel[t] = bx;
                if (t == D - 1) atomicMin(ub_key, okey(bv));
            }
        }
        __syncthreads();
        if (sel[t] < 0) return;
    }
}

// padded FP32 copies for the tiled enumeration: row i of Gp holds kTC zero columns, then
// (float)G[i][0..n), then zeros up to the stride ldp; bp, diag: (float)b, G[x][x] (padding 0, 1)
__global__ void k_pad_gram(const double* __restrict__ G, const double* __restrict__ b, int ld, int n, int ldp,
                           float* __restrict__ Gp, float* __restrict__ bp, float* __restrict__ dg) {
    const int64_t total = (int64_t)n * ldp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldp), x = (int)(e % ldp) - kTC;
        Gp[e] = x >= 0 && x < n ? (float)G[(size_t)i * ld + x] : 0.f;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ldp; j += gridDim.x * blockDim.x) {
        bp[j] = j < n ? (float)b[j] : 0.f;
        dg[j] = j < n ? (float)G[(size_t)j * ld + j] : 1.f;
    }
}

}  // namespace
}  // namespace sg
