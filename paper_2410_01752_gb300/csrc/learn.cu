// learn.cu — learned subset proposal for the l0 search (§2.3, Eq. 7) at D = 5.
//
// Scoring every D-subset with a network costs about 1e3 exact solves each, so the search's
// prefixes are ranked instead: for every 3-subset {p0 < p1 < p2} of the n screened features,
// its greedy completion (the two features above p2 that lower its RSS most) gives a base
// score, log10 of that 5-subset's RSS/SST, and the network predicts from the completion's
// statistics how much lower the prefix's best completion goes; the prefixes are taken by
// base + correction, best first, until their extensions make up a given fraction of
// C(n, 5), and only those extensions are solved, exactly (the same FP32
// enumeration with FP64 confirmation as the full search).  The full search stays the
// fallback and the judge.
//
// The network: 20 inputs describing a candidate 5-subset (the upper triangle of its 5 x 5
// standardised sub-Gram in row order and its 5 correlations with the target); for a prefix
// the candidate is the prefix completed greedily by the two features that lower its RSS
// most.  Two hidden layers of 256 with ReLU, one output.  Weights are FP32 masters
// with BF16 copies; activations and gradients are BF16; products accumulate in FP32.  The
// three 256-wide contractions of a step (forward H1 W2^T, backward dZ2 W2 and dZ2^T H1) and
// the input layer (K padded to 64) run on the tcgen05 tensor cores: C = A B^T with A and B
// BF16, K-major, staged by TMA into a 4-stage ring, one elected thread issuing tcgen05.mma
// into a TMEM accumulator, the epilogue reading TMEM (tcgen05.ld) and applying bias + ReLU
// (BF16 out, plus a transposed copy for the backward pass) or storing FP32.  Training is
// MSE with Adam, all on the device.
#include "l0_device.cuh"
#include "tc_device.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

namespace sg {
namespace {

constexpr int kIn = SISSO_MLP_IN;          // 20
constexpr int kInPad = 64;                 // K of the input layer (one 128-byte TMA row)
constexpr int kHid = SISSO_MLP_HIDDEN;     // 256
constexpr int GT = 128;                    // output tile (M = N = 128)
constexpr int GBK = 64;                    // K per stage
constexpr int GST = 2;                     // stages (2 CTAs per SM)
constexpr int kGemmThreads = 128;

// parameter layout (FP32 masters): W1 [256 x 20], b1 [256], W2 [256 x 256], b2 [256], w3 [256], b3
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid, kParams = oB3 + 1;
static_assert(kParams == SISSO_MLP_PARAMS, "parameter layout");

// one CTA: a 128 x BN output tile over all of K, in 64-wide stages through a 2-slot ring
template <int BN>
struct GemmSmem {
    uint8_t a[GST][GT * GBK * 2];
    uint8_t b[GST][BN * GBK * 2];
    uint64_t full[GST], empty[GST], done;
    uint32_t tmem_base;
};

enum : int { EPI_F32 = 0, EPI_RELU = 1 };

struct GemmArgs {
    int nk;                   // K / 64
    int m_tiles;              // output row tiles
    int rows;                 // valid output rows (M before padding)
    // EPI_F32
    float* C;
    int ldc;
    int cols;                 // valid output columns (a multiple of 32)
    // EPI_RELU
    const float* bias;
    __nv_bfloat16* H;         // rows x ldh
    int ldh;
    __nv_bfloat16* HT;        // optional transposed copy (cols x ldt)
    int ldt;
    int* err;
    uint32_t idesc;
};

// C[M x N] = A[M x K] B[N x K]^T: warp 0 streams the A and B tiles of each K stage with TMA,
// warp 1 issues tcgen05.mma (M = 128, N = BN, K = 16) into a BN-column TMEM accumulator,
// all four warps read it back (warp w: rows 32w..32w+31) and store it, each lane writing
// its row's 32 consecutive values with 16-byte stores
template <int EPI, int BN>
__global__ void __launch_bounds__(kGemmThreads, 2)
k_gemm_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, GemmArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using SM = GemmSmem<BN>;
    SM& S = *reinterpret_cast<SM*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t kA = GT * GBK * 2, kB = BN * GBK * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x % A.m_tiles, tj = blockIdx.x / A.m_tiles;
    const int nk = A.nk;
    if (threadIdx.x == 0) {
        for (int s = 0; s < GST; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 1); }
        mbar_init(&S.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    __shared__ int failed;
    if (threadIdx.x == 0) failed = 0;
    __syncthreads();
    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % GST;
            const uint32_t ph = (uint32_t)(ks / GST) & 1u;
            if (ks >= GST && !mbar_wait(&S.empty[s], ph ^ 1u)) { failed = 1; break; }
            mbar_expect_tx(&S.full[s], kA + kB);
            tma_load_2d(S.a[s], &map_a, ks * GBK, ti * GT, &S.full[s]);
            tma_load_2d(S.b[s], &map_b, ks * GBK, tj * BN, &S.full[s]);
            ++issued;
        }
        if (failed)
            for (int ks = (issued > GST ? issued - GST : 0); ks < issued; ++ks)
                mbar_wait(&S.full[ks % GST], (uint32_t)(ks / GST) & 1u);
    } else if (warp == 1 && lane == 0) {
        bool ok = true;
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % GST;
            if (!mbar_wait(&S.full[s], (uint32_t)(ks / GST) & 1u)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = desc_sw128(smem_u32(S.a[s])), db = desc_sw128(smem_u32(S.b[s]));
#pragma unroll
            for (int k = 0; k < GBK / 16; ++k)
                mma_f16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), A.idesc, (ks > 0 || k > 0) ? 1u : 0u);
            mma_commit(&S.empty[s]);
        }
        if (!ok) failed = 1;
        mma_commit(&S.done);
    }
    __syncwarp();
    const bool ready = mbar_wait(&S.done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ready || failed) {
        if (threadIdx.x == 0) atomicExch(A.err, 1);
    } else {
        const int row = ti * GT + warp * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < BN / 32; ++cb) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), r);
            const int col0 = tj * BN + cb * 32;
            if (EPI == EPI_F32) {
                if (row < A.rows && col0 < A.cols) {
                    float4* dst = reinterpret_cast<float4*>(A.C + (size_t)row * A.ldc + col0);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                             __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                }
            } else {
                uint32_t pk[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float h0 = row < A.rows ? fmaxf(__uint_as_float(r[2 * q]) + A.bias[col0 + 2 * q], 0.f) : 0.f;
                    const float h1 = row < A.rows ? fmaxf(__uint_as_float(r[2 * q + 1]) + A.bias[col0 + 2 * q + 1], 0.f) : 0.f;
                    const __nv_bfloat162 hb = __floats2bfloat162_rn(h0, h1);
                    pk[q] = *reinterpret_cast<const uint32_t*>(&hb);
                    if (A.HT) {
                        A.HT[(size_t)(col0 + 2 * q) * A.ldt + row] = hb.x;       // lanes = rows: coalesced
                        A.HT[(size_t)(col0 + 2 * q + 1) * A.ldt + row] = hb.y;
                    }
                }
                uint4* dst = reinterpret_cast<uint4*>(A.H + (size_t)row * A.ldh + col0);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// ---------------------------------------------------------------------------------
// CUDA-core parts of the network
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// inputs FP32 [M x 20] -> BF16 [Mpad x 64] (zero padded) and, for training, the transposed
// copy XT [128 x Mpad] (rows 20..127 zero) for the input layer's weight gradient
__global__ void k_pack_x(const float* __restrict__ X, int64_t M, int64_t Mpad, __nv_bfloat16* __restrict__ Xb,
                         __nv_bfloat16* __restrict__ XT) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Mpad * kInPad; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / kInPad;
        const int c = (int)(e % kInPad);
        const float v = (r < M && c < kIn) ? X[r * kIn + c] : 0.f;
        Xb[e] = __float2bfloat16(v);
        if (XT && c < GT) XT[(size_t)c * Mpad + r] = __float2bfloat16(v);
    }
    if (XT)
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)(GT - kInPad) * Mpad;
             e += (int64_t)gridDim.x * blockDim.x)
            XT[(size_t)kInPad * Mpad + e] = __float2bfloat16(0.f);
}

// output layer: out[r] = H2[r] . w3 + b3 (warp per row)
__global__ void k_head_fwd(const __nv_bfloat16* __restrict__ H2, int64_t M, const float* __restrict__ w3,
                           const float* __restrict__ b3, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < M;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int j = lane; j < kHid; j += 32) s += __bfloat162float(H2[r * kHid + j]) * w3[j];
        s = wsum(s);
        if (lane == 0) out[r] = s + b3[0];
    }
}

// loss and the output layer's backward: dout = 2 (out - t) / B; dZ2 = dout w3 (where H2 > 0)
// as BF16 with its transpose; grad of w3 and b3 accumulated
__global__ void k_head_bwd(const __nv_bfloat16* __restrict__ H2, const float* __restrict__ out,
                           const float* __restrict__ t, int B, const float* __restrict__ w3,
                           __nv_bfloat16* __restrict__ dZ2, __nv_bfloat16* __restrict__ dZ2T,
                           float* __restrict__ g_w3, float* __restrict__ g_b3, float* __restrict__ loss) {
    __shared__ float gw[kHid];
    __shared__ float red[32];
    for (int j = threadIdx.x; j < kHid; j += blockDim.x) gw[j] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float gb = 0.f, ls = 0.f;
    for (int r = blockIdx.x * nw + w; r < B; r += gridDim.x * nw) {
        const float e = out[r] - t[r];
        const float d = 2.f * e / (float)B;
        if (lane == 0) { gb += d; ls += e * e; }    // once per row
        for (int j = lane; j < kHid; j += 32) {
            const float h = __bfloat162float(H2[(size_t)r * kHid + j]);
            atomicAdd(&gw[j], d * h);
            const __nv_bfloat16 g = __float2bfloat16(h > 0.f ? d * w3[j] : 0.f);
            dZ2[(size_t)r * kHid + j] = g;
            dZ2T[(size_t)j * B + r] = g;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kHid; j += blockDim.x) atomicAdd(&g_w3[j], gw[j]);
    gb = wsum(gb);
    ls = wsum(ls);
    if (lane == 0) red[w] = gb;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int q = 0; q < nw; ++q) s += red[q];
        atomicAdd(g_b3, s);
    }
    __syncthreads();
    if (lane == 0) red[w] = ls;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int q = 0; q < nw; ++q) s += red[q];
        atomicAdd(loss, s / (float)B);
    }
}

// dZ1 = dH1 (where H1 > 0), BF16 and transposed
__global__ void k_relu_bwd(const float* __restrict__ dH1, const __nv_bfloat16* __restrict__ H1, int B,
                           __nv_bfloat16* __restrict__ dZ1T) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)B * kHid; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / kHid), j = (int)(e % kHid);
        const float h = __bfloat162float(H1[e]);
        dZ1T[(size_t)j * B + r] = __float2bfloat16(h > 0.f ? dH1[e] : 0.f);
    }
}

// bias gradient: row sums of a transposed BF16 gradient [256 x B] (warp per row)
__global__ void k_rowsum(const __nv_bfloat16* __restrict__ T, int B, float* __restrict__ g) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= kHid) return;
    float s = 0.f;
    for (int r = lane; r < B; r += 32) s += __bfloat162float(T[(size_t)j * B + r]);
    s = wsum(s);
    if (lane == 0) g[j] += s;
}

// the weight gradients from the GEMM outputs into the flat gradient vector
__global__ void k_collect_grads(const float* __restrict__ gW1, const float* __restrict__ gW2, float* __restrict__ g) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kHid * kHid; e += gridDim.x * blockDim.x) {
        g[oW2 + e] = gW2[e];
        if (e < kHid * kIn) {
            const int i = e / kIn, c = e % kIn;
            g[oW1 + e] = gW1[(size_t)i * GT + c];
        }
    }
}

// BF16 copies of the weights: W1 [256 x 64] (padded), W2 [256 x 256], W2^T
__global__ void k_weights_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ W1b,
                               __nv_bfloat16* __restrict__ W2b, __nv_bfloat16* __restrict__ W2Tb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kHid * kHid; e += gridDim.x * blockDim.x) {
        const int i = e / kHid, j = e % kHid;
        const __nv_bfloat16 w = __float2bfloat16(p[oW2 + e]);
        W2b[e] = w;
        W2Tb[(size_t)j * kHid + i] = w;
        if (e < kHid * kInPad) {
            const int r = e / kInPad, c = e % kInPad;
            W1b[e] = __float2bfloat16(c < kIn ? p[oW1 + r * kIn + c] : 0.f);
        }
    }
}

// one training batch gathered by a permutation
__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ t, const int64_t* __restrict__ idx,
                         int B, float* __restrict__ xb, float* __restrict__ tb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * kIn; e += gridDim.x * blockDim.x) {
        const int r = e / kIn, c = e % kIn;
        const int64_t i = idx[r];
        xb[e] = X[i * kIn + c];
        if (c == 0) tb[r] = t[i];
    }
}

// Adam (decoupled moments, bias correction by step)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// ---------------------------------------------------------------------------------
// prefixes: features, labels, selection
// ---------------------------------------------------------------------------------
__device__ __forceinline__ int64_t c3(int64_t m) { return m * (m - 1) * (m - 2) / 6; }
__device__ __forceinline__ int64_t c2(int64_t m) { return m * (m - 1) / 2; }

__device__ __forceinline__ void prefix_of(int64_t r, int& p0, int& p1, int& p2) {
    int64_t m = (int64_t)cbrt(6.0 * (double)r) + 1;
    while (m > 2 && c3(m) > r) --m;
    while (c3(m + 1) <= r) ++m;
    p2 = (int)m;
    r -= c3(m);
    int64_t q = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)r)) * 0.5);
    while (q > 1 && c2(q) > r) --q;
    while (c2(q + 1) <= r) ++q;
    p1 = (int)q;
    p0 = (int)(r - c2(q));
}

// Greedy completion of a prefix: with E the current positions (m of them) and L, w its
// Cholesky factor and forward solution, adding feature j lowers RSS / N by c_j^2 / d_j with
// v = L^-1 G[E][j], d_j = G[j][j] - |v|^2, c_j = b[j] - v . w.  Returns the j > lo that
// lowers it most (-1 if none) and extends L, w by it.
template <int M>
__device__ __forceinline__ int greedy_next(const double* __restrict__ G, const double* __restrict__ b, int n,
                                           const int (&E)[5], float (&L)[5][5], float (&w)[5], int lo, int skip) {
    int best = -1;
    float best_gain = -1.f, bv[5] = {0, 0, 0, 0, 0}, bd = 1.f, bc = 0.f;
    for (int j = lo + 1; j < n; ++j) {
        if (j == skip) continue;
        float v[5];
        float d = (float)G[(size_t)j * n + j], c = (float)b[j];
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float x = (float)G[(size_t)E[q] * n + j];
#pragma unroll
            for (int r = 0; r < q; ++r) x -= L[q][r] * v[r];
            v[q] = x / L[q][q];
            d -= v[q] * v[q];
            c -= v[q] * w[q];
        }
        if (!(d > 1e-6f)) continue;
        const float gain = c * c / d;
        if (gain > best_gain) {
            best_gain = gain; best = j; bd = d; bc = c;
#pragma unroll
            for (int q = 0; q < M; ++q) bv[q] = v[q];
        }
    }
    if (best >= 0) {
#pragma unroll
        for (int q = 0; q < M; ++q) L[M][q] = bv[q];
        L[M][M] = sqrtf(bd);
        w[M] = bc / L[M][M];
    }
    return best;
}

// network inputs of every 3-prefix (colex rank r): the prefix completed greedily by the two
// features that lower its RSS most (positions above p2), as a candidate 5-subset
// E = (p0, p1, p2, j1, j2): the upper triangle of its standardised sub-Gram in row order,
// then its correlations b_i / sqrt(syy).  A prefix without two such features keeps zeros
// in the missing slots (it has no extension either).  base (optional): log10 of the
// completion's RSS / SST, the score the network corrects.
__global__ void k_prefix_features(const double* __restrict__ G, const double* __restrict__ b, double inv_sy, int n,
                                  int64_t n_pre, float* __restrict__ X, int* __restrict__ plist,
                                  float* __restrict__ base) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_pre; r += (int64_t)gridDim.x * blockDim.x) {
        int E[5] = {0, 0, 0, -1, -1};
        prefix_of(r, E[0], E[1], E[2]);
        // Cholesky of the prefix (FP32; a singular prefix gets no completion)
        float L[5][5] = {}, w[5] = {};
        bool ok = true;
        for (int q = 0; q < 3 && ok; ++q) {
            float d = (float)G[(size_t)E[q] * n + E[q]];
            for (int m = 0; m < q; ++m) d -= L[q][m] * L[q][m];
            if (!(d > 1e-6f)) { ok = false; break; }
            L[q][q] = sqrtf(d);
            for (int i = q + 1; i < 3; ++i) {
                float x = (float)G[(size_t)E[i] * n + E[q]];
                for (int m = 0; m < q; ++m) x -= L[i][m] * L[q][m];
                L[i][q] = x / L[q][q];
            }
            float v = (float)b[E[q]];
            for (int m = 0; m < q; ++m) v -= L[q][m] * w[m];
            w[q] = v / L[q][q];
        }
        if (ok) {
            E[3] = greedy_next<3>(G, b, n, E, L, w, E[2], -1);
            if (E[3] >= 0) E[4] = greedy_next<4>(G, b, n, E, L, w, E[2], E[3]);
        }
        // base score: log10 of the greedy completion's RSS / SST = 1 - |w|^2 syy^-1
        if (base) {
            float q = 0.f;
            for (int i = 0; i < 5; ++i) q += (ok && E[4] >= 0) ? w[i] * w[i] : 0.f;
            const float frac = (ok && E[4] >= 0) ? 1.f - q * (float)(inv_sy * inv_sy) : 1.f;
            base[r] = log10f(fmaxf(frac, 1e-12f));
        }
        float* x = X + r * kIn;
        int q = 0;
        for (int i = 0; i < 5; ++i)
            for (int j = i; j < 5; ++j, ++q)
                x[q] = (E[i] >= 0 && E[j] >= 0) ? (float)G[(size_t)E[i] * n + E[j]] : 0.f;
        for (int i = 0; i < 5; ++i) x[15 + i] = E[i] >= 0 ? (float)(b[E[i]] * inv_sy) : 0.f;
        if (plist) { plist[3 * r] = E[0]; plist[3 * r + 1] = E[1]; plist[3 * r + 2] = E[2]; }
    }
}

__device__ __forceinline__ unsigned fkey32(float v) {
    const unsigned u = __float_as_uint(v);
    return (u >> 31) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey32_inv(unsigned k) {
    return __uint_as_float((k >> 31) ? (k & 0x7FFFFFFFu) : ~k);
}

// labels: per prefix, the lowest FP32 RSS over its extensions (enumeration items of D = 5)
template <int MODE_UNUSED>
__global__ void __launch_bounds__(kWarps * 32) k_prefix_labels(EnumArgs<float> A, unsigned* __restrict__ lab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tab = reinterpret_cast<float*>(smem_raw) + (size_t)w * 5 * A.n;
    while (true) {
        int item;
        if (lane == 0) item = atomicAdd(A.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= A.n_items) break;
        float best = INFINITY;
        unsigned long long key = 0, ex = 0;
        enum_item<float, 3, 0>(A, tab, item, best, key, 0.0, ex);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0 && best < INFINITY) atomicMin(&lab[item / A.cpp], fkey32(best));
    }
}

__global__ void k_add(float* __restrict__ a, const float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// weight of a prefix: its number of extensions C(n - 1 - p2, 2)
__device__ __forceinline__ uint64_t ext_count(int n, int p2) {
    const int64_t m = n - 1 - p2;
    return m >= 2 ? (uint64_t)(m * (m - 1) / 2) : 0;
}

// weighted radix select (one pass of 11 or 10 bits of the ordered key, lowest scores first)
__global__ void k_wsel_hist(const float* __restrict__ score, const int* __restrict__ plist, int n, int64_t n_pre,
                            int pass, const unsigned* __restrict__ state, unsigned long long* __restrict__ hist) {
    __shared__ unsigned long long h[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned prefix = state[0];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_pre; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = fkey32(score[r]);
        const uint64_t wgt = ext_count(n, plist[3 * r + 2]);
        if (pass == 0) atomicAdd(&h[k >> 21], wgt);
        else if (pass == 1) { if ((k >> 21) == prefix) atomicAdd(&h[(k >> 10) & 0x7FFu], wgt); }
        else { if ((k >> 10) == prefix) atomicAdd(&h[k & 0x3FFu], wgt); }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[pass * 2048 + i], h[i]);
}

// state (32-bit words): [0] prefix bits, [1] threshold key, [2..3] weight still to take
// (one 64-bit value, 8-byte aligned), [4] compacted count
__global__ void k_wsel_find(const unsigned long long* __restrict__ hist, int pass, unsigned* state,
                            unsigned long long budget) {
    if (threadIdx.x != 0) return;
    unsigned long long* rest = reinterpret_cast<unsigned long long*>(state + 2);
    const int nb = pass == 2 ? 1024 : 2048;
    const unsigned long long need = pass == 0 ? budget : *rest;
    unsigned long long cum = 0;
    int bin = nb - 1;
    for (int q = 0; q < nb; ++q) {
        const unsigned long long c = hist[pass * 2048 + q];
        if (cum + c >= need) { bin = q; break; }
        cum += c;
    }
    const unsigned pre = pass == 0 ? (unsigned)bin : pass == 1 ? ((state[0] << 11) | (unsigned)bin)
                                                               : ((state[0] << 10) | (unsigned)bin);
    state[0] = pre;
    *rest = need > cum ? need - cum : 0;
    if (pass == 2) state[1] = pre;
}

__global__ void k_wsel_compact(const float* __restrict__ score, const int* __restrict__ plist, int64_t n_pre,
                               const unsigned* __restrict__ state, int* __restrict__ out, unsigned* __restrict__ count,
                               int64_t cap, unsigned long long* __restrict__ taken) {
    const unsigned thr = state[1];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_pre; r += (int64_t)gridDim.x * blockDim.x) {
        if (fkey32(score[r]) <= thr) {
            const unsigned slot = atomicAdd(count, 1u);
            if (slot < cap) {
                out[3 * (int64_t)slot] = plist[3 * r];
                out[3 * (int64_t)slot + 1] = plist[3 * r + 1];
                out[3 * (int64_t)slot + 2] = plist[3 * r + 2];
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// host: GEMM launch
// ---------------------------------------------------------------------------------
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {GBK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI, int BN>
cudaError_t gemm_launch(cudaStream_t st, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& g,
                        int64_t grid) {
    const size_t smem = sizeof(GemmSmem<BN>) + 1024;
    cudaFuncSetAttribute(k_gemm_tc<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gemm_tc<EPI, BN><<<(unsigned)grid, kGemmThreads, smem, st>>>(ma, mb, g);
    return cudaGetLastError();
}

// C = A B^T with A [Mpad x K], B [Npad x K] (BF16, row-major = K-major); M, N multiples of
// 128; tiles 128 x 256 when N is a multiple of 256
cudaError_t gemm(cudaStream_t st, const __nv_bfloat16* Am, int64_t Mpad, const __nv_bfloat16* Bm, int64_t Npad, int K,
                 int epi, GemmArgs g) {
    const int bn = Npad % 256 == 0 ? 256 : GT;
    CUtensorMap ma, mb;
    if (!make_map(&ma, Am, Mpad, K, GT) || !make_map(&mb, Bm, Npad, K, bn)) return cudaErrorInvalidValue;
    g.nk = K / GBK;
    g.m_tiles = (int)(Mpad / GT);
    g.idesc = idesc_f16(1u, GT, bn);
    const int64_t grid = (Mpad / GT) * (Npad / bn);
    if (epi == EPI_F32) return bn == 256 ? gemm_launch<EPI_F32, 256>(st, ma, mb, g, grid) : gemm_launch<EPI_F32, GT>(st, ma, mb, g, grid);
    return bn == 256 ? gemm_launch<EPI_RELU, 256>(st, ma, mb, g, grid) : gemm_launch<EPI_RELU, GT>(st, ma, mb, g, grid);
}

int64_t pad128(int64_t m) { return (m + GT - 1) / GT * GT; }

}  // namespace
}  // namespace sg

// ===================================================================================
// the network object
// ===================================================================================
struct sisso_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float* p = nullptr;         // FP32 masters (kParams)
    float* g = nullptr;         // gradients
    float* m = nullptr;         // Adam moments
    float* v = nullptr;
    __nv_bfloat16* W1b = nullptr;   // [256 x 64]
    __nv_bfloat16* W2b = nullptr;   // [256 x 256]
    __nv_bfloat16* W2Tb = nullptr;
    int* err = nullptr;
    float* loss = nullptr;
    int64_t step = 0;
    // activations for a batch of up to cap rows
    int64_t cap = 0;
    __nv_bfloat16 *Xb = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *dZ2 = nullptr,
                  *dZ2T = nullptr, *dZ1T = nullptr;
    float *out = nullptr, *dH1 = nullptr, *gW1 = nullptr, *gW2 = nullptr, *tgt = nullptr, *xin = nullptr;
};

namespace sg {
namespace {

void mlp_free_acts(sisso_mlp* m) {
    void* ps[] = {m->Xb, m->XT, m->H1, m->H1T, m->H2, m->dZ2, m->dZ2T, m->dZ1T, m->out, m->dH1, m->gW1, m->gW2,
                  m->tgt, m->xin};
    for (void* q : ps) if (q) cudaFree(q);
    m->Xb = m->XT = m->H1 = m->H1T = m->H2 = m->dZ2 = m->dZ2T = m->dZ1T = nullptr;
    m->out = m->dH1 = m->gW1 = m->gW2 = m->tgt = m->xin = nullptr;
    m->cap = 0;
}

sisso_status mlp_reserve(sisso_mlp* m, int64_t rows, bool train) {
    const int64_t R = pad128(rows);
    if (R <= m->cap && (!train || m->dZ2)) return SISSO_OK;
    mlp_free_acts(m);
    bool ok = true;
    auto al = [&](void** q, size_t bytes) { if (ok && cudaMalloc(q, bytes) != cudaSuccess) ok = false; };
    al((void**)&m->xin, sizeof(float) * R * kIn);
    al((void**)&m->Xb, 2 * R * kInPad);
    al((void**)&m->H1, 2 * R * kHid);
    al((void**)&m->H2, 2 * R * kHid);
    al((void**)&m->out, sizeof(float) * R);
    if (train) {
        al((void**)&m->XT, 2 * (size_t)GT * R);
        al((void**)&m->H1T, 2 * (size_t)kHid * R);
        al((void**)&m->dZ2, 2 * R * kHid);
        al((void**)&m->dZ2T, 2 * (size_t)kHid * R);
        al((void**)&m->dZ1T, 2 * (size_t)kHid * R);
        al((void**)&m->dH1, sizeof(float) * R * kHid);
        al((void**)&m->gW1, sizeof(float) * kHid * GT);
        al((void**)&m->gW2, sizeof(float) * kHid * kHid);
        al((void**)&m->tgt, sizeof(float) * R);
    }
    if (!ok) { cudaGetLastError(); mlp_free_acts(m); return SISSO_ERR_OOM; }
    m->cap = R;
    return SISSO_OK;
}

// forward on rows already packed in m->Xb (Mpad rows); train: keep H1^T for the backward
cudaError_t mlp_forward_dev(sisso_mlp* m, int64_t M, bool train) {
    const int64_t Mpad = pad128(M);
    GemmArgs g{};
    g.rows = (int)std::min<int64_t>(M, INT32_MAX); g.err = m->err;
    g.bias = m->p + oB1; g.H = m->H1; g.ldh = kHid; g.HT = train ? m->H1T : nullptr; g.ldt = (int)Mpad;
    cudaError_t e = gemm(m->stream, m->Xb, Mpad, m->W1b, kHid, kInPad, EPI_RELU, g);
    if (e) return e;
    g.bias = m->p + oB2; g.H = m->H2; g.HT = nullptr;
    if ((e = gemm(m->stream, m->H1, Mpad, m->W2b, kHid, kHid, EPI_RELU, g))) return e;
    k_head_fwd<<<(unsigned)std::min<int64_t>((M * 32 + 255) / 256, 1 << 20), 256, 0, m->stream>>>(m->H2, M, m->p + oW3,
                                                                                                    m->p + oB3, m->out);
    return cudaGetLastError();
}

// gradients of the mean squared error on one batch (rows in Xb/XT, targets in tgt) into m->g
cudaError_t mlp_backward_dev(sisso_mlp* m, int B) {
    cudaMemsetAsync(m->g, 0, sizeof(float) * kParams, m->stream);
    k_head_bwd<<<std::max(1, std::min(1024, (B + 7) / 8)), 256, 0, m->stream>>>(m->H2, m->out, m->tgt, B, m->p + oW3,
                                                                                m->dZ2, m->dZ2T, m->g + oW3, m->g + oB3,
                                                                                m->loss);
    // dW2 = dZ2^T H1 ([256 x B] . [256 x B]^T), dH1 = dZ2 W2 ([B x 256] . (W2^T)^T)
    GemmArgs g{};
    g.err = m->err;
    g.rows = kHid; g.C = m->gW2; g.ldc = kHid; g.cols = kHid;
    cudaError_t e = gemm(m->stream, m->dZ2T, kHid, m->H1T, kHid, B, EPI_F32, g);
    if (e) return e;
    g.rows = B; g.C = m->dH1; g.ldc = kHid; g.cols = kHid;
    if ((e = gemm(m->stream, m->dZ2, B, m->W2Tb, kHid, kHid, EPI_F32, g))) return e;
    k_relu_bwd<<<std::max(1, std::min(4096, (B * kHid + 255) / 256)), 256, 0, m->stream>>>(m->dH1, m->H1, B, m->dZ1T);
    // dW1 = dZ1^T X ([256 x B] . [128 x B]^T, columns 0..19 used)
    g.rows = kHid; g.C = m->gW1; g.ldc = GT; g.cols = GT;
    if ((e = gemm(m->stream, m->dZ1T, kHid, m->XT, GT, B, EPI_F32, g))) return e;
    k_rowsum<<<(kHid * 32 + 255) / 256, 256, 0, m->stream>>>(m->dZ2T, B, m->g + oB2);
    k_rowsum<<<(kHid * 32 + 255) / 256, 256, 0, m->stream>>>(m->dZ1T, B, m->g + oB1);
    k_collect_grads<<<256, 256, 0, m->stream>>>(m->gW1, m->gW2, m->g);
    return cudaGetLastError();
}

void refresh_bf16(sisso_mlp* m) {
    k_weights_bf16<<<256, 256, 0, m->stream>>>(m->p, m->W1b, m->W2b, m->W2Tb);
}

sisso_status mlp_status(sisso_mlp* m, cudaError_t e) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return SISSO_ERR_CUDA; }
    int h = 0;
    cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost);
    return h ? SISSO_ERR_TIMEOUT : SISSO_OK;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" {

sisso_status sisso_mlp_create(uint64_t seed, sisso_mlp** out) {
    if (!out) return SISSO_ERR_ARG;
    *out = nullptr;
    sisso_mlp* m = new sisso_mlp();
    cudaGetDevice(&m->device);
    bool ok = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) == cudaSuccess;
    auto al = [&](void** q, size_t bytes) { if (ok && cudaMalloc(q, bytes) != cudaSuccess) ok = false; };
    al((void**)&m->p, sizeof(float) * kParams);
    al((void**)&m->g, sizeof(float) * kParams);
    al((void**)&m->m, sizeof(float) * kParams);
    al((void**)&m->v, sizeof(float) * kParams);
    al((void**)&m->W1b, 2 * kHid * kInPad);
    al((void**)&m->W2b, 2 * kHid * kHid);
    al((void**)&m->W2Tb, 2 * kHid * kHid);
    al((void**)&m->err, sizeof(int));
    al((void**)&m->loss, sizeof(float));
    if (!ok) { cudaGetLastError(); sisso_mlp_destroy(m); return SISSO_ERR_OOM; }
    // He-uniform initialisation from a seeded host generator; zero biases
    std::vector<float> p(kParams, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int n, int fan_in) {
        const float a = std::sqrt(6.f / (float)fan_in);
        std::uniform_real_distribution<float> u(-a, a);
        for (int i = 0; i < n; ++i) p[off + i] = u(rng);
    };
    fill(oW1, kHid * kIn, kIn);
    fill(oW2, kHid * kHid, kHid);
    fill(oW3, kHid, kHid);
    cudaMemcpy(m->p, p.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
    cudaMemset(m->m, 0, sizeof(float) * kParams);
    cudaMemset(m->v, 0, sizeof(float) * kParams);
    cudaMemset(m->err, 0, sizeof(int));
    refresh_bf16(m);
    if (mlp_status(m, cudaGetLastError())) { sisso_mlp_destroy(m); return SISSO_ERR_CUDA; }
    *out = m;
    return SISSO_OK;
}

void sisso_mlp_destroy(sisso_mlp* m) {
    if (!m) return;
    mlp_free_acts(m);
    void* ps[] = {m->p, m->g, m->m, m->v, m->W1b, m->W2b, m->W2Tb, m->err, m->loss};
    for (void* q : ps) if (q) cudaFree(q);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

sisso_status sisso_mlp_get_params(sisso_mlp* m, float* params) {
    if (!m || !params) return SISSO_ERR_ARG;
    return cudaMemcpy(params, m->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost) == cudaSuccess ? SISSO_OK
                                                                                                       : SISSO_ERR_CUDA;
}

sisso_status sisso_mlp_set_params(sisso_mlp* m, const float* params) {
    if (!m || !params) return SISSO_ERR_ARG;
    if (cudaMemcpy(m->p, params, sizeof(float) * kParams, cudaMemcpyDefault) != cudaSuccess) return SISSO_ERR_CUDA;
    refresh_bf16(m);
    m->step = 0;
    cudaMemsetAsync(m->m, 0, sizeof(float) * kParams, m->stream);
    cudaMemsetAsync(m->v, 0, sizeof(float) * kParams, m->stream);
    return mlp_status(m, cudaGetLastError());
}

sisso_status sisso_mlp_forward(sisso_mlp* m, const float* X, int64_t M, float* out) {
    if (!m || !X || !out || M < 1) return SISSO_ERR_ARG;
    sisso_status st = mlp_reserve(m, M, false);
    if (st) return st;
    cudaMemcpyAsync(m->xin, X, sizeof(float) * M * kIn, cudaMemcpyDefault, m->stream);
    const int64_t Mpad = pad128(M);
    k_pack_x<<<(unsigned)std::min<int64_t>((Mpad * kInPad + 255) / 256, 65535), 256, 0, m->stream>>>(m->xin, M, Mpad,
                                                                                                      m->Xb, nullptr);
    cudaError_t e = mlp_forward_dev(m, M, false);
    if (!e) e = cudaMemcpyAsync(out, m->out, sizeof(float) * M, cudaMemcpyDefault, m->stream);
    return mlp_status(m, e);
}

sisso_status sisso_mlp_gradients(sisso_mlp* m, const float* X, const float* t, int B, float* loss, float* grad) {
    if (!m || !X || !t || !grad || B < 1 || B % GT) return SISSO_ERR_ARG;
    sisso_status st = mlp_reserve(m, B, true);
    if (st) return st;
    cudaMemcpyAsync(m->xin, X, sizeof(float) * (size_t)B * kIn, cudaMemcpyDefault, m->stream);
    cudaMemcpyAsync(m->tgt, t, sizeof(float) * B, cudaMemcpyDefault, m->stream);
    k_pack_x<<<(unsigned)std::min<int64_t>(((int64_t)B * GT + 255) / 256, 65535), 256, 0, m->stream>>>(m->xin, B, B,
                                                                                                        m->Xb, m->XT);
    cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
    cudaError_t e = mlp_forward_dev(m, B, true);
    if (!e) e = mlp_backward_dev(m, B);
    if (!e) e = cudaMemcpyAsync(grad, m->g, sizeof(float) * kParams, cudaMemcpyDefault, m->stream);
    if (!e && loss) e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDefault, m->stream);
    return mlp_status(m, e);
}

sisso_status sisso_mlp_train(sisso_mlp* m, const float* X, const float* t, int64_t M, int epochs, int batch, float lr,
                             uint64_t seed, float* final_loss) {
    if (!m || !X || !t || M < batch || epochs < 1 || batch < GT || batch % GT || !(lr > 0.f)) return SISSO_ERR_ARG;
    sisso_status st = mlp_reserve(m, batch, true);
    if (st) return st;
    float *dX = nullptr, *dT = nullptr;
    int64_t* dI = nullptr;
    if (cudaMalloc((void**)&dX, sizeof(float) * M * kIn) != cudaSuccess ||
        cudaMalloc((void**)&dT, sizeof(float) * M) != cudaSuccess ||
        cudaMalloc((void**)&dI, sizeof(int64_t) * M) != cudaSuccess) {
        cudaFree(dX); cudaFree(dT); cudaFree(dI); cudaGetLastError();
        return SISSO_ERR_OOM;
    }
    cudaMemcpyAsync(dX, X, sizeof(float) * M * kIn, cudaMemcpyDefault, m->stream);
    cudaMemcpyAsync(dT, t, sizeof(float) * M, cudaMemcpyDefault, m->stream);
    std::vector<int64_t> order(M);
    for (int64_t i = 0; i < M; ++i) order[i] = i;
    std::mt19937_64 rng(seed);
    const int64_t steps = M / batch;
    float last = 0.f;
    cudaError_t e = cudaSuccess;
    for (int ep = 0; ep < epochs && !e; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        cudaMemcpyAsync(dI, order.data(), sizeof(int64_t) * M, cudaMemcpyHostToDevice, m->stream);
        cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
        for (int64_t s = 0; s < steps && !e; ++s) {
            k_gather<<<std::max(1, std::min(1024, (batch * kIn + 255) / 256)), 256, 0, m->stream>>>(
                dX, dT, dI + s * batch, batch, m->xin, m->tgt);
            k_pack_x<<<(unsigned)std::min<int64_t>(((int64_t)batch * GT + 255) / 256, 65535), 256, 0, m->stream>>>(
                m->xin, batch, batch, m->Xb, m->XT);
            e = mlp_forward_dev(m, batch, true);
            if (!e) e = mlp_backward_dev(m, batch);
            if (!e) {
                ++m->step;
                const float b1 = 0.9f, b2 = 0.999f;
                k_adam<<<256, 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, kParams, lr, b1, b2, 1e-8f,
                                                   1.f - std::pow(b1, (float)m->step), 1.f - std::pow(b2, (float)m->step));
                refresh_bf16(m);
                e = cudaGetLastError();
            }
        }
        if (!e) {
            cudaMemcpyAsync(&last, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
            e = cudaStreamSynchronize(m->stream);   // the order buffer is rewritten next epoch
            last /= (float)std::max<int64_t>(steps, 1);
        }
    }
    cudaFree(dX);
    cudaFree(dT);
    cudaFree(dI);
    if (final_loss) *final_loss = last;
    return mlp_status(m, e);
}

sisso_status sisso_prefix_features(const double* G, const double* b, double syy, int n, float* out, int* prefixes,
                                   float* base) {
    if (!G || !b || !out || n < 3 || n > 4095 || !(syy > 0.0)) return SISSO_ERR_ARG;
    const int64_t np = (int64_t)n * (n - 1) * (n - 2) / 6;
    double *dG = nullptr, *db = nullptr;
    float *dX = nullptr, *dB = nullptr;
    int* dP = nullptr;
    bool ok = cudaMalloc((void**)&dG, sizeof(double) * n * n) == cudaSuccess &&
              cudaMalloc((void**)&db, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc((void**)&dX, sizeof(float) * np * kIn) == cudaSuccess &&
              (!prefixes || cudaMalloc((void**)&dP, sizeof(int) * 3 * np) == cudaSuccess) &&
              (!base || cudaMalloc((void**)&dB, sizeof(float) * np) == cudaSuccess);
    sisso_status st = ok ? SISSO_OK : SISSO_ERR_OOM;
    if (ok) {
        cudaMemcpy(dG, G, sizeof(double) * n * n, cudaMemcpyDefault);
        cudaMemcpy(db, b, sizeof(double) * n, cudaMemcpyDefault);
        k_prefix_features<<<(unsigned)std::min<int64_t>((np + 255) / 256, 65535), 256>>>(dG, db, 1.0 / std::sqrt(syy), n,
                                                                                          np, dX, dP, dB);
        if (cudaMemcpy(out, dX, sizeof(float) * np * kIn, cudaMemcpyDefault) != cudaSuccess) st = SISSO_ERR_CUDA;
        if (!st && prefixes && cudaMemcpy(prefixes, dP, sizeof(int) * 3 * np, cudaMemcpyDefault) != cudaSuccess)
            st = SISSO_ERR_CUDA;
        if (!st && base && cudaMemcpy(base, dB, sizeof(float) * np, cudaMemcpyDefault) != cudaSuccess) st = SISSO_ERR_CUDA;
    }
    cudaGetLastError();
    cudaFree(dG); cudaFree(db); cudaFree(dX); cudaFree(dP); cudaFree(dB);
    return st;
}

}  // extern "C"

namespace sg {
namespace {
// labels of every 3-prefix from the enumeration's ordered keys: the lowest RSS / SST of its
// extensions (+inf: none); with base (the greedy completion's log10 RSS/SST) also the
// training target log10(max(label, 1e-12)) - base (NaN for a prefix without extensions)
__global__ void k_prefix_targets(const unsigned* __restrict__ keys, int64_t np, double sst,
                                 const float* __restrict__ base, float* __restrict__ label,
                                 float* __restrict__ target) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < np; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = keys[r];
        const unsigned u = (k >> 31) ? (k & 0x7FFFFFFFu) : ~k;
        const float lab = k == 0xFFFFFFFFu ? INFINITY : (float)((double)__uint_as_float(u) / sst);
        label[r] = lab;
        if (target) target[r] = isinf(lab) ? NAN : log10f(fmaxf(lab, 1e-12f)) - base[r];
    }
}
}  // namespace

// labels (and, with base_dev, training targets) of every 3-prefix on the current device;
// outputs HOST
static sisso_status prefix_labels_dev(const double* G, const double* b, double syy, int N, int n,
                                      const float* base_dev, float* labels, float* targets) {
    const int64_t np = (int64_t)n * (n - 1) * (n - 2) / 6;
    std::vector<float> G32((size_t)n * n), b32(n);
    std::vector<double> hG((size_t)n * n), hb(n);
    cudaMemcpy(hG.data(), G, sizeof(double) * n * n, cudaMemcpyDefault);
    cudaMemcpy(hb.data(), b, sizeof(double) * n, cudaMemcpyDefault);
    for (size_t i = 0; i < hG.size(); ++i) G32[i] = (float)hG[i];
    for (int i = 0; i < n; ++i) b32[i] = (float)hb[i];
    float *dG = nullptr, *db = nullptr, *dl = nullptr, *dt = nullptr;
    unsigned* lab = nullptr;
    int* ctr = nullptr;
    sisso_status st = SISSO_OK;
    if (cudaMalloc((void**)&dG, sizeof(float) * n * n) != cudaSuccess || cudaMalloc((void**)&db, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc((void**)&lab, sizeof(unsigned) * np) != cudaSuccess || cudaMalloc((void**)&ctr, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&dl, sizeof(float) * np) != cudaSuccess ||
        (targets && cudaMalloc((void**)&dt, sizeof(float) * np) != cudaSuccess))
        st = SISSO_ERR_OOM;
    if (!st) {
        cudaMemcpy(dG, G32.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice);
        cudaMemcpy(db, b32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        cudaMemset(lab, 0xFF, sizeof(unsigned) * np);
        cudaMemset(ctr, 0, sizeof(int));
        EnumArgs<float> A{};
        A.G = dG; A.b = db; A.ld = n; A.n = n; A.N = N; A.syy = (float)syy; A.sst = syy * N;
        A.cpp = std::max(1, (n - 1 - 3 + kRows - 1) / kRows);
        A.n_items = (int64_t)(n - 2) * (n - 3) * (n - 4) / 6 * A.cpp;
        A.counter = ctr; A.tau = kPivotMin32; A.fp32 = 1;
        const size_t smem = (size_t)kWarps * 5 * n * sizeof(float);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_prefix_labels<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_prefix_labels<0><<<sms * 2, kWarps * 32, smem>>>(A, lab);
        // prefixes of [0, n-2) only have extensions; the rest keep the +inf key
        k_prefix_targets<<<(unsigned)std::min<int64_t>((np + 255) / 256, 4096), 256>>>(lab, np, syy * N, base_dev, dl,
                                                                                       targets ? dt : nullptr);
        if (cudaMemcpy(labels, dl, sizeof(float) * np, cudaMemcpyDeviceToHost) != cudaSuccess) st = SISSO_ERR_CUDA;
        if (!st && targets && cudaMemcpy(targets, dt, sizeof(float) * np, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = SISSO_ERR_CUDA;
    }
    cudaGetLastError();
    cudaFree(dG); cudaFree(db); cudaFree(lab); cudaFree(ctr); cudaFree(dl); cudaFree(dt);
    return st;
}

}  // namespace sg

extern "C" {

sisso_status sisso_prefix_labels(const double* G, const double* b, double syy, int N, int n, float* out) {
    // the enumeration keeps 5 n FP32 values per warp in shared memory
    if (!G || !b || !out || n < 5 || n > 1400 || N < 1 || !(syy > 0.0)) return SISSO_ERR_ARG;
    return sg::prefix_labels_dev(G, b, syy, N, n, nullptr, out, nullptr);
}

sisso_status sisso_prefix_training(const double* G, const double* b, double syy, int N, int n, float* inputs,
                                   float* labels, float* targets) {
    if (!G || !b || !inputs || !labels || !targets || n < 5 || n > 1400 || N < 1 || !(syy > 0.0))
        return SISSO_ERR_ARG;
    const int64_t np = (int64_t)n * (n - 1) * (n - 2) / 6;
    double *dG = nullptr, *db = nullptr;
    float *dX = nullptr, *dB = nullptr;
    sisso_status st = SISSO_OK;
    if (cudaMalloc((void**)&dG, sizeof(double) * n * n) != cudaSuccess || cudaMalloc((void**)&db, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc((void**)&dX, sizeof(float) * np * kIn) != cudaSuccess || cudaMalloc((void**)&dB, sizeof(float) * np) != cudaSuccess)
        st = SISSO_ERR_OOM;
    if (!st) {
        cudaMemcpy(dG, G, sizeof(double) * n * n, cudaMemcpyDefault);
        cudaMemcpy(db, b, sizeof(double) * n, cudaMemcpyDefault);
        k_prefix_features<<<(unsigned)std::min<int64_t>((np + 255) / 256, 65535), 256>>>(dG, db, 1.0 / std::sqrt(syy), n,
                                                                                          np, dX, nullptr, dB);
        if (cudaMemcpy(inputs, dX, sizeof(float) * np * kIn, cudaMemcpyDeviceToHost) != cudaSuccess) st = SISSO_ERR_CUDA;
        if (!st) st = sg::prefix_labels_dev(G, b, syy, N, n, dB, labels, targets);
    }
    cudaGetLastError();
    cudaFree(dG); cudaFree(db); cudaFree(dX); cudaFree(dB);
    return st;
}


}  // extern "C"

// ===================================================================================
// the learned l0 search on a context
// ===================================================================================
namespace sg {

// D = 5 over n standardised features (G, b FP64 on the device, G32/b32 their FP32 copies):
// network scores of every 3-prefix, the best prefixes up to frac of C(n, 5) subsets, their
// extensions solved exactly.  On return *examined is the number of subsets enumerated.
sisso_status l0_learned(sisso_ctx* c, sisso_mlp* mlp, const double* G, const double* b, const float* G32,
                        const float* b32, int ld, double syy, int n, const int64_t* gid_dev, double frac, Winner& w,
                        int64_t* n_selected) {
    if (n < 5 || n > 1400) return fail(c, SISSO_ERR_ARG, "learned l0: n must be in 5..1400");
    const int64_t np = (int64_t)n * (n - 1) * (n - 2) / 6;
    // the network reads a dense n x n Gram
    double* Gd = nullptr;
    float* X = nullptr;
    int* plist = nullptr;
    int* sel = nullptr;
    float* score = nullptr;
    unsigned long long* hist = nullptr;
    unsigned* state = nullptr;
    unsigned* count = nullptr;
    sisso_status st = SISSO_OK;
    auto ck = [&](cudaError_t e, const char* what) { if (!st && e != cudaSuccess) st = check_cuda(c, e, what); };
    ck(cudaMallocAsync((void**)&Gd, sizeof(double) * n * n, c->stream), "learned: G");
    ck(cudaMallocAsync((void**)&X, sizeof(float) * np * kIn, c->stream), "learned: inputs");
    ck(cudaMallocAsync((void**)&plist, sizeof(int) * 3 * np, c->stream), "learned: prefixes");
    ck(cudaMallocAsync((void**)&sel, sizeof(int) * 3 * np, c->stream), "learned: selection");
    float* base = nullptr;
    ck(cudaMallocAsync((void**)&base, sizeof(float) * np, c->stream), "learned: base");
    ck(cudaMallocAsync((void**)&hist, sizeof(unsigned long long) * 3 * 2048, c->stream), "learned: histogram");
    ck(cudaMallocAsync((void**)&state, sizeof(unsigned) * 8, c->stream), "learned: state");
    if (st) return st;
    count = state + 4;
    ck(cudaMemcpy2DAsync(Gd, sizeof(double) * n, G, sizeof(double) * ld, sizeof(double) * n, n, cudaMemcpyDeviceToDevice,
                         c->stream), "learned: G copy");
    k_prefix_features<<<(unsigned)std::min<int64_t>((np + 255) / 256, 65535), 256, 0, c->stream>>>(
        Gd, b, 1.0 / std::sqrt(syy), n, np, X, plist, base);
    // network scores (on the network's stream, ordered after the features)
    sisso_status sm = mlp_reserve(mlp, np, false);
    if (sm) return fail(c, sm, "learned: network buffers");
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, c->stream);
    cudaStreamWaitEvent(mlp->stream, ev, 0);
    const int64_t Mpad = pad128(np);
    k_pack_x<<<(unsigned)std::min<int64_t>((Mpad * kInPad + 255) / 256, 65535), 256, 0, mlp->stream>>>(X, np, Mpad,
                                                                                                          mlp->Xb, nullptr);
    ck(mlp_forward_dev(mlp, np, false), "learned: network");
    score = mlp->out;
    cudaEventRecord(ev, mlp->stream);
    cudaStreamWaitEvent(c->stream, ev, 0);
    cudaEventDestroy(ev);
    // score = base (greedy completion) + the network's correction
    k_add<<<(unsigned)std::min<int64_t>((np + 255) / 256, 65535), 256, 0, c->stream>>>(score, base, np);
    // weighted selection of the lowest predicted RSS up to frac of the subsets
    const double total = (double)n * (n - 1) * (n - 2) * (n - 3) * (n - 4) / 120.0;
    const unsigned long long budget = (unsigned long long)std::max(1.0, std::ceil(frac * total));
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 3 * 2048, c->stream);
    cudaMemsetAsync(state, 0, sizeof(unsigned) * 8, c->stream);
    const int gs = std::max(1, std::min(c->sms * 4, (int)((np + 255) / 256)));
    for (int pass = 0; pass < 3; ++pass) {
        k_wsel_hist<<<gs, 256, 0, c->stream>>>(score, plist, n, np, pass, state, hist);
        k_wsel_find<<<1, 32, 0, c->stream>>>(hist, pass, state, budget);
    }
    k_wsel_compact<<<gs, 256, 0, c->stream>>>(score, plist, np, state, sel, count, np, nullptr);
    c->stats.launches += 13;   // features, pack, 2 layers + head, add, 3 x (histogram, find), compact
    unsigned h_count = 0;
    cudaMemcpyAsync(&h_count, count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    ck(cudaStreamSynchronize(c->stream), "learned: selection");
    if (!st) {
        int h_err = 0;
        cudaMemcpy(&h_err, mlp->err, sizeof(int), cudaMemcpyDeviceToHost);
        if (h_err) st = fail(c, SISSO_ERR_TIMEOUT, "learned: a bounded wait in the network ran out");
    }
    if (!st) {
        *n_selected = h_count;
        st = l0_solve(c, G, b, G32, b32, ld, syy, n, 5, gid_dev, SISSO_PREC_FP32, w, sel, (int64_t)h_count);
    }
    cudaFreeAsync(Gd, c->stream); cudaFreeAsync(X, c->stream); cudaFreeAsync(plist, c->stream);
    cudaFreeAsync(sel, c->stream); cudaFreeAsync(hist, c->stream); cudaFreeAsync(state, c->stream);
    cudaFreeAsync(base, c->stream);
    return st;
}

}  // namespace sg
