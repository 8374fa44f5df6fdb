// gram_tc.cu — the subspace Gram G = Z Z^T / N on the tcgen05 tensor cores (§2.3 Eq. 7).
//
// 16-bit form (mixed precision; the 3xTF32 form of FP32 precision follows further down).
// Z (rows of standardised features, plus the centred target scaled to unit variance as the
// last row) is rounded to BF16 or FP16 and stored K-major (rows of samples), zero-padded to
// multiples of 128 rows and 64 samples.  A CTA computes one 128 x 128 output tile over a
// range of samples (split-K):
//   - one thread (warp 0) streams 128 x 64 tiles of both operands into a 4-stage
//     shared-memory ring with TMA (cp.async.bulk.tensor, 128-byte swizzle), completion
//     counted on an mbarrier per stage;
//   - one thread (warp 1) issues tcgen05.mma (M = 128, N = 128, K = 16, FP32 accumulate)
//     from shared-memory descriptors into a 128-column TMEM accumulator and releases each
//     stage with tcgen05.commit;
//   - all four warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes
//     32w..32w+31, i.e. output rows) and add it into the FP32 result.
// Every mbarrier wait is bounded; on timeout the kernel raises an error flag, waits
// (bounded) for its own copies, frees its TMEM and returns.
#include "tc_device.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace sg {
namespace {

constexpr int TMT = 128, TNT = 128, BK = 64;        // output tile; samples per stage (128 B of 16-bit)
constexpr int STAGES = 4;
constexpr int kTcThreads = 128;
constexpr uint32_t kTileBytes = TMT * BK * 2;        // 16 KB per operand tile
constexpr uint32_t kTmemCols = 128;                  // FP32 accumulator: 128 lanes x 128 columns

struct TcSmem {
    uint8_t a[STAGES][kTileBytes];
    uint8_t b[STAGES][kTileBytes];
    uint64_t full[STAGES], empty[STAGES], done;
    uint32_t tmem_base;
};

struct TcArgs {
    int rows;          // real rows (features + target row)
    int tiles;         // 128-row tiles per side
    int splits;        // K splits
    int nk;            // 64-sample stages in total
    float scale;       // 1 / N
    float* C;          // rows x ld FP32 result (accumulated with atomics; zeroed before)
    int ld;
    int* err;          // error flag (bounded waits)
    uint32_t idesc;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const __grid_constant__ CUtensorMap map, TcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_tile = A.splits;
    const int t = blockIdx.x / per_tile, split = blockIdx.x % per_tile;
    const int ti = t / A.tiles, tj = t % A.tiles;
    const int k_lo = (int)((int64_t)A.nk * split / A.splits), k_hi = (int)((int64_t)A.nk * (split + 1) / A.splits);
    const int nk = k_hi - k_lo;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 1); }
        mbar_init(&S.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {      // TMEM accumulator (whole warp)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
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

    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            // producer: TMA both operand tiles of every stage
            int issued = 0;
            for (int ks = 0; ks < nk; ++ks) {
                const int s = ks % STAGES;
                const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
                if (ks >= STAGES && !mbar_wait(&S.empty[s], ph ^ 1u)) { failed = 1; break; }
                mbar_expect_tx(&S.full[s], 2 * kTileBytes);
                const int x = (k_lo + ks) * BK;
                tma_load_2d(S.a[s], &map, x, ti * TMT, &S.full[s]);
                tma_load_2d(S.b[s], &map, x, tj * TNT, &S.full[s]);
                ++issued;
            }
            // on failure, wait (bounded) for the copies already in flight
            if (failed)
                for (int ks = (issued > STAGES ? issued - STAGES : 0); ks < issued; ++ks)
                    mbar_wait(&S.full[ks % STAGES], (uint32_t)(ks / STAGES) & 1u);
        } else if (warp == 1 && lane == 0) {
            // MMA issuer
            bool ok = true;
            for (int ks = 0; ks < nk; ++ks) {
                const int s = ks % STAGES;
                if (!mbar_wait(&S.full[s], (uint32_t)(ks / STAGES) & 1u)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t da = desc_sw128(smem_u32(S.a[s])), db = desc_sw128(smem_u32(S.b[s]));
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)   // 16 values = 32 B further along the swizzled row
                    mma_f16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), A.idesc, (ks > 0 || k > 0) ? 1u : 0u);
                mma_commit(&S.empty[s]);
            }
            if (!ok) failed = 1;
            mma_commit(&S.done);
        }
        __syncwarp();
        // epilogue: every warp reads its 32 TMEM lanes (output rows)
        const bool ready = mbar_wait(&S.done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (!ready || failed) {
            if (threadIdx.x == 0) atomicExch(A.err, 1);
        } else {
            const int row = ti * TMT + warp * 32 + lane;
#pragma unroll 1
            for (int cb = 0; cb < TNT / 32; ++cb) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), r);
                if (row < A.rows) {
                    float* dst = A.C + (size_t)row * A.ld + tj * TNT + cb * 32;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (tj * TNT + cb * 32 + q < A.rows) atomicAdd(dst + q, __uint_as_float(r[q]) * A.scale);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// rows of Z (FP64, n x N) and the centred target / sd (row n) -> 16-bit, zero-padded
template <typename H>
__global__ void k_to_half(const double* __restrict__ Z, const double* __restrict__ yc, double inv_sdy, int n, int N,
                          int Rpad, int Kpad, H* __restrict__ out) {
    const int64_t total = (int64_t)Rpad * Kpad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Kpad), s = (int)(e % Kpad);
        double v = 0.0;
        if (s < N) {
            if (r < n) v = Z[(size_t)r * N + s];
            else if (r == n) v = yc[s] * inv_sdy;
        }
        if constexpr (sizeof(H) == 2 && std::is_same<H, __nv_bfloat16>::value) out[e] = __double2bfloat16(v);
        else out[e] = __double2half(v);
    }
}

// C (rows x ld, rows = n + 1) -> G32 (n x n, leading dimension ldg), b32 (n, times sd_y)
__global__ void k_unpack_gram(const float* __restrict__ C, int ld, int n, float sdy, float* __restrict__ G32, int ldg,
                              float* __restrict__ b32) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * (n + 1); e += gridDim.x * blockDim.x) {
        const int i = e / (n + 1), j = e % (n + 1);
        if (j < n) G32[(size_t)i * ldg + j] = C[(size_t)i * ld + j];
        else b32[i] = C[(size_t)i * ld + n] * sdy;
    }
}

// ---------------------------------------------------------------------------------
// 3xTF32 form (FP32 precision).  Every value z of Z is split into two TF32 parts,
// h = tf32(z) and l = tf32(z - h) (10 explicit mantissa bits each, so h + l carries about
// 22 bits), and z_i z_j is taken as h_i h_j + h_i l_j + l_i h_j: the dropped l_i l_j and
// the rounding of l are below 2^-21 |z_i z_j|.  The parts are stored as FP32 words whose
// low 13 bits are zero, rows [0, Rpad) holding h and [Rpad, 2 Rpad) holding l.
// A CTA owns one 128 x 128 output tile (ti <= tj: the Gram is symmetric) and one run of
// at most kSplitSamples samples; its TMEM accumulator goes to a partial buffer of its own,
// and a second kernel adds the partials of every run in FP64 (no atomics, the same
// result on every run).  The tensor cores' FP32 accumulation drops up to about one unit
// in the last place per MMA (measured: with 2048-sample runs the entries came out 1.7e-5
// low), so the error of a run grows with its length: 512-sample runs (192 MMAs of
// K = 8) bound it by 192 x 2^-23 of the run's sum of |z_i z_j|, 2.3e-5 of G's scale.
// ---------------------------------------------------------------------------------
constexpr int BKT = 32;                              // samples per stage (128 B of FP32)
constexpr int STAGES_T = 3;
constexpr int kSplitSamples = 512;                   // samples per CTA: one accumulator run
constexpr uint32_t kTfTileBytes = TMT * BKT * 4;     // 16 KB per part tile

struct TfSmem {
    uint8_t t[STAGES_T][4][kTfTileBytes];            // h rows ti, l rows ti, h rows tj, l rows tj
    uint64_t full[STAGES_T], empty[STAGES_T], done;
    uint32_t tmem_base;
};

struct TfArgs {
    int tiles;         // 128-row tiles per side
    int rpad;          // tiles * 128: first row of the l parts
    int pairs;         // tile pairs ti <= tj
    int splits;        // sample runs
    int nk;            // BKT-sample stages in total
    float* P;          // partials: [split][pair][128][128]
    int* err;          // error flag (bounded waits)
    uint32_t idesc;
};

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// pair index p -> (ti, tj), pairs listed by ti, then tj >= ti
__device__ __forceinline__ void tile_pair(int p, int tiles, int& ti, int& tj) {
    ti = 0;
    while (p >= tiles - ti) { p -= tiles - ti; ++ti; }
    tj = ti + p;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tf32(const __grid_constant__ CUtensorMap map, TfArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TfSmem& S = *reinterpret_cast<TfSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = blockIdx.x % A.pairs, split = blockIdx.x / A.pairs;
    int ti, tj;
    tile_pair(pair, A.tiles, ti, tj);
    const int k_lo = (int)((int64_t)A.nk * split / A.splits), k_hi = (int)((int64_t)A.nk * (split + 1) / A.splits);
    const int nk = k_hi - k_lo;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES_T; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 1); }
        mbar_init(&S.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
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

    float* out = A.P + ((size_t)split * A.pairs + pair) * (TMT * TNT);
    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            int issued = 0;
            for (int ks = 0; ks < nk; ++ks) {
                const int s = ks % STAGES_T;
                if (ks >= STAGES_T && !mbar_wait(&S.empty[s], ((uint32_t)(ks / STAGES_T) & 1u) ^ 1u)) { failed = 1; break; }
                mbar_expect_tx(&S.full[s], 4 * kTfTileBytes);
                const int x = (k_lo + ks) * BKT;
                tma_load_2d(S.t[s][0], &map, x, ti * TMT, &S.full[s]);
                tma_load_2d(S.t[s][1], &map, x, A.rpad + ti * TMT, &S.full[s]);
                tma_load_2d(S.t[s][2], &map, x, tj * TNT, &S.full[s]);
                tma_load_2d(S.t[s][3], &map, x, A.rpad + tj * TNT, &S.full[s]);
                ++issued;
            }
            if (failed)
                for (int ks = (issued > STAGES_T ? issued - STAGES_T : 0); ks < issued; ++ks)
                    mbar_wait(&S.full[ks % STAGES_T], (uint32_t)(ks / STAGES_T) & 1u);
        } else if (warp == 1 && lane == 0) {
            bool ok = true;
            for (int ks = 0; ks < nk; ++ks) {
                const int s = ks % STAGES_T;
                if (!mbar_wait(&S.full[s], (uint32_t)(ks / STAGES_T) & 1u)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dh_i = desc_sw128(smem_u32(S.t[s][0])), dl_i = desc_sw128(smem_u32(S.t[s][1]));
                const uint64_t dh_j = desc_sw128(smem_u32(S.t[s][2])), dl_j = desc_sw128(smem_u32(S.t[s][3]));
#pragma unroll
                for (int k = 0; k < BKT / 8; ++k) {   // 8 TF32 values = 32 B further along the swizzled row
                    const uint64_t o = (uint64_t)(2 * k);
                    mma_tf32(tmem, dh_i + o, dh_j + o, A.idesc, (ks > 0 || k > 0) ? 1u : 0u);
                    mma_tf32(tmem, dh_i + o, dl_j + o, A.idesc, 1u);
                    mma_tf32(tmem, dl_i + o, dh_j + o, A.idesc, 1u);
                }
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
            const int r = warp * 32 + lane;
#pragma unroll 1
            for (int cb = 0; cb < TNT / 32; ++cb) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v);
                float4* dst = reinterpret_cast<float4*>(out + (size_t)r * TNT + cb * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                         __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            }
        }
    } else {
        // an empty run (more runs than stages never happens; kept for safety): zeros
        for (int e = threadIdx.x; e < TMT * TNT; e += blockDim.x) out[e] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// round to TF32 (10 explicit mantissa bits), nearest with ties to even, on the FP32 word
__device__ __forceinline__ float tf32_rne(float x) {
    uint32_t u = __float_as_uint(x);
    u += 0xFFFu + ((u >> 13) & 1u);
    return __uint_as_float(u & ~0x1FFFu);
}

// rows of Z and the scaled target (row n) -> TF32 parts h (rows [0, Rpad)) and l (rows
// [Rpad, 2 Rpad)), zero-padded
__global__ void k_to_tf32x2(const double* __restrict__ Z, const double* __restrict__ yc, double inv_sdy, int n, int N,
                            int Rpad, int Kpad, float* __restrict__ out) {
    const int64_t total = (int64_t)Rpad * Kpad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Kpad), s = (int)(e % Kpad);
        double v = 0.0;
        if (s < N) {
            if (r < n) v = Z[(size_t)r * N + s];
            else if (r == n) v = yc[s] * inv_sdy;
        }
        const float h = tf32_rne((float)v);
        out[e] = h;
        out[total + e] = tf32_rne((float)(v - (double)h));
    }
}

// sum of the runs' partials in FP64: G32 (n x n) and b32 (n, times sd_y) from the tiles
// ti <= tj (the lower triangle read from its mirror)
__global__ void k_reduce_tf32(const float* __restrict__ P, int tiles, int pairs, int splits, int n, double scale,
                              double sdy, float* __restrict__ G32, int ldg, float* __restrict__ b32) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * (n + 1); e += gridDim.x * blockDim.x) {
        const int i = e / (n + 1), j = e % (n + 1);
        const int r = min(i, j), q = max(i, j);
        const int tr = r / TMT, tq = q / TNT;
        const int p = tr * tiles - tr * (tr - 1) / 2 + (tq - tr);
        const size_t off = (size_t)p * (TMT * TNT) + (size_t)(r % TMT) * TNT + (q % TNT);
        double s = 0.0;
        for (int k = 0; k < splits; ++k) s += (double)P[(size_t)k * pairs * (TMT * TNT) + off];
        s *= scale;
        if (j < n) G32[(size_t)i * ldg + j] = (float)s;
        else b32[i] = (float)(s * sdy);
    }
}

// G32 / b32 in the 3xTF32 form
static sisso_status gram_tf32x3(sisso_ctx* c, const double* Z, const double* yc, double sdy, int n, int N, float* G32,
                                int ldg, float* b32) {
    const int rows = n + 1;
    const int tiles = (rows + TMT - 1) / TMT;
    const int Rpad = tiles * TMT;
    const int Kpad = ((N + BKT - 1) / BKT) * BKT;
    const int nk = Kpad / BKT;
    const int pairs = tiles * (tiles + 1) / 2;
    // runs of kSplitSamples; fewer, longer runs when the partials would pass 512 MB
    // (pairs x runs <= 8192 tiles of 64 KB: above about 1000 features at 65 536 samples)
    const int splits = std::max(1, std::min((Kpad + kSplitSamples - 1) / kSplitSamples, 8192 / pairs));
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(c, SISSO_ERR_CUDA, "gram_tc: cuTensorMapEncodeTiled unavailable");
    float* parts = nullptr;
    float* P = nullptr;
    int* err = nullptr;
    sisso_status st;
    if ((st = check_cuda(c, cudaMallocAsync((void**)&parts, (size_t)2 * Rpad * Kpad * sizeof(float), c->stream),
                         "gram_tc tf32 parts")) ||
        (st = check_cuda(c, cudaMallocAsync((void**)&P, (size_t)splits * pairs * TMT * TNT * sizeof(float), c->stream),
                         "gram_tc tf32 partials")) ||
        (st = check_cuda(c, cudaMallocAsync((void**)&err, sizeof(int), c->stream), "gram_tc err")))
        return st;
    const int g = std::max(1, std::min(c->sms * 8, (int)(((int64_t)Rpad * Kpad + 255) / 256)));
    k_to_tf32x2<<<g, 256, 0, c->stream>>>(Z, yc, 1.0 / sdy, n, N, Rpad, Kpad, parts);
    cudaMemsetAsync(err, 0, sizeof(int), c->stream);
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)Kpad, (cuuint64_t)(2 * Rpad)};
    const cuuint64_t gstride[1] = {(cuuint64_t)Kpad * 4};
    const cuuint32_t box[2] = {BKT, TMT};
    const cuuint32_t estride[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, parts, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        cudaFreeAsync(parts, c->stream); cudaFreeAsync(P, c->stream); cudaFreeAsync(err, c->stream);
        return fail(c, SISSO_ERR_CUDA, "gram_tc: tensor map encoding failed");
    }
    TfArgs A{};
    A.tiles = tiles; A.rpad = Rpad; A.pairs = pairs; A.splits = splits; A.nk = nk; A.P = P; A.err = err;
    A.idesc = idesc_f16(2u, TMT, TNT);     // A and B format 2: TF32 (kind::tf32)
    const size_t smem = sizeof(TfSmem) + 1024;
    cudaFuncSetAttribute(k_gram_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gram_tf32<<<pairs * splits, kTcThreads, smem, c->stream>>>(map, A);
    k_reduce_tf32<<<std::max(1, std::min(c->sms * 4, (rows * rows + 255) / 256)), 256, 0, c->stream>>>(
        P, tiles, pairs, splits, n, 1.0 / (double)N, sdy, G32, ldg, b32);
    c->stats.launches += 3;
    int h_err = 0;
    cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(parts, c->stream);
    cudaFreeAsync(P, c->stream);
    cudaFreeAsync(err, c->stream);
    if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "gram_tc tf32"))) return st;
    if (h_err) return fail(c, SISSO_ERR_TIMEOUT, "gram_tc: a bounded wait ran out");
    return SISSO_OK;
}

}  // namespace

// G32 (n x n, leading dimension ldg) and b32 (n) of the n standardised rows of Z and the
// centred target yc (population sd sdy) on the tensor cores; kind: SISSO_PREC_MIXED_BF16
// or SISSO_PREC_MIXED_FP16 (16-bit operands), or SISSO_PREC_FP32 (3xTF32 split).  Scratch
// comes from the caller's stream-ordered allocator.
sisso_status gram_tc(sisso_ctx* c, const double* Z, const double* yc, double sdy, int n, int N, int kind,
                     float* G32, int ldg, float* b32) {
    if (kind == SISSO_PREC_FP32) return gram_tf32x3(c, Z, yc, sdy, n, N, G32, ldg, b32);
    const int rows = n + 1;
    const int tiles = (rows + TMT - 1) / TMT;
    const int Rpad = tiles * TMT;
    const int Kpad = ((N + BK - 1) / BK) * BK;
    const int nk = Kpad / BK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(c, SISSO_ERR_CUDA, "gram_tc: cuTensorMapEncodeTiled unavailable");
    void* half = nullptr;
    float* C = nullptr;
    int* err = nullptr;
    sisso_status st;
    if ((st = check_cuda(c, cudaMallocAsync(&half, (size_t)Rpad * Kpad * 2, c->stream), "gram_tc half")) ||
        (st = check_cuda(c, cudaMallocAsync((void**)&C, (size_t)Rpad * Rpad * sizeof(float), c->stream), "gram_tc C")) ||
        (st = check_cuda(c, cudaMallocAsync((void**)&err, sizeof(int), c->stream), "gram_tc err")))
        return st;
    const bool bf16 = kind == SISSO_PREC_MIXED_BF16;
    const int g = std::max(1, std::min(c->sms * 8, (int)(((int64_t)Rpad * Kpad + 255) / 256)));
    if (bf16) k_to_half<__nv_bfloat16><<<g, 256, 0, c->stream>>>(Z, yc, 1.0 / sdy, n, N, Rpad, Kpad, (__nv_bfloat16*)half);
    else k_to_half<__half><<<g, 256, 0, c->stream>>>(Z, yc, 1.0 / sdy, n, N, Rpad, Kpad, (__half*)half);
    cudaMemsetAsync(C, 0, (size_t)Rpad * Rpad * sizeof(float), c->stream);
    cudaMemsetAsync(err, 0, sizeof(int), c->stream);
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)Kpad, (cuuint64_t)Rpad};
    const cuuint64_t gstride[1] = {(cuuint64_t)Kpad * 2};
    const cuuint32_t box[2] = {BK, TMT};
    const cuuint32_t estride[2] = {1, 1};
    if (enc(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, half, gdim, gstride, box,
            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        cudaFreeAsync(half, c->stream); cudaFreeAsync(C, c->stream); cudaFreeAsync(err, c->stream);
        return fail(c, SISSO_ERR_CUDA, "gram_tc: tensor map encoding failed");
    }
    TcArgs A{};
    A.rows = rows; A.tiles = tiles; A.nk = nk; A.scale = 1.0f / (float)N; A.C = C; A.ld = Rpad; A.err = err;
    A.idesc = idesc_f16(bf16 ? 1u : 0u, TMT, TNT);
    const int out_tiles = tiles * tiles;
    A.splits = std::max(1, std::min(nk, (c->sms + out_tiles - 1) / out_tiles));
    const size_t smem = sizeof(TcSmem) + 1024;
    cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gram_tc<<<out_tiles * A.splits, kTcThreads, smem, c->stream>>>(map, A);
    k_unpack_gram<<<std::max(1, std::min(c->sms * 4, (rows * rows + 255) / 256)), 256, 0, c->stream>>>(C, Rpad, n, (float)sdy,
                                                                                                       G32, ldg, b32);
    c->stats.launches += 3;
    int h_err = 0;
    cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(half, c->stream);
    cudaFreeAsync(C, c->stream);
    cudaFreeAsync(err, c->stream);
    if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "gram_tc"))) return st;
    if (h_err) return fail(c, SISSO_ERR_TIMEOUT, "gram_tc: a bounded wait ran out");
    return SISSO_OK;
}

}  // namespace sg

extern "C" sisso_status sisso_gram_tc(const double* Z, const double* yc, double sdy, int n, int N, int kind, float* G,
                                      float* b) {
    using namespace sg;
    if (!Z || !yc || !G || !b || n < 1 || N < 1 || !(sdy > 0.0) ||
        (kind != SISSO_PREC_MIXED_BF16 && kind != SISSO_PREC_MIXED_FP16 && kind != SISSO_PREC_FP32))
        return SISSO_ERR_ARG;
    sisso_ctx c;
    c.stream = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
    double *dZ = nullptr, *dy = nullptr;
    float *dG = nullptr, *db = nullptr;
    sisso_status st = SISSO_OK;
    auto ck = [&](cudaError_t e) { if (!st && e != cudaSuccess) st = SISSO_ERR_CUDA; };
    ck(cudaMalloc((void**)&dZ, sizeof(double) * (size_t)n * N));
    ck(cudaMalloc((void**)&dy, sizeof(double) * (size_t)N));
    ck(cudaMalloc((void**)&dG, sizeof(float) * (size_t)n * n));
    ck(cudaMalloc((void**)&db, sizeof(float) * (size_t)n));
    if (!st) {
        ck(cudaMemcpy(dZ, Z, sizeof(double) * (size_t)n * N, cudaMemcpyDefault));
        ck(cudaMemcpy(dy, yc, sizeof(double) * (size_t)N, cudaMemcpyDefault));
    }
    if (!st) st = gram_tc(&c, dZ, dy, sdy, n, N, kind, dG, n, db);
    if (!st) {
        ck(cudaMemcpy(G, dG, sizeof(float) * (size_t)n * n, cudaMemcpyDeviceToHost));
        ck(cudaMemcpy(b, db, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
    }
    cudaFree(dZ); cudaFree(dy); cudaFree(dG); cudaFree(db);
    return st;
}
