// gram_tc.cu — the subspace Gram G = Z Z^T / N on the tcgen05 tensor cores.
//
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

}  // namespace

// G32 (n x n, leading dimension ldg) and b32 (n) of the n standardised rows of Z and the
// centred target yc (population sd sdy) on the tensor cores; kind: SISSO_PREC_MIXED_BF16
// or SISSO_PREC_MIXED_FP16.  Scratch comes from the caller's stream-ordered allocator.
sisso_status gram_tc(sisso_ctx* c, const double* Z, const double* yc, double sdy, int n, int N, int kind,
                     float* G32, int ldg, float* b32) {
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
        (kind != SISSO_PREC_MIXED_BF16 && kind != SISSO_PREC_MIXED_FP16))
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
