// screen_tc.cu — SIS scores of the top level's binary candidates from bilinear sums on the
// tcgen05 tensor cores (the mixed-precision forms; §2.2 Eq. 5 as a contraction).
//
// A candidate f = x (op) z over operands of phi_{L-1} scores |sum (f - fbar) r| /
// sqrt(sum (f - fbar)^2 * sum r^2) (r: the centred target).  With each operand centred in
// FP64 (x' = x - xbar) and g = z for *, g = 1/z for x/z, the candidate's two sums are
//   U = xbar sum g'r + gbar sum x'r + P5 - P1 sum(r) / N
//   V = xbar^2 sum g'^2 + gbar^2 sum x'^2 + P2 - P1^2 / N + 2 xbar gbar P1 + 2 xbar P3 + 2 gbar P4
// with P1 = sum x'g', P2 = sum x'^2 g'^2, P3 = sum x'g'^2, P4 = sum x'^2 g', P5 = sum (x'r) g',
// and for x +/- z: U = sum x'r +/- sum z'r, V = sum x'^2 + sum z'^2 +/- 2 P1.  The per-operand
// sums are FP64; P1..P4 do not depend on the target (one product per fit), P5 does (one
// product per SIS step).  The products run as C = L R^T over the samples:
//   L rows [x' | x'^2 | x'r],  R rows [z' | (1/z)' | z'^2 | ((1/z)')^2]   (blocks of Pp rows)
// each row scaled by a power of two and split into 16-bit parts (FP16: hi + lo, BF16:
// hi + mid + lo); the part products kept (FP16: hh, hl, lh; BF16: hh, hm, mh, hl, lh, mm)
// give every sum to about 2^-21 of its Cauchy-Schwarz scale.  A CTA computes one 128 x 128
// tile over a chunk of 1024 samples (FP32 accumulation in TMEM) and stores it; chunks are
// added in FP64.  Each candidate's score carries an error bound from eps_tc times the
// Cauchy-Schwarz scale of every product it uses; where the bound exceeds the FP32 screening
// margin the stored key is raised by the excess, so that key + margin bounds the exact
// score and the FP64 re-score of the selection window stays exact.
#include "tc_device.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace sg {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;            // output tile; samples per stage
constexpr int kThreads = 128;
constexpr uint32_t kTileBytes = BM * BK * 2;
constexpr int kAcc = 4;                                // TMEM accumulators per tile, 128 columns each
constexpr uint32_t kTmemCols = 128 * kAcc;
constexpr int kAccBlocks = 4;                          // 64-sample blocks summed in one accumulator
constexpr int kChunkBlocks = kAcc * kAccBlocks;        // 64-sample blocks per chunk (1024 samples)
constexpr double kTcEps = 1.0 / (1 << 17);            // bound on |error| / Cauchy-Schwarz scale
constexpr int kMaxParts = 6;

// one stage = one 64-sample block: every 16-bit part of the L tile and of the R tile
// (FP16: 2 + 2 tiles, 64 KB, three stages; BF16: 3 + 3 tiles, 96 KB, two stages), so each
// part is loaded once per block and the block's part products are issued back to back
template <int NP>
struct Smem {
    static constexpr int ST = NP == 2 ? 3 : 2;
    uint8_t a[ST][NP][kTileBytes];
    uint8_t b[ST][NP][kTileBytes];
    uint64_t full[ST], empty[ST], done;
    uint32_t tmem_base;
};

struct BilinArgs {
    int tiles_m, tiles_n;        // output tiles of this product
    int chunks, kb_per_chunk;    // sample chunks (in 64-sample blocks) and their length
    int nkb;                     // 64-sample blocks in all
    int l_row0, r_row0;          // first row of the product within a part block
    int l_part_rows, r_part_rows;// rows of one part block (the stride between parts)
    int npairs;                  // part products summed
    int lp[kMaxParts], rp[kMaxParts];
    float* C;                    // C[chunk * chunk_stride + row * ldc + col]
    int ldc;
    size_t chunk_stride;
    int* err;
    uint32_t idesc;
};

// One 128 x 128 tile of one sample chunk: TMA producer (warp 0), MMA issuer (warp 1), all
// four warps store the tile (warp w: rows 32w..32w+31).  The tensor cores' FP32 accumulation
// loses up to about one unit in the last place per MMA, so every run of kAccBlocks blocks
// goes to its own TMEM accumulator and the accumulators are added in FP64 before the store.
// Bounded waits; on timeout the error flag is raised and nothing is stored.
template <int NP>
__global__ void __launch_bounds__(kThreads, 1) k_bilin_tc(const __grid_constant__ CUtensorMap mapL,
                                                          const __grid_constant__ CUtensorMap mapR, BilinArgs A) {
    using SM = Smem<NP>;
    constexpr int ST = SM::ST;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SM& S = *reinterpret_cast<SM*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_chunk = A.tiles_m * A.tiles_n;
    const int chunk = blockIdx.x / per_chunk, t = blockIdx.x % per_chunk;
    const int tm = t / A.tiles_n, tn = t % A.tiles_n;
    const int kb_lo = chunk * A.kb_per_chunk, kb_hi = min(A.nkb, kb_lo + A.kb_per_chunk);
    const int nk = max(0, kb_hi - kb_lo);

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 1); }
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

    float* out = A.C + (size_t)chunk * A.chunk_stride + (size_t)(tm * BM + warp * 32 + lane) * A.ldc + tn * BN;
    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            int issued = 0;
            for (int ks = 0; ks < nk; ++ks) {
                const int s = ks % ST;
                const uint32_t ph = (uint32_t)(ks / ST) & 1u;
                if (ks >= ST && !mbar_wait(&S.empty[s], ph ^ 1u)) { failed = 1; break; }
                mbar_expect_tx(&S.full[s], 2 * NP * kTileBytes);
                const int x = (kb_lo + ks) * BK;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    tma_load_2d(S.a[s][q], &mapL, x, q * A.l_part_rows + A.l_row0 + tm * BM, &S.full[s]);
                    tma_load_2d(S.b[s][q], &mapR, x, q * A.r_part_rows + A.r_row0 + tn * BN, &S.full[s]);
                }
                ++issued;
            }
            if (failed)
                for (int ks = (issued > ST ? issued - ST : 0); ks < issued; ++ks)
                    mbar_wait(&S.full[ks % ST], (uint32_t)(ks / ST) & 1u);
        } else if (warp == 1 && lane == 0) {
            bool ok = true;
            for (int ks = 0; ks < nk; ++ks) {
                const int s = ks % ST;
                if (!mbar_wait(&S.full[s], (uint32_t)(ks / ST) & 1u)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)((ks / kAccBlocks) * 128);
                const bool first = ks % kAccBlocks == 0;
                for (int p = 0; p < A.npairs; ++p) {
                    const uint64_t da = desc_sw128(smem_u32(S.a[s][A.lp[p]])), db = desc_sw128(smem_u32(S.b[s][A.rp[p]]));
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        mma_f16(acc, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), A.idesc,
                                (!first || p > 0 || k > 0) ? 1u : 0u);
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
            const int used = (kb_hi - kb_lo + kAccBlocks - 1) / kAccBlocks;
#pragma unroll 1
            for (int cb = 0; cb < BN / 32; ++cb) {
                double v[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.0;
#pragma unroll 1
                for (int a = 0; a < used; ++a) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * 128 + cb * 32), r);
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] += (double)__uint_as_float(r[q]);
                }
                float4* dst = reinterpret_cast<float4*>(out + cb * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4((float)v[4 * q], (float)v[4 * q + 1], (float)v[4 * q + 2], (float)v[4 * q + 3]);
            }
        }
    } else {
        float4* dst = reinterpret_cast<float4*>(out);
        for (int q = 0; q < BN / 4; ++q) dst[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---- 16-bit parts --------------------------------------------------------------------
// x (already scaled, rounded once to FP32) as NP 16-bit parts whose sum is x to about 2^-22
// (FP16: two parts of 11 bits) or 2^-24 (BF16: three parts of 8 bits); the residuals are
// exact in FP32
template <typename H> __device__ __forceinline__ H to_h(float v);
template <> __device__ __forceinline__ __half to_h<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_h<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from_h(__half v) { return __half2float(v); }
__device__ __forceinline__ float from_h(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename H, int NP>
__device__ __forceinline__ void split_parts(double xd, H (&h)[NP]) {
    float x = (float)xd;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        h[p] = to_h<H>(x);
        x -= from_h(h[p]);
    }
}

template <typename H, int NP>
__device__ __forceinline__ void put_parts(const H (&h)[NP], H* dst, size_t part_stride) {
#pragma unroll
    for (int p = 0; p < NP; ++p) dst[(size_t)p * part_stride] = h[p];
}

template <typename H, int NP>
__device__ __forceinline__ void store_parts(double x, H* dst, size_t part_stride) {
    H h[NP];
    split_parts<H, NP>(x, h);
    put_parts<H, NP>(h, dst, part_stride);
}

// power-of-two exponent e with max * 2^e in [2^14, 2^15) (0 for max = 0)
__device__ __forceinline__ int scale_exp(double mx) {
    if (!(mx > 0.0) || !isfinite(mx)) return 0;
    int q;
    frexp(mx, &q);
    return 15 - q;
}

__device__ __forceinline__ double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double wmax(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kPrepThreads = 512;          // one CTA per operand or row, threads over samples
constexpr int kPrepWarps = kPrepThreads / 32;

// CTA-wide sums (op 0) or maxima (op 1) of K values, the same in every thread (warps
// combined in a fixed order, so results do not depend on timing)
template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], const int (&op)[K], double (*sh)[K]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = op[k] ? wmax(v[k]) : wsum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[w][k] = v[k];
    __syncthreads();
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double t = sh[0][k];
        for (int q = 1; q < nw; ++q) t = op[k] ? fmax(t, sh[q][k]) : t + sh[q][k];
        v[k] = t;
    }
}

// threads per CTA of the per-operand and per-row kernels: enough samples per thread to
// amortise the CTA-wide reductions
inline int prep_threads(int N) { return N >= 8192 ? kPrepThreads : N >= 2048 ? 256 : 128; }

// row kinds: x', x'^2, (1/x)', ((1/x)')^2, x' r, (1/x)' r
enum RowKind { RK_X = 0, RK_X2 = 1, RK_C = 2, RK_C2 = 3, RK_XR = 4, RK_CR = 5 };

struct MomArgs {
    const double* val;            // operand values, feature-major (P rows of N)
    const unsigned char* valid;   // operand validity (recursive rules)
    int P, N;
    double* mom;                  // per operand: xbar, sum x'^2, sum x'^4, gbar, sum g'^2, sum g'^4,
                                  // 1/x state (0 rows built, 1 x has a zero, 2 rows unusable), valid
    double* recip;                // 1/x of every operand value (P rows of N)
    int write_recip;              // 0: recip already holds 1/x
    int* mex;                     // per operand and row kind: power-of-two exponent of the row
};

// Target-independent moments of every operand (one CTA per operand), with g = 1/x.  An
// operand with a zero (or a 1/x that overflows) has no 1/x rows; 1/x rows whose fourth powers
// overflow (|x| below about 1e-77 somewhere) are not used either: the keys of candidates
// divided by it are then 1, left to the FP64 re-score.
__global__ void __launch_bounds__(kPrepThreads) k_tc_moments(MomArgs A) {
    __shared__ double sh[kPrepWarps][8];
    const int f = blockIdx.x, t = threadIdx.x;
    const bool ok = f < A.P && A.valid[f];
    const double* v = A.val + (size_t)(ok ? f : 0) * A.N;
    double* rc = A.recip + (size_t)(ok ? f : 0) * A.N;
    double m1[3] = {0.0, 0.0, 0.0};          // sum x, zero flag, sum 1/x
    if (ok)
        for (int i = t; i < A.N; i += blockDim.x) {
            const double x = v[i];
            m1[0] += x;
            const double c = A.write_recip ? 1.0 / x : rc[i];       // stored reciprocals when there are
            if (A.write_recip) rc[i] = c;
            if (!(x != 0.0) || !isfinite(c)) m1[1] = 1.0;
            else m1[2] += c;
        }
    block_reduce<3>(m1, {0, 1, 0}, reinterpret_cast<double (*)[3]>(&sh[0][0]));
    const bool zero = m1[1] != 0.0;
    const double mean = m1[0] / A.N, meanc = zero ? 0.0 : m1[2] / A.N;
    double m2[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // x'^2, x'^4, c'^2, c'^4, max |x'|, x'^2, |c'|, c'^2
    if (ok)
        for (int i = t; i < A.N; i += blockDim.x) {
            const double a = v[i] - mean, a2 = a * a;
            m2[0] += a2; m2[1] += a2 * a2;
            m2[4] = fmax(m2[4], fabs(a)); m2[5] = fmax(m2[5], a2);
            if (!zero) {
                const double c = (A.write_recip ? 1.0 / v[i] : rc[i]) - meanc, cc = c * c;
                m2[2] += cc; m2[3] += cc * cc;
                m2[6] = fmax(m2[6], fabs(c)); m2[7] = fmax(m2[7], cc);
            }
        }
    block_reduce<8>(m2, {0, 0, 0, 0, 1, 1, 1, 1}, sh);
    const bool unusable = !zero && !(isfinite(m2[2]) && isfinite(m2[3]));
    if (t == 0 && f < A.P) {
        int* ex = A.mex + (size_t)f * 6;
        ex[RK_X] = scale_exp(m2[4]); ex[RK_X2] = scale_exp(m2[5]);
        ex[RK_C] = zero || unusable ? 0 : scale_exp(m2[6]);
        ex[RK_C2] = zero || unusable ? 0 : scale_exp(m2[7]);
        double* m = A.mom + (size_t)f * 8;
        m[0] = mean; m[1] = m2[0]; m[2] = m2[1];
        m[3] = zero || unusable ? 0.0 : meanc;
        m[4] = zero || unusable ? 0.0 : m2[2];
        m[5] = zero || unusable ? 0.0 : m2[3];
        m[6] = zero ? 1.0 : unusable ? 2.0 : 0.0;
        m[7] = ok;
    }
}

// Target moments of every operand (one CTA per operand): sum x'r, sum (x'r)^2, sum g'r,
// sum (g'r)^2 with g = 1/x
__global__ void __launch_bounds__(kPrepThreads) k_tc_tmoments(const double* __restrict__ val,
                                                              const double* __restrict__ recip,
                                                              const double* __restrict__ mom, int P, int N,
                                                              const double* __restrict__ r, double* __restrict__ tgt,
                                                              int* __restrict__ mex) {
    __shared__ double sh[kPrepWarps][6];
    const int f = blockIdx.x, t = threadIdx.x;
    const double* m = mom + (size_t)f * 8;
    const bool ok = m[7] != 0.0, crow = m[6] == 0.0;
    const double* v = val + (size_t)(ok ? f : 0) * N;
    const double* rc = recip + (size_t)(ok ? f : 0) * N;
    double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};      // sums, then max |x'r|, max |c'r|
    if (ok)
        for (int i = t; i < N; i += blockDim.x) {
            const double a = (v[i] - m[0]) * r[i];
            q[0] += a; q[1] += a * a;
            q[4] = fmax(q[4], fabs(a));
            if (crow) {
                const double c = (rc[i] - m[3]) * r[i];
                q[2] += c; q[3] += c * c;
                q[5] = fmax(q[5], fabs(c));
            }
        }
    block_reduce<6>(q, {0, 0, 0, 0, 1, 1}, sh);
    if (t == 0) {
        for (int k = 0; k < 4; ++k) tgt[(size_t)f * 4 + k] = q[k];
        mex[(size_t)f * 6 + RK_XR] = scale_exp(q[4]);
        mex[(size_t)f * 6 + RK_CR] = scale_exp(q[5]);
    }
}

struct RowArgs {
    const double* val;
    const double* recip;
    const double* mom;
    const int* mex;               // per operand and kind: power-of-two exponent
    const double* r;              // centred target (row kinds 4, 5)
    int N, Kpad;
    int set0, nset, setp;         // the operands of this matrix side: set0 .. set0 + nset, padded to setp
    int nblk;                     // row blocks written by this launch
    int kind[8];                  // their kinds
    int row0;                     // matrix row of the first block's operand 0
    size_t part_stride;           // elements between part planes
    void* dst;                    // parts x rows x Kpad
    int* ex;                      // per matrix row: power-of-two exponent
};

// one CTA per operand of the set: its rows of every requested block in one pass over the
// samples (values scaled by the row's power of two, then split into 16-bit parts); rows of
// padding, of invalid operands and of unusable 1/x rows are zero
template <typename H, int NP>
__global__ void __launch_bounds__(kPrepThreads) k_tc_rows(RowArgs A) {
    const int fl = blockIdx.x, t = threadIdx.x;
    const int f = A.set0 + fl;
    const bool in = fl < A.nset;
    const double* m = A.mom + (size_t)(in ? f : 0) * 8;
    const bool okx = in && m[7] != 0.0, okc = okx && m[6] == 0.0;
    const double* v = A.val + (size_t)(okx ? f : 0) * A.N;
    const double* rc = A.recip + (size_t)(okx ? f : 0) * A.N;
    double sc[8];
    bool ok[8];
    H* dst[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b >= A.nblk) break;
        const int k = A.kind[b];
        ok[b] = (k == RK_C || k == RK_C2 || k == RK_CR) ? okc : okx;
        const int e = ok[b] ? A.mex[(size_t)f * 6 + k] : 0;
        sc[b] = ldexp(1.0, e);
        const int row = A.row0 + b * A.setp + fl;
        dst[b] = static_cast<H*>(A.dst) + (size_t)row * A.Kpad;
        if (t == 0) A.ex[row] = e;
    }
    for (int i = t; i < A.Kpad; i += blockDim.x) {
        const bool live = i < A.N;
        const double u = okx && live ? v[i] - m[0] : 0.0;
        const double c = okc && live ? rc[i] - m[3] : 0.0;
        const double r = live ? A.r[i] : 0.0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (b >= A.nblk) break;
            double x;
            switch (A.kind[b]) {
                case RK_X: x = u; break;
                case RK_X2: x = u * u; break;
                case RK_C: x = c; break;
                case RK_C2: x = c * c; break;
                case RK_XR: x = u * r; break;
                default: x = c * r; break;
            }
            store_parts<H, NP>(ok[b] ? x * sc[b] : 0.0, dst[b] + i, A.part_stride);
        }
    }
}

// out[r][c] = sum over chunks of C (FP64, in chunk order), unscaled by the rows' exponents
__global__ void k_bilin_reduce(const float* __restrict__ C, int chunks, size_t chunk_stride, int rows, int cols, int ldc,
                               const int* __restrict__ eL, const int* __restrict__ eR, double* __restrict__ out,
                               int ldo) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const float* p = C + (size_t)r * ldc + c;
        double s = 0.0;
        for (int q = 0; q < chunks; ++q) s += (double)p[(size_t)q * chunk_stride];
        out[(size_t)r * ldo + c] = ldexp(s, -(eL[r] + eR[c]));
    }
}

struct ScoreArgs {
    const Space* sp;
    int sec[4];
    int P, Q, N;
    int rect;               // 0: operand pairs i < j of one set (Pp = Ap = Bp); 1: i in [0, Q) x j in [Q, P)
    int Ap, Bp;             // padded operand counts of the L and R sides
    const double* mom;      // P x 8
    const double* tgt;      // P x 4
    const double* C1;       // target-independent products (ld1 columns)
    const double* C2;       // per-step products (ld2 columns)
    size_t ld1, ld2;
    const TargetStats* st;
    double eps_tc, eps_sel;
    float* scores;
    unsigned long long* raised;
};

// U, V and their error bounds for f = x g from the moments of x (mean, sum x'^2, sum x'^4,
// sum x'r) and of g (mean, sum g'^2, sum g'^4, sum g'r), the products P1..P5 and the
// Cauchy-Schwarz scale of the P5 product as computed; see the header comment for the formulas
struct UV { double U, V, dU, dV; };

__device__ __forceinline__ UV uv_product(double xb, double X2, double X4, double XR, double gb, double G2, double G4,
                                         double GR, double P1, double P2, double P3, double P4, double P5, double cs5,
                                         double N, double ts, double eps) {
    UV o;
    const double t1 = xb * xb * G2, t2 = gb * gb * X2, t3 = 2.0 * xb * gb * P1, t4 = 2.0 * xb * P3, t5 = 2.0 * gb * P4;
    o.V = t1 + t2 + P2 - P1 * P1 / N + t3 + t4 + t5;
    o.U = xb * GR + gb * XR + P5 - P1 * ts / N;
    const double cs11 = sqrt(X2 * G2);
    o.dV = eps * ((2.0 * fabs(P1) / N + 2.0 * fabs(xb * gb)) * cs11 + sqrt(X4 * G4) + 2.0 * fabs(xb) * sqrt(X2 * G4) +
                  2.0 * fabs(gb) * sqrt(X4 * G2)) +
           1e-15 * (t1 + t2 + fabs(P2) + P1 * P1 / N + fabs(t3) + fabs(t4) + fabs(t5));
    o.dU = eps * (cs5 + fabs(ts / N) * cs11) + 1e-15 * (fabs(xb * GR) + fabs(gb * XR) + fabs(P5));
    return o;
}

// one operand pair of one set: x = operand xi, g = operand zi (gs = 0) or its 1/x rows (gs = 1)
__device__ __forceinline__ UV prod_uv(const ScoreArgs& A, int xi, int zi, int gs) {
    const int Pp = A.Ap;
    const double* mx = A.mom + (size_t)xi * 8;
    const double* mz = A.mom + (size_t)zi * 8;
    const double* tx = A.tgt + (size_t)xi * 4;
    const double* tz = A.tgt + (size_t)zi * 4;
    const double P1 = A.C1[(size_t)xi * A.ld1 + gs * Pp + zi];
    const double P2 = A.C1[(size_t)(Pp + xi) * A.ld1 + (2 + gs) * Pp + zi];
    const double P3 = A.C1[(size_t)xi * A.ld1 + (2 + gs) * Pp + zi];
    const double P4 = A.C1[(size_t)(Pp + xi) * A.ld1 + gs * Pp + zi];
    const double P5 = A.C2[(size_t)xi * A.ld2 + gs * Pp + zi];
    const double G2 = gs ? mz[4] : mz[1];
    return uv_product(mx[0], mx[1], mx[2], tx[0], gs ? mz[3] : mz[0], G2, gs ? mz[5] : mz[2], gs ? tz[2] : tz[0],
                      P1, P2, P3, P4, P5, sqrt(tx[1] * G2), (double)A.N, A.st->tsum, A.eps_tc);
}

// stored key: the estimate, raised to (upper bound - margin) where the bound exceeds it by
// more than the margin; 1 (the largest |rho|) where V is not resolved
__device__ __forceinline__ float key_of(const UV& o, double srr, double eps_sel, unsigned long long* raised) {
    if (!(o.V - o.dV > 0.0)) {
        atomicAdd(raised, 1ull);
        return 1.0f;
    }
    const double est = fabs(o.U) / sqrt(o.V * srr);
    const double ub = (fabs(o.U) + o.dU) / sqrt((o.V - o.dV) * srr);
    double key = est;
    if (ub - eps_sel > est) {
        key = ub - eps_sel;
        atomicAdd(raised, 1ull);
    }
    return __double2float_ru(fmin(key, 1.0));
}

// key of x / z: -1 where z has a zero (division by zero), 1 where the 1/z rows are unusable
__device__ __forceinline__ bool div_state(const ScoreArgs& A, bool ok, int zi, float& key) {
    const double st = A.mom[(size_t)zi * 8 + 6];
    if (!ok || st == 1.0) { key = -1.f; return false; }
    if (st == 2.0) { atomicAdd(A.raised, 1ull); key = 1.f; return false; }
    return true;
}

__device__ __forceinline__ float key_sum(const ScoreArgs& A, double P1, int xi, int zi, double sg, double srr) {
    const double X2 = A.mom[(size_t)xi * 8 + 1], Z2 = A.mom[(size_t)zi * 8 + 1];
    const double XR = A.tgt[(size_t)xi * 4], ZR = A.tgt[(size_t)zi * 4];
    UV u;
    u.V = X2 + Z2 + 2.0 * sg * P1;
    u.U = XR + sg * ZR;
    u.dV = 2.0 * A.eps_tc * sqrt(X2 * Z2) + 1e-15 * (X2 + Z2 + 2.0 * fabs(P1));
    u.dU = 1e-15 * (fabs(XR) + fabs(ZR));
    return key_of(u, srr, A.eps_sel, A.raised);
}

// one thread per operand pair i < j (j >= Q) of one set: the keys of i+j, i-j, i*j, i/j, j/i
__global__ void k_score_bilin(ScoreArgs A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)A.P * A.P) return;
    const int i = (int)(e / A.P), j = (int)(e % A.P);
    if (!(i < j && j >= A.Q)) return;
    const bool ok = A.mom[(size_t)i * 8 + 7] != 0.0 && A.mom[(size_t)j * 8 + 7] != 0.0;
    const double srr = (double)A.N * A.st->sd * A.st->sd;
    const double P1 = A.C1[(size_t)i * A.ld1 + j];
    for (int o = 0; o < 2; ++o) {
        if (A.sec[o] < 0) continue;
        const Section& sc = A.sp->sec[A.sec[o]];
        A.scores[sc.base + rank_of(sc, i, j)] = ok ? key_sum(A, P1, i, j, o == 0 ? 1.0 : -1.0, srr) : -1.f;
    }
    if (A.sec[2] >= 0) {
        const Section& sc = A.sp->sec[A.sec[2]];
        A.scores[sc.base + rank_of(sc, i, j)] = ok ? key_of(prod_uv(A, i, j, 0), srr, A.eps_sel, A.raised) : -1.f;
    }
    if (A.sec[3] >= 0) {
        const Section& sc = A.sp->sec[A.sec[3]];
        float k1, k2;
        if (div_state(A, ok, j, k1)) k1 = key_of(prod_uv(A, i, j, 1), srr, A.eps_sel, A.raised);
        if (div_state(A, ok, i, k2)) k2 = key_of(prod_uv(A, j, i, 1), srr, A.eps_sel, A.raised);
        A.scores[sc.base + rank_of(sc, i, j)] = k1;
        A.scores[sc.base + rank_of(sc, j, i)] = k2;
    }
}

// One thread per pair i in [0, Q) x j in [Q, P) (the NEW_X_PREV top level): the keys of i+j,
// i-j, i*j, i/j, j/i.  L side: the operands [0, Q), row blocks x', x'^2, c', c'^2 (products
// C1, Ap rows each) and x'r, c'r (C2); R side: the operands [Q, P), row blocks z', c_z',
// z'^2, c_z'^2 (Bp columns each; C2 uses the first two).  j/i = z (1/x) is read as
// sum z' c_x' = C1[c'][z'], sum z'^2 c_x'^2 = C1[c'^2][z'^2], sum z' c_x'^2 = C1[c'^2][z'],
// sum z'^2 c_x' = C1[c'][z'^2] and sum (z'r) c_x' = C2[c'r][z'].
__global__ void k_score_bilin_rect(ScoreArgs A) {
    const int nB = A.P - A.Q;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)A.Q * nB) return;
    const int i = (int)(e / nB), jl = (int)(e % nB), j = A.Q + jl;
    const double* mi = A.mom + (size_t)i * 8;
    const double* mj = A.mom + (size_t)j * 8;
    const double* ti = A.tgt + (size_t)i * 4;
    const double* tj = A.tgt + (size_t)j * 4;
    const bool ok = mi[7] != 0.0 && mj[7] != 0.0;
    const double srr = (double)A.N * A.st->sd * A.st->sd;
    const double N = (double)A.N, ts = A.st->tsum;
    auto c1 = [&](int rb, int cb) { return A.C1[(size_t)(rb * A.Ap + i) * A.ld1 + (size_t)cb * A.Bp + jl]; };
    auto c2 = [&](int rb, int cb) { return A.C2[(size_t)(rb * A.Ap + i) * A.ld2 + (size_t)cb * A.Bp + jl]; };
    const double P1 = c1(0, 0);
    for (int o = 0; o < 2; ++o) {
        if (A.sec[o] < 0) continue;
        const Section& sc = A.sp->sec[A.sec[o]];
        A.scores[sc.base + rank_of(sc, i, j)] = ok ? key_sum(A, P1, i, j, o == 0 ? 1.0 : -1.0, srr) : -1.f;
    }
    // x = operand i, g = operand j (gs = 0) or 1/j (gs = 1)
    auto uv_ij = [&](int gs) {
        const double G2 = gs ? mj[4] : mj[1];
        return uv_product(mi[0], mi[1], mi[2], ti[0], gs ? mj[3] : mj[0], G2, gs ? mj[5] : mj[2], gs ? tj[2] : tj[0],
                          c1(0, gs), c1(1, 2 + gs), c1(0, 2 + gs), c1(1, gs), c2(0, gs), sqrt(ti[1] * G2), N, ts,
                          A.eps_tc);
    };
    if (A.sec[2] >= 0) {
        const Section& sc = A.sp->sec[A.sec[2]];
        A.scores[sc.base + rank_of(sc, i, j)] = ok ? key_of(uv_ij(0), srr, A.eps_sel, A.raised) : -1.f;
    }
    if (A.sec[3] >= 0) {
        const Section& sc = A.sp->sec[A.sec[3]];
        float k1, k2;
        if (div_state(A, ok, j, k1)) k1 = key_of(uv_ij(1), srr, A.eps_sel, A.raised);
        if (div_state(A, ok, i, k2)) {
            // x = operand j, g = 1/i; P5 computed as sum (c_i' r) z_j'
            const UV u = uv_product(mj[0], mj[1], mj[2], tj[0], mi[3], mi[4], mi[5], ti[2], c1(2, 0), c1(3, 2),
                                    c1(3, 0), c1(2, 2), c2(1, 0), sqrt(ti[3] * mj[1]), N, ts, A.eps_tc);
            k2 = key_of(u, srr, A.eps_sel, A.raised);
        }
        A.scores[sc.base + rank_of(sc, i, j)] = k1;
        A.scores[sc.base + rank_of(sc, j, i)] = k2;
    }
}

// rows (FP64, row stride N) -> NP parts of 16 bits, scaled per row (one warp per row)
template <typename H, int NP>
__global__ void k_rows_parts(const double* __restrict__ src, int rows, int N, int rows_pad, int Kpad, H* __restrict__ dst,
                             int* __restrict__ ex) {
    const int f = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (f >= rows_pad) return;
    const size_t K = (size_t)Kpad, ps = (size_t)rows_pad * K;
    double mx = 0.0;
    if (f < rows)
        for (int i = lane; i < N; i += 32) mx = fmax(mx, fabs(src[(size_t)f * N + i]));
    const int e = scale_exp(wmax(mx));
    const double s = ldexp(1.0, e);
    for (int i = lane; i < Kpad; i += 32)
        store_parts<H, NP>(f < rows && i < N ? src[(size_t)f * N + i] * s : 0.0, dst + (size_t)f * K + i, ps);
    if (lane == 0) ex[f] = e;
}

// ---- host -----------------------------------------------------------------------------
struct Parts {
    int n;
    int lp[kMaxParts], rp[kMaxParts];
};
Parts parts_of(bool bf16) {
    if (bf16) return Parts{6, {0, 0, 1, 0, 2, 1}, {0, 1, 0, 2, 0, 1}};
    return Parts{3, {0, 0, 1}, {0, 1, 0}};
}
int nparts(bool bf16) { return bf16 ? 3 : 2; }

bool encode_map(EncodeTiledFn enc, CUtensorMap* map, bool bf16, void* base, int rows, int Kpad) {
    const cuuint64_t gdim[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)Kpad * 2};
    const cuuint32_t box[2] = {BK, BM};
    const cuuint32_t estride[2] = {1, 1};
    return enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, gdim, gstride, box,
               estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int chunks_of(int nkb, int& per) {
    const int ch = std::max(1, (nkb + kChunkBlocks - 1) / kChunkBlocks);
    per = (nkb + ch - 1) / ch;
    return (nkb + per - 1) / per;
}

// C (m_rows x n_rows of the product, FP64 into out) = L[l_row0 ..] R[r_row0 ..]^T over the
// samples, both sides given as parts; out is unscaled by eL / eR (offset to the product's rows)
cudaError_t bilin(cudaStream_t s, int sms, bool bf16, void* L, int l_part_rows, int l_row0, int m_rows, void* R,
                  int r_part_rows, int r_row0, int n_rows, int Kpad, float* part, int* err, const int* eL,
                  const int* eR, double* out, int ldo, int& launches) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int np = nparts(bf16);
    CUtensorMap mL, mR;
    if (!encode_map(enc, &mL, bf16, L, np * l_part_rows, Kpad) || !encode_map(enc, &mR, bf16, R, np * r_part_rows, Kpad))
        return cudaErrorInvalidValue;
    const Parts pp = parts_of(bf16);
    BilinArgs A{};
    A.tiles_m = m_rows / BM;
    A.tiles_n = n_rows / BN;
    A.nkb = Kpad / BK;
    A.chunks = chunks_of(A.nkb, A.kb_per_chunk);
    A.l_row0 = l_row0; A.r_row0 = r_row0;
    A.l_part_rows = l_part_rows; A.r_part_rows = r_part_rows;
    A.npairs = pp.n;
    for (int q = 0; q < pp.n; ++q) { A.lp[q] = pp.lp[q]; A.rp[q] = pp.rp[q]; }
    A.C = part;
    A.ldc = n_rows;
    A.chunk_stride = (size_t)m_rows * n_rows;
    A.err = err;
    A.idesc = idesc_f16(bf16 ? 1u : 0u, BM, BN);
    const unsigned grid = (unsigned)A.tiles_m * A.tiles_n * A.chunks;
    if (bf16) {
        const size_t smem = sizeof(Smem<3>) + 1024;
        cudaFuncSetAttribute(k_bilin_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_bilin_tc<3><<<grid, kThreads, smem, s>>>(mL, mR, A);
    } else {
        const size_t smem = sizeof(Smem<2>) + 1024;
        cudaFuncSetAttribute(k_bilin_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_bilin_tc<2><<<grid, kThreads, smem, s>>>(mL, mR, A);
    }
    const int64_t total = (int64_t)m_rows * n_rows;
    k_bilin_reduce<<<(int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, (total + 255) / 256)), 256, 0, s>>>(
        part, A.chunks, A.chunk_stride, m_rows, n_rows, n_rows, eL + l_row0, eR + r_row0, out, ldo);
    launches += 2;
    return cudaGetLastError();
}

// layout of the tensor-core screening for a context: one operand set (pairs i < j) or two
// (NEW_X_PREV at rung >= 3: [0, Q) x [Q, P)); L and R row blocks, product sizes
struct TcLayout {
    bool rect;
    int P, Q, Ap, Bp, Kpad, chunks;
    int lblk, rblk;               // row blocks per part plane of L and R
    int m1, n1, m2, n2;           // the two products' rows and columns
};

TcLayout tc_layout(const sisso_ctx* c) {
    TcLayout t{};
    const int L = c->space.rung;
    t.P = (int)c->space.phi[L - 1];
    t.Q = L >= 2 ? (int)c->space.phi[L - 2] : 0;
    t.rect = c->space.grammar == SISSO_GRAMMAR_NEW_X_PREV && L >= 3;
    t.Kpad = ((c->N + BK - 1) / BK) * BK;
    int per;
    t.chunks = chunks_of(t.Kpad / BK, per);
    if (t.rect) {
        t.Ap = (t.Q + BM - 1) / BM * BM;
        t.Bp = (t.P - t.Q + BM - 1) / BM * BM;
        t.lblk = 6; t.rblk = 4;
        t.m1 = 4 * t.Ap; t.n1 = 4 * t.Bp; t.m2 = 2 * t.Ap; t.n2 = 2 * t.Bp;
    } else {
        t.Ap = t.Bp = (t.P + BM - 1) / BM * BM;
        t.lblk = 3; t.rblk = 4;
        t.m1 = 2 * t.Ap; t.n1 = 4 * t.Bp; t.m2 = t.Ap; t.n2 = 2 * t.Bp;
    }
    return t;
}

size_t tc_bytes(const sisso_ctx* c, const TcLayout& t, bool bf16) {
    const size_t np = nparts(bf16);
    const size_t part = (size_t)t.chunks * std::max((size_t)t.m1 * t.n1, (size_t)t.m2 * t.n2);
    return np * ((size_t)t.lblk * t.Ap + (size_t)t.rblk * t.Bp) * t.Kpad * 2 + part * 4 +
           ((size_t)t.m1 * t.n1 + (size_t)t.m2 * t.n2) * 8 + (c->opinv64 ? 0 : (size_t)t.P * c->N * 8) +
           (size_t)t.P * 12 * 8;
}

}  // namespace

// the rectangular (NEW_X_PREV) layout only on request: on lognormal rung-3 data about 5% of
// its keys carry bounds above the screening margin, and the windows they open cost more
// FP64 re-scoring than the products save
bool tc_screen_possible(const sisso_ctx* c, int screen) {
    const TcLayout t = tc_layout(c);
    if (t.rect && screen != SISSO_SCREEN_TENSOR) return false;
    if (t.rect ? t.Q > 4096 : t.P > 4096) return false;
    if ((int64_t)t.rblk * t.Bp * 3 > (int64_t)INT32_MAX / 2) return false;
    return tc_bytes(c, t, c->opts.precision == SISSO_PREC_MIXED_BF16) <= ((size_t)48 << 30);
}

sisso_status tc_screen_alloc(sisso_ctx* c) {
    const TcLayout t = tc_layout(c);
    const bool bf16 = c->opts.precision == SISSO_PREC_MIXED_BF16;
    const size_t np = nparts(bf16);
    c->tc_P = t.P; c->tc_Pp = t.Ap; c->tc_Kpad = t.Kpad;
    c->tc_part_cap = (size_t)t.chunks * std::max((size_t)t.m1 * t.n1, (size_t)t.m2 * t.n2);
    sisso_status st;
    auto al = [&](void** p, size_t bytes, const char* what) {
        return check_cuda(c, cudaMalloc(p, bytes), what);
    };
    if ((st = al(&c->tc_L, np * t.lblk * t.Ap * t.Kpad * 2, "tc L")) ||
        (st = al(&c->tc_R, np * t.rblk * t.Bp * t.Kpad * 2, "tc R")) ||
        (st = al((void**)&c->tc_eL, sizeof(int) * t.lblk * t.Ap, "tc eL")) ||
        (st = al((void**)&c->tc_eR, sizeof(int) * t.rblk * t.Bp, "tc eR")) ||
        (st = al((void**)&c->tc_mom, sizeof(double) * 8 * (size_t)t.P, "tc mom")) ||
        (st = al((void**)&c->tc_tgt, sizeof(double) * 4 * (size_t)t.P, "tc tgt")) ||
        (st = al((void**)&c->tc_mex, sizeof(int) * 6 * (size_t)t.P, "tc row exponents")) ||
        (st = al((void**)&c->tc_part, sizeof(float) * c->tc_part_cap, "tc partials")) ||
        (st = al((void**)&c->tc_C1, sizeof(double) * t.m1 * (size_t)t.n1, "tc C1")) ||
        (st = al((void**)&c->tc_C2, sizeof(double) * t.m2 * (size_t)t.n2, "tc C2")) ||
        (st = al((void**)&c->tc_err, 16, "tc err")))
        return st;
    if (!c->opinv64 && (st = al((void**)&c->tc_recip, sizeof(double) * (size_t)t.P * c->N, "tc reciprocals")))
        return st;
    c->tc_raised = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(c->tc_err) + 8);
    cudaMemsetAsync(c->tc_err, 0, 16, c->stream);
    c->tc_on = true;
    c->tc_ready = false;
    return SISSO_OK;
}

namespace {
// the rows of one side for the given blocks (one launch)
void tc_rows(sisso_ctx* c, bool bf16, void* dst, int* ex, int setp, int lblk_total, int set0, int nset, int blk0,
             std::initializer_list<int> kinds) {
    RowArgs R{};
    R.val = c->opval64;
    R.recip = c->opinv64 ? c->opinv64 : c->tc_recip;
    R.mom = c->tc_mom;
    R.r = c->tc64;
    R.N = c->N; R.Kpad = c->tc_Kpad;
    R.mex = c->tc_mex;
    R.set0 = set0; R.nset = nset; R.setp = setp;
    R.nblk = 0;
    for (int k : kinds) R.kind[R.nblk++] = k;
    R.row0 = blk0 * setp;
    R.part_stride = (size_t)lblk_total * setp * c->tc_Kpad;
    R.dst = dst;
    R.ex = ex;
    const int grid = setp;
    if (bf16) k_tc_rows<__nv_bfloat16, 3><<<grid, prep_threads(c->N), 0, c->stream>>>(R);
    else k_tc_rows<__half, 2><<<grid, prep_threads(c->N), 0, c->stream>>>(R);
    c->stats.launches++;
}
}  // namespace

// keys of the top level's binary sections for the current target (tc64 / tstats); the
// target-independent rows, moments and product run on the first call after tc_ready was
// cleared
sisso_status tc_screen_pairs(sisso_ctx* c, const int sec[4]) {
    const bool bf16 = c->opts.precision == SISSO_PREC_MIXED_BF16;
    const TcLayout t = tc_layout(c);
    const double* recip = c->opinv64 ? c->opinv64 : c->tc_recip;
    cudaError_t e = cudaSuccess;
    const int nA = t.rect ? t.Q : t.P, nB = t.rect ? t.P - t.Q : t.P, b0 = t.rect ? t.Q : 0;
    if (!c->tc_ready) {
        MomArgs M{};
        M.val = c->opval64; M.valid = c->subvalid; M.P = t.P; M.N = c->N; M.mom = c->tc_mom;
        M.recip = const_cast<double*>(recip); M.write_recip = c->opinv64 ? 0 : 1; M.mex = c->tc_mex;
        k_tc_moments<<<t.P, prep_threads(c->N), 0, c->stream>>>(M);
        c->stats.launches++;
        if (t.rect) tc_rows(c, bf16, c->tc_L, c->tc_eL, t.Ap, t.lblk, 0, nA, 0, {RK_X, RK_X2, RK_C, RK_C2});
        else tc_rows(c, bf16, c->tc_L, c->tc_eL, t.Ap, t.lblk, 0, nA, 0, {RK_X, RK_X2});
        tc_rows(c, bf16, c->tc_R, c->tc_eR, t.Bp, t.rblk, b0, nB, 0, {RK_X, RK_C, RK_X2, RK_C2});
        e = bilin(c->stream, c->sms, bf16, c->tc_L, t.lblk * t.Ap, 0, t.m1, c->tc_R, t.rblk * t.Bp, 0, t.n1, t.Kpad,
                  c->tc_part, c->tc_err, c->tc_eL, c->tc_eR, c->tc_C1, t.n1, c->stats.launches);
        if (e != cudaSuccess) return check_cuda(c, e, "tc product (target-independent)");
        c->tc_ready = true;
    }
    k_tc_tmoments<<<t.P, prep_threads(c->N), 0, c->stream>>>(c->opval64, recip, c->tc_mom, t.P, c->N, c->tc64, c->tc_tgt,
                                                                  c->tc_mex);
    c->stats.launches++;
    if (t.rect) tc_rows(c, bf16, c->tc_L, c->tc_eL, t.Ap, t.lblk, 0, nA, 4, {RK_XR, RK_CR});
    else tc_rows(c, bf16, c->tc_L, c->tc_eL, t.Ap, t.lblk, 0, nA, 2, {RK_XR});
    const int l2 = t.rect ? 4 * t.Ap : 2 * t.Ap;
    e = bilin(c->stream, c->sms, bf16, c->tc_L, t.lblk * t.Ap, l2, t.m2, c->tc_R, t.rblk * t.Bp, 0, t.n2, t.Kpad,
              c->tc_part, c->tc_err, c->tc_eL, c->tc_eR, c->tc_C2, t.n2, c->stats.launches);
    if (e != cudaSuccess) return check_cuda(c, e, "tc product (target)");
    ScoreArgs S{};
    S.sp = c->space_dev;
    for (int o = 0; o < 4; ++o) S.sec[o] = sec[o];
    S.P = t.P; S.Q = t.Q; S.N = c->N;
    S.rect = t.rect; S.Ap = t.Ap; S.Bp = t.Bp;
    S.mom = c->tc_mom; S.tgt = c->tc_tgt; S.C1 = c->tc_C1; S.C2 = c->tc_C2;
    S.ld1 = (size_t)t.n1; S.ld2 = (size_t)t.n2;
    S.st = c->tstats;
    S.eps_tc = kTcEps;
    S.eps_sel = kScoreErr32;
    S.scores = c->scores;
    S.raised = c->tc_raised;
    if (t.rect) {
        const int64_t n = (int64_t)nA * nB;
        k_score_bilin_rect<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(S);
    } else {
        const int64_t n = (int64_t)t.P * t.P;
        k_score_bilin<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(S);
    }
    c->stats.launches++;
    return check_cuda(c, cudaGetLastError(), "tc keys");
}

// the error flag and the raised-key count since the last call (both then cleared)
sisso_status tc_screen_status(sisso_ctx* c) {
    int h[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(h, c->tc_err, 16, cudaMemcpyDeviceToHost, c->stream);
    cudaMemsetAsync(c->tc_err, 0, 16, c->stream);
    sisso_status st = check_cuda(c, cudaStreamSynchronize(c->stream), "tc status");
    if (st) return st;
    unsigned long long raised;
    std::memcpy(&raised, &h[2], 8);
    c->stats.tc_keys_raised += (int64_t)raised;
    if (h[0]) return fail(c, SISSO_ERR_TIMEOUT, "tensor-core screening: a bounded wait ran out");
    return SISSO_OK;
}

void tc_screen_free(sisso_ctx* c) {
    void* bufs[] = {c->tc_L,  c->tc_R,  c->tc_eL,    c->tc_eR,  c->tc_mom, c->tc_tgt, c->tc_mex,
                    c->tc_part, c->tc_C1, c->tc_C2, c->tc_recip, c->tc_err};
    for (void* p : bufs)
        if (p) cudaFree(p);
}

}  // namespace sg

// sum_s L[i][s] R[j][s] (FP64 in and out, host memory) through the split 16-bit tensor-core
// product the mixed forms' screening uses
extern "C" sisso_status sisso_bilinear_tc(const double* Lrows, const double* Rrows, int m, int n, int N, int kind,
                                          double* out) {
    using namespace sg;
    if (!Lrows || !Rrows || !out || m < 1 || n < 1 || N < 1 ||
        (kind != SISSO_PREC_MIXED_BF16 && kind != SISSO_PREC_MIXED_FP16) || m > 65536 || n > 65536)
        return SISSO_ERR_ARG;
    const bool bf16 = kind == SISSO_PREC_MIXED_BF16;
    const int np = nparts(bf16);
    const int mp = (m + BM - 1) / BM * BM, npad = (n + BN - 1) / BN * BN, Kpad = (N + BK - 1) / BK * BK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per;
    const int ch = chunks_of(Kpad / BK, per);
    double *dL = nullptr, *dR = nullptr, *dout = nullptr;
    void *hL = nullptr, *hR = nullptr;
    int *eL = nullptr, *eR = nullptr, *err = nullptr;
    float* part = nullptr;
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t x) { if (e == cudaSuccess && x != cudaSuccess) e = x; };
    ck(cudaMalloc((void**)&dL, sizeof(double) * (size_t)m * N));
    ck(cudaMalloc((void**)&dR, sizeof(double) * (size_t)n * N));
    ck(cudaMalloc(&hL, (size_t)np * mp * Kpad * 2));
    ck(cudaMalloc(&hR, (size_t)np * npad * Kpad * 2));
    ck(cudaMalloc((void**)&eL, sizeof(int) * mp));
    ck(cudaMalloc((void**)&eR, sizeof(int) * npad));
    ck(cudaMalloc((void**)&err, sizeof(int)));
    ck(cudaMalloc((void**)&part, sizeof(float) * (size_t)ch * mp * npad));
    ck(cudaMalloc((void**)&dout, sizeof(double) * (size_t)mp * npad));
    int h_err = 0, launches = 0;
    if (e == cudaSuccess) {
        ck(cudaMemcpy(dL, Lrows, sizeof(double) * (size_t)m * N, cudaMemcpyHostToDevice));
        ck(cudaMemcpy(dR, Rrows, sizeof(double) * (size_t)n * N, cudaMemcpyHostToDevice));
        ck(cudaMemset(err, 0, sizeof(int)));
        if (bf16) {
            k_rows_parts<__nv_bfloat16, 3><<<(mp * 32 + 255) / 256, 256>>>(dL, m, N, mp, Kpad, (__nv_bfloat16*)hL, eL);
            k_rows_parts<__nv_bfloat16, 3><<<(npad * 32 + 255) / 256, 256>>>(dR, n, N, npad, Kpad, (__nv_bfloat16*)hR, eR);
        } else {
            k_rows_parts<__half, 2><<<(mp * 32 + 255) / 256, 256>>>(dL, m, N, mp, Kpad, (__half*)hL, eL);
            k_rows_parts<__half, 2><<<(npad * 32 + 255) / 256, 256>>>(dR, n, N, npad, Kpad, (__half*)hR, eR);
        }
        ck(cudaGetLastError());
        if (e == cudaSuccess)
            ck(bilin(0, sms, bf16, hL, mp, 0, mp, hR, npad, 0, npad, Kpad, part, err, eL, eR, dout, npad, launches));
        ck(cudaDeviceSynchronize());
        if (e == cudaSuccess) {
            ck(cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost));
            ck(cudaMemcpy2D(out, sizeof(double) * n, dout, sizeof(double) * npad, sizeof(double) * n, m,
                            cudaMemcpyDeviceToHost));
        }
    }
    cudaFree(dL); cudaFree(dR); cudaFree(hL); cudaFree(hR); cudaFree(eL); cudaFree(eR); cudaFree(err);
    cudaFree(part); cudaFree(dout);
    if (e != cudaSuccess) return SISSO_ERR_CUDA;
    return h_err ? SISSO_ERR_TIMEOUT : SISSO_OK;
}
