// whiten.cu — SISSO on whitened data (§2.4: W = Sigma^-1/2, y~ = W y, Phi~ = W Phi).
//
// Whitening maps every candidate column v (N samples) to W v, which mixes the samples: a
// whitened candidate is no longer a pointwise function of its operands, so the fused
// scoring kernels do not apply.  This path (FP64 precision) evaluates candidates in chunks
// of rows instead:
//   1. k_w_raw: one warp per id evaluates the candidate on the samples in FP64 with the
//      re-score's exact rules (finite, |v| <= 1e12, not cancelled, not near-constant, valid
//      operands) and keeps the raw row;
//   2. k_w_gemm: U = R W^T (row r of U is W applied to raw row r), FP64, 64 x 64 output
//      tiles staged through shared memory;
//   3. k_w_moments: one warp per row: the whitened column passes the same value rules, and
//      its Pearson score against the (whitened) target, its mean and std, its standardised
//      values and probes go wherever the caller asks (the score buffer, the selection
//      window, the subspace rows Z).
// The target is whitened once at context creation (y <- W y); the residuals of later
// steps are formed from the whitened rows, so they live in the whitened space too.
// Selection, duplicate checks, the Gram, l0 and the model then run unchanged on these
// values.
#include "sis_device.cuh"

#include <algorithm>

namespace sg {
namespace {

constexpr int kWB = 64, kWK = 16;       // GEMM output tile and K step

// U (n x N) = R (n x N) W^T, W N x N row-major: U[r][s] = sum_k R[r][k] W[s][k]
__global__ void __launch_bounds__(256) k_w_gemm(const double* __restrict__ R, int n, const double* __restrict__ W, int N,
                                                double* __restrict__ U) {
    __shared__ double Rs[kWK][kWB + 1], Ws[kWK][kWB + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * kWB, s0 = blockIdx.x * kWB;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < N; k0 += kWK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int m = e >> 4, kk = e & 15;
            const int k = k0 + kk;
            Rs[kk][m] = (r0 + m < n && k < N) ? R[(size_t)(r0 + m) * N + k] : 0.0;
            Ws[kk][m] = (s0 + m < N && k < N) ? W[(size_t)(s0 + m) * N + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kWK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = Rs[kk][ty + 16 * i]; b[i] = Ws[kk][tx + 16 * i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = s0 + tx + 16 * j;
            if (s < N) U[(size_t)r * N + s] = acc[i][j];
        }
    }
}

// raw values and raw validity of ids[w] (or lo + w): the FP64 re-score's evaluation and
// rules, its raw row kept in raw + w N; its score / mean / std / probes are scratch here
__global__ void k_w_raw(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, const double* __restrict__ tc,
                        const TargetStats* __restrict__ st, const int64_t* __restrict__ ids, int64_t lo, int n,
                        const unsigned char* __restrict__ subvalid, const double* __restrict__ V,
                        const double* __restrict__ Vinv, double* scr, int* ok, double* probe, double* raw) {
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= n) return;
    const int64_t id = ids ? ids[w] : lo + w;
    rescore_one(sp, Xc, N, N, tc, st, id, w, subvalid, V, scr, scr + n, scr + 2 * (size_t)n, ok, probe, raw, true, Vinv);
}

// whitened rows: the value rules (finite, |u| <= 1e12, std > 1e-6 max|u|), the Pearson score
// against the centred target tc (sums shifted by the sample-0 value, as the re-score), and
// the outputs the caller passes (any may be null)
__global__ void k_w_moments(const double* __restrict__ U, int n, int N, const int* __restrict__ ok_raw,
                            const double* __restrict__ tc, const TargetStats* __restrict__ st,
                            const int64_t* __restrict__ ids, int64_t lo, float* scores32, double* score,
                            double* mean_out, double* sd_out, int* valid_out, double* probe, double* z_out) {
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const double* u = U + (size_t)w * N;
    int bad = !ok_raw[w];
    double s1 = 0.0, s2 = 0.0, sc = 0.0, mx = 0.0;
    const double u0 = u[0];
    if (!bad)
        for (int i = lane; i < N; i += 32) {
            const double v = u[i];
            if (!isfinite(v) || fabs(v) > kValueCap) bad = 1;
            const double d = v - u0;
            s1 += d;
            s2 += d * d;
            sc += d * tc[i];
            mx = fmax(mx, fabs(v));
        }
    bad = warp_or(bad);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    sc = warp_sum(sc);
    mx = warp_max(mx);
    const double mean = u0 + s1 / N;
    const double var = s2 / N - (s1 / N) * (s1 / N);
    const double sd = bad || !(var > 0.0) ? 0.0 : sqrt(var);
    const int valid = !bad && sd > kConstRel * mx;
    const double inv = valid ? 1.0 / sd : 0.0;
    if (z_out)
        for (int i = lane; i < N; i += 32) z_out[(size_t)w * N + i] = valid ? (u[i] - mean) * inv : 0.0;
    if (probe && lane < kProbes) {
        const int i = (int)(((int64_t)lane * N) / kProbes);
        probe[(size_t)w * kProbes + lane] = valid ? (u[i] - mean) * inv : 0.0;
    }
    if (lane == 0) {
        const double r = valid ? fabs(sc - (s1 / N) * st->tsum) / ((double)N * sd * st->sd) : -1.0;
        if (scores32) scores32[ids ? ids[w] : lo + w] = valid ? (float)r : -1.f;
        if (score) score[w] = r;
        if (mean_out) mean_out[w] = valid ? mean : 0.0;
        if (sd_out) sd_out[w] = sd;
        if (valid_out) valid_out[w] = valid;
    }
}

void w_gemm(sisso_ctx* c, const double* R, int n) {
    dim3 grid((c->N + kWB - 1) / kWB, (n + kWB - 1) / kWB);
    k_w_gemm<<<grid, 256, 0, c->stream>>>(R, n, c->Wm, c->N, c->w_u);
    c->stats.launches++;
}

// raw rows, whitened rows and their moments for n ids (device list, or lo.. when null)
sisso_status w_rows(sisso_ctx* c, const int64_t* ids, int64_t lo, int n, float* scores32, double* score,
                    double* mean, double* sd, int* valid, double* probe, double* z) {
    const int N = c->N;
    for (int off = 0; off < n; off += c->w_chunk) {
        const int m = std::min(c->w_chunk, n - off);
        const int64_t* idc = ids ? ids + off : nullptr;
        const int g = (int)(((int64_t)m * 32 + 255) / 256);
        k_w_raw<<<g, 256, 0, c->stream>>>(c->space_dev, c->Xc64, N, c->tc64, c->tstats, idc, lo + off, m, c->subvalid,
                                          c->opval64, c->opinv64, c->w_scr, c->w_ok, c->w_probe, c->w_raw);
        w_gemm(c, c->w_raw, m);
        k_w_moments<<<g, 256, 0, c->stream>>>(c->w_u, m, N, c->w_ok, c->tc64, c->tstats, idc, lo + off, scores32,
                                              score ? score + off : nullptr, mean ? mean + off : nullptr,
                                              sd ? sd + off : nullptr, valid ? valid + off : nullptr,
                                              probe ? probe + (size_t)off * kProbes : nullptr,
                                              z ? z + (size_t)off * N : nullptr);
        c->stats.launches += 2;
    }
    return check_cuda(c, cudaGetLastError(), "whitened rows");
}

}  // namespace

// W to the device, the chunk buffers, and the target whitened in place (y <- W y)
sisso_status whiten_setup(sisso_ctx* c, const double* W) {
    const int N = c->N;
    const int64_t rows = std::max<int64_t>({c->n_feat, c->surv_cap, (int64_t)c->n_cap, 1});
    c->w_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(rows, ((int64_t)256 << 20) / ((int64_t)16 * N)));
    const size_t C = (size_t)c->w_chunk;
    sisso_status st;
    if ((st = check_cuda(c, cudaMalloc((void**)&c->Wm, sizeof(double) * (size_t)N * N), "whiten W")) ||
        (st = check_cuda(c, cudaMalloc((void**)&c->w_raw, sizeof(double) * C * N), "whiten raw")) ||
        (st = check_cuda(c, cudaMalloc((void**)&c->w_u, sizeof(double) * C * N), "whiten rows")) ||
        (st = check_cuda(c, cudaMalloc((void**)&c->w_scr, sizeof(double) * 3 * C), "whiten scratch")) ||
        (st = check_cuda(c, cudaMalloc((void**)&c->w_probe, sizeof(double) * kProbes * C), "whiten probes")) ||
        (st = check_cuda(c, cudaMalloc((void**)&c->w_ok, sizeof(int) * C), "whiten flags")))
        return st;
    cudaMemcpyAsync(c->Wm, W, sizeof(double) * (size_t)N * N, cudaMemcpyDefault, c->stream);
    w_gemm(c, c->y64, 1);
    cudaMemcpyAsync(c->y64, c->w_u, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, c->stream);
    return check_cuda(c, cudaGetLastError(), "whiten setup");
}

void whiten_free(sisso_ctx* c) {
    void* bufs[] = {c->Wm, c->w_raw, c->w_u, c->w_scr, c->w_probe, c->w_ok};
    for (void* p : bufs)
        if (p) cudaFree(p);
    c->Wm = c->w_raw = c->w_u = c->w_scr = c->w_probe = nullptr;
    c->w_ok = nullptr;
}

// scores of every id of phi_rung against the prepared (whitened) target
sisso_status whiten_score_all(sisso_ctx* c) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    sisso_status st = SISSO_OK;
    for (int64_t lo = 0; lo < c->n_feat && !st; lo += (int64_t)c->w_chunk) {
        const int n = (int)std::min<int64_t>(c->w_chunk, c->n_feat - lo);
        st = w_rows(c, nullptr, lo, n, c->scores, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    if (!st) apply_unit_mask(c);
    cudaEventRecord(e1, c->stream);
    if (!st) st = check_cuda(c, cudaEventSynchronize(e1), "whitened scores");
    if (!st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->stats.ms_screen += ms;
        c->stats.candidates_scored += c->n_feat;
    }
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    return st;
}

// the selection window's FP64 scores, means, stds, flags, probes and standardised vectors
sisso_status whiten_rescore(sisso_ctx* c, const int64_t* ids, int n, double* score, double* mean, double* sd,
                            int* valid, double* probe, double* zc) {
    return w_rows(c, ids, 0, n, nullptr, score, mean, sd, valid, probe, zc);
}

// standardised whitened rows of n subspace ids (Z rows, their means and stds)
sisso_status whiten_standardise(sisso_ctx* c, const int64_t* ids, int n, double* Z, double* Zmean, double* Zsd) {
    return w_rows(c, ids, 0, n, nullptr, nullptr, Zmean, Zsd, nullptr, nullptr, Z);
}

}  // namespace sg
