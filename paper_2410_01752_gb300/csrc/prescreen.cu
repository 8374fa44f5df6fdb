// prescreen.cu — pre-screening of the primary features for large d (§3.1; §3.3,
// initial_screening): every primary x_i is scored against the target y by mutual
// information MI(y; x_i) (Eq. MI, approximated with Gaussian kernel density estimates) or
// by the Spearman rank correlation, and only the primaries in the top quantile of the
// scores enter the expansion.
//
//  MI: p(y_s), p(x_s) and p(x_s, y_s) are kernel density estimates at the samples
//  themselves, with Scott's rule for the kernel covariance (N^(-2/(dim+4)) times the
//  sample covariance, the full 2 x 2 covariance for the joint density), and
//  MI = mean_s log(p(x_s, y_s) / (p(x_s) p(y_s))).  A CTA takes one primary and 256
//  samples s; the samples t stream through shared memory; kernel values are evaluated in
//  FP32 (exp of a non-positive argument) and summed in FP64.
//  Spearman: average ranks by counting (2 rank = 2 #less + #equal + 1, exact integers), then
//  the FP64 Pearson correlation of the ranks.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace sg {
namespace {

constexpr int kPsBlock = 256;

template <typename T> __device__ __forceinline__ T ps_warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// per primary (column i of X, row-major N x d) and for y (i = d): mean, unbiased variance,
// covariance with y
__global__ void k_ps_moments(const double* __restrict__ X, const double* __restrict__ y, int N, int d,
                             double* __restrict__ mom) {
    const int i = blockIdx.x;
    __shared__ double red[3][32];
    double s = 0.0, sy = 0.0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        s += i < d ? X[(size_t)t * d + i] : y[t];
        sy += y[t];
    }
    s = ps_warp_sum(s);
    sy = ps_warp_sum(sy);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][w] = s; red[1][w] = sy; }
    __syncthreads();
    s = sy = 0.0;
    for (int q = 0; q < nw; ++q) { s += red[0][q]; sy += red[1][q]; }
    const double m = s / N, my = sy / N;
    __syncthreads();
    double vv = 0.0, cv = 0.0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const double e = (i < d ? X[(size_t)t * d + i] : y[t]) - m;
        vv += e * e;
        cv += e * (y[t] - my);
    }
    vv = ps_warp_sum(vv);
    cv = ps_warp_sum(cv);
    if (lane == 0) { red[0][w] = vv; red[1][w] = cv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        vv = cv = 0.0;
        for (int q = 0; q < nw; ++q) { vv += red[0][q]; cv += red[1][q]; }
        mom[3 * i] = m;
        mom[3 * i + 1] = vv / (N - 1);
        mom[3 * i + 2] = cv / (N - 1);
    }
}

// p(y_s) for every sample
__global__ void k_ps_kde_y(const double* __restrict__ y, int N, const double* __restrict__ mom, int d,
                           double* __restrict__ py) {
    __shared__ float ys[kPsBlock];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const double hy2 = pow((double)N, -2.0 / 5.0) * mom[3 * d + 1];
    const float inv = (float)(-0.5 / hy2);
    const double my = mom[3 * d];
    const float yv = s < N ? (float)(y[s] - my) : 0.f;
    double acc = 0.0;
    for (int t0 = 0; t0 < N; t0 += kPsBlock) {
        __syncthreads();
        if (t0 + threadIdx.x < N) ys[threadIdx.x] = (float)(y[t0 + threadIdx.x] - my);
        __syncthreads();
        const int tn = min(kPsBlock, N - t0);
        float part = 0.f;
        for (int t = 0; t < tn; ++t) {
            const float u = yv - ys[t];
            part += expf(inv * u * u);
        }
        acc += part;
    }
    if (s < N) py[s] = acc / (N * sqrt(2.0 * M_PI * hy2));
}

// MI of primary blockIdx.y over the samples of this block: sum of log(pxy / (px py))
__global__ void k_ps_mi(const double* __restrict__ X, const double* __restrict__ y, int N, int d,
                        const double* __restrict__ mom, const double* __restrict__ py, double* __restrict__ mi_sum,
                        int* __restrict__ bad) {
    __shared__ float xs[kPsBlock], ys[kPsBlock];
    __shared__ double red[32];
    const int i = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const double vx = mom[3 * i + 1], cxy = mom[3 * i + 2], vy = mom[3 * d + 1];
    const double f1 = pow((double)N, -2.0 / 5.0), f2 = pow((double)N, -2.0 / 6.0);
    const double hx2 = f1 * vx;
    const double a = f2 * vx, b = f2 * cxy, c = f2 * vy, det = a * c - b * b;
    if (!(vx > 0.0) || !(det > 0.0)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(bad, 1);
        return;
    }
    const float ia = (float)(-0.5 * c / det), ib = (float)(b / det), ic = (float)(-0.5 * a / det);
    const float ix = (float)(-0.5 / hx2);
    // values centred in FP64 before the FP32 differences
    const double mx = mom[3 * i], my = mom[3 * d];
    const float xv = s < N ? (float)(X[(size_t)s * d + i] - mx) : 0.f, yv = s < N ? (float)(y[s] - my) : 0.f;
    double kx = 0.0, kxy = 0.0;
    for (int t0 = 0; t0 < N; t0 += kPsBlock) {
        __syncthreads();
        if (t0 + threadIdx.x < N) {
            xs[threadIdx.x] = (float)(X[(size_t)(t0 + threadIdx.x) * d + i] - mx);
            ys[threadIdx.x] = (float)(y[t0 + threadIdx.x] - my);
        }
        __syncthreads();
        const int tn = min(kPsBlock, N - t0);
        float px = 0.f, pxy = 0.f;
        for (int t = 0; t < tn; ++t) {
            const float u = xv - xs[t], v = yv - ys[t];
            px += expf(ix * u * u);
            // -0.5 (u, v) H^-1 (u, v)^T with H^-1 = [[c, -b], [-b, a]] / det
            pxy += expf(ia * u * u + ib * u * v + ic * v * v);
        }
        kx += px;
        kxy += pxy;
    }
    double term = 0.0;
    if (s < N) {
        const double px = kx / (N * sqrt(2.0 * M_PI * hx2));
        const double pxy = kxy / (N * 2.0 * M_PI * sqrt(det));
        term = log(pxy / (px * py[s]));
    }
    term = ps_warp_sum(term);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(&mi_sum[i], t);
    }
}

// twice the average rank of every sample of column i (i = d: y): 2 #less + #equal + 1
__global__ void k_ps_ranks(const double* __restrict__ X, const double* __restrict__ y, int N, int d,
                           int64_t* __restrict__ r2) {
    __shared__ double vs[kPsBlock];
    const int i = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const double v = s < N ? (i < d ? X[(size_t)s * d + i] : y[s]) : 0.0;
    int64_t less = 0, equal = 0;
    for (int t0 = 0; t0 < N; t0 += kPsBlock) {
        __syncthreads();
        if (t0 + threadIdx.x < N) vs[threadIdx.x] = i < d ? X[(size_t)(t0 + threadIdx.x) * d + i] : y[t0 + threadIdx.x];
        __syncthreads();
        const int tn = min(kPsBlock, N - t0);
        for (int t = 0; t < tn; ++t) {
            less += vs[t] < v;
            equal += vs[t] == v;
        }
    }
    if (s < N) r2[(size_t)i * N + s] = 2 * less + equal + 1;
}

// Pearson correlation of the ranks of column i with those of y (one block per column)
__global__ void k_ps_rank_corr(const int64_t* __restrict__ r2, int N, int d, double* __restrict__ rho) {
    const int i = blockIdx.x;
    __shared__ double red[3][32];
    const int64_t* rx = r2 + (size_t)i * N;
    const int64_t* ry = r2 + (size_t)d * N;
    // mean of 2 * rank is N + 1 for any column
    const double m = (double)(N + 1);
    double sxy = 0.0, sxx = 0.0, syy = 0.0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const double a = (double)rx[t] - m, b = (double)ry[t] - m;
        sxy += a * b; sxx += a * a; syy += b * b;
    }
    sxy = ps_warp_sum(sxy); sxx = ps_warp_sum(sxx); syy = ps_warp_sum(syy);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = sxy; red[1][w] = sxx; red[2][w] = syy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        sxy = sxx = syy = 0.0;
        for (int q = 0; q < nw; ++q) { sxy += red[0][q]; sxx += red[1][q]; syy += red[2][q]; }
        rho[i] = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
    }
}

}  // namespace

// The top-quantile rule of §3.3: keep the primaries scoring strictly above the
// (1 - q)-quantile of the scores (linear interpolation between order statistics at
// position (d - 1)(1 - q)); q = 1 keeps every primary.  Returns the number kept.
int prescreen_keep(const double* score, int d, double q, int* keep) {
    if (q >= 1.0) {
        std::fill(keep, keep + d, 1);
        return d;
    }
    std::vector<double> s(score, score + d);
    std::sort(s.begin(), s.end());
    const double pos = (double)(d - 1) * (1.0 - q);
    const int lo = (int)std::floor(pos);
    const double cut = lo + 1 < d ? s[lo] + (pos - lo) * (s[lo + 1] - s[lo]) : s[lo];
    int n = 0;
    for (int i = 0; i < d; ++i) {
        keep[i] = score[i] > cut ? 1 : 0;
        n += keep[i];
    }
    return n;
}

// scores (HOST, d) of the primaries by method (SISSO_PRESCREEN_MI or _SPEARMAN; Spearman
// as |rho|), on the current device
sisso_status prescreen_scores(const double* X, const double* y, int N, int d, int method, double* scores,
                              std::string& why) {
    double *dX = nullptr, *dy = nullptr, *mom = nullptr, *py = nullptr, *out = nullptr;
    int64_t* r2 = nullptr;
    int* bad = nullptr;
    auto fail_cuda = [&](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return false;
        why = std::string(what) + ": " + cudaGetErrorString(e);
        return true;
    };
    sisso_status st = SISSO_OK;
    cudaStream_t s0 = 0;
    if (fail_cuda(cudaMalloc(&dX, sizeof(double) * (size_t)N * d), "prescreen X") ||
        fail_cuda(cudaMalloc(&dy, sizeof(double) * (size_t)N), "prescreen y") ||
        fail_cuda(cudaMalloc(&mom, sizeof(double) * 3 * (size_t)(d + 1)), "prescreen moments") ||
        fail_cuda(cudaMalloc(&out, sizeof(double) * (size_t)d), "prescreen scores") ||
        fail_cuda(cudaMalloc(&bad, sizeof(int)), "prescreen flag")) {
        st = SISSO_ERR_OOM;
    } else {
        cudaMemcpyAsync(dX, X, sizeof(double) * (size_t)N * d, cudaMemcpyDefault, s0);
        cudaMemcpyAsync(dy, y, sizeof(double) * (size_t)N, cudaMemcpyDefault, s0);
        cudaMemsetAsync(bad, 0, sizeof(int), s0);
        const dim3 grid((N + kPsBlock - 1) / kPsBlock, d);
        if (method == SISSO_PRESCREEN_MI) {
            if (fail_cuda(cudaMalloc(&py, sizeof(double) * (size_t)N), "prescreen p(y)")) {
                st = SISSO_ERR_OOM;
            } else {
                k_ps_moments<<<d + 1, 256, 0, s0>>>(dX, dy, N, d, mom);
                k_ps_kde_y<<<(N + kPsBlock - 1) / kPsBlock, kPsBlock, 0, s0>>>(dy, N, mom, d, py);
                cudaMemsetAsync(out, 0, sizeof(double) * (size_t)d, s0);
                k_ps_mi<<<grid, kPsBlock, 0, s0>>>(dX, dy, N, d, mom, py, out, bad);
            }
        } else {
            if (fail_cuda(cudaMalloc(&r2, sizeof(int64_t) * (size_t)N * (d + 1)), "prescreen ranks")) {
                st = SISSO_ERR_OOM;
            } else {
                k_ps_ranks<<<dim3((N + kPsBlock - 1) / kPsBlock, d + 1), kPsBlock, 0, s0>>>(dX, dy, N, d, r2);
                k_ps_rank_corr<<<d, 256, 0, s0>>>(r2, N, d, out);
            }
        }
        int h_bad = 0;
        if (!st && (fail_cuda(cudaGetLastError(), "prescreen kernels") ||
                    fail_cuda(cudaMemcpy(scores, out, sizeof(double) * (size_t)d, cudaMemcpyDeviceToHost), "prescreen") ||
                    fail_cuda(cudaMemcpy(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost), "prescreen")))
            st = SISSO_ERR_CUDA;
        if (!st && h_bad) {
            why = "prescreen: a primary (or the target) has zero variance or a degenerate joint density";
            st = SISSO_ERR_ARG;
        }
        if (!st) {
            for (int i = 0; i < d; ++i) scores[i] = method == SISSO_PRESCREEN_MI ? scores[i] / N : std::fabs(scores[i]);
        }
    }
    cudaFree(dX); cudaFree(dy); cudaFree(mom); cudaFree(py); cudaFree(out); cudaFree(r2); cudaFree(bad);
    return st;
}

}  // namespace sg

extern "C" sisso_status sisso_prescreen(const double* X, const double* y, int N, int d, int method, double quantile,
                                        double* scores, int* keep, int* n_keep) {
    if (!X || !y || !scores || N < 3 || d < 1 || (method != SISSO_PRESCREEN_MI && method != SISSO_PRESCREEN_SPEARMAN) ||
        !(quantile > 0.0 && quantile <= 1.0))
        return SISSO_ERR_ARG;
    std::string why;
    const sisso_status st = sg::prescreen_scores(X, y, N, d, method, scores, why);
    if (st) return st;
    std::vector<int> k((size_t)d);
    const int n = sg::prescreen_keep(scores, d, quantile, k.data());
    if (keep) std::copy(k.begin(), k.end(), keep);
    if (n_keep) *n_keep = n;
    return SISSO_OK;
}
