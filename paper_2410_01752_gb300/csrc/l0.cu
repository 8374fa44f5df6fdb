// l0.cu — the sparsifying operator (§2.3, Eqs. 7-8) on the device.
//
//  Subspace: each new S member is evaluated in FP64 from the primaries and standardised
//  (rows of Z); the FP64 Gram G = Z Z^T / N and b = Z y~ / N grow by the new rows only.
//
//  Enumeration (k_l0_enum): every D-subset {p_0 < ... < p_{D-3} < i1 < i2} is one FP32
//  (or FP64) Cholesky solve.  A warp owns a prefix (p_0..p_{D-3}) and a run of i1 rows.
//  It first tabulates, for every x > i1_start, the prefix-reduced row of x:
//      R[m][x] = (G[x][p_m] - sum_{m'<m} R[m'][x] L[m][m']) / L[m][m],
//      dpart[x] = G[x][x] - sum_m R[m][x]^2,   npart[x] = b[x] - sum_m R[m][x] w[m],
//  so that for a pair (i1, i2) only
//      r = (G[i1][i2] - sum_m R[m][i1] R[m][i2]) / sqrt(dpart[i1]),
//      d = dpart[i2] - r^2,   num = npart[i2] - r * npart[i1] / sqrt(dpart[i1])
//  remain, and RSS = N (syy - |w_prefix|^2 - w_i1^2 - num^2 / d).  Lanes own i2 (row i1
//  of G is read coalesced), i1 is warp-uniform.
//
//  FP32 exactness: pass 1 finds UB = the FP64 RSS of the best FP32 subset (an upper bound
//  of the minimum); pass 2 takes every subset with RSS32_E - err_E <= UB + tie (err_E an a
//  posteriori bound from the subset's coefficients) and every subset with an FP32 pivot
//  <= 1e-5, solves each in FP64 and keeps it when its FP64 RSS is within UB + tie.  The
//  winner is the lowest FP64 RSS of the band, ties (1e-12 SST) to the smallest ascending
//  global-id tuple — the same rule as a full FP64 search.  In FP64 mode pass 1 gives the
//  minimum and pass 2 the tie window directly.
#include "l0_device.cuh"
#include "l0_tile.cuh"

#include <algorithm>
#include <cfloat>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace sg {
namespace {

template <typename T> __device__ __forceinline__ T warp_sum(T v) { return l0_warp_sum(v); }


// ---------------------------------------------------------------------------------
// subspace: standardised rows and Gram growth
// ---------------------------------------------------------------------------------
__global__ void k_standardise(const Space* __restrict__ sp, const double* __restrict__ Xc, int N, const int64_t* __restrict__ ids,
                              int row0, const double* __restrict__ V, double* __restrict__ Z,
                              double* __restrict__ mean_out, double* __restrict__ sd_out) {
    __shared__ double red[32];
    __shared__ double sh_mean, sh_sd;
    const int row = row0 + blockIdx.x;
    Prog p;
    OpRef ref{};
    const bool ok = V ? make_opref(*sp, ids[row], ref) : build_prog(*sp, ids[row], p);
    double* z = Z + (size_t)row * N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double mg;
        const double v = !ok ? 0.0 : V ? opref_val(ref, V, N, i, mg) : eval_prog<double>(p, [&](int c) { return Xc[(size_t)c * N + i]; });
        z[i] = v;
        s += v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        sh_mean = t / N;
    }
    __syncthreads();
    const double m = sh_mean;
    double ss = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) { const double v = z[i] - m; ss += v * v; }
    ss = warp_sum(ss);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        sh_sd = sqrt(t / N);
        mean_out[row] = m;
        sd_out[row] = sh_sd;
    }
    __syncthreads();
    const double inv = sh_sd > 0.0 ? 1.0 / sh_sd : 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) z[i] = (z[i] - m) * inv;
}

// G[i][j] = G[j][i] = Z_i . Z_j / N for i in [n_old, n), j in [0, n); b[i] = Z_i . y~ / N
__global__ void k_gram_rows(const double* __restrict__ Z, const double* __restrict__ yc, int N, int n_old,
                            int n, int ld, double* __restrict__ G, double* __restrict__ b,
                            float* __restrict__ G32, float* __restrict__ b32) {
    const int i = n_old + blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* zi = Z + (size_t)i * N;
    for (int j = blockIdx.y * kWarps + w; j <= n; j += gridDim.y * kWarps) {
        // column n is the moment vector b
        const double* zj = j < n ? Z + (size_t)j * N : yc;
        if (j < n && j > i && j >= n_old) continue;   // computed by row j
        double s = 0.0;
        for (int t = lane; t < N; t += 32) s += zi[t] * zj[t];
        s = warp_sum(s) / N;
        if (lane == 0) {
            if (j < n) {
                G[(size_t)i * ld + j] = s;
                G[(size_t)j * ld + i] = s;
                G32[(size_t)i * ld + j] = (float)s;
                G32[(size_t)j * ld + i] = (float)s;
            } else {
                b[i] = s;
                b32[i] = (float)s;
            }
        }
    }
}

template <typename T, int DP, int MODE>
__global__ void __launch_bounds__(kWarps * 32) k_l0_enum(EnumArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* tab = reinterpret_cast<T*>(smem_raw) + (size_t)w * (DP + 2) * A.n;
    T best = T(INFINITY);                 // pass 1: this lane's best subset
    unsigned long long best_key = 0;
    const double thr = MODE == 1 ? A.win->thr : 0.0;
    unsigned long long my_examined = 0;
    while (true) {
        int item;
        if (lane == 0) item = atomicAdd(A.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= A.n_items) break;
        enum_item<T, DP, MODE>(A, tab, item, best, best_key, thr, my_examined);
    }
    if (MODE == 0) enum_flush(A, DP + 2, best, best_key, my_examined);
}

// D = 1: RSS_i = N (syy - b_i^2 / G_ii)
template <typename T, int MODE>
__global__ void k_l0_single(EnumArgs<T> A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    single_subset<T, MODE>(A, i, MODE == 1 ? A.win->thr : 0.0);
}

// threshold of pass 2: the bound (+ the FP64 tie window)
__global__ void k_set_thr(Winner* w, const unsigned long long* ub_key, double add) {
    const double ub = okey_inv(*ub_key);
    w->thr = ub + add;
    w->min_key = *ub_key;
}

// ---------------------------------------------------------------------------------
// FP64 refit of the band and the tie-broken winner
// ---------------------------------------------------------------------------------
__global__ void k_refit(const double* __restrict__ G, const double* __restrict__ b, int ld, double syy, int N,
                        int D, const uint64_t* __restrict__ band, const unsigned* __restrict__ count, int64_t cap,
                        double* __restrict__ rss, unsigned long long* min_key) {
    const int64_t n = (int64_t)*count < cap ? (int64_t)*count : cap;
    double local = INFINITY;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int pos[kMaxDim];
        unpack(band[e], D, pos);
        const double r = rss64(G, b, ld, syy, N, D, pos, nullptr);
        rss[e] = r;
        local = fmin(local, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local = fmin(local, __shfl_xor_sync(0xffffffffu, local, o));
    if ((threadIdx.x & 31) == 0 && local < INFINITY) atomicMin(min_key, okey(local));
}

// one block: among refit entries within the tie window of the minimum, the smallest
// ascending global-id tuple (block-strided scan, then a shared-memory reduction)
__global__ void k_winner(const uint64_t* __restrict__ band, const double* __restrict__ rss,
                         const unsigned* __restrict__ count, int64_t cap, const unsigned long long* min_key,
                         double tie, const int64_t* __restrict__ gid, int D, Winner* W) {
    __shared__ int64_t best_e[1024];
    const int64_t n = (int64_t)*count < cap ? (int64_t)*count : cap;
    const double mn = okey_inv(*min_key);
    int64_t be = -1;
    int64_t bt[kMaxDim];
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        if (!(rss[e] <= mn + tie)) continue;
        int pos[kMaxDim];
        int64_t t[kMaxDim];
        unpack(band[e], D, pos);
        gid_tuple(gid, pos, D, t);
        if (be < 0 || tuple_less(t, bt, D)) { be = e; for (int j = 0; j < D; ++j) bt[j] = t[j]; }
    }
    best_e[threadIdx.x] = be;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t w = -1;
        int64_t wt[kMaxDim];
        for (int q = 0; q < (int)blockDim.x; ++q) {
            const int64_t e = best_e[q];
            if (e < 0) continue;
            int pos[kMaxDim];
            int64_t t[kMaxDim];
            unpack(band[e], D, pos);
            gid_tuple(gid, pos, D, t);
            if (w < 0 || tuple_less(t, wt, D)) { w = e; for (int j = 0; j < D; ++j) wt[j] = t[j]; }
        }
        W->found = w >= 0;
        if (w >= 0) {
            unpack(band[w], D, W->pos);
            W->rss_gram = rss[w];
        }
    }
}

// winner's coefficients (original units), residual r* = y~ - Z_E gamma, RMSE, R^2
__global__ void k_model(const double* __restrict__ G, const double* __restrict__ b, int ld, double syy, int N,
                        int D, const double* __restrict__ Z, const double* __restrict__ Zmean,
                        const double* __restrict__ Zsd, const double* __restrict__ yc, double ybar,
                        const int64_t* __restrict__ gid, Winner* W, double* __restrict__ resid) {
    __shared__ double gamma[kMaxDim];
    __shared__ double red[32];
    if (!W->found) return;
    if (threadIdx.x == 0) rss64(G, b, ld, syy, N, D, W->pos, gamma);
    __syncthreads();
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double f = yc[i];
        for (int j = 0; j < D; ++j) f -= gamma[j] * Z[(size_t)W->pos[j] * N + i];
        resid[i] = f;
        s += f * f;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double rss = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rss += red[w];
        // ids ascending with their coefficients
        int order[kMaxDim];
        for (int j = 0; j < D; ++j) order[j] = j;
        for (int a = 1; a < D; ++a)
            for (int c = a; c > 0 && gid[W->pos[order[c - 1]]] > gid[W->pos[order[c]]]; --c) {
                const int t = order[c]; order[c] = order[c - 1]; order[c - 1] = t;
            }
        double c0 = ybar;
        for (int j = 0; j < D; ++j) {
            const int q = order[j], p = W->pos[q];
            const double cj = gamma[q] / Zsd[p];
            W->ids[j] = gid[p];
            W->coef[j + 1] = cj;
            W->gamma[j] = gamma[q];
            c0 -= cj * Zmean[p];
        }
        W->coef[0] = c0;
        W->rss = rss;
        W->rmse = sqrt(rss / N);
        W->r2 = 1.0 - rss / (syy * N);
    }
}

// ---------------------------------------------------------------------------------
// mixed precision: the band's K best FP32 RSS (plus every entry flagged by a pivot) are
// re-solved in FP64 from the standardised FP64 rows, without an FP64 Gram
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned fkey(float v) {
    const unsigned u = __float_as_uint(v);
    return (u >> 31) ? ~u : (u | 0x80000000u);
}

// one block: the K-th smallest key among finite band RSS32 (binary search on the key), then
// the selection flags (key <= threshold, or flagged)
__global__ void k_select_top(const float* __restrict__ r32, const unsigned* __restrict__ count, int64_t cap, int K,
                             unsigned char* __restrict__ sel) {
    __shared__ unsigned red[32];
    __shared__ unsigned thr_s;
    const int64_t n = (int64_t)*count < cap ? (int64_t)*count : cap;
    auto count_le = [&](unsigned t) -> unsigned {
        unsigned c = 0;
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
            const float v = r32[e];
            if (v == v && fkey(v) <= t) ++c;
        }
        c = warp_sum(c);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        unsigned tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        __syncthreads();
        return tot;
    };
    // smallest threshold t with count(key <= t) >= K (all finite entries if fewer than K)
    unsigned lo = 0, hi = 0xFFFFFFFFu;
    if (count_le(hi) < (unsigned)K) lo = hi;
    while (lo < hi) {
        const unsigned mid = lo + ((hi - lo) >> 1);
        if (count_le(mid) >= (unsigned)K) hi = mid; else lo = mid + 1;
    }
    if (threadIdx.x == 0) thr_s = lo;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const float v = r32[e];
        sel[e] = (v != v) || fkey(v) <= thr_s;
    }
}

// one warp per band entry: FP64 sub-Gram and moments from Z rows, Cholesky, RSS
__global__ void k_refit_z(const double* __restrict__ Z, const double* __restrict__ yc, int N, double syy, int D,
                          const uint64_t* __restrict__ band, const unsigned* __restrict__ count, int64_t cap,
                          const unsigned char* __restrict__ sel, double* __restrict__ rss_out,
                          unsigned long long* min_key) {
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)*count < cap ? (int64_t)*count : cap;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n;
         e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        if (!sel[e]) { if (lane == 0) rss_out[e] = INFINITY; continue; }
        int pos[kMaxDim];
        unpack(band[e], D, pos);
        double g[kMaxDim][kMaxDim], bv[kMaxDim];
        for (int i = 0; i < D; ++i) {
            const double* zi = Z + (size_t)pos[i] * N;
            for (int j = 0; j <= i; ++j) {
                const double* zj = Z + (size_t)pos[j] * N;
                double acc = 0.0;
                for (int t = lane; t < N; t += 32) acc += zi[t] * zj[t];
                g[i][j] = g[j][i] = warp_sum(acc) / N;
            }
            double acc = 0.0;
            for (int t = lane; t < N; t += 32) acc += zi[t] * yc[t];
            bv[i] = warp_sum(acc) / N;
        }
        if (lane == 0) {
            double L[kMaxDim][kMaxDim], w[kMaxDim], q = 0.0;
            bool ok = true;
            for (int j = 0; j < D && ok; ++j) {
                double dj = g[j][j];
                for (int m = 0; m < j; ++m) dj -= L[j][m] * L[j][m];
                if (!(dj > kPivotMin)) { ok = false; break; }
                L[j][j] = sqrt(dj);
                for (int i = j + 1; i < D; ++i) {
                    double v = g[i][j];
                    for (int m = 0; m < j; ++m) v -= L[i][m] * L[j][m];
                    L[i][j] = v / L[j][j];
                }
                double v = bv[j];
                for (int m = 0; m < j; ++m) v -= L[j][m] * w[m];
                w[j] = v / L[j][j];
                q += w[j] * w[j];
            }
            const double r = ok ? (double)N * (syy - q) : INFINITY;
            rss_out[e] = r;
            if (r < INFINITY) atomicMin(min_key, okey(r));
        }
    }
}

// the winner's model from Z rows (one block): coefficients in original units, residual
__global__ void k_model_z(const double* __restrict__ Z, const double* __restrict__ Zmean,
                          const double* __restrict__ Zsd, const double* __restrict__ yc, double ybar, int N, double syy,
                          int D, const int64_t* __restrict__ gid, Winner* W, double* __restrict__ resid) {
    __shared__ double g[kMaxDim][kMaxDim], bv[kMaxDim], gamma[kMaxDim];
    __shared__ double red[32];
    if (!W->found) return;
    // lower triangle of the sub-Gram, then the moments with the target (column D)
    for (int i = 0; i < D; ++i) {
        const double* zi = Z + (size_t)W->pos[i] * N;
        for (int j = 0; j <= D; ++j) {
            if (j < D && j > i) continue;
            const double* zj = j < D ? Z + (size_t)W->pos[j] * N : yc;
            double acc = 0.0;
            for (int t = threadIdx.x; t < N; t += blockDim.x) acc += zi[t] * zj[t];
            acc = warp_sum(acc);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
                if (j < D) g[i][j] = g[j][i] = tot / N;
                else bv[i] = tot / N;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {   // Cholesky solve G gamma = b
        double L[kMaxDim][kMaxDim], w[kMaxDim];
        for (int j = 0; j < D; ++j) {
            double dj = g[j][j];
            for (int m = 0; m < j; ++m) dj -= L[j][m] * L[j][m];
            L[j][j] = sqrt(dj > 0 ? dj : 1e-300);
            for (int i = j + 1; i < D; ++i) {
                double v = g[i][j];
                for (int m = 0; m < j; ++m) v -= L[i][m] * L[j][m];
                L[i][j] = v / L[j][j];
            }
            double v = bv[j];
            for (int m = 0; m < j; ++m) v -= L[j][m] * w[m];
            w[j] = v / L[j][j];
        }
        for (int j = D - 1; j >= 0; --j) {
            double v = w[j];
            for (int m = j + 1; m < D; ++m) v -= L[m][j] * gamma[m];
            gamma[j] = v / L[j][j];
        }
    }
    __syncthreads();
    double ssr = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double f = yc[i];
        for (int j = 0; j < D; ++j) f -= gamma[j] * Z[(size_t)W->pos[j] * N + i];
        resid[i] = f;
        ssr += f * f;
    }
    ssr = warp_sum(ssr);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ssr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double rss = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rss += red[w];
        int order[kMaxDim];
        for (int j = 0; j < D; ++j) order[j] = j;
        for (int a = 1; a < D; ++a)
            for (int c = a; c > 0 && gid[W->pos[order[c - 1]]] > gid[W->pos[order[c]]]; --c) {
                const int t = order[c]; order[c] = order[c - 1]; order[c - 1] = t;
            }
        double c0 = ybar;
        for (int j = 0; j < D; ++j) {
            const int q = order[j], p = W->pos[q];
            const double cj = gamma[q] / Zsd[p];
            W->ids[j] = gid[p];
            W->coef[j + 1] = cj;
            W->gamma[j] = gamma[q];
            c0 -= cj * Zmean[p];
        }
        W->coef[0] = c0;
        W->rss = rss;
        W->rmse = sqrt(rss / N);
        W->r2 = 1.0 - rss / (syy * N);
    }
}

}  // namespace

// ===================================================================================
// host side
// ===================================================================================

sisso_status append_subspace(sisso_ctx* c, int n_old, int n_new, bool gram64) {
    if (n_new <= 0) return SISSO_OK;
    const int n = n_old + n_new;
    if (c->Wm) {       // whitened data (§2.4): the standardised rows of W v
        sisso_status st = whiten_standardise(c, c->S_dev + n_old, n_new, c->Z + (size_t)n_old * c->N,
                                             c->Zmean + n_old, c->Zsd + n_old);
        if (st) return st;
    } else {
        k_standardise<<<n_new, 256, 0, c->stream>>>(c->space_dev, c->Xc64, c->N, c->S_dev, n_old, c->opval64, c->Z,
                                                     c->Zmean, c->Zsd);
        c->stats.launches++;
    }
    if (gram64) {
        dim3 grid(n_new, std::max(1, std::min(64, (n + 1 + kWarps - 1) / kWarps)));
        k_gram_rows<<<grid, kWarps * 32, 0, c->stream>>>(c->Z, c->yc64, c->N, n_old, n, c->n_cap, c->G64, c->b64,
                                                          c->G32, c->b32);
        c->stats.launches++;
    }
    return check_cuda(c, cudaGetLastError(), "append_subspace");
}


static int64_t binom_host(int64_t n, int k) {
    if (k < 0 || n < k) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

template <typename T>
static sisso_status run_enum(sisso_ctx* c, EnumArgs<T> A, int D, int mode) {
    const int DP = D - 2;
    const size_t smem = (size_t)kWarps * (DP + 2) * A.n * sizeof(T);
    const int grid = c->sms * 2;
    cudaMemsetAsync(A.counter, 0, sizeof(int), c->stream);
#define SG_LAUNCH(DPV, MV)                                                                              \
    do {                                                                                                \
        cudaFuncSetAttribute(k_l0_enum<T, DPV, MV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_l0_enum<T, DPV, MV><<<grid, kWarps * 32, smem, c->stream>>>(A);                               \
    } while (0)
    if (D == 1) {
        if (mode == 0) k_l0_single<T, 0><<<(A.n + 255) / 256, 256, 0, c->stream>>>(A);
        else k_l0_single<T, 1><<<(A.n + 255) / 256, 256, 0, c->stream>>>(A);
    } else if (DP == 0) { if (mode == 0) SG_LAUNCH(0, 0); else SG_LAUNCH(0, 1); }
    else if (DP == 1) { if (mode == 0) SG_LAUNCH(1, 0); else SG_LAUNCH(1, 1); }
    else if (DP == 2) { if (mode == 0) SG_LAUNCH(2, 0); else SG_LAUNCH(2, 1); }
    else if (DP == 3) { if (mode == 0) SG_LAUNCH(3, 0); else SG_LAUNCH(3, 1); }
    else return fail(c, SISSO_ERR_ARG, "descriptor dimension above SISSO_MAX_DIM");
#undef SG_LAUNCH
    c->stats.launches++;
    return check_cuda(c, cudaGetLastError(), "l0_enum");
}

// padded FP32 copies and the tile list of the tiled enumeration, for up to n features
sisso_status ensure_tile_buffers(sisso_ctx* c, int n) {
    const int ld = kTC + (n + 31) / 32 * 32;                  // kTC zero columns, then the row
    const int n_tiles = ((n + kTR - 1) / kTR) * ((n + kTC - 1) / kTC);
    if (n <= c->tile_rows && ld <= c->tile_ld && n_tiles <= c->tile_info_cap) return SISSO_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->tile_G); cudaFree(c->tile_b); cudaFree(c->tile_diag); cudaFree(c->tile_info);
    c->tile_G = c->tile_b = c->tile_diag = nullptr;
    c->tile_info = nullptr;
    c->tile_rows = c->tile_ld = c->tile_info_cap = 0;
    sisso_status st;
    if ((st = check_cuda(c, cudaMalloc(&c->tile_G, sizeof(float) * (size_t)n * ld), "tile_G")) ||
        (st = check_cuda(c, cudaMalloc(&c->tile_b, sizeof(float) * (size_t)ld), "tile_b")) ||
        (st = check_cuda(c, cudaMalloc(&c->tile_diag, sizeof(float) * (size_t)ld), "tile_diag")) ||
        (st = check_cuda(c, cudaMalloc(&c->tile_info, sizeof(TileInfo) * (size_t)n_tiles), "tile_info")))
        return st;
    c->tile_rows = n; c->tile_ld = ld; c->tile_info_cap = n_tiles;
    return SISSO_OK;
}

// Exhaustive FP32 l0 (D >= 2) by the single-pass tiled enumeration (l0_tile.cuh): padded
// FP32 copies, a greedy FP64 bound, one enumeration launch, FP64 refit of the band and the
// tie-broken winner.
__global__ void k_set_bound(unsigned long long* key, double v) { *key = okey(v); }

// prefix_mask (optional): only the prefixes whose bit is set are enumerated; bound0 >= 0:
// the search starts from this FP64 RSS (an upper bound of the minimum) instead of the greedy one
static sisso_status l0_solve_tiled(sisso_ctx* c, const double* G, const double* b, int ld, double syy, int n, int D,
                                   const int64_t* gid_dev, Winner& w, const unsigned* prefix_mask = nullptr,
                                   double bound0 = -1.0) {
    sisso_status st;
    if ((st = ensure_tile_buffers(c, n))) return st;
    const int DP = D - 2;
    const int ldp = kTC + (n + 31) / 32 * 32;
    // tiles (a, c): a row block [a, a + kTR) and a column block [c, c + kTC) starting at the
    // row block (columns left of it hold no subsets); a tile's prefixes are the colex ranks
    // below C(m, DP), m the largest row of the tile with a column to its right; one work
    // unit per (tile, prefix)
    std::vector<TileInfo> tiles;
    int64_t items = 0;
    for (int a = 0; a < n - 1; a += kTR)
        for (int cc = a; cc < n; cc += kTC) {
            const int m = std::min({a + kTR - 1, n - 2, cc + kTC - 2});
            if (m < a || m < DP) continue;
            const int64_t np = binom_host(m, DP);
            if (np <= 0) continue;
            tiles.push_back(TileInfo{a, cc, np, items});
            items += np;
        }
    if ((int)tiles.size() > c->tile_info_cap) return fail(c, SISSO_ERR_CAPACITY, "l0: tile list");
    cudaMemcpyAsync(c->tile_info, tiles.data(), sizeof(TileInfo) * tiles.size(), cudaMemcpyHostToDevice, c->stream);
    const double sst = syy * c->N;
    unsigned long long* ub_key = reinterpret_cast<unsigned long long*>(c->work + 2);
    unsigned long long* examined = ub_key + 1;
    unsigned long long* min_key = ub_key + 2;
    unsigned long long* cand = ub_key + 3;
    cudaEvent_t e0, e1, e2, e3, e4;
    cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2); cudaEventCreate(&e3); cudaEventCreate(&e4);
    cudaEventRecord(e0, c->stream);
    cudaMemsetAsync(c->work, 0, sizeof(unsigned long long), c->stream);   // 64-bit unit counter
    cudaMemsetAsync(ub_key, 0xFF, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(min_key, 0xFF, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(examined, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(cand, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->band_count, 0, sizeof(unsigned), c->stream);
    const int64_t tot = (int64_t)n * ldp;
    k_pad_gram<<<std::max(1, (int)std::min<int64_t>(c->sms * 8, (tot + 255) / 256)), 256, 0, c->stream>>>(
        G, b, ld, n, ldp, c->tile_G, c->tile_b, c->tile_diag);
    if (bound0 >= 0.0) k_set_bound<<<1, 1, 0, c->stream>>>(ub_key, bound0);
    else k_greedy_bound<<<1, 256, 0, c->stream>>>(G, b, ld, syy, c->N, n, D, ub_key);
    TileArgs A{};
    A.G = c->tile_G + kTC; A.b = c->tile_b; A.diag = c->tile_diag; A.ldp = ldp; A.n = n; A.N = c->N; A.D = D;
    A.syy = (float)syy; A.tau = kPivotMin32; A.sst = sst; A.sqrt_syy = std::sqrt(syy);
    // filter: coefficient 1-norm bound Smax = 16 sqrt(syy); E1 = twice the a posteriori bound
    // at Smax (|RSS| <= 2 SST) plus the rounding of the filter's own comparison
    {
        const double u = 5.9604644775390625e-8, c1 = 1.0 + 3.1 * (D + 1);
        const double smax = 16.0 * std::sqrt(syy);
        const double err = 2.0 * u * (c->N * (2.0 * std::sqrt(syy) * smax + c1 * smax * smax) + (D + 3) * 4.0 * sst);
        A.Smax = (float)smax;
        A.E1 = (float)(2.0 * err + 64.0 * u * sst);
    }
    A.tiles = reinterpret_cast<const TileInfo*>(c->tile_info); A.n_tiles = (int)tiles.size(); A.n_items = items;
    A.counter = c->work; A.ub_key = ub_key; A.tie64 = 2.0 * kRssTie * sst;
    A.G64 = G; A.b64 = b; A.ld64 = ld; A.syy64 = syy;
    A.band = c->band; A.band_count = c->band_count; A.band_cap = c->band_cap; A.band_r32 = nullptr;
    A.examined = examined; A.candidates = cand; A.prefix_mask = prefix_mask;
    cudaEventRecord(e1, c->stream);
    const int grid = c->sms * 2;
#define SG_TILE(DPV)                                                                                   \
    do {                                                                                               \
        const size_t sm = tile_smem_bytes(DPV);                                                        \
        cudaFuncSetAttribute(k_l0_tile<DPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);   \
        k_l0_tile<DPV><<<grid, kTW * 32, sm, c->stream>>>(A);                                          \
    } while (0)
    switch (DP) {
        case 0: SG_TILE(0); break;
        case 1: SG_TILE(1); break;
        case 2: SG_TILE(2); break;
        default: SG_TILE(3); break;
    }
#undef SG_TILE
    cudaEventRecord(e2, c->stream);
    k_refit<<<c->sms * 4, 256, 0, c->stream>>>(G, b, ld, syy, c->N, D, c->band, c->band_count, c->band_cap,
                                              c->band_rss, min_key);
    k_winner<<<1, 1024, 0, c->stream>>>(c->band, c->band_rss, c->band_count, c->band_cap, min_key, kRssTie * sst,
                                        gid_dev, D, c->win);
    c->stats.launches += 5;
    c->stats.l0_enum_launches++;
    cudaEventRecord(e3, c->stream);
    if ((st = check_cuda(c, cudaGetLastError(), "l0_tile"))) return st;
    unsigned cnt = 0;
    unsigned long long ex[2] = {0, 0};
    cudaMemcpyAsync(&cnt, c->band_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&ex[0], examined, sizeof(ex[0]), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&ex[1], cand, sizeof(ex[1]), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(c->win_h, c->win, sizeof(Winner), cudaMemcpyDeviceToHost, c->stream);
    cudaEventRecord(e4, c->stream);
    if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "l0 tiled"))) return st;
    c->stats.ms_l0 += event_ms(e0, e2);
    c->stats.ms_l0_enum += event_ms(e1, e2);
    c->stats.ms_refit += event_ms(e2, e3);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2); cudaEventDestroy(e3); cudaEventDestroy(e4);
    if ((int64_t)cnt > c->band_cap)
        return fail(c, SISSO_ERR_CAPACITY, "l0: FP64 refit band exceeds max_band (" + std::to_string(cnt) + ")");
    c->stats.subsets_fit += (int64_t)ex[0];
    c->stats.l0_candidates += (int64_t)ex[1];
    c->stats.subsets_refit += cnt;
    w = *c->win_h;
    w.examined = (int64_t)ex[0];
    if (!w.found) return fail(c, SISSO_ERR_NUMERIC, "l0: every subset is singular");
    return SISSO_OK;
}

// Certificate of a D = 5 incumbent (FP64 RSS bound0, e.g. the learned search's winner):
// every 3-prefix whose superset bound (l0_tile.cuh) exceeds bound0 + tie + margin cannot
// extend to the minimum or a tie of it and is skipped; the other prefixes are enumerated
// exactly by the tiled search started from bound0, whose winner is then the exhaustive
// search's.  The bounds are FP64 (margin 1e-9 SST + 1e-7 relative); suffix sets whose
// reversed Cholesky meets a pivot at or below 1e-6 are never pruned.
sisso_status l0_certify(sisso_ctx* c, const double* G, const double* b, int ld, double syy, int n,
                        const int64_t* gid_dev, double bound0, Winner& w, int64_t* prefixes_kept) {
    if (n < 5 || n > 4095) return fail(c, SISSO_ERR_ARG, "certificate: n must be in 5..4095");
    const int64_t np = (int64_t)n * (n - 1) * (n - 2) / 6;
    const int64_t words = (np + 31) / 32;
    double *L = nullptr, *wv = nullptr, *q = nullptr;
    int* m_ok = nullptr;
    unsigned* mask = nullptr;
    unsigned long long* kept = nullptr;
    sisso_status st = SISSO_OK;
    auto ck = [&](cudaError_t e, const char* what) { if (!st && e != cudaSuccess) st = check_cuda(c, e, what); };
    ck(cudaMallocAsync((void**)&L, sizeof(double) * (size_t)n * n, c->stream), "certificate: factor");
    ck(cudaMallocAsync((void**)&wv, sizeof(double) * (size_t)n, c->stream), "certificate: w");
    ck(cudaMallocAsync((void**)&q, sizeof(double) * (size_t)(n + 1), c->stream), "certificate: q");
    ck(cudaMallocAsync((void**)&m_ok, sizeof(int), c->stream), "certificate: m");
    ck(cudaMallocAsync((void**)&mask, sizeof(unsigned) * (size_t)words, c->stream), "certificate: mask");
    ck(cudaMallocAsync((void**)&kept, sizeof(unsigned long long), c->stream), "certificate: count");
    if (!st) {
        const double sst = syy * c->N;
        const double thr = bound0 + 2.0 * kRssTie * sst + 1e-9 * sst + 1e-7 * std::fabs(bound0);
        cudaMemsetAsync(mask, 0, sizeof(unsigned) * (size_t)words, c->stream);
        cudaMemsetAsync(kept, 0, sizeof(unsigned long long), c->stream);
        k_rev_chol<<<1, 1024, 0, c->stream>>>(G, b, ld, n, 1e-6, L, wv, m_ok);
        k_prefix_sq<<<1, 32, 0, c->stream>>>(wv, n, m_ok, q);
        const int64_t npair = (int64_t)n * (n - 1) / 2;
        k_superset_mask<<<(unsigned)((npair + 255) / 256), 256, 0, c->stream>>>(G, b, ld, n, c->N, syy, L, wv, q, m_ok,
                                                                                  thr, mask, kept);
        c->stats.launches += 3;
        ck(cudaGetLastError(), "certificate");
        unsigned long long h_kept = 0;
        ck(cudaMemcpyAsync(&h_kept, kept, sizeof(h_kept), cudaMemcpyDeviceToHost, c->stream), "certificate: count");
        ck(cudaStreamSynchronize(c->stream), "certificate");
        if (!st) {
            if (prefixes_kept) *prefixes_kept = (int64_t)h_kept;
            st = l0_solve_tiled(c, G, b, ld, syy, n, 5, gid_dev, w, mask, bound0);
        }
    }
    cudaFreeAsync(L, c->stream); cudaFreeAsync(wv, c->stream); cudaFreeAsync(q, c->stream);
    cudaFreeAsync(m_ok, c->stream); cudaFreeAsync(mask, c->stream); cudaFreeAsync(kept, c->stream);
    (void)np;
    return st;
}

sisso_status l0_solve(sisso_ctx* c, const double* G, const double* b, const float* G32, const float* b32,
                      int ld, double syy, int n, int D, const int64_t* gid_dev, int precision, Winner& w,
                      const int* prefix_list, int64_t n_prefixes) {
    if (D < 1 || D > kMaxDim || n < D) return fail(c, SISSO_ERR_ARG, "l0: bad D or n");
    if (n > (D <= 4 ? 65535 : 4095)) return fail(c, SISSO_ERR_ARG, "l0: too many features for D");
    const bool fp32 = precision != SISSO_PREC_FP64;
    if (fp32 && !prefix_list && D >= 2) return l0_solve_tiled(c, G, b, ld, syy, n, D, gid_dev, w);
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
    cudaEventRecord(e0, c->stream);
    // work items: (D-2)-prefixes of [0, n-2) in colex order x chunks of kRows i1 rows,
    // decoded in the kernel
    const int DPh = D - 2;
    const int cpp = D >= 2 ? std::max(1, (n - 1 - DPh + kRows - 1) / kRows) : 1;
    if (prefix_list && D < 3) return fail(c, SISSO_ERR_ARG, "l0: a prefix list needs D >= 3");
    const int64_t n_items = D >= 2 ? (prefix_list ? n_prefixes : binom_host(n - 2, DPh)) * cpp : 0;
    unsigned long long* ub_key = reinterpret_cast<unsigned long long*>(c->work + 2);
    unsigned long long* examined = ub_key + 1;
    unsigned long long* min_key = ub_key + 2;
    cudaMemsetAsync(ub_key, 0xFF, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(min_key, 0xFF, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(examined, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->band_count, 0, sizeof(unsigned), c->stream);
    const double sst = syy * c->N;
    sisso_status st;
    if (fp32) {
        EnumArgs<float> A{};
        A.G = G32; A.b = b32; A.ld = ld; A.n = n; A.N = c->N; A.syy = (float)syy; A.sst = sst;
        A.cpp = cpp; A.n_items = n_items; A.counter = c->work;
        A.tau = kPivotMin32; A.fp32 = 1; A.sqrt_syy = std::sqrt(syy); A.ub_key = ub_key; A.win = c->win; A.band = c->band;
        A.G64 = G; A.b64 = b; A.syy64 = syy; A.tie64 = 2.0 * kRssTie * sst; A.prefix_list = prefix_list;
        A.band_count = c->band_count; A.band_cap = c->band_cap; A.examined = examined;
        if ((st = run_enum(c, A, D, 0))) return st;
        k_set_thr<<<1, 1, 0, c->stream>>>(c->win, ub_key, 0.0);
        cudaEventRecord(e1, c->stream);
        if ((st = run_enum(c, A, D, 1))) return st;
    } else {
        EnumArgs<double> A{};
        A.G = G; A.b = b; A.ld = ld; A.n = n; A.N = c->N; A.syy = syy; A.sst = sst;
        A.cpp = cpp; A.n_items = n_items; A.counter = c->work; A.prefix_list = prefix_list;
        A.tau = (float)kPivotMin; A.fp32 = 0; A.ub_key = ub_key; A.win = c->win; A.band = c->band;
        A.band_count = c->band_count; A.band_cap = c->band_cap; A.examined = examined;
        if ((st = run_enum(c, A, D, 0))) return st;
        // the FP64 tie window, widened so that rounding differences between this
        // enumeration and the refit cannot drop a tied subset
        k_set_thr<<<1, 1, 0, c->stream>>>(c->win, ub_key, 2.0 * kRssTie * sst + 1e-14 * sst);
        cudaEventRecord(e1, c->stream);
        if ((st = run_enum(c, A, D, 1))) return st;
    }
    c->stats.launches++;
    cudaEventRecord(e2, c->stream);
    // FP64 refit of the band, minimum, tie-broken winner
    k_refit<<<c->sms * 4, 256, 0, c->stream>>>(G, b, ld, syy, c->N, D, c->band, c->band_count, c->band_cap,
                                              c->band_rss, min_key);
    k_winner<<<1, 1024, 0, c->stream>>>(c->band, c->band_rss, c->band_count, c->band_cap, min_key, kRssTie * sst,
                                        gid_dev, D, c->win);
    c->stats.launches += 2;
    if ((st = check_cuda(c, cudaGetLastError(), "l0_refit"))) return st;
    unsigned cnt = 0;
    unsigned long long ex = 0;
    cudaMemcpyAsync(&cnt, c->band_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&ex, examined, sizeof(ex), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(c->win_h, c->win, sizeof(Winner), cudaMemcpyDeviceToHost, c->stream);
    if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "l0"))) return st;
    cudaEvent_t e3;
    cudaEventCreate(&e3);
    cudaEventRecord(e3, c->stream);
    cudaEventSynchronize(e3);
    c->stats.ms_l0 += event_ms(e0, e2);
    c->stats.ms_refit += event_ms(e2, e3);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2); cudaEventDestroy(e3);
    if ((int64_t)cnt > c->band_cap)
        return fail(c, SISSO_ERR_CAPACITY, "l0: FP64 refit band exceeds max_band (" + std::to_string(cnt) + ")");
    c->stats.subsets_fit += (int64_t)ex;
    c->stats.subsets_refit += cnt;
    w = *c->win_h;
    w.examined = (int64_t)ex;
    if (!w.found) return fail(c, SISSO_ERR_NUMERIC, "l0: every subset is singular");
    return SISSO_OK;
}

// Mixed precision l0: FP32 enumeration on the tensor-core Gram (G32, b32), then the K = 100
// best subsets by FP32 RSS and every subset with a pivot <= 1e-6 (condition estimate above
// 1e6) re-solved in FP64 from the standardised rows; the winner is the lowest FP64 RSS
// with the same tie rule as the exact forms.
sisso_status l0_solve_mixed(sisso_ctx* c, int n, int D, Winner& w) {
    constexpr int kTop = 100;
    if (D < 1 || D > kMaxDim || n < D) return fail(c, SISSO_ERR_ARG, "l0: bad D or n");
    cudaEvent_t e0, e2, e3;
    cudaEventCreate(&e0); cudaEventCreate(&e2); cudaEventCreate(&e3);
    cudaEventRecord(e0, c->stream);
    const int DPh = D - 2;
    const int cpp = D >= 2 ? std::max(1, (n - 1 - DPh + kRows - 1) / kRows) : 1;
    const int64_t n_items = D >= 2 ? binom_host(n - 2, DPh) * cpp : 0;
    unsigned long long* ub_key = reinterpret_cast<unsigned long long*>(c->work + 2);
    unsigned long long* examined = ub_key + 1;
    unsigned long long* min_key = ub_key + 2;
    cudaMemsetAsync(ub_key, 0xFF, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(examined, 0, sizeof(unsigned long long), c->stream);
    const double sst = c->syy * c->N;
    EnumArgs<float> A{};
    A.G = c->G32; A.b = c->b32; A.ld = c->n_cap; A.n = n; A.N = c->N; A.syy = (float)c->syy; A.sst = sst;
    A.cpp = cpp; A.n_items = n_items; A.counter = c->work; A.tau = 1e-6f; A.fp32 = 1; A.sqrt_syy = 0.0;
    A.ub_key = ub_key; A.win = c->win; A.band = c->band; A.band_count = c->band_count; A.band_cap = c->band_cap;
    A.examined = examined; A.band_r32 = c->band_r32;
    sisso_status st;
    if ((st = run_enum(c, A, D, 0))) return st;
    // widen the band until it holds at least kTop subsets (or everything)
    unsigned cnt = 0;
    for (double delta = 1e-4 * sst;; delta *= 10.0) {
        cudaMemsetAsync(c->band_count, 0, sizeof(unsigned), c->stream);
        k_set_thr<<<1, 1, 0, c->stream>>>(c->win, ub_key, delta);
        if ((st = run_enum(c, A, D, 1))) return st;
        cudaMemcpyAsync(&cnt, c->band_count, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
        if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "l0 mixed band"))) return st;
        if ((int64_t)cnt > c->band_cap)
            return fail(c, SISSO_ERR_CAPACITY, "l0: mixed-precision band exceeds max_band");
        if (cnt >= (unsigned)kTop || delta > 2.0 * sst) break;
    }
    cudaEventRecord(e2, c->stream);
    cudaMemsetAsync(min_key, 0xFF, sizeof(unsigned long long), c->stream);
    k_select_top<<<1, 1024, 0, c->stream>>>(c->band_r32, c->band_count, c->band_cap, kTop, c->band_sel);
    k_refit_z<<<c->sms * 8, 256, 0, c->stream>>>(c->Z, c->yc64, c->N, c->syy, D, c->band, c->band_count, c->band_cap,
                                                 c->band_sel, c->band_rss, min_key);
    k_winner<<<1, 1024, 0, c->stream>>>(c->band, c->band_rss, c->band_count, c->band_cap, min_key, kRssTie * sst,
                                        c->S_dev, D, c->win);
    c->stats.launches += 3;
    unsigned long long ex = 0;
    cudaMemcpyAsync(&ex, examined, sizeof(ex), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(c->win_h, c->win, sizeof(Winner), cudaMemcpyDeviceToHost, c->stream);
    cudaEventRecord(e3, c->stream);
    if ((st = check_cuda(c, cudaStreamSynchronize(c->stream), "l0 mixed"))) return st;
    c->stats.ms_l0 += event_ms(e0, e2);
    c->stats.ms_refit += event_ms(e2, e3);
    cudaEventDestroy(e0); cudaEventDestroy(e2); cudaEventDestroy(e3);
    c->stats.subsets_fit += (int64_t)ex;
    c->stats.subsets_refit += std::min<int64_t>(cnt, kTop);
    w = *c->win_h;
    w.examined = (int64_t)ex;
    if (!w.found) return fail(c, SISSO_ERR_NUMERIC, "l0: every refit subset is singular");
    return SISSO_OK;
}

sisso_status winner_model_z(sisso_ctx* c, int n, int D, Winner& w) {
    (void)n;
    k_model_z<<<1, 1024, 0, c->stream>>>(c->Z, c->Zmean, c->Zsd, c->yc64, c->ybar, c->N, c->syy, D, c->S_dev, c->win,
                                         c->resid);
    c->stats.launches++;
    cudaMemcpyAsync(c->win_h, c->win, sizeof(Winner), cudaMemcpyDeviceToHost, c->stream);
    sisso_status st = check_cuda(c, cudaStreamSynchronize(c->stream), "winner_model_z");
    if (st) return st;
    w = *c->win_h;
    return SISSO_OK;
}

sisso_status winner_model(sisso_ctx* c, int n, int D, Winner& w) {
    (void)n;
    k_model<<<1, 1024, 0, c->stream>>>(c->G64, c->b64, c->n_cap, c->syy, c->N, D, c->Z, c->Zmean, c->Zsd, c->yc64,
                                       c->ybar, c->S_dev, c->win, c->resid);
    c->stats.launches++;
    cudaMemcpyAsync(c->win_h, c->win, sizeof(Winner), cudaMemcpyDeviceToHost, c->stream);
    sisso_status st = check_cuda(c, cudaStreamSynchronize(c->stream), "winner_model");
    if (st) return st;
    w = *c->win_h;
    return SISSO_OK;
}

}  // namespace sg

// =====================================================================================
// allocation-free l0 search: the kernels above, with their working memory in one
// file-scope device array instead of context buffers
// =====================================================================================
namespace sg {
namespace {

constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaN = SISSO_NOALLOC_MAX_N;
constexpr size_t kNaBand = SISSO_NOALLOC_MAX_BAND;
constexpr size_t kNaG64 = 0;                                              // n x n FP64
constexpr size_t kNaG32 = na_align(kNaG64 + kNaN * kNaN * sizeof(double)); // n x n FP32
constexpr size_t kNaB64 = na_align(kNaG32 + kNaN * kNaN * sizeof(float));
constexpr size_t kNaB32 = na_align(kNaB64 + kNaN * sizeof(double));
constexpr size_t kNaGid = na_align(kNaB32 + kNaN * sizeof(float));
constexpr size_t kNaBandOff = na_align(kNaGid + kNaN * sizeof(int64_t));
constexpr size_t kNaRss = na_align(kNaBandOff + kNaBand * sizeof(uint64_t));
constexpr size_t kNaCtr = na_align(kNaRss + kNaBand * sizeof(double));    // counters (64 B)
constexpr size_t kNaWin = na_align(kNaCtr + 64);
constexpr size_t kNaTotal = na_align(kNaWin + sizeof(Winner));

// the working array: reserved on every device that loads the library
static __device__ __align__(256) unsigned char g_l0_scratch[kNaTotal];

std::mutex g_na_mu;
unsigned char* g_na_addr[256] = {};    // device address of g_l0_scratch, per device ordinal

__global__ void k_na_cast(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

template <typename T>
cudaError_t na_enum(const EnumArgs<T>& A, int D, int mode, int sms, cudaStream_t st) {
    const int DP = D - 2;
    const size_t smem = (size_t)kWarps * (DP + 2) * A.n * sizeof(T);
    const int grid = sms * 2;
#define SG_NA(DPV, MV)                                                                                   \
    do {                                                                                                 \
        cudaFuncSetAttribute(k_l0_enum<T, DPV, MV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_l0_enum<T, DPV, MV><<<grid, kWarps * 32, smem, st>>>(A);                                       \
    } while (0)
    if (D == 1) {
        if (mode == 0) k_l0_single<T, 0><<<(A.n + 255) / 256, 256, 0, st>>>(A);
        else k_l0_single<T, 1><<<(A.n + 255) / 256, 256, 0, st>>>(A);
    } else if (DP == 0) { if (mode == 0) SG_NA(0, 0); else SG_NA(0, 1); }
    else if (DP == 1) { if (mode == 0) SG_NA(1, 0); else SG_NA(1, 1); }
    else if (DP == 2) { if (mode == 0) SG_NA(2, 0); else SG_NA(2, 1); }
    else { if (mode == 0) SG_NA(3, 0); else SG_NA(3, 1); }
#undef SG_NA
    return cudaGetLastError();
}

}  // namespace
}  // namespace sg

extern "C" sisso_status sisso_l0_search_noalloc(const double* G, const double* b, double syy, int N, int n, int D,
                                                const int64_t* gid, int precision, void* stream, int* best_pos,
                                                double* best_rss, int64_t* examined) {
    using namespace sg;
    if (!G || !b || !gid || !best_pos || N < 1 || n < 1 || D < 1 || D > SISSO_MAX_DIM || n < D ||
        (precision != SISSO_PREC_FP32 && precision != SISSO_PREC_FP64) || !(syy > 0.0))
        return SISSO_ERR_ARG;
    if (n > SISSO_NOALLOC_MAX_N) return SISSO_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SISSO_ERR_CUDA;
    unsigned char* base = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_l0_scratch) != cudaSuccess || !p) return SISSO_ERR_CUDA;
            g_na_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_na_addr[dev];
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SISSO_ERR_CUDA;
    double* dG = reinterpret_cast<double*>(base + kNaG64);
    float* dG32 = reinterpret_cast<float*>(base + kNaG32);
    double* db = reinterpret_cast<double*>(base + kNaB64);
    float* db32 = reinterpret_cast<float*>(base + kNaB32);
    int64_t* dgid = reinterpret_cast<int64_t*>(base + kNaGid);
    uint64_t* band = reinterpret_cast<uint64_t*>(base + kNaBandOff);
    double* band_rss = reinterpret_cast<double*>(base + kNaRss);
    int* counter = reinterpret_cast<int*>(base + kNaCtr);
    unsigned long long* ub_key = reinterpret_cast<unsigned long long*>(base + kNaCtr + 8);
    unsigned long long* ex_key = ub_key + 1;
    unsigned long long* min_key = ub_key + 2;
    unsigned int* band_count = reinterpret_cast<unsigned int*>(base + kNaCtr + 32);
    Winner* win = reinterpret_cast<Winner*>(base + kNaWin);

    const size_t nn = (size_t)n * n;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    ok(cudaMemcpyAsync(dG, G, sizeof(double) * nn, cudaMemcpyDefault, st));
    ok(cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyDefault, st));
    ok(cudaMemcpyAsync(dgid, gid, sizeof(int64_t) * n, cudaMemcpyDefault, st));
    // what must start at zero (or at the maximum key) for this call
    ok(cudaMemsetAsync(base + kNaCtr, 0, 64, st));
    ok(cudaMemsetAsync(ub_key, 0xFF, sizeof(unsigned long long), st));
    ok(cudaMemsetAsync(min_key, 0xFF, sizeof(unsigned long long), st));
    if (e != cudaSuccess) return SISSO_ERR_CUDA;
    k_na_cast<<<std::max(1, std::min(sms * 4, (int)((nn + 255) / 256))), 256, 0, st>>>(dG, dG32, (int64_t)nn);
    k_na_cast<<<1, 256, 0, st>>>(db, db32, n);
    const bool fp32 = precision != SISSO_PREC_FP64;
    const double sst = syy * N;
    const int DPh = D - 2;
    const int cpp = D >= 2 ? std::max(1, (n - 1 - DPh + kRows - 1) / kRows) : 1;
    const int64_t n_items = D >= 2 ? binom_host(n - 2, DPh) * cpp : 0;
    if (fp32) {
        EnumArgs<float> A{};
        A.G = dG32; A.b = db32; A.ld = n; A.n = n; A.N = N; A.syy = (float)syy; A.sst = sst;
        A.cpp = cpp; A.n_items = n_items; A.counter = counter; A.tau = kPivotMin32; A.fp32 = 1; A.sqrt_syy = std::sqrt(syy);
        A.G64 = dG; A.b64 = db; A.syy64 = syy; A.tie64 = 2.0 * kRssTie * sst;
        A.ub_key = ub_key; A.win = win; A.band = band; A.band_count = band_count;
        A.band_cap = (int64_t)kNaBand; A.examined = ex_key;
        ok(na_enum(A, D, 0, sms, st));
        k_set_thr<<<1, 1, 0, st>>>(win, ub_key, 0.0);
        ok(cudaMemsetAsync(counter, 0, sizeof(int), st));
        ok(na_enum(A, D, 1, sms, st));
    } else {
        EnumArgs<double> A{};
        A.G = dG; A.b = db; A.ld = n; A.n = n; A.N = N; A.syy = syy; A.sst = sst;
        A.cpp = cpp; A.n_items = n_items; A.counter = counter; A.tau = (float)kPivotMin; A.fp32 = 0;
        A.ub_key = ub_key; A.win = win; A.band = band; A.band_count = band_count;
        A.band_cap = (int64_t)kNaBand; A.examined = ex_key;
        ok(na_enum(A, D, 0, sms, st));
        k_set_thr<<<1, 1, 0, st>>>(win, ub_key, 2.0 * kRssTie * sst + 1e-14 * sst);
        ok(cudaMemsetAsync(counter, 0, sizeof(int), st));
        ok(na_enum(A, D, 1, sms, st));
    }
    k_refit<<<sms * 4, 256, 0, st>>>(dG, db, n, syy, N, D, band, band_count, (int64_t)kNaBand, band_rss, min_key);
    k_winner<<<1, 1024, 0, st>>>(band, band_rss, band_count, (int64_t)kNaBand, min_key, kRssTie * sst, dgid, D, win);
    ok(cudaGetLastError());
    unsigned cnt = 0;
    unsigned long long ex = 0;
    Winner w{};
    ok(cudaMemcpyAsync(&cnt, band_count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(&ex, ex_key, sizeof(ex), cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(&w, win, sizeof(Winner), cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
    if (e != cudaSuccess) return SISSO_ERR_CUDA;
    if ((size_t)cnt > kNaBand) return SISSO_ERR_CAPACITY;
    if (!w.found) return SISSO_ERR_NUMERIC;
    for (int j = 0; j < D; ++j) best_pos[j] = w.pos[j];
    if (best_rss) *best_rss = w.rss_gram;
    if (examined) *examined = (int64_t)ex;
    return SISSO_OK;
}
