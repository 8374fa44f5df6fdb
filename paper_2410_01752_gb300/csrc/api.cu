// api.cu — the C ABI declared in include/sisso.h: context lifetime, the SISSO iteration
// of §2.3 (Eq. 8) driving the screening (sis.cu) and l0 (l0.cu) kernels, and the
// kernel-level entry points used by the parity tests and the benchmark.
#include "common.cuh"

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

using namespace sg;

namespace {

// X (N x d row-major, FP64) -> column-major FP64 and FP32 copies; flags non-finite input
__global__ void k_ingest(const double* __restrict__ X, const double* __restrict__ y, int N, int d,
                         double* __restrict__ Xc64, float* __restrict__ Xc32, double* __restrict__ y64,
                         int* bad) {
    const int64_t total = (int64_t)N * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / d), c = (int)(e % d);
        const double v = X[e];
        if (!isfinite(v)) atomicOr(bad, 1);
        Xc64[(size_t)c * N + s] = v;
        Xc32[(size_t)c * N + s] = (float)v;
    }
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const double v = y[s];
        if (!isfinite(v)) atomicOr(bad, 2);
        y64[s] = v;
    }
}

__global__ void k_cast(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// A context's buffers (several GB at rung 3) come from a stream-ordered pool per device that
// is private to the library and keeps up to kPoolKeep bytes of freed memory for the next
// context: mapping and unmapping them at every create / destroy took a large share of a
// create-fit-destroy cycle.  sisso_release_memory hands the kept memory back.
constexpr uint64_t kPoolKeep = (uint64_t)32 << 30;
std::mutex g_pool_mutex;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t ctx_pool(int dev, bool create) {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    if (!create) return nullptr;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = kPoolKeep;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    return pool;
}

template <typename T>
sisso_status dalloc(sisso_ctx* c, T*& p, size_t count, const char* what) {
    p = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = ctx_pool(c->opts.device, true);
    if (!pool) return check_cuda(c, cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * count), what);
    const sisso_status st = check_cuda(
        c, cudaMallocFromPoolAsync(reinterpret_cast<void**>(&p), sizeof(T) * count, pool, c->stream), what);
    if (!st) c->pooled.insert(p);
    return st;
}

void free_all(sisso_ctx* c) {
    void* bufs[] = {c->Xc64, c->Xc32, c->y64, c->yc64, c->scores, c->target64, c->tc64, c->tc32, c->tstats,
                    c->hist, c->sel_state, c->surv_ids, c->surv_count, c->surv_score, c->surv_mean, c->surv_sd,
                    c->surv_valid, c->sort_score, c->sort_id, c->sort_src, c->removed, c->walk, c->S_dev,
                    c->S_sorted, c->Z, c->Zmean, c->Zsd, c->G64, c->b64, c->G32, c->b32, c->resid, c->ymom,
                    c->band, c->band_rss, c->band_count, c->prefixes, c->work, c->win, c->blk_best,
                    c->space_dev, c->surv_probe, c->zcache, c->subvalid, c->dup_list, c->dup_ok,
                    c->dup_cnt, c->accepted, c->opcache32, c->opcache64, c->opsum, c->opval64,
                    c->band_r32, c->band_sel, c->tile_G, c->tile_b, c->tile_diag, c->tile_info,
                    c->unit_ok, c->unit_mask, c->opinv64, c->fix_ids, c->fix_count};
    for (void* p : bufs) {
        if (!p) continue;
        if (c->pooled.count(p)) cudaFreeAsync(p, c->stream);    // back to the library's pool
        else cudaFree(p);
    }
    c->pooled.clear();
    tc_screen_free(c);
    whiten_free(c);
    if (c->walk_h) cudaFreeHost(c->walk_h);
    if (c->win_h) cudaFreeHost(c->win_h);
    if (c->stream) cudaStreamSynchronize(c->stream);          // the frees done before the stream goes
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

sisso_status validate(int N, int d, uint32_t ops, int rung, int k, int max_dim, const sisso_opts& o,
                      std::string& why) {
    if (d < 1) { why = "d < 1"; return SISSO_ERR_ARG; }
    if (rung < 1 || rung > SISSO_MAX_RUNG) { why = "rung must be in 1..3"; return SISSO_ERR_ARG; }
    if (max_dim < 1 || max_dim > SISSO_MAX_DIM) { why = "max_dim must be in 1..5"; return SISSO_ERR_ARG; }
    if (k < 1 || k > SISSO_MAX_SIS) { why = "sis_size must be in 1..1024"; return SISSO_ERR_ARG; }
    if (N < max_dim + 1 || N < 2) { why = "N must be at least max_dim + 1"; return SISSO_ERR_ARG; }
    if ((ops & SISSO_OP_ALL) == 0 || (ops & ~SISSO_OP_ALL)) { why = "bad operator mask"; return SISSO_ERR_ARG; }
    if (o.precision < SISSO_PREC_FP64 || o.precision > SISSO_PREC_MIXED_FP16) { why = "bad precision"; return SISSO_ERR_ARG; }
    if (o.grammar != SISSO_GRAMMAR_EQ2 && o.grammar != SISSO_GRAMMAR_NEW_X_PREV) { why = "bad grammar"; return SISSO_ERR_ARG; }
    if ((int64_t)max_dim * k > (max_dim <= 4 ? 65535 : 4095)) { why = "subspace too large"; return SISSO_ERR_ARG; }
    if (!(o.sis_threshold >= 0.0 && o.sis_threshold < 1.0)) { why = "sis_threshold must be in [0, 1)"; return SISSO_ERR_ARG; }
    if (!(o.stop_rmse >= 0.0)) { why = "stop_rmse must be >= 0"; return SISSO_ERR_ARG; }
    if (o.screen < SISSO_SCREEN_AUTO || o.screen > SISSO_SCREEN_TENSOR) { why = "bad screen option"; return SISSO_ERR_ARG; }
    if (o.whiten && (o.precision != SISSO_PREC_FP64 || o.prescreen != SISSO_PRESCREEN_NONE)) {
        why = "whitening needs SISSO_PREC_FP64 and no pre-screening";
        return SISSO_ERR_ARG;
    }
    if (o.gram < SISSO_GRAM_AUTO || o.gram > SISSO_GRAM_TF32X3 ||
        (o.gram == SISSO_GRAM_TF32X3 && o.precision != SISSO_PREC_FP32)) {
        why = "bad gram option (the 3xTF32 Gram is an FP32-precision form)";
        return SISSO_ERR_ARG;
    }
    if (o.units)
        for (int j = 0; j < d; ++j)
            if (o.units[j] < -1 || o.units[j] >= d) { why = "unit labels must be in -1..d-1"; return SISSO_ERR_ARG; }
    if (o.prescreen < SISSO_PRESCREEN_NONE || o.prescreen > SISSO_PRESCREEN_SPEARMAN) { why = "bad prescreen"; return SISSO_ERR_ARG; }
    if (o.prescreen != SISSO_PRESCREEN_NONE && !(o.prescreen_quantile > 0.0 && o.prescreen_quantile <= 1.0)) {
        why = "prescreen_quantile must be in (0, 1]";
        return SISSO_ERR_ARG;
    }
    return SISSO_OK;
}

}  // namespace

extern "C" {

void sisso_default_opts(sisso_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = SISSO_PREC_FP32;
    o->grammar = SISSO_GRAMMAR_EQ2;
    o->survivors = 0;
    o->band_rel = 0.0;
    o->max_band = 0;
    o->cuda_stream = nullptr;
    o->device = 0;
}

sisso_status sisso_create(const double* X, const double* y, int N, int d, uint32_t op_set, int rung,
                          int sis_size, int max_dim, const sisso_opts* opts, sisso_ctx** out) {
    if (!out) return SISSO_ERR_ARG;
    *out = nullptr;
    if (!X || !y) return SISSO_ERR_ARG;
    sisso_opts o;
    sisso_default_opts(&o);
    if (opts) o = *opts;
    std::string why;
    sisso_status st = validate(N, d, op_set, rung, sis_size, max_dim, o, why);
    if (st) return st;
    if (o.prescreen != SISSO_PRESCREEN_NONE) {
        // pre-screening (§3.1): score the primaries, keep the top quantile and build the
        // context on those columns only (renumbered; their unit labels renumbered too)
        if (cudaSetDevice(o.device) != cudaSuccess) return SISSO_ERR_CUDA;
        std::vector<double> score((size_t)d);
        std::vector<int> keep((size_t)d);
        if ((st = prescreen_scores(X, y, N, d, o.prescreen, score.data(), why))) return st;
        const int dk = prescreen_keep(score.data(), d, o.prescreen_quantile, keep.data());
        if (dk < 1) return SISSO_ERR_NUMERIC;
        std::vector<double> Xh((size_t)N * d), Xk((size_t)N * dk);
        if (cudaMemcpy(Xh.data(), X, sizeof(double) * Xh.size(), cudaMemcpyDefault) != cudaSuccess) return SISSO_ERR_CUDA;
        std::vector<int> idx, lab, relabel((size_t)d + 1, -2);
        for (int j = 0; j < d; ++j)
            if (keep[j]) idx.push_back(j);
        for (int r = 0; r < N; ++r)
            for (int q = 0; q < dk; ++q) Xk[(size_t)r * dk + q] = Xh[(size_t)r * d + idx[q]];
        sisso_opts o2 = o;
        o2.prescreen = SISSO_PRESCREEN_NONE;
        if (o.units) {
            int next = 0;
            for (int q = 0; q < dk; ++q) {
                const int u = o.units[idx[q]];
                if (u < 0) { lab.push_back(-1); continue; }
                if (relabel[u] == -2) relabel[u] = next++;
                lab.push_back(relabel[u]);
            }
            o2.units = lab.data();
        }
        st = sisso_create(Xk.data(), y, N, dk, op_set, rung, sis_size, max_dim, &o2, out);
        if (!st) (*out)->primaries = idx;
        return st;
    }
    sisso_ctx* c = new (std::nothrow) sisso_ctx();
    if (!c) return SISSO_ERR_OOM;
    c->N = N; c->d = d; c->rung = rung; c->k = sis_size; c->max_dim = max_dim; c->ops = op_set; c->opts = o;
    if (o.units) c->units.assign(o.units, o.units + d);
    for (int j = 0; j < d; ++j) c->primaries.push_back(j);
    c->opts.units = nullptr;        // the labels live in the context
    if (!plan_space(d, op_set, rung, o.grammar, c->space)) { delete c; return SISSO_ERR_ARG; }
    c->n_feat = c->space.phi[rung];
    if (c->space.phi[rung - 1] >= (int64_t)1 << 31) { delete c; return SISSO_ERR_ARG; }
    auto bail = [&](sisso_status s) { free_all(c); delete c; return s; };
    if ((st = check_cuda(c, cudaSetDevice(o.device), "cudaSetDevice"))) return bail(st);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    if (o.cuda_stream) { c->stream = (cudaStream_t)o.cuda_stream; c->own_stream = false; }
    else {
        if ((st = check_cuda(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream"))) return bail(st);
        c->own_stream = true;
    }
    const size_t Nn = (size_t)N;
    c->n_cap = max_dim * sis_size;
    const int64_t base_window = std::max<int64_t>(16384, 64LL * sis_size);
    c->surv_cap = std::min<int64_t>(base_window * 64, c->n_feat) + c->n_cap;
    int64_t sp = 1;
    while (sp < c->surv_cap) sp <<= 1;
    c->sort_cap = sp;
    c->band_cap = o.max_band > 0 ? o.max_band : ((int64_t)1 << 22);
    if ((st = dalloc(c, c->Xc64, Nn * d, "X")) || (st = dalloc(c, c->Xc32, Nn * d, "X32")) ||
        (st = dalloc(c, c->y64, Nn, "y")) || (st = dalloc(c, c->yc64, Nn, "yc")) ||
        (st = dalloc(c, c->scores, (size_t)c->n_feat, "scores")) || (st = dalloc(c, c->target64, Nn, "target")) ||
        (st = dalloc(c, c->tc64, Nn, "tc64")) || (st = dalloc(c, c->tc32, Nn, "tc32")) ||
        (st = dalloc(c, c->tstats, 1, "tstats")) || (st = dalloc(c, c->hist, 3 * 4096, "hist")) ||
        (st = dalloc(c, c->sel_state, 4, "sel")) || (st = dalloc(c, c->surv_ids, (size_t)c->surv_cap, "surv")) ||
        (st = dalloc(c, c->surv_count, 1, "surv_count")) ||
        (st = dalloc(c, c->surv_score, (size_t)c->surv_cap, "surv_score")) ||
        (st = dalloc(c, c->surv_mean, (size_t)c->surv_cap, "surv_mean")) ||
        (st = dalloc(c, c->surv_sd, (size_t)c->surv_cap, "surv_sd")) ||
        (st = dalloc(c, c->surv_valid, (size_t)c->surv_cap, "surv_valid")) ||
        (st = dalloc(c, c->surv_probe, (size_t)c->surv_cap * kProbes, "surv_probe")) ||
        (st = dalloc(c, c->sort_score, (size_t)c->sort_cap, "sort")) ||
        (st = dalloc(c, c->sort_id, (size_t)c->sort_cap, "sort_id")) ||
        (st = dalloc(c, c->sort_src, (size_t)c->sort_cap, "sort_src")) ||
        (st = dalloc(c, c->removed, (size_t)c->sort_cap, "removed")) || (st = dalloc(c, c->walk, 1, "walk")) ||
        (st = dalloc(c, c->S_dev, (size_t)c->n_cap, "S")) || (st = dalloc(c, c->S_sorted, (size_t)c->n_cap, "S_sorted")) ||
        (st = dalloc(c, c->Z, (size_t)c->n_cap * Nn, "Z")) || (st = dalloc(c, c->Zmean, (size_t)c->n_cap, "Zmean")) ||
        (st = dalloc(c, c->Zsd, (size_t)c->n_cap, "Zsd")) ||
        (st = dalloc(c, c->G64, (size_t)c->n_cap * c->n_cap, "G64")) || (st = dalloc(c, c->b64, (size_t)c->n_cap, "b64")) ||
        (st = dalloc(c, c->G32, (size_t)c->n_cap * c->n_cap, "G32")) || (st = dalloc(c, c->b32, (size_t)c->n_cap, "b32")) ||
        (st = dalloc(c, c->resid, Nn, "resid")) || (st = dalloc(c, c->ymom, 4, "ymom")) ||
        (st = dalloc(c, c->band, (size_t)c->band_cap, "band")) ||
        (st = dalloc(c, c->band_rss, (size_t)c->band_cap, "band_rss")) ||
        (st = dalloc(c, c->band_count, 1, "band_count")) || (st = dalloc(c, c->work, 16, "work")) ||
        (st = dalloc(c, c->band_r32, (size_t)c->band_cap, "band_r32")) ||
        (st = dalloc(c, c->band_sel, (size_t)c->band_cap, "band_sel")) ||
        (st = dalloc(c, c->win, 1, "win")) || (st = dalloc(c, c->space_dev, 1, "space")))
        return bail(st);
    cudaMemcpyAsync(c->space_dev, &c->space, sizeof(Space), cudaMemcpyHostToDevice, c->stream);
    if ((st = ensure_tile_buffers(c, c->n_cap))) return bail(st);
    // standardised FP64 vectors of the screening window, for the duplicate rule: up to
    // 4 GB (the walk evaluates on the fly when a window does not fit)
    c->zcap = std::min<int64_t>(c->surv_cap, ((int64_t)16 << 30) / ((int64_t)8 * N));
    if ((st = dalloc(c, c->zcache, (size_t)c->zcap * Nn, "zcache")) ||
        (st = dalloc(c, c->subvalid, (size_t)c->space.phi[rung - 1], "subvalid")) ||
        (st = dalloc(c, c->dup_list, (size_t)c->sort_cap * kDupSlots, "dup_list")) ||
        (st = dalloc(c, c->dup_ok, (size_t)c->sort_cap * kDupSlots, "dup_ok")) ||
        (st = dalloc(c, c->dup_cnt, (size_t)c->sort_cap, "dup_cnt")) ||
        (st = dalloc(c, c->accepted, (size_t)c->surv_cap, "accepted")))
        return bail(st);
    // operand cache (phi_{L-1} values): kept when it fits 8 GB, otherwise the screening
    // kernels rebuild operands from the primaries on the fly
    {
        const size_t elt = o.precision == SISSO_PREC_FP64 ? sizeof(double) : sizeof(float);
        const size_t bytes = (size_t)c->space.phi[rung - 1] * Nn * elt;
        if (bytes <= ((size_t)8 << 30)) {
            if (o.precision == SISSO_PREC_FP64) st = dalloc(c, c->opcache64, (size_t)c->space.phi[rung - 1] * Nn, "opcache");
            else st = dalloc(c, c->opcache32, (size_t)c->space.phi[rung - 1] * Nn, "opcache");
            if (!st) st = dalloc(c, c->opsum, 3 * (size_t)c->space.phi[rung - 1], "opsum");
            if (!st && o.precision != SISSO_PREC_FP64) {
                c->fix_cap = 1 << 20;
                st = dalloc(c, c->fix_ids, (size_t)c->fix_cap, "fix_ids");
                if (!st) st = dalloc(c, c->fix_count, 1, "fix_count");
            }
            if (st) return bail(st);
        }
        // FP64 operand values (feature-major) for the exact re-score and duplicate checks
        if ((size_t)c->space.phi[rung - 1] * Nn * sizeof(double) <= ((size_t)16 << 30)) {
            if ((st = dalloc(c, c->opval64, (size_t)c->space.phi[rung - 1] * Nn, "opval64"))) return bail(st);
            // their reciprocals when they fit 8 GB (the FP64 re-score divides by operands)
            if ((size_t)c->space.phi[rung - 1] * Nn * sizeof(double) <= ((size_t)8 << 30) &&
                (st = dalloc(c, c->opinv64, (size_t)c->space.phi[rung - 1] * Nn, "opinv64")))
                return bail(st);
        }
    }
    if ((st = check_cuda(c, cudaMallocHost(&c->walk_h, sizeof(WalkResult)), "walk_h")) ||
        (st = check_cuda(c, cudaMallocHost(&c->win_h, sizeof(Winner)), "win_h")))
        return bail(st);
    // inputs: may be host or device memory (unified addressing)
    double *Xraw = nullptr, *yraw = nullptr;
    int* bad = nullptr;
    if ((st = dalloc(c, Xraw, Nn * d, "Xraw")) || (st = dalloc(c, yraw, Nn, "yraw")) || (st = dalloc(c, bad, 1, "bad")))
        return bail(st);
    cudaMemcpyAsync(Xraw, X, sizeof(double) * Nn * d, cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(yraw, y, sizeof(double) * Nn, cudaMemcpyDefault, c->stream);
    cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    k_ingest<<<std::max(1, std::min(c->sms * 8, (int)((Nn * d + 255) / 256))), 256, 0, c->stream>>>(
        Xraw, yraw, N, d, c->Xc64, c->Xc32, c->y64, bad);
    int h_bad = 0;
    cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    // validity of the operand features (depends on X only), moments of y, y~ = y - mean(y)
    st = fill_val64(c);
    if (!st) st = build_units(c);
    if (!st) st = compute_subvalid(c);
    if (!st) st = fill_opcache(c);
    const bool mixed_form = o.precision == SISSO_PREC_MIXED_BF16 || o.precision == SISSO_PREC_MIXED_FP16;
    if (!st && mixed_form && o.screen != SISSO_SCREEN_CORES && c->opval64 && tc_screen_possible(c, o.screen))
        st = tc_screen_alloc(c);
    if (!st && o.whiten) {
        // whitening (§2.4) runs row by row from the FP64 operand values and keeps every
        // window vector
        if (!c->opval64 || c->zcap < c->surv_cap)
            st = fail(c, SISSO_ERR_CAPACITY, "whitening: FP64 operand values or window vectors do not fit");
        else
            st = whiten_setup(c, o.whiten);
    }
    if (!st) st = prepare_target(c, c->y64);
    cudaMemcpyAsync(c->yc64, c->tc64, sizeof(double) * Nn, cudaMemcpyDeviceToDevice, c->stream);
    TargetStats ts{};
    cudaMemcpyAsync(&ts, c->tstats, sizeof(ts), cudaMemcpyDeviceToHost, c->stream);
    sisso_status st2 = check_cuda(c, cudaStreamSynchronize(c->stream), "create");
    cudaFree(Xraw); cudaFree(yraw); cudaFree(bad);
    if (st || st2) return bail(st ? st : st2);
    if (h_bad) return bail(SISSO_ERR_ARG);
    if (!(ts.sd > 0.0)) return bail(SISSO_ERR_ARG);     // constant target
    c->ybar = ts.mean;
    c->syy = ts.sd * ts.sd;
    *out = c;
    return SISSO_OK;
}

sisso_status sisso_fit(sisso_ctx* c) {
    if (!c) return SISSO_ERR_ARG;
    cudaSetDevice(c->opts.device);
    const int prec = c->opts.precision;
    const bool mixed = prec == SISSO_PREC_MIXED_BF16 || prec == SISSO_PREC_MIXED_FP16;
    // tensor-core Gram: the mixed forms' 16-bit one, or FP32 precision's 3xTF32 one on request;
    // either way the l0 step refits its best subsets in FP64 from the standardised rows
    const bool tc_gram = mixed || (prec == SISSO_PREC_FP32 && c->opts.gram == SISSO_GRAM_TF32X3);
    c->stats = sisso_stats{};
    c->tc_ready = false;
    c->S.clear(); c->n_sis.clear(); c->res_ids.clear(); c->res_coef.clear(); c->res_rmse.clear(); c->res_r2.clear();
    c->n_dims = 0;
    c->fitted = false;
    cudaEvent_t f0, f1;
    cudaEventCreate(&f0); cudaEventCreate(&f1);
    cudaEventRecord(f0, c->stream);
    const double* target = c->y64;
    sisso_status st = SISSO_OK;
    for (int t = 1; t <= c->max_dim; ++t) {
        if ((st = prepare_target(c, target))) break;
        if ((st = score_all(c, prec))) break;
        std::vector<int64_t> acc;
        if ((st = sis_select(c, c->k, c->S.data(), (int)c->S.size(), acc))) break;
        const int n_old = (int)c->S.size();
        if (!acc.empty())
            cudaMemcpyAsync(c->S_dev + n_old, acc.data(), sizeof(int64_t) * acc.size(), cudaMemcpyHostToDevice, c->stream);
        c->S.insert(c->S.end(), acc.begin(), acc.end());
        c->n_sis.push_back((int)acc.size());
        const int n = (int)c->S.size();
        if (n < t) {
            // nothing valid to screen is an error; nothing above the SIS threshold ends the fit
            if (t == 1 && !(c->opts.sis_threshold > 0.0)) st = fail(c, SISSO_ERR_NUMERIC, "no valid feature");
            break;
        }
        cudaEvent_t g0, g1;
        cudaEventCreate(&g0); cudaEventCreate(&g1);
        cudaEventRecord(g0, c->stream);
        if ((st = append_subspace(c, n_old, (int)acc.size(), !tc_gram))) break;
        if (tc_gram && (st = gram_tc(c, c->Z, c->yc64, std::sqrt(c->syy), n, c->N, prec, c->G32, c->n_cap, c->b32))) break;
        cudaEventRecord(g1, c->stream);
        Winner w{};
        if (tc_gram) st = l0_solve_mixed(c, n, t, w);
        else if (c->proposal && t == 5 && n >= 5 && n <= 1400) {
            st = l0_learned(c, c->proposal, c->G64, c->b64, c->G32, c->b32, c->n_cap, c->syy, n, c->S_dev,
                            c->prune_frac, w, &c->learned_prefixes);
            if (!st && c->certify_proposal) {
                // certificate: the prefixes the learned winner cannot rule out are enumerated
                // exactly, so the step's winner is the exhaustive search's
                Winner w2{};
                int64_t kept = 0;
                st = l0_certify(c, c->G64, c->b64, c->n_cap, c->syy, n, c->S_dev, w.rss_gram, w2, &kept);
                if (!st) w = w2;
                c->certified_prefixes = kept;
                c->stats.certified_prefixes += kept;
            }
            // the exhaustive search is the fallback when the proposed subsets are all singular
            if (st == SISSO_ERR_NUMERIC)
                st = l0_solve(c, c->G64, c->b64, c->G32, c->b32, c->n_cap, c->syy, n, t, c->S_dev, prec, w);
        } else st = l0_solve(c, c->G64, c->b64, c->G32, c->b32, c->n_cap, c->syy, n, t, c->S_dev, prec, w);
        if (st) break;
        c->stats.ms_gram += event_ms(g0, g1);
        cudaEventDestroy(g0); cudaEventDestroy(g1);
        if ((st = tc_gram ? winner_model_z(c, n, t, w) : winner_model(c, n, t, w))) break;
        c->res_ids.emplace_back(w.ids, w.ids + t);
        c->res_coef.emplace_back(w.coef, w.coef + t + 1);
        c->res_rmse.push_back(w.rmse);
        c->res_r2.push_back(w.r2);
        c->n_dims = t;
        target = c->resid;
        if (w.rmse <= kStopRel * std::sqrt(c->syy)) break;   // exact fit
        if (c->opts.stop_rmse > 0.0 && w.rmse <= c->opts.stop_rmse) break;   // low enough error (§2.3)
    }
    cudaEventRecord(f1, c->stream);
    cudaEventSynchronize(f1);
    c->stats.ms_fit = event_ms(f0, f1);
    cudaEventDestroy(f0); cudaEventDestroy(f1);
    if (st) return st;
    c->fitted = true;
    return SISSO_OK;
}

sisso_status sisso_get_primaries(const sisso_ctx* c, int* idx, int cap, int* n) {
    if (!c || !n) return SISSO_ERR_ARG;
    *n = (int)c->primaries.size();
    if (idx) {
        if (cap < *n) return SISSO_ERR_CAPACITY;
        std::copy(c->primaries.begin(), c->primaries.end(), idx);
    }
    return SISSO_OK;
}

sisso_status sisso_get_n_dims(const sisso_ctx* c, int* n_dims) {
    if (!c || !n_dims) return SISSO_ERR_ARG;
    if (!c->fitted) return SISSO_ERR_STATE;
    *n_dims = c->n_dims;
    return SISSO_OK;
}

sisso_status sisso_get_descriptor(const sisso_ctx* c, int dim, int64_t* ids, double* coef, double* rmse, double* r2) {
    if (!c) return SISSO_ERR_ARG;
    if (!c->fitted) return SISSO_ERR_STATE;
    if (dim < 1 || dim > c->n_dims) return SISSO_ERR_ARG;
    const int q = dim - 1;
    if (ids) std::copy(c->res_ids[q].begin(), c->res_ids[q].end(), ids);
    if (coef) std::copy(c->res_coef[q].begin(), c->res_coef[q].end(), coef);
    if (rmse) *rmse = c->res_rmse[q];
    if (r2) *r2 = c->res_r2[q];
    return SISSO_OK;
}

sisso_status sisso_get_sis(const sisso_ctx* c, int step, int64_t* ids, int cap, int* n) {
    if (!c || !n) return SISSO_ERR_ARG;
    if (!c->fitted) return SISSO_ERR_STATE;
    if (step < 1 || step > (int)c->n_sis.size()) return SISSO_ERR_ARG;
    int off = 0;
    for (int s = 0; s < step - 1; ++s) off += c->n_sis[s];
    const int cnt = c->n_sis[step - 1];
    *n = cnt;
    if (ids) for (int i = 0; i < cnt && i < cap; ++i) ids[i] = c->S[off + i];
    return SISSO_OK;
}

sisso_status sisso_feature_count(const sisso_ctx* c, int64_t* n_features, int64_t* sizes) {
    if (!c) return SISSO_ERR_ARG;
    if (n_features) *n_features = c->n_feat;
    if (sizes) for (int l = 0; l <= c->rung; ++l) sizes[l] = c->space.phi[l];
    return SISSO_OK;
}

sisso_status sisso_feature_expr(const sisso_ctx* c, int64_t id, char* buf, size_t len) {
    if (!c || !buf || len == 0) return SISSO_ERR_ARG;
    if (id < 0 || id >= c->n_feat) return SISSO_ERR_ARG;
    const std::string s = feature_expr(c->space, id);
    if (s.size() + 1 > len) return SISSO_ERR_CAPACITY;
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return SISSO_OK;
}

sisso_status sisso_get_stats(const sisso_ctx* c, sisso_stats* out) {
    if (!c || !out) return SISSO_ERR_ARG;
    *out = c->stats;
    return SISSO_OK;
}

const char* sisso_last_error(const sisso_ctx* c) { return c ? c->err.c_str() : "null context"; }

void sisso_destroy(sisso_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->opts.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

sisso_status sisso_release_memory(int device) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SISSO_ERR_ARG;
    cudaMemPool_t pool = ctx_pool(device, false);
    if (!pool) return SISSO_OK;
    if (cudaSetDevice(device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemPoolTrimTo(pool, 0) != cudaSuccess)
        return SISSO_ERR_CUDA;
    return SISSO_OK;
}

// ---- feature space without a context -----------------------------------------------------

sisso_status sisso_space_sizes(int d, uint32_t op_set, int rung, int grammar, int64_t* sizes) {
    if (!sizes || rung < 1 || rung > SISSO_MAX_RUNG || (op_set & SISSO_OP_ALL) == 0 || (op_set & ~SISSO_OP_ALL))
        return SISSO_ERR_ARG;
    Space sp;
    if (!plan_space(d, op_set, rung, grammar, sp)) return SISSO_ERR_ARG;
    for (int l = 0; l <= rung; ++l) sizes[l] = sp.phi[l];
    return SISSO_OK;
}

sisso_status sisso_space_expr(int d, uint32_t op_set, int rung, int grammar, int64_t id, char* buf, size_t len) {
    if (!buf || len == 0 || rung < 1 || rung > SISSO_MAX_RUNG || (op_set & SISSO_OP_ALL) == 0) return SISSO_ERR_ARG;
    Space sp;
    if (!plan_space(d, op_set, rung, grammar, sp)) return SISSO_ERR_ARG;
    if (id < 0 || id >= sp.phi[rung]) return SISSO_ERR_ARG;
    const std::string s = feature_expr(sp, id);
    if (s.size() + 1 > len) return SISSO_ERR_CAPACITY;
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return SISSO_OK;
}

// ---- kernel-level entry points --------------------------------------------------------

sisso_status sisso_eval_features(sisso_ctx* c, const int64_t* ids, int64_t n, int precision, double* out) {
    if (!c || !ids || !out || n < 0) return SISSO_ERR_ARG;
    if (n == 0) return SISSO_OK;
    cudaSetDevice(c->opts.device);
    int64_t* d_ids = nullptr;
    double* d_out = nullptr;
    sisso_status st;
    if ((st = dalloc(c, d_ids, (size_t)n, "ids")) || (st = dalloc(c, d_out, (size_t)n * c->N, "out"))) {
        cudaFree(d_ids);
        return st;
    }
    cudaMemcpyAsync(d_ids, ids, sizeof(int64_t) * n, cudaMemcpyDefault, c->stream);
    st = eval_features(c, d_ids, n, precision, d_out);
    if (!st) {
        cudaMemcpyAsync(out, d_out, sizeof(double) * n * c->N, cudaMemcpyDefault, c->stream);
        st = check_cuda(c, cudaStreamSynchronize(c->stream), "eval_features");
    }
    cudaFree(d_ids);
    cudaFree(d_out);
    return st;
}

sisso_status sisso_score_all(sisso_ctx* c, const double* target, int precision, float* scores) {
    if (!c || !target || !scores) return SISSO_ERR_ARG;
    cudaSetDevice(c->opts.device);
    cudaMemcpyAsync(c->target64, target, sizeof(double) * c->N, cudaMemcpyDefault, c->stream);
    sisso_status st = prepare_target(c, c->target64);
    if (!st) st = score_all(c, precision);
    if (!st) {
        cudaMemcpyAsync(scores, c->scores, sizeof(float) * c->n_feat, cudaMemcpyDefault, c->stream);
        st = check_cuda(c, cudaStreamSynchronize(c->stream), "score_all");
    }
    return st;
}

sisso_status sisso_sis_step(sisso_ctx* c, const double* target, const int64_t* S_prev, int n_prev, int k,
                            int64_t* acc, int* n_acc) {
    if (!c || !target || !acc || !n_acc || k < 1 || k > SISSO_MAX_SIS || n_prev < 0 || n_prev > c->n_cap - k ||
        (n_prev > 0 && !S_prev))
        return SISSO_ERR_ARG;
    cudaSetDevice(c->opts.device);
    std::vector<int64_t> prev(S_prev, S_prev + n_prev);
    cudaMemcpyAsync(c->target64, target, sizeof(double) * c->N, cudaMemcpyDefault, c->stream);
    sisso_status st = prepare_target(c, c->target64);
    if (!st) st = score_all(c, c->opts.precision);
    std::vector<int64_t> out;
    if (!st) st = sis_select(c, k, prev.data(), n_prev, out);
    if (st) return st;
    *n_acc = (int)out.size();
    std::copy(out.begin(), out.end(), acc);
    return SISSO_OK;
}

sisso_status sisso_l0_search(sisso_ctx* c, const double* G, const double* b, double syy, int n, int D,
                             const int64_t* gid, int precision, int* best_pos, double* best_rss, int64_t* examined) {
    if (!c || !G || !b || !gid || !best_pos || n < 1 || D < 1 || D > SISSO_MAX_DIM || n < D ||
        n > (D <= 4 ? 65535 : 4095))
        return SISSO_ERR_ARG;
    cudaSetDevice(c->opts.device);
    double *dG = nullptr, *db = nullptr;
    float *dG32 = nullptr, *db32 = nullptr;
    int64_t* dgid = nullptr;
    sisso_status st;
    const size_t nn = (size_t)n * n;
    if ((st = dalloc(c, dG, nn, "G")) || (st = dalloc(c, db, (size_t)n, "b")) || (st = dalloc(c, dG32, nn, "G32")) ||
        (st = dalloc(c, db32, (size_t)n, "b32")) || (st = dalloc(c, dgid, (size_t)n, "gid"))) {
        cudaFree(dG); cudaFree(db); cudaFree(dG32); cudaFree(db32); cudaFree(dgid);
        return st;
    }
    cudaMemcpyAsync(dG, G, sizeof(double) * nn, cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(dgid, gid, sizeof(int64_t) * n, cudaMemcpyDefault, c->stream);
    k_cast<<<std::max(1, std::min(c->sms * 4, (int)((nn + 255) / 256))), 256, 0, c->stream>>>(dG, dG32, (int64_t)nn);
    k_cast<<<1, 256, 0, c->stream>>>(db, db32, n);
    Winner w{};
    st = l0_solve(c, dG, db, dG32, db32, n, syy, n, D, dgid, precision, w);
    if (!st) {
        std::copy(w.pos, w.pos + D, best_pos);
        if (best_rss) *best_rss = w.rss_gram;
        if (examined) *examined = w.examined;
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(dG); cudaFree(db); cudaFree(dG32); cudaFree(db32); cudaFree(dgid);
    return st;
}

}  // extern "C"

extern "C" sisso_status sisso_set_proposal_ex(sisso_ctx* c, sisso_mlp* mlp, double frac, int certify) {
    if (!c || (mlp && !(frac > 0.0 && frac <= 1.0))) return SISSO_ERR_ARG;
    c->proposal = mlp;
    if (mlp) c->prune_frac = frac;
    c->certify_proposal = certify != 0;
    return SISSO_OK;
}

extern "C" sisso_status sisso_set_proposal(sisso_ctx* c, sisso_mlp* mlp, double frac) {
    return sisso_set_proposal_ex(c, mlp, frac, 1);
}

static sisso_status l0_learned_entry(sisso_ctx* c, const double* G, const double* b, double syy, int n,
                                     const int64_t* gid, sisso_mlp* mlp, double frac, int* best_pos, double* best_rss,
                                     int64_t* examined, int64_t* n_prefixes, bool certify, int64_t* kept) {
    using namespace sg;
    if (!c || !G || !b || !gid || !mlp || !best_pos || n < 5 || n > 1400 || !(frac > 0.0 && frac <= 1.0) ||
        !(syy > 0.0))
        return SISSO_ERR_ARG;
    cudaSetDevice(c->opts.device);
    double *dG = nullptr, *db = nullptr;
    float *dG32 = nullptr, *db32 = nullptr;
    int64_t* dgid = nullptr;
    sisso_status st;
    const size_t nn = (size_t)n * n;
    if ((st = dalloc(c, dG, nn, "G")) || (st = dalloc(c, db, (size_t)n, "b")) || (st = dalloc(c, dG32, nn, "G32")) ||
        (st = dalloc(c, db32, (size_t)n, "b32")) || (st = dalloc(c, dgid, (size_t)n, "gid"))) {
        cudaFree(dG); cudaFree(db); cudaFree(dG32); cudaFree(db32); cudaFree(dgid);
        return st;
    }
    cudaMemcpyAsync(dG, G, sizeof(double) * nn, cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(dgid, gid, sizeof(int64_t) * n, cudaMemcpyDefault, c->stream);
    k_cast<<<std::max(1, std::min(c->sms * 4, (int)((nn + 255) / 256))), 256, 0, c->stream>>>(dG, dG32, (int64_t)nn);
    k_cast<<<1, 256, 0, c->stream>>>(db, db32, n);
    Winner w{};
    int64_t sel = 0;
    st = l0_learned(c, mlp, dG, db, dG32, db32, n, syy, n, dgid, frac, w, &sel);
    int64_t ex = w.examined;
    if (!st && certify) {
        Winner w2{};
        st = l0_certify(c, dG, db, n, syy, n, dgid, w.rss_gram, w2, kept);
        if (!st) { ex += w2.examined; w = w2; }
    }
    if (!st) {
        std::copy(w.pos, w.pos + 5, best_pos);
        if (best_rss) *best_rss = w.rss_gram;
        if (examined) *examined = ex;
        if (n_prefixes) *n_prefixes = sel;
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(dG); cudaFree(db); cudaFree(dG32); cudaFree(db32); cudaFree(dgid);
    return st;
}

extern "C" sisso_status sisso_l0_learned(sisso_ctx* c, const double* G, const double* b, double syy, int n,
                                         const int64_t* gid, sisso_mlp* mlp, double frac, int* best_pos,
                                         double* best_rss, int64_t* examined, int64_t* n_prefixes) {
    return l0_learned_entry(c, G, b, syy, n, gid, mlp, frac, best_pos, best_rss, examined, n_prefixes, false, nullptr);
}

extern "C" sisso_status sisso_l0_learned_certified(sisso_ctx* c, const double* G, const double* b, double syy, int n,
                                                   const int64_t* gid, sisso_mlp* mlp, double frac, int* best_pos,
                                                   double* best_rss, int64_t* examined, int64_t* n_prefixes,
                                                   int64_t* prefixes_kept) {
    return l0_learned_entry(c, G, b, syy, n, gid, mlp, frac, best_pos, best_rss, examined, n_prefixes, true,
                            prefixes_kept);
}

extern "C" sisso_status sisso_subspace_gram(sisso_ctx* c, const int64_t* ids, int n, double* G, double* b, double* syy) {
    using namespace sg;
    if (!c || !ids || !G || !b || n < 1 || n > c->n_cap) return SISSO_ERR_ARG;
    cudaSetDevice(c->opts.device);
    cudaMemcpyAsync(c->S_dev, ids, sizeof(int64_t) * n, cudaMemcpyDefault, c->stream);
    sisso_status st = append_subspace(c, 0, n, true);
    if (st) return st;
    cudaMemcpy2DAsync(G, sizeof(double) * n, c->G64, sizeof(double) * c->n_cap, sizeof(double) * n, n,
                      cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(b, c->b64, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    st = check_cuda(c, cudaStreamSynchronize(c->stream), "subspace_gram");
    if (!st && syy) *syy = c->syy;
    return st;
}
