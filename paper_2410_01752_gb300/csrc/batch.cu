// batch.cu — the batched multi-task form: many independent SISSO problems (§2.1-2.3,
// Eqs. 2-8) solved by one persistent kernel launch.
//
// Each task runs the same method, with the same numerics, as the per-problem FP32 path
// (FP32 screening with an FP64 re-scored window, FP32 l0 enumeration with an
// error-bounded band refit in FP64), written as a chain of stages:
//
//   START    (serial)   primaries: values, validity; moments of y (target of step 1)
//   LEVEL l  (parallel) phi_l for 0 < l < L: FP64 rows, FP32 sample-major cache, validity
//   OPSUM t  (parallel) per-operand sums for the + and - pairs: sum(x - x0) once per task,
//                       sum((x - x0) r) against the step-t target
//   SCORE t  (parallel) every candidate of phi_L scored against the step-t target (FP32)
//   SELECT t (serial)   the best FP32 scores re-scored in FP64, sorted, walked with the tie
//                       and duplicate rules; accepted features standardised into Z
//   GRAM t   (parallel) FP64 Gram rows and moments of the new subspace members
//   BOUND t  (parallel) l0 pass 1: FP32 bound over every t-subset
//   BAND t   (parallel) l0 pass 2: subsets within the error band of the bound
//   REFIT t  (serial)   FP64 refit of the band, tie-broken winner, model, residual and the
//                       target of step t + 1
//
// Parallel stages are cut into work items that any CTA may take from a queue; the CTA that
// completes a stage's last item runs the following serial stage itself and queues the next
// parallel one.  CTAs take queued items first and start a new task (in the order given,
// longest first) only when nothing is queued, so that few tasks are in flight and each
// finishes soon after it starts.  The only waits are on the queue, and they are bounded.
//
// Memory discipline: every region written inside the launch is written by one stage and
// read only by later stages, per-step products have one region per step, and regions are
// 256-byte aligned, so no cache line is read before the stage writing it has completed.
// Small shared words (queue, per-task counters) are accessed with atomics or L2 loads.
#include "sis_device.cuh"
#include "l0_device.cuh"

#include <algorithm>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

namespace sg {
namespace {

constexpr int kBT = NG * 32;                     // threads per CTA (the pair tile's shape)
constexpr int kWinMax = 4096;                    // screening window cap (sorted in shared memory)
constexpr int kInitIds = 32;                     // ids per LEVEL unit
constexpr int kLowIds = kBT;                     // lower-level ids per SCORE unit
constexpr int kMaxSub = 1024;                    // subspace size cap (max_dim * k)
constexpr int kZRaw = 512;                       // window entries whose FP64 values are kept
constexpr unsigned long long kIdleNs = 10000000000ull;  // default: 10 s with no progress anywhere, give up
constexpr unsigned long long kExit = ~0ull;

enum : int { WK_NONE = 0, WK_START, WK_LEVEL, WK_SCORE, WK_GRAM, WK_BOUND, WK_BAND, WK_OPSUM = 11 };
// stage ids of the profile counters (parallel items by kind; serial stages after them)
enum : int { PS_FLAT = 7, PS_SELECT = 8, PS_REFIT = 9, PS_IDLE = 10,
             PS_SEL_RADIX = 12, PS_SEL_RESCORE = 13, PS_SEL_SORT = 14, PS_SEL_WALK = 15 };

__device__ __forceinline__ void prof_add(const unsigned long long* prof_c, int s, unsigned long long dt) {
    unsigned long long* prof = const_cast<unsigned long long*>(prof_c);
    atomicAdd(prof + s, dt);
    atomicAdd(prof + 16 + s, 1ull);
    atomicMax(prof + 32 + s, dt);
}

// queue word: kind (4 bits) | step or level (4) | task (20) | item index within the stage (36)
__host__ __device__ __forceinline__ unsigned long long item_word(int kind, int t, int task, long long q) {
    return (unsigned long long)kind | ((unsigned long long)t << 4) | ((unsigned long long)task << 8) |
           ((unsigned long long)q << 28);
}
__device__ __forceinline__ int item_kind(unsigned long long w) { return (int)(w & 15); }
__device__ __forceinline__ int item_t(unsigned long long w) { return (int)((w >> 4) & 15); }
__device__ __forceinline__ int item_task(unsigned long long w) { return (int)((w >> 8) & 0xFFFFF); }
__device__ __forceinline__ long long item_q(unsigned long long w) { return (long long)(w >> 28); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// per task and step t (regions written once per launch)
struct BDim {
    float* scores;              // |phi_L| FP32 scores against the step-t target
    double* tc64;               // centred target (N)
    float* tc32;
    TargetStats* ts;
    int64_t* w_ids;             // screening window (kWinMax entries)
    double* w_score;
    double* w_mean;
    double* w_sd;
    int* w_valid;
    double* w_probe;            // kProbes per entry
    int64_t* gid;               // subspace ids after step t (acceptance order)
    double* zmean;              // per subspace member: mean and std of its values
    double* zsd;
    double* G64;                // Gram of the subspace after step t (n_t x n_t) and moments
    double* b64;
    float* G32;
    float* b32;
    uint64_t* band;             // l0 band (band_cap)
    double* band_rss;
    double* resid;              // residual of the step-t model (N)
    double* AR;                 // per operand: sum_s (x_s - x_0) r_s with r the step-t target (P)
};

// per task, written by the host at creation
struct BTask {
    int N, ldv, d, rung;        // samples, row stride of V and Z (N rounded up to 32), primaries
    int P, Q;                   // |phi_{L-1}|, |phi_{L-2}| (operands of the top level)
    int64_t n_feat;             // |phi_L|
    int n_low, n_un, n_tiles;   // SCORE units: 256 lower ids, 32-operand unary blocks, pair tiles
    int n_units;
    int lvl_first[kMaxRung + 1];   // LEVEL units of level l: [lvl_first[l], lvl_first[l + 1])
    const Space* sp;
    PairArgs pa;                // top-level binary sections (scores pointer set per step)
    UnaryArgs ua;
    const int2* tiles;
    const double* X;            // N x d row-major
    const double* y;
    double* V;                  // P rows of FP64 values (stride ldv)
    float* cache;               // N x P FP32 values, sample-major
    unsigned char* vlvl[kMaxRung];   // validity of level l ids (region per level)
    unsigned char* valid;       // validity of ids [0, P), one array
    double* yc;                 // y - mean(y)
    double* Z;                  // standardised subspace members (kMaxSub rows, stride ldv)
    double* zraw;               // FP64 values of the first kZRaw window entries (stride N)
    double* A1;                 // per operand: sum_s (x_s - x_0) (P), written with the step-1 sums
    BDim dim[kMaxDim + 1];      // index t = 1..max_dim
};

// per task, mutable (cleared before each launch)
struct BState {
    int pending;                // items of the running parallel stage not yet done
    int status;                 // SISSO_OK or the task's error
    int n_dims;
    int saturated;              // a screening window could not grow to exactness
    int grown;                  // screening windows grown
    int visits;                 // walk: candidates visited
    int checks;                 // walk: full duplicate comparisons
    int n_S[kMaxDim + 1];       // subspace size after step t
    unsigned band_count[kMaxDim + 1];
    unsigned long long ub_key[kMaxDim + 1];
    unsigned long long examined[kMaxDim + 1];
    unsigned long long t_start, t_end;
    double ybar, syy;
    double thr[kMaxDim + 1];    // l0 pass-2 threshold per step
};

struct BatchArgs {
    const BTask* tasks;
    BState* state;
    sisso_task_result* res;
    int n_tasks;
    const int* order;           // task start order
    unsigned long long* slots;  // work queue (0 = not yet written)
    long long cap;
    int* ctr;                   // [0] head, [1] tail, [2] next task, [3] tasks done, [4] error
    unsigned long long* t0;     // launch start (min over CTAs)
    unsigned long long* prof;   // per stage: [s] ns summed over CTAs, [16 + s] count, [32 + s] max ns
    int k, max_dim;
    int score_units;            // SCORE units per item
    int enum_items;             // l0 enumeration items per BOUND/BAND item
    int gram_rows;              // new subspace rows per GRAM item
    int win0;                   // first screening window
    int band_cap;
    unsigned long long idle_ns; // no progress anywhere for this long: give up (error word)
};

// shared memory of one CTA: one layout per stage
struct SelectSmem {
    union {
        unsigned hist[8 * 1024];            // radix select: one histogram per warp
        struct {
            double sk[kWinMax];             // sorted window: FP64 score (or -1/-2), id, entry
            int64_t sid[kWinMax];
            int ssrc[kWinMax];
        } srt;
    } u;
    unsigned part[kBT];
    unsigned char removed[kWinMax];
    int64_t S_sorted[kMaxSub];
};struct UnarySmem {
    float xs[32][33];
    float r[32];
};
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kL0Smem = (size_t)8 * 4 * 512 * sizeof(float);   // per-warp tables: D <= 4, n <= 512
constexpr size_t kBatchSmem = cmax(cmax(sizeof(PairSmem<float>), sizeof(SelectSmem)), cmax(sizeof(UnarySmem), kL0Smem));

struct Ctl {                    // small per-CTA control block (static shared memory)
    unsigned long long item;
    int flag, n, cur, done, n_acc, visited, n_match, acc_row;
    int ival[8];
    unsigned long long ukey;
    double dval[8];
    double red[32];
    int match[kMaxSub];
};

__device__ __forceinline__ int ldcg_i(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_d(const double* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------------
// the queue
// ---------------------------------------------------------------------------------
// thread 0: the next item (queued work first, else a new task), or kExit
__device__ unsigned long long acquire(const BatchArgs& B) {
    volatile int* head = B.ctr;
    volatile int* tail = B.ctr + 1;
    unsigned long long since = gtimer();
    int seen_tail = -1, seen_done = -1;
    unsigned ns = 64;
    while (true) {
        const int h = *head, t = *tail;
        const int dn = *(volatile int*)(B.ctr + 3);
        if (t != seen_tail || dn != seen_done) { seen_tail = t; seen_done = dn; since = gtimer(); }
        if (h < t) {
            if (atomicCAS(B.ctr, h, h + 1) == h) {
                // slot h is reserved by a producer that is writing it now
                const volatile unsigned long long* slot = B.slots + h;
                const unsigned long long w0 = gtimer();
                while (true) {
                    const unsigned long long v = *slot;
                    if (v) { __threadfence(); return v; }
                    if (*(volatile int*)(B.ctr + 4) || gtimer() - w0 > B.idle_ns) { atomicOr(B.ctr + 4, 1); return kExit; }
                }
            }
            continue;
        }
        if (*(volatile int*)(B.ctr + 2) < B.n_tasks) {
            const int c = atomicAdd(B.ctr + 2, 1);
            if (c < B.n_tasks) return item_word(WK_START, 0, B.order[c], 0);
        }
        if (*(volatile int*)(B.ctr + 3) >= B.n_tasks || *(volatile int*)(B.ctr + 4)) return kExit;
        if (gtimer() - since > B.idle_ns) { atomicOr(B.ctr + 4, 2); return kExit; }
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
    }
}

// whole CTA: queue n items of a parallel stage (pending set first)
__device__ void push(const BatchArgs& B, Ctl& C, int task, int kind, int t, long long n) {
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicExch(&B.state[task].pending, (int)n);
        __threadfence();
        const long long base = atomicAdd(B.ctr + 1, (int)n);
        if (base + n > B.cap) {
            atomicOr(B.ctr + 4, 4);     // queue overflow: every CTA stops
        } else {
            for (long long q = 0; q < n; ++q)
                atomicExch(B.slots + base + q, item_word(kind, t, task, q));
        }
    }
    __syncthreads();
}

__device__ void finish(const BatchArgs& B, int task, int status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        BState& S = B.state[task];
        if (status != SISSO_OK) atomicCAS(&S.status, 0, status);
        const int stt = ldcg_i(&S.status);
        const int nd = ldcg_i(&S.n_dims);
        B.res[task].status = stt;
        B.res[task].n_dims = nd;
        S.t_end = gtimer();
        __threadfence();
        atomicAdd(B.ctr + 3, 1);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// START: primaries and the moments of y
// ---------------------------------------------------------------------------------
__device__ __noinline__ void run_start(const BatchArgs& B, Ctl& C, int task) {
    const BTask& T = B.tasks[task];
    BState& S = B.state[task];
    const int N = T.N, d = T.d, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        S.t_start = gtimer();
        for (int t = 0; t <= kMaxDim; ++t) S.ub_key[t] = ~0ull;
    }
    // primary c: FP64 row, FP32 cache column, validity (finite, |v| <= 1e12, std > 1e-6 max|v|)
    for (int c = w; c < d; c += kBT / 32) {
        double* row = T.V + (size_t)c * T.ldv;
        double s = 0.0, mx = 0.0;
        int bad = 0;
        for (int i = lane; i < N; i += 32) {
            const double v = T.X[(size_t)i * d + c];
            row[i] = v;
            T.cache[(size_t)i * T.P + c] = (float)v;
            if (!isfinite(v) || fabs(v) > kValueCap) bad = 1;
            s += v;
            mx = fmax(mx, fabs(v));
        }
        bad = warp_or(bad);
        s = warp_sum(s);
        mx = warp_max(mx);
        const double mean = s / N;
        double ss = 0.0;
        if (!bad)
            for (int i = lane; i < N; i += 32) { const double u = row[i] - mean; ss += u * u; }
        ss = warp_sum(ss);
        if (lane == 0) T.vlvl[0][c] = !bad && sqrt(ss / N) > kConstRel * mx;
    }
    // step-1 target: y; y~ = y - mean(y) is its centred copy
    const BDim& D1 = T.dim[1];
    prepare_target_block(T.y, N, D1.tc64, D1.tc32, D1.ts, C.red);
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += kBT) T.yc[i] = D1.tc64[i];
    if (threadIdx.x == 0) {
        S.ybar = D1.ts->mean;
        S.syy = D1.ts->sd * D1.ts->sd;
    }
    __syncthreads();
}

// validity of an id below P from its level's region
__device__ __forceinline__ bool valid_lvl(const BTask& T, int64_t id) {
    const Space& sp = *T.sp;
    int l = 0;
    while (id >= sp.phi[l]) ++l;
    return T.vlvl[l][id - (l ? sp.phi[l - 1] : 0)];
}

// ---------------------------------------------------------------------------------
// LEVEL: 32 ids of level l per item; values from their operands' rows
// ---------------------------------------------------------------------------------
__device__ __noinline__ void run_level(const BatchArgs& B, Ctl& C, int task, int l, long long q, float (*tile)[33]) {
    const BTask& T = B.tasks[task];
    const Space& sp = *T.sp;
    const int N = T.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t lo = sp.phi[l - 1], hi = sp.phi[l];
    const int64_t id0 = lo + q * kInitIds;
    // warp w: ids id0 + w + 8 m (m = 0..3)
    int64_t ids[4];
    int ops[4];
    int64_t oa[4], ob[4];
    bool live[4], opok[4];
    double s[4], mx[4], mo[4];
    int bad[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        ids[m] = id0 + w + 8 * m;
        live[m] = ids[m] < hi;
        int level = 0;
        ops[m] = -1; oa[m] = 0; ob[m] = -1;
        opok[m] = false;
        if (live[m] && decode(sp, ids[m], level, ops[m], oa[m], ob[m]) && ops[m] >= 0)
            opok[m] = valid_lvl(T, oa[m]) && (ob[m] < 0 || valid_lvl(T, ob[m]));
        else { ops[m] = -1; oa[m] = 0; ob[m] = -1; }
        s[m] = 0.0; mx[m] = 0.0; mo[m] = 0.0; bad[m] = 0;
    }
    for (int s0 = 0; s0 < N; s0 += 32) {
        const int i = s0 + lane;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float f = 0.f;
            if (live[m] && i < N && ops[m] < 0) T.V[(size_t)ids[m] * T.ldv + i] = 0.0;
            if (live[m] && i < N && ops[m] >= 0) {
                const double x = T.V[(size_t)oa[m] * T.ldv + i];
                double v, mag;
                if (ob[m] < 0) { v = op_unary<double>(ops[m], x); mag = fabs(v); }
                else {
                    const double yv = T.V[(size_t)ob[m] * T.ldv + i];
                    v = op_binary<double>(ops[m], x, yv);
                    mag = (ops[m] == ADD || ops[m] == SUB) ? fabs(x) + fabs(yv) : fabs(v);
                }
                T.V[(size_t)ids[m] * T.ldv + i] = v;
                if (!isfinite(v) || fabs(v) > kValueCap) bad[m] = 1;
                s[m] += v;
                mx[m] = fmax(mx[m], fabs(v));
                mo[m] = fmax(mo[m], mag);
                f = (float)v;
            }
            tile[w + 8 * m][lane] = f;
        }
        __syncthreads();
        // transpose: warp w writes samples s0 + w + 8 r, lanes over the 32 ids
        for (int r = w; r < 32; r += 8) {
            const int si = s0 + r;
            const int64_t id = id0 + lane;
            if (si < N && id < hi) T.cache[(size_t)si * T.P + id] = tile[lane][r];
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int b = warp_or(bad[m]);
        const double sm = warp_sum(s[m]);
        const double mxm = warp_max(mx[m]);
        const double mom = warp_max(mo[m]);
        const double mean = sm / N;
        double ss = 0.0;
        if (live[m] && !b)
            for (int i = lane; i < N; i += 32) { const double u = T.V[(size_t)ids[m] * T.ldv + i] - mean; ss += u * u; }
        ss = warp_sum(ss);
        if (lane == 0 && live[m]) {
            const bool cancelled = (ops[m] == ADD || ops[m] == SUB) && mxm <= kCancelRel * mom;
            T.vlvl[l][ids[m] - lo] = opok[m] && !b && !cancelled && sqrt(ss / N) > kConstRel * mxm;
        }
    }
}

// after the last level: validity of [0, P) as one array
__device__ __noinline__ void run_flat(const BTask& T) {
    for (int64_t id = threadIdx.x; id < T.P; id += kBT) T.valid[id] = valid_lvl(T, id);
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// OPSUM: per-operand sums for the pair tiles' + and - (256 operands per item), FP32 runs of
// 32 samples accumulated in FP64
// ---------------------------------------------------------------------------------
__device__ __noinline__ void run_opsum(const BatchArgs& B, int task, int t, long long q) {
    const BTask& T = B.tasks[task];
    const BDim& D = T.dim[t];
    const int64_t f = q * kBT + threadIdx.x;
    if (f >= T.P) return;
    const float x0 = T.cache[f];
    const int N = T.N;
    double a = 0.0, ar = 0.0;
    for (int s0 = 0; s0 < N; s0 += 32) {
        const int e = s0 + 32 < N ? s0 + 32 : N;
        float pa = 0.f, pr = 0.f;
        for (int sidx = s0; sidx < e; ++sidx) {
            const float v = T.cache[(size_t)sidx * T.P + f] - x0;
            pa += v;
            pr = fmaf(v, D.tc32[sidx], pr);
        }
        a += (double)pa;
        ar += (double)pr;
    }
    if (t == 1) T.A1[f] = a;
    D.AR[f] = ar;
}

// ---------------------------------------------------------------------------------
// SCORE: units [u0, u1) of step t
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void run_score(const BatchArgs& B, int task, int t, long long q, unsigned char* smem) {
    const BTask& T = B.tasks[task];
    const BDim& D = T.dim[t];
    const int64_t u0 = q * B.score_units;
    const int64_t u1 = min((int64_t)T.n_units, u0 + B.score_units);
    for (int64_t u = u0; u < u1; ++u) {
        if (u < T.n_low) {
            const int64_t id = u * kLowIds + threadIdx.x;
            if (id < T.P) score_cached_id<float>(T.cache, T.N, T.P, D.tc32, D.tc64, D.ts, id, T.valid, D.scores);
        } else if (u < T.n_low + T.n_un) {
            UnarySmem& U = *reinterpret_cast<UnarySmem*>(smem);
            __syncthreads();
            unary_block<float>(T.ua, T.cache, D.tc32, D.tc64, D.ts, T.valid, D.scores, u - T.n_low, U.xs, U.r);
            __syncthreads();
        } else {
            PairArgs A = T.pa;
            A.scores = D.scores;
            const int2 tl = T.tiles[u - T.n_low - T.n_un];
            pair_tile<float, true>(A, nullptr, D.tc32, D.tc64, D.ts, T.valid, T.cache, T.A1, D.AR,
                                    *reinterpret_cast<PairSmem<float>*>(smem), tl.x, tl.y);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------------
// SELECT: window, FP64 re-score, sort, walk (one CTA)
// ---------------------------------------------------------------------------------

// the bin holding the need-th largest key of a 4096- (or 256-) bin histogram: returns
// the bin and the rank still needed inside it; bin -1 when fewer keys exist
__device__ void hist_find(SelectSmem& M, Ctl& C, int nb, unsigned need) {
    const int per = nb / kBT > 0 ? nb / kBT : 1;
    const int tid = threadIdx.x;
    unsigned p = 0;
    if (tid * per < nb)
        for (int b = 0; b < per; ++b) p += M.u.hist[tid * per + b];
    M.part[tid] = p;
    __syncthreads();
    if (tid == 0) {
        unsigned cum = 0;
        int bin = -1;
        unsigned rest = 0;
        const int nparts = nb / per;
        for (int g = nparts - 1; g >= 0 && bin < 0; --g) {
            const unsigned c = M.part[g];
            if (cum + c >= need) {
                for (int b = g * per + per - 1; b >= g * per; --b) {
                    const unsigned cb = M.u.hist[b];
                    if (cum + cb >= need) { bin = b; rest = need - cum; break; }
                    cum += cb;
                }
            } else {
                cum += c;
            }
        }
        C.ival[0] = bin;
        C.ival[1] = (int)rest;
    }
    __syncthreads();
}

// radix select over the step's scores: C.ukey = key of the M-th best; C.flag = 1 when fewer
// than M keys are nonzero (then every nonzero key is taken).  Keys are the float bits of
// positive scores, capped below 2.0, so bits 31-30 are zero: three passes of 10 bits, with
// per-warp histograms and vector loads (the scan is one CTA's, so it must keep many loads
// in flight).
__device__ __forceinline__ unsigned rkey(float s) {
    const unsigned k = s > 0.f ? __float_as_uint(s) : 0u;
    return k < 0x3FFFFFFFu ? k : 0x3FFFFFFFu;
}

template <typename F>
__device__ __forceinline__ void scan_keys(const float* scores, int64_t n, F f) {
    const int64_t n4 = n >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(scores);
    int64_t v = threadIdx.x;
    for (; v + kBT < n4; v += 2 * kBT) {
        const float4 a = __ldcg(s4 + v), b = __ldcg(s4 + v + kBT);
        f(rkey(a.x)); f(rkey(a.y)); f(rkey(a.z)); f(rkey(a.w));
        f(rkey(b.x)); f(rkey(b.y)); f(rkey(b.z)); f(rkey(b.w));
    }
    for (; v < n4; v += kBT) {
        const float4 a = __ldcg(s4 + v);
        f(rkey(a.x)); f(rkey(a.y)); f(rkey(a.z)); f(rkey(a.w));
    }
    for (int64_t i = (n4 << 2) + threadIdx.x; i < n; i += kBT) f(rkey(__ldcg(scores + i)));
}

__device__ void radix_select(SelectSmem& M, Ctl& C, const float* scores, int64_t n, unsigned Mw) {
    unsigned prefix = 0, need = Mw;
    int all = 0;
    const int w = threadIdx.x >> 5;
    unsigned* hw = M.u.hist + w * 1024;               // this warp's histogram
    for (int pass = 0; pass < 3 && !all; ++pass) {
        for (int i = threadIdx.x; i < 8 * 1024; i += kBT) M.u.hist[i] = 0;
        __syncthreads();
        const int sh = 20 - 10 * pass;
        const unsigned pre = prefix;
        scan_keys(scores, n, [&](unsigned k) {
            if (k != 0u && (pass == 0 || (k >> (sh + 10)) == pre)) atomicAdd(&hw[(k >> sh) & 0x3FFu], 1u);
        });
        __syncthreads();
        for (int b = threadIdx.x; b < 1024; b += kBT) {
            unsigned t = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) t += M.u.hist[q * 1024 + b];
            M.u.hist[b] = t;
        }
        __syncthreads();
        hist_find(M, C, 1024, need);
        const int bin = C.ival[0];
        if (bin < 0) { all = 1; break; }
        prefix = (prefix << 10) | (unsigned)bin;
        need = (unsigned)C.ival[1];
        __syncthreads();
    }
    if (threadIdx.x == 0) { C.ukey = all ? 1u : prefix; C.flag = all; }
    __syncthreads();
}

__device__ __forceinline__ bool before(double sa, int64_t ia, double sb, int64_t ib) {
    return sa > sb || (sa == sb && ia < ib);
}

// block bitonic sort of n_pad (power of two) entries by (score desc, id asc)
__device__ void block_sort(SelectSmem& M, int n_pad) {
    for (int kk = 2; kk <= n_pad; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pad; i += kBT) {
                const int l = i ^ j;
                if (l <= i) continue;
                const bool up = (i & kk) == 0;
                const double si = M.u.srt.sk[i], sl = M.u.srt.sk[l];
                const int64_t ii = M.u.srt.sid[i], il = M.u.srt.sid[l];
                if (up ? before(sl, il, si, ii) : before(si, ii, sl, il)) {
                    M.u.srt.sk[i] = sl; M.u.srt.sk[l] = si;
                    M.u.srt.sid[i] = il; M.u.srt.sid[l] = ii;
                    const int x = M.u.srt.ssrc[i]; M.u.srt.ssrc[i] = M.u.srt.ssrc[l]; M.u.srt.ssrc[l] = x;
                }
            }
            __syncthreads();
        }
}

// standardised row of window entry e into Z row r (two passes, as the per-problem path)
__device__ void standardise_into(const BTask& T, Ctl& C, const OpRef& ref, double* z, double& mean, double& sd) {
    const int N = T.N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) {
        double mg;
        const double v = opref_val(ref, T.V, T.ldv, i, mg);
        z[i] = v;
        s += v;
    }
    const double m = block_sum(s, C.red) / N;
    double ss = 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) { const double u = z[i] - m; ss += u * u; }
    const double sdv = sqrt(block_sum(ss, C.red) / N);
    const double inv = sdv > 0.0 ? 1.0 / sdv : 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) z[i] = (z[i] - m) * inv;
    mean = m;
    sd = sdv;
    __syncthreads();
}

// the same from a row of values already computed (two passes, as the per-problem path)
__device__ void standardise_from(const BTask& T, Ctl& C, const double* raw, double* z, double& mean, double& sd) {
    const int N = T.N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) s += raw[i];
    const double m = block_sum(s, C.red) / N;
    double ss = 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) { const double u = raw[i] - m; ss += u * u; }
    const double sdv = sqrt(block_sum(ss, C.red) / N);
    const double inv = sdv > 0.0 ? 1.0 / sdv : 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) z[i] = (raw[i] - m) * inv;
    mean = m;
    sd = sdv;
    __syncthreads();
}

// returns SISSO_OK, or an error status for the task
__device__ __noinline__ int run_select(const BatchArgs& B, Ctl& C, int task, int t, unsigned char* smem) {
    const BTask& T = B.tasks[task];
    BState& St = B.state[task];
    const BDim& D = T.dim[t];
    SelectSmem& M = *reinterpret_cast<SelectSmem*>(smem);
    const int N = T.N, w = threadIdx.x >> 5, tid = threadIdx.x;
    const int n_prev = t > 1 ? ldcg_i(&St.n_S[t - 1]) : 0;
    const int64_t* gprev = t > 1 ? T.dim[t - 1].gid : nullptr;
    const int k = B.k;
    // S, ascending, for the membership test; previous members carried into this step's lists
    for (int i = tid; i < n_prev; i += kBT) {
        M.S_sorted[i] = gprev[i];
        D.gid[i] = gprev[i];
        D.zmean[i] = T.dim[t - 1].zmean[i];
        D.zsd[i] = T.dim[t - 1].zsd[i];
    }
    __syncthreads();
    if (tid == 0)
        for (int a = 1; a < n_prev; ++a)
            for (int c = a; c > 0 && M.S_sorted[c - 1] > M.S_sorted[c]; --c) {
                const int64_t x = M.S_sorted[c]; M.S_sorted[c] = M.S_sorted[c - 1]; M.S_sorted[c - 1] = x;
            }
    __syncthreads();
    int Mw = B.win0 < k ? k : B.win0;
    if (Mw > kWinMax) Mw = kWinMax;
    int n_acc = 0;
    while (true) {
        unsigned long long ts0 = gtimer();
        radix_select(M, C, D.scores, T.n_feat, (unsigned)Mw);
        const unsigned thr = (unsigned)C.ukey;
        const int all = C.flag;
        float t32 = 0.f;
        if (!all) t32 = __uint_as_float(thr);
        // compact the window
        if (tid == 0) C.n = 0;
        __syncthreads();
        for (int64_t i = tid; i < T.n_feat; i += kBT) {
            const unsigned kk = rkey(__ldcg(D.scores + i));
            if (kk != 0u && kk >= thr) {
                const int slot = atomicAdd(&C.n, 1);
                if (slot < kWinMax) D.w_ids[slot] = i;
            }
        }
        __syncthreads();
        const int ns = C.n;
        if (ns > kWinMax) return SISSO_ERR_CAPACITY;    // tied scores overflow the window
        unsigned long long ts1 = gtimer();
        if (tid == 0) prof_add(B.prof, PS_SEL_RADIX, ts1 - ts0);
        // FP64 re-score, one warp per entry
        for (int e = w; e < ns; e += kBT / 32)
            rescore_one(T.sp, nullptr, N, T.ldv, D.tc64, D.ts, D.w_ids[e], e, T.valid, T.V, D.w_score, D.w_mean,
                        D.w_sd, D.w_valid, D.w_probe, e < kZRaw ? T.zraw : nullptr, true);
        __syncthreads();
        ts0 = gtimer();
        if (tid == 0) prof_add(B.prof, PS_SEL_RESCORE, ts0 - ts1);
        int n_pad = 1;
        while (n_pad < (ns > 0 ? ns : 1)) n_pad <<= 1;
        for (int i = tid; i < n_pad; i += kBT) {
            if (i >= ns) { M.u.srt.sk[i] = -2.0; M.u.srt.sid[i] = INT64_MAX; M.u.srt.ssrc[i] = -1; }
            else {
                const int64_t id = D.w_ids[i];
                int lo = 0, hi = n_prev;
                while (lo < hi) { const int m = (lo + hi) >> 1; if (M.S_sorted[m] < id) lo = m + 1; else hi = m; }
                const bool inS = lo < n_prev && M.S_sorted[lo] == id;
                M.u.srt.sk[i] = (D.w_valid[i] && !inS) ? D.w_score[i] : -1.0;
                M.u.srt.sid[i] = id;
                M.u.srt.ssrc[i] = i;
            }
            M.removed[i] = 0;
        }
        __syncthreads();
        block_sort(M, n_pad);
        ts1 = gtimer();
        if (tid == 0) prof_add(B.prof, PS_SEL_SORT, ts1 - ts0);
        // the walk
        if (tid == 0) { C.n_acc = 0; C.done = 0; C.visited = 0; C.dval[0] = -1.0; C.ival[2] = 0; }
        __syncthreads();
        int p = 0;                                    // thread 0: first entry not yet visited
        while (true) {
            if (tid == 0) {
                while (p < n_pad && M.removed[p]) ++p;
                if (C.n_acc >= k || p >= n_pad || M.u.srt.sk[p] < 0.0) {
                    C.done = 1;
                } else {
                    // among the entries within kScoreTie of the maximum, the lowest id
                    const double mxs = M.u.srt.sk[p];
                    int best = p;
                    for (int e = p + 1; e < n_pad && M.u.srt.sk[e] >= 0.0 && M.u.srt.sk[e] >= mxs - kScoreTie; ++e)
                        if (!M.removed[e] && M.u.srt.sid[e] < M.u.srt.sid[best]) best = e;
                    M.removed[best] = 1;
                    C.cur = best;
                    C.dval[0] = M.u.srt.sk[best];
                    ++C.visited;
                }
                C.n_match = 0;
            }
            __syncthreads();
            if (C.done) break;
            const int row = n_prev + C.n_acc;         // Z row the candidate takes if accepted
            const int src = M.u.srt.ssrc[C.cur];
            // probe test (a necessary condition) against every S member and every id accepted
            // in this step, with the candidate's probes from the re-score
            const double* pc = D.w_probe + (size_t)src * kProbes;
            for (int r = tid; r < row; r += kBT) {
                const double* zr = T.Z + (size_t)r * T.ldv;
                bool same = true, flip = true;
#pragma unroll
                for (int q = 0; q < kProbes; ++q) {
                    const double zq = zr[(int)(((int64_t)q * N) / kProbes)];
                    same = same && fabs(pc[q] - zq) <= kDupTol;
                    flip = flip && fabs(pc[q] + zq) <= kDupTol;
                }
                if (same || flip) C.match[atomicAdd(&C.n_match, 1)] = r;
            }
            __syncthreads();
            const int nm = C.n_match;
            const double* raw = src < kZRaw ? T.zraw + (size_t)src * N : nullptr;
            OpRef ref{};
            if (!raw) make_opref(*T.sp, M.u.srt.sid[C.cur], ref);
            bool dup = false;
            if (tid == 0) { St.visits += 1; St.checks += nm; }
            if (nm > 0) {
                // full comparison on every sample, the candidate standardised by its re-score moments
                const double mc = D.w_mean[src], dc = D.w_sd[src];
                for (int q = 0; q < nm && !dup; ++q) {
                    const double* zr = T.Z + (size_t)C.match[q] * T.ldv;
                    double e1 = 0.0, e2 = 0.0;
                    for (int i = tid; i < N; i += kBT) {
                        double mg;
                        const double zc = ((raw ? raw[i] : opref_val(ref, T.V, T.ldv, i, mg)) - mc) / dc;
                        e1 = fmax(e1, fabs(zc - zr[i]));
                        e2 = fmax(e2, fabs(zc + zr[i]));
                    }
                    e1 = block_max(e1, C.red);
                    e2 = block_max(e2, C.red);
                    dup = e1 <= kDupTol || e2 <= kDupTol;
                }
            }
            double zm = 0.0, zs = 0.0;
            if (!dup) {
                double* z = T.Z + (size_t)row * T.ldv;
                if (raw) standardise_from(T, C, raw, z, zm, zs);
                else standardise_into(T, C, ref, z, zm, zs);
            }
            if (tid == 0 && !dup) {
                D.gid[row] = M.u.srt.sid[C.cur];
                D.zmean[row] = zm;
                D.zsd[row] = zs;
                ++C.n_acc;
            }
            __syncthreads();
        }
        if (tid == 0) prof_add(B.prof, PS_SEL_WALK, gtimer() - ts1);
        n_acc = C.n_acc;
        const double last = C.dval[0];
        // exact iff every candidate outside the window scores below the last visited one by
        // more than the tie tolerance (FP32 scores within kScoreErr32 of FP64)
        const bool safe = all || (n_acc == k && last - kScoreTie > (double)t32 + kScoreErr32);
        if (safe || Mw >= kWinMax) {
            if (!safe && tid == 0) St.saturated = 1;
            break;
        }
        Mw = Mw * 4 > kWinMax ? kWinMax : Mw * 4;
        if (tid == 0) St.grown += 1;
        __syncthreads();
    }
    if (tid == 0) St.n_S[t] = n_prev + n_acc;
    __syncthreads();
    return SISSO_OK;
}

// ---------------------------------------------------------------------------------
// GRAM: new rows [r0, r1) of step t; row i < n_old copies of the previous step's block
// ---------------------------------------------------------------------------------
__device__ __noinline__ void run_gram(const BatchArgs& B, int task, int t, long long q) {
    const BTask& T = B.tasks[task];
    BState& St = B.state[task];
    const BDim& D = T.dim[t];
    const int n = ldcg_i(&St.n_S[t]);
    const int n_old = t > 1 ? ldcg_i(&St.n_S[t - 1]) : 0;
    const int n_new = n - n_old;
    const int items = n_new > 0 ? (n_new + B.gram_rows - 1) / B.gram_rows : 1;
    const int N = T.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // copy of the previous block, rows split among the items
    if (n_old > 0) {
        const BDim& P = T.dim[t - 1];
        const int c0 = (int)((int64_t)n_old * q / items), c1 = (int)((int64_t)n_old * (q + 1) / items);
        for (int e = threadIdx.x; e < (c1 - c0) * n_old; e += kBT) {
            const int i = c0 + e / n_old, j = e % n_old;
            D.G64[(size_t)i * n + j] = P.G64[(size_t)i * n_old + j];
            D.G32[(size_t)i * n + j] = P.G32[(size_t)i * n_old + j];
        }
        for (int i = c0 + threadIdx.x; i < c1; i += kBT) { D.b64[i] = P.b64[i]; D.b32[i] = P.b32[i]; }
    }
    const int r0 = n_old + (int)q * B.gram_rows, r1 = min(n, r0 + B.gram_rows);
    // entries (i, j) with i new and j < n_old or n_old <= j <= i, and the moment b_i
    for (int i = r0; i < r1; ++i) {
        const double* zi = T.Z + (size_t)i * T.ldv;
        for (int j = w; j <= i + 1; j += kBT / 32) {
            const int jj = j <= i ? j : n;            // j = i + 1 stands for the moment column
            const double* zj = jj < n ? T.Z + (size_t)jj * T.ldv : T.yc;
            double s = 0.0;
            for (int u = lane; u < N; u += 32) s += zi[u] * zj[u];
            s = warp_sum(s) / N;
            if (lane == 0) {
                if (jj < n) {
                    D.G64[(size_t)i * n + jj] = s;
                    D.G64[(size_t)jj * n + i] = s;
                    D.G32[(size_t)i * n + jj] = (float)s;
                    D.G32[(size_t)jj * n + i] = (float)s;
                } else {
                    D.b64[i] = s;
                    D.b32[i] = (float)s;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// BOUND / BAND: l0 enumeration items [e0, e1) of step t
// ---------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t binom_hd(int64_t n, int k) {
    if (k < 0 || n < k) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

__device__ __forceinline__ int enum_cpp(int n, int D) {
    const int DP = D - 2;
    const int c = (n - 1 - DP + kRows - 1) / kRows;
    return c > 1 ? c : 1;
}

// enumeration items of step t: D = t >= 2: prefixes x chunks; D = 1: blocks of 256 features
__device__ __forceinline__ int64_t enum_total(int n, int D) {
    if (D == 1) return (n + kBT - 1) / kBT;
    return binom_hd(n - 2, D - 2) * enum_cpp(n, D);
}

__device__ EnumArgs<float> enum_args(const BatchArgs& B, int task, int t, int n) {
    const BTask& T = B.tasks[task];
    BState& St = B.state[task];
    const BDim& D = T.dim[t];
    const double syy = ldcg_d(&St.syy);
    EnumArgs<float> A{};
    A.G = D.G32; A.b = D.b32; A.ld = n; A.n = n; A.N = T.N; A.syy = (float)syy; A.sst = syy * T.N;
    A.cpp = t >= 2 ? enum_cpp(n, t) : 1;
    A.n_items = enum_total(n, t);
    A.counter = nullptr;
    A.tau = kPivotMin32; A.fp32 = 1; A.sqrt_syy = sqrt(syy);
    A.ub_key = &St.ub_key[t]; A.win = nullptr; A.band = D.band; A.band_count = &St.band_count[t];
    A.band_cap = B.band_cap; A.examined = &St.examined[t]; A.band_r32 = nullptr;
    A.G64 = D.G64; A.b64 = D.b64; A.syy64 = syy; A.tie64 = 2.0 * kRssTie * A.sst;
    return A;
}

template <int DP, int MODE>
__device__ void enum_range(const EnumArgs<float>& A, Ctl& C, float* tabs, int64_t e0, int64_t e1, double thr) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tab = tabs + (size_t)w * (DP + 2) * A.n;
    float best = INFINITY;
    unsigned long long best_key = 0;
    unsigned long long ex = 0;
    if (threadIdx.x == 0) C.n = 0;
    __syncthreads();
    while (true) {
        int it;
        if (lane == 0) it = atomicAdd(&C.n, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        const int64_t item = e0 + it;
        if (item >= e1) break;
        enum_item<float, DP, MODE>(A, tab, item, best, best_key, thr, ex);
    }
    if (MODE == 0) enum_flush(A, DP + 2, best, best_key, ex);
    __syncthreads();
}

__device__ __noinline__ void run_enum(const BatchArgs& B, Ctl& C, int task, int t, long long q, int mode, unsigned char* smem) {
    BState& St = B.state[task];
    const int n = ldcg_i(&St.n_S[t]);
    const EnumArgs<float> A = enum_args(B, task, t, n);
    const int64_t e0 = q * B.enum_items;
    const int64_t e1 = min(A.n_items, e0 + B.enum_items);
    const double thr = mode == 1 ? ldcg_d(&St.thr[t]) : 0.0;
    float* tabs = reinterpret_cast<float*>(smem);
    if (t == 1) {
        for (int64_t e = e0; e < e1; ++e) {
            const int i0 = (int)(e * kBT), i1 = min(n, i0 + kBT);
            const int i = i0 + threadIdx.x;
            if (i < i1) {
                if (mode == 0) single_subset<float, 0>(A, i, 0.0); else single_subset<float, 1>(A, i, thr);
            }
        }
        __syncthreads();
        return;
    }
    switch ((t - 2) * 2 + mode) {
        case 0: enum_range<0, 0>(A, C, tabs, e0, e1, thr); break;
        case 1: enum_range<0, 1>(A, C, tabs, e0, e1, thr); break;
        case 2: enum_range<1, 0>(A, C, tabs, e0, e1, thr); break;
        case 3: enum_range<1, 1>(A, C, tabs, e0, e1, thr); break;
        case 4: enum_range<2, 0>(A, C, tabs, e0, e1, thr); break;
        default: enum_range<2, 1>(A, C, tabs, e0, e1, thr); break;
    }
}

// ---------------------------------------------------------------------------------
// REFIT: FP64 refit of the band, winner, model; next target
// ---------------------------------------------------------------------------------
__device__ __noinline__ int run_refit(const BatchArgs& B, Ctl& C, int task, int t, unsigned char* smem) {
    const BTask& T = B.tasks[task];
    BState& St = B.state[task];
    const BDim& D = T.dim[t];
    const int n = ldcg_i(&St.n_S[t]);
    const int N = T.N, tid = threadIdx.x;
    const double syy = ldcg_d(&St.syy), ybar = ldcg_d(&St.ybar);
    const double sst = syy * N;
    const unsigned cnt = atomicAdd(&St.band_count[t], 0u);
    if ((int64_t)cnt > B.band_cap) return SISSO_ERR_CAPACITY;
    // FP64 RSS of every band entry and the minimum
    double local = INFINITY;
    for (unsigned e = tid; e < cnt; e += kBT) {
        int pos[kMaxDim];
        unpack(D.band[e], t, pos);
        const double r = rss64(D.G64, D.b64, n, syy, N, t, pos, nullptr);
        D.band_rss[e] = r;
        local = fmin(local, r);
    }
    const double mn = -block_max(-local, C.red);
    if (!(mn < INFINITY)) return SISSO_ERR_NUMERIC;     // every subset singular
    // within the tie window: the smallest ascending global-id tuple
    int64_t bt[kMaxDim];
    int be = -1;
    for (unsigned e = tid; e < cnt; e += kBT) {
        if (!(D.band_rss[e] <= mn + kRssTie * sst)) continue;
        int pos[kMaxDim];
        int64_t tu[kMaxDim];
        unpack(D.band[e], t, pos);
        gid_tuple(D.gid, pos, t, tu);
        if (be < 0 || tuple_less(tu, bt, t)) { be = (int)e; for (int j = 0; j < t; ++j) bt[j] = tu[j]; }
    }
    int* cand = reinterpret_cast<int*>(smem);
    cand[tid] = be;
    __syncthreads();
    if (tid == 0) {
        int wbest = -1;
        int64_t wt[kMaxDim];
        for (int q = 0; q < kBT; ++q) {
            const int e = cand[q];
            if (e < 0) continue;
            int pos[kMaxDim];
            int64_t tu[kMaxDim];
            unpack(D.band[e], t, pos);
            gid_tuple(D.gid, pos, t, tu);
            if (wbest < 0 || tuple_less(tu, wt, t)) { wbest = e; for (int j = 0; j < t; ++j) wt[j] = tu[j]; }
        }
        C.ival[3] = wbest;
        if (wbest >= 0) {
            int pos[kMaxDim];
            unpack(D.band[wbest], t, pos);
            for (int j = 0; j < t; ++j) C.ival[4 + j] = pos[j];
            rss64(D.G64, D.b64, n, syy, N, t, pos, C.dval);   // gamma in dval[0..t)
        }
    }
    __syncthreads();
    if (C.ival[3] < 0) return SISSO_ERR_NUMERIC;
    int pos[kMaxDim];
    double gamma[kMaxDim];
    for (int j = 0; j < t; ++j) { pos[j] = C.ival[4 + j]; gamma[j] = C.dval[j]; }
    // residual r* = y~ - Z_E gamma, RSS
    double s = 0.0;
    for (int i = tid; i < N; i += kBT) {
        double f = T.yc[i];
        for (int j = 0; j < t; ++j) f -= gamma[j] * T.Z[(size_t)pos[j] * T.ldv + i];
        D.resid[i] = f;
        s += f * f;
    }
    const double rss = block_sum(s, C.red);
    if (tid == 0) {
        int order[kMaxDim];
        for (int j = 0; j < t; ++j) order[j] = j;
        for (int a = 1; a < t; ++a)
            for (int c = a; c > 0 && D.gid[pos[order[c - 1]]] > D.gid[pos[order[c]]]; --c) {
                const int x = order[c]; order[c] = order[c - 1]; order[c - 1] = x;
            }
        sisso_task_result& R = B.res[task];
        double c0 = ybar;
        for (int j = 0; j < t; ++j) {
            const int qj = order[j], p = pos[qj];
            const double cj = gamma[qj] / D.zsd[p];
            R.ids[t - 1][j] = D.gid[p];
            R.coef[t - 1][j + 1] = cj;
            c0 -= cj * D.zmean[p];
        }
        R.coef[t - 1][0] = c0;
        R.rmse[t - 1] = sqrt(rss / N);
        R.r2[t - 1] = 1.0 - rss / (syy * N);
        St.n_dims = t;
        C.flag = sqrt(rss / N) <= kStopRel * sqrt(syy);
    }
    __syncthreads();
    return SISSO_OK;
}

// ---------------------------------------------------------------------------------
// stage transitions
// ---------------------------------------------------------------------------------
enum : int { NX_LEVEL = 0, NX_SCORE, NX_SELECT, NX_BOUND, NX_BAND, NX_REFIT, NX_OPSUM };

// Run serial stages from `next` on and queue the next parallel stage (or finish the task).
__device__ void advance(const BatchArgs& B, Ctl& C, int task, int next, int t, unsigned char* smem) {
    const BTask& T = B.tasks[task];
    BState& St = B.state[task];
    while (true) {
        if (next == NX_LEVEL) {                          // t = level
            if (t < T.rung) {
                const int nu = T.lvl_first[t + 1] - T.lvl_first[t];
                if (nu > 0) { push(B, C, task, WK_LEVEL, t, nu); return; }
                ++t;
                continue;
            }
            const unsigned long long f0 = gtimer();
            run_flat(T);
            if (threadIdx.x == 0) prof_add(B.prof, PS_FLAT, gtimer() - f0);
            next = NX_OPSUM;
            t = 1;
            continue;
        }
        if (next == NX_OPSUM) {
            if (T.n_tiles > 0) { push(B, C, task, WK_OPSUM, t, (T.P + kBT - 1) / kBT); return; }
            next = NX_SCORE;
            continue;
        }
        if (next == NX_SCORE) {
            push(B, C, task, WK_SCORE, t, (T.n_units + B.score_units - 1) / B.score_units);
            return;
        }
        if (next == NX_SELECT) {
            const unsigned long long s0 = gtimer();
            const int st = run_select(B, C, task, t, smem);
            if (threadIdx.x == 0) prof_add(B.prof, PS_SELECT, gtimer() - s0);
            if (st != SISSO_OK) { finish(B, task, st); return; }
            const int n = ldcg_i(&St.n_S[t]);
            if (n < t) { finish(B, task, t == 1 ? SISSO_ERR_NUMERIC : SISSO_OK); return; }
            const int n_new = n - (t > 1 ? ldcg_i(&St.n_S[t - 1]) : 0);
            // (nothing new: one item copies the previous step's Gram)
            push(B, C, task, WK_GRAM, t, n_new > 0 ? (n_new + B.gram_rows - 1) / B.gram_rows : 1);
            return;
        }
        if (next == NX_BOUND) {
            const int n = ldcg_i(&St.n_S[t]);
            const int64_t tot = enum_total(n, t);
            push(B, C, task, WK_BOUND, t, (tot + B.enum_items - 1) / B.enum_items);
            return;
        }
        if (next == NX_BAND) {
            if (threadIdx.x == 0) {
                const unsigned long long kk = atomicAdd(&St.ub_key[t], 0ull);
                St.thr[t] = okey_inv(kk);
            }
            const int n = ldcg_i(&St.n_S[t]);
            const int64_t tot = enum_total(n, t);
            push(B, C, task, WK_BAND, t, (tot + B.enum_items - 1) / B.enum_items);
            return;
        }
        // NX_REFIT
        const unsigned long long r0 = gtimer();
        const int st = run_refit(B, C, task, t, smem);
        if (threadIdx.x == 0) prof_add(B.prof, PS_REFIT, gtimer() - r0);
        if (st != SISSO_OK) { finish(B, task, st); return; }
        if (C.flag || t >= B.max_dim) { finish(B, task, SISSO_OK); return; }
        const BDim& Dn = T.dim[t + 1];
        prepare_target_block(T.dim[t].resid, T.N, Dn.tc64, Dn.tc32, Dn.ts, C.red);
        __syncthreads();
        next = NX_OPSUM;
        ++t;
    }
}

// MINB resident CTAs per SM: 2 (registers capped at 128) or 1 (the pair tile unspilled)
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB) k_batch(BatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Ctl C;
    if (threadIdx.x == 0) atomicMin(B.t0, gtimer());
    while (true) {
        if (threadIdx.x == 0) {
            const unsigned long long a0 = gtimer();
            C.item = acquire(B);
            prof_add(B.prof, PS_IDLE, gtimer() - a0);
        }
        __syncthreads();
        const unsigned long long it = C.item;
        __syncthreads();
        if (it == kExit) break;
        const int kind = item_kind(it), t = item_t(it), task = item_task(it);
        const long long q = item_q(it);
        const unsigned long long i0 = gtimer();
        if (kind == WK_START) {
            run_start(B, C, task);
            if (threadIdx.x == 0) prof_add(B.prof, WK_START, gtimer() - i0);
            advance(B, C, task, NX_LEVEL, 1, smem);
            continue;
        }
        if (ldcg_i(&B.state[task].status) == SISSO_OK) {
            if (kind == WK_LEVEL) run_level(B, C, task, t, q, reinterpret_cast<float (*)[33]>(smem));
            else if (kind == WK_SCORE) run_score(B, task, t, q, smem);
            else if (kind == WK_OPSUM) run_opsum(B, task, t, q);
            else if (kind == WK_GRAM) run_gram(B, task, t, q);
            else run_enum(B, C, task, t, q, kind == WK_BAND, smem);
        }
        // stage completion: the CTA finishing the last item moves the task on
        __syncthreads();
        if (threadIdx.x == 0) prof_add(B.prof, kind, gtimer() - i0);
        if (threadIdx.x == 0) {
            __threadfence();
            const int left = atomicSub(&B.state[task].pending, 1) - 1;
            if (left == 0) __threadfence();
            C.flag = left == 0;
        }
        __syncthreads();
        if (!C.flag) continue;
        if (kind == WK_LEVEL) advance(B, C, task, NX_LEVEL, t + 1, smem);
        else if (kind == WK_SCORE) advance(B, C, task, NX_SELECT, t, smem);
        else if (kind == WK_OPSUM) advance(B, C, task, NX_SCORE, t, smem);
        else if (kind == WK_GRAM) advance(B, C, task, NX_BOUND, t, smem);
        else if (kind == WK_BOUND) advance(B, C, task, NX_BAND, t, smem);
        else advance(B, C, task, NX_REFIT, t, smem);
    }
}

}  // namespace
}  // namespace sg

// ===================================================================================
// host side
// ===================================================================================

struct sisso_batch {
    int n_tasks = 0, rung = 0, k = 0, max_dim = 0, grammar = 0;
    unsigned long long idle_ns = 0;     // work-queue no-progress limit (0: the default)
    uint32_t ops = 0;
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int band_cap = 0;
    // device memory
    void* arena = nullptr;
    size_t arena_bytes = 0;
    sg::Space* plans = nullptr;
    sg::BTask* tasks_dev = nullptr;
    sg::BState* state = nullptr;
    sisso_task_result* res_dev = nullptr;
    int* order_dev = nullptr;
    int2* tiles_dev = nullptr;
    unsigned long long* slots = nullptr;
    long long cap = 0;
    int* ctr = nullptr;
    unsigned long long* t0 = nullptr;
    unsigned long long* prof = nullptr;
    double* in_dev = nullptr;
    size_t in_count = 0;
    // pinned host memory
    double* in_host = nullptr;
    sisso_task_result* res_host = nullptr;
    sg::BState* state_host = nullptr;
    int* ctr_host = nullptr;
    unsigned long long* t0_host = nullptr;
    unsigned long long* prof_host = nullptr;
    // plan
    std::vector<int> Ns, ds;
    std::vector<size_t> in_off;        // offset (doubles) of each task's X; y follows X
    std::vector<sg::BTask> th;
    std::vector<int64_t> n_feat;
    sisso_batch_tune tune{};
    cudaGraphExec_t g_dev = nullptr, g_e2e = nullptr;
    sisso_batch_stats stats{};
    bool ran = false;
    bool fetched = false;
};

namespace sg {
namespace {

std::string g_batch_create_err;
std::mutex g_batch_err_mu;

sisso_status bfail(sisso_batch* b, sisso_status st, const std::string& msg) {
    b->err = msg;
    return st;
}
sisso_status bcuda(sisso_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SISSO_OK;
    cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? SISSO_ERR_OOM : SISSO_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// LEVEL units of one task and SCORE units
struct TaskPlan {
    Space sp;
    int P, Q;
    int64_t n_feat;
    int n_low, n_un, n_tiles;
    int lvl_units[kMaxRung + 1];
    std::vector<int2> tiles;
    UnaryArgs ua;
    int sec_bin[4];
};

bool plan_task(int N, int d, uint32_t ops, int rung, int grammar, TaskPlan& T) {
    if (!plan_space(d, ops, rung, grammar, T.sp)) return false;
    const Space& sp = T.sp;
    const int L = sp.rung;
    T.P = (int)sp.phi[L - 1];
    T.Q = L >= 2 ? (int)sp.phi[L - 2] : 0;
    T.n_feat = sp.phi[L];
    for (int l = 0; l <= kMaxRung; ++l) T.lvl_units[l] = 0;
    for (int l = 1; l < L; ++l) T.lvl_units[l] = (int)((sp.phi[l] - sp.phi[l - 1] + kInitIds - 1) / kInitIds);
    for (int o = 0; o < 4; ++o) T.sec_bin[o] = -1;
    T.ua = UnaryArgs{};
    T.ua.Q = T.Q; T.ua.P = T.P; T.ua.N = N;
    bool any_bin = false;
    for (int s = 0; s < sp.nsec; ++s) {
        const Section& sc = sp.sec[s];
        if (sc.level != L) continue;
        if (sc.op <= DIV) { T.sec_bin[sc.op] = s; any_bin = true; }
        else if (T.ua.n_ops < kUnaryMax) { T.ua.op[T.ua.n_ops] = sc.op; T.ua.base[T.ua.n_ops] = sc.base; ++T.ua.n_ops; }
        else return false;
    }
    T.tiles.clear();
    if (any_bin) pair_tiles(T.P, T.Q, sp.grammar == SISSO_GRAMMAR_NEW_X_PREV && L >= 3, T.tiles);
    T.n_low = (T.P + kLowIds - 1) / kLowIds;
    T.n_un = T.ua.n_ops > 0 ? (T.P - T.Q + 31) / 32 : 0;
    T.n_tiles = (int)T.tiles.size();
    (void)N;
    return true;
}

int64_t enum_total_host(int n, int D) {
    if (n < D) return 0;
    if (D == 1) return (n + kBT - 1) / kBT;
    const int DP = D - 2;
    const int cpp = std::max(1, (n - 1 - DP + kRows - 1) / kRows);
    return binom_hd(n - 2, DP) * cpp;
}

// upper bound on the work items one task queues
long long queue_items(const TaskPlan& T, int rung, int k, int max_dim, const sisso_batch_tune& tu) {
    long long n = 0;
    for (int l = 1; l < rung; ++l) n += T.lvl_units[l];
    const int units = T.n_low + T.n_un + T.n_tiles;
    for (int t = 1; t <= max_dim; ++t) {
        n += (T.P + kBT - 1) / kBT;
        n += (units + tu.score_units - 1) / tu.score_units;
        n += std::max(1, (k + tu.gram_rows - 1) / tu.gram_rows);
        n += 2 * ((enum_total_host(t * k, t) + tu.enum_items - 1) / tu.enum_items);
    }
    return n;
}

sisso_status capture(sisso_batch* b, bool copies, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    // a persistent grid: never more CTAs than can be resident at once
    int resident = 0;
    if (b->tune.ctas_per_sm == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_batch<1>, kBT, kBatchSmem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_batch<2>, kBT, kBatchSmem);
    const int grid = b->sms * std::max(1, std::min(resident, b->tune.ctas_per_sm));

    sisso_status st = bcuda(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "capture");
    if (st) return st;
    if (copies) cudaMemcpyAsync(b->in_dev, b->in_host, sizeof(double) * b->in_count, cudaMemcpyHostToDevice, b->stream);
    cudaMemsetAsync(b->state, 0, sizeof(BState) * b->n_tasks, b->stream);
    cudaMemsetAsync(b->ctr, 0, sizeof(int) * 8, b->stream);
    cudaMemsetAsync(b->t0, 0xFF, sizeof(unsigned long long), b->stream);
    cudaMemsetAsync(b->prof, 0, sizeof(unsigned long long) * 48, b->stream);
    cudaMemsetAsync(b->slots, 0, sizeof(unsigned long long) * b->cap, b->stream);
    cudaMemsetAsync(b->res_dev, 0, sizeof(sisso_task_result) * b->n_tasks, b->stream);
    BatchArgs A{};
    A.tasks = b->tasks_dev; A.state = b->state; A.res = b->res_dev; A.n_tasks = b->n_tasks;
    A.order = b->order_dev; A.slots = b->slots; A.cap = b->cap; A.ctr = b->ctr; A.t0 = b->t0; A.prof = b->prof;
    A.k = b->k; A.max_dim = b->max_dim;
    A.score_units = b->tune.score_units; A.enum_items = b->tune.enum_items; A.gram_rows = b->tune.gram_rows;
    A.win0 = b->tune.window; A.band_cap = b->band_cap;
    A.idle_ns = b->idle_ns > 0 ? b->idle_ns : kIdleNs;
    if (b->tune.ctas_per_sm == 1) k_batch<1><<<grid, kBT, kBatchSmem, b->stream>>>(A);
    else k_batch<2><<<grid, kBT, kBatchSmem, b->stream>>>(A);
    cudaMemcpyAsync(b->ctr_host, b->ctr, sizeof(int) * 8, cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(b->prof_host, b->prof, sizeof(unsigned long long) * 48, cudaMemcpyDeviceToHost, b->stream);
    if (copies) {
        cudaMemcpyAsync(b->res_host, b->res_dev, sizeof(sisso_task_result) * b->n_tasks, cudaMemcpyDeviceToHost, b->stream);
        cudaMemcpyAsync(b->state_host, b->state, sizeof(BState) * b->n_tasks, cudaMemcpyDeviceToHost, b->stream);
        cudaMemcpyAsync(b->t0_host, b->t0, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream);
    }
    st = bcuda(b, cudaStreamEndCapture(b->stream, &g), "capture end");
    if (st) return st;
    st = bcuda(b, cudaGraphInstantiate(out, g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    b->stats.grid = grid;
    return st;
}

sisso_status rebuild(sisso_batch* b) {
    if (b->g_dev) { cudaGraphExecDestroy(b->g_dev); b->g_dev = nullptr; }
    if (b->g_e2e) { cudaGraphExecDestroy(b->g_e2e); b->g_e2e = nullptr; }
    sisso_status st = capture(b, false, &b->g_dev);
    if (!st) st = capture(b, true, &b->g_e2e);
    return st;
}

void free_batch(sisso_batch* b) {
    if (b->g_dev) cudaGraphExecDestroy(b->g_dev);
    if (b->g_e2e) cudaGraphExecDestroy(b->g_e2e);
    void* dev[] = {b->arena, b->plans, b->tasks_dev, b->state, b->res_dev, b->order_dev, b->tiles_dev,
                   b->slots, b->ctr, b->t0, b->prof, b->in_dev};
    for (void* p : dev) if (p) cudaFree(p);
    void* host[] = {b->in_host, b->res_host, b->state_host, b->ctr_host, b->t0_host, b->prof_host};
    for (void* p : host) if (p) cudaFreeHost(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" {

const char* sisso_batch_create_error(void) {
    std::lock_guard<std::mutex> lk(g_batch_err_mu);
    return g_batch_create_err.c_str();
}

sisso_status sisso_batch_create(const sisso_task* tasks, int n_tasks, uint32_t op_set, int rung, int sis_size,
                                int max_dim, const sisso_opts* opts, sisso_batch** out) {
    auto set_err = [](const std::string& m) {
        std::lock_guard<std::mutex> lk(g_batch_err_mu);
        g_batch_create_err = m;
    };
    if (!out) { set_err("out is NULL"); return SISSO_ERR_ARG; }
    *out = nullptr;
    sisso_opts o;
    sisso_default_opts(&o);
    if (opts) o = *opts;
    if (!tasks || n_tasks < 1 || n_tasks > (1 << 20)) { set_err("n_tasks must be 1..2^20"); return SISSO_ERR_ARG; }
    if (rung < 1 || rung > kMaxRung || max_dim < 1 || max_dim > 4 || sis_size < 1 ||
        (op_set & SISSO_OP_ALL) == 0 || max_dim * sis_size > 512) {
        set_err("bad rung, max_dim (1..4), sis_size (max_dim * sis_size <= 512) or op_set");
        return SISSO_ERR_ARG;
    }
    if (o.precision != SISSO_PREC_FP32) { set_err("the batched form computes in FP32 (SISSO_PREC_FP32)"); return SISSO_ERR_ARG; }
    if (o.wait_limit_ns < 0) { set_err("wait_limit_ns must be >= 0"); return SISSO_ERR_ARG; }
    if (o.sis_threshold != 0.0 || o.stop_rmse != 0.0 || o.units) {
        set_err("the batched form screens the top sis_size without units and stops at exact fits (sis_threshold = stop_rmse = 0, units = NULL)");
        return SISSO_ERR_ARG;
    }
    if (o.grammar != SISSO_GRAMMAR_EQ2 && o.grammar != SISSO_GRAMMAR_NEW_X_PREV) { set_err("bad grammar"); return SISSO_ERR_ARG; }
    sisso_batch* b = new sisso_batch();
    b->n_tasks = n_tasks; b->rung = rung; b->k = sis_size; b->max_dim = max_dim; b->grammar = o.grammar;
    b->ops = op_set; b->device = o.device;
    b->band_cap = o.max_band > 0 ? (int)std::min<int64_t>(o.max_band, 1 << 24) : 16384;
    b->idle_ns = o.wait_limit_ns > 0 ? (unsigned long long)o.wait_limit_ns : 0;
    b->tune.score_units = 2; b->tune.enum_items = 32; b->tune.gram_rows = 2; b->tune.ctas_per_sm = 2;
    b->tune.window = std::max(256, 4 * sis_size);
    auto bail = [&](sisso_status st, const std::string& m) {
        set_err(m.empty() ? b->err : m);
        free_batch(b);
        return st;
    };
    // validate and plan every task
    std::vector<TaskPlan> plans(n_tasks);
    b->Ns.resize(n_tasks); b->ds.resize(n_tasks); b->in_off.resize(n_tasks); b->n_feat.resize(n_tasks);
    size_t in_count = 0;
    for (int i = 0; i < n_tasks; ++i) {
        const sisso_task& t = tasks[i];
        const std::string tag = "task " + std::to_string(i) + ": ";
        if (!t.X || !t.y || t.N < max_dim + 1 || t.d < 1 || t.d > 4096)
            return bail(SISSO_ERR_ARG, tag + "needs X, y, N >= max_dim + 1 and 1 <= d <= 4096");
        const size_t nx = (size_t)t.N * t.d;
        for (size_t e = 0; e < nx; ++e)
            if (!std::isfinite(t.X[e])) return bail(SISSO_ERR_ARG, tag + "non-finite X");
        double ymin = t.y[0], ymax = t.y[0];
        for (int s = 0; s < t.N; ++s) {
            if (!std::isfinite(t.y[s])) return bail(SISSO_ERR_ARG, tag + "non-finite y");
            ymin = std::min(ymin, t.y[s]); ymax = std::max(ymax, t.y[s]);
        }
        if (!(ymax > ymin)) return bail(SISSO_ERR_ARG, tag + "constant y");
        if (!plan_task(t.N, t.d, op_set, rung, o.grammar, plans[i])) return bail(SISSO_ERR_ARG, tag + "feature space plan failed");
        const TaskPlan& P = plans[i];
        if (P.n_low + P.n_un + P.n_tiles >= (1 << 18)) return bail(SISSO_ERR_ARG, tag + "too many screening units for the batched form");
        b->Ns[i] = t.N; b->ds[i] = t.d; b->n_feat[i] = P.n_feat;
        b->in_off[i] = in_count;
        in_count += align256(sizeof(double) * (nx + t.N)) / sizeof(double);
    }
    if (cudaSetDevice(o.device) != cudaSuccess) return bail(SISSO_ERR_CUDA, "cudaSetDevice failed");
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, o.device);
    b->sms = prop.multiProcessorCount;
    if (o.cuda_stream) b->stream = (cudaStream_t)o.cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(SISSO_ERR_CUDA, "stream");
        b->own_stream = true;
    }
    b->in_count = in_count;
    // arena layout
    const int W = kWinMax;
    const int ncap = max_dim * sis_size;
    std::vector<size_t> base(n_tasks);
    size_t total = 0;
    auto region = [&](size_t bytes) { const size_t at = total; total += align256(bytes); return at; };
    struct Off {
        size_t V, cache, vlvl[kMaxRung], valid, yc, Z, zraw, A1;
        size_t scores[kMaxDim + 1], tc64[kMaxDim + 1], tc32[kMaxDim + 1], ts[kMaxDim + 1], w_ids[kMaxDim + 1],
            w_score[kMaxDim + 1], w_mean[kMaxDim + 1], w_sd[kMaxDim + 1], w_valid[kMaxDim + 1], w_probe[kMaxDim + 1],
            gid[kMaxDim + 1], zmean[kMaxDim + 1], zsd[kMaxDim + 1], G64[kMaxDim + 1], b64[kMaxDim + 1],
            G32[kMaxDim + 1], b32[kMaxDim + 1], band[kMaxDim + 1], band_rss[kMaxDim + 1], resid[kMaxDim + 1],
            AR[kMaxDim + 1];
    };
    std::vector<Off> off(n_tasks);
    for (int i = 0; i < n_tasks; ++i) {
        const TaskPlan& P = plans[i];
        const int N = b->Ns[i];
        const size_t ldv = (size_t)((N + 31) / 32) * 32;
        Off& f = off[i];
        f.V = region(sizeof(double) * ldv * P.P);
        f.cache = region(sizeof(float) * (size_t)N * P.P);
        for (int l = 0; l < kMaxRung; ++l) {
            const int64_t cnt = l < rung ? P.sp.phi[l] - (l ? P.sp.phi[l - 1] : 0) : 0;
            f.vlvl[l] = region((size_t)std::max<int64_t>(cnt, 1));
        }
        f.valid = region((size_t)P.P);
        f.yc = region(sizeof(double) * N);
        f.Z = region(sizeof(double) * ldv * ncap);
        f.zraw = region(sizeof(double) * (size_t)N * kZRaw);
        f.A1 = region(sizeof(double) * P.P);
        for (int t = 1; t <= max_dim; ++t) {
            const size_t nt = (size_t)t * sis_size;
            f.scores[t] = region(sizeof(float) * P.n_feat);
            f.tc64[t] = region(sizeof(double) * N);
            f.tc32[t] = region(sizeof(float) * N);
            f.ts[t] = region(sizeof(TargetStats));
            f.w_ids[t] = region(sizeof(int64_t) * W);
            f.w_score[t] = region(sizeof(double) * W);
            f.w_mean[t] = region(sizeof(double) * W);
            f.w_sd[t] = region(sizeof(double) * W);
            f.w_valid[t] = region(sizeof(int) * W);
            f.w_probe[t] = region(sizeof(double) * W * kProbes);
            f.gid[t] = region(sizeof(int64_t) * nt);
            f.zmean[t] = region(sizeof(double) * nt);
            f.zsd[t] = region(sizeof(double) * nt);
            f.G64[t] = region(sizeof(double) * nt * nt);
            f.b64[t] = region(sizeof(double) * nt);
            f.G32[t] = region(sizeof(float) * nt * nt);
            f.b32[t] = region(sizeof(float) * nt);
            f.band[t] = region(sizeof(uint64_t) * b->band_cap);
            f.band_rss[t] = region(sizeof(double) * b->band_cap);
            f.resid[t] = region(sizeof(double) * N);
            f.AR[t] = region(sizeof(double) * P.P);
        }
    }
    b->arena_bytes = total;
    sisso_status st;
    if ((st = bcuda(b, cudaMalloc(&b->arena, total), "batch arena"))) return bail(st, "");
    size_t n_tiles_all = 0;
    for (auto& P : plans) n_tiles_all += P.tiles.size();
    if ((st = bcuda(b, cudaMalloc(&b->plans, sizeof(Space) * n_tasks), "plans")) ||
        (st = bcuda(b, cudaMalloc(&b->tasks_dev, sizeof(BTask) * n_tasks), "tasks")) ||
        (st = bcuda(b, cudaMalloc(&b->state, sizeof(BState) * n_tasks), "state")) ||
        (st = bcuda(b, cudaMalloc(&b->res_dev, sizeof(sisso_task_result) * n_tasks), "results")) ||
        (st = bcuda(b, cudaMalloc(&b->order_dev, sizeof(int) * n_tasks), "order")) ||
        (st = bcuda(b, cudaMalloc(&b->tiles_dev, sizeof(int2) * std::max<size_t>(n_tiles_all, 1)), "tiles")) ||
        (st = bcuda(b, cudaMalloc(&b->ctr, sizeof(int) * 8), "counters")) ||
        (st = bcuda(b, cudaMalloc(&b->t0, sizeof(unsigned long long)), "t0")) ||
        (st = bcuda(b, cudaMalloc(&b->prof, sizeof(unsigned long long) * 48), "profile")) ||
        (st = bcuda(b, cudaMallocHost(&b->prof_host, sizeof(unsigned long long) * 48), "pinned profile")) ||
        (st = bcuda(b, cudaMalloc(&b->in_dev, sizeof(double) * in_count), "inputs")) ||
        (st = bcuda(b, cudaMallocHost(&b->in_host, sizeof(double) * in_count), "pinned inputs")) ||
        (st = bcuda(b, cudaMallocHost(&b->res_host, sizeof(sisso_task_result) * n_tasks), "pinned results")) ||
        (st = bcuda(b, cudaMallocHost(&b->state_host, sizeof(BState) * n_tasks), "pinned state")) ||
        (st = bcuda(b, cudaMallocHost(&b->ctr_host, sizeof(int) * 8), "pinned counters")) ||
        (st = bcuda(b, cudaMallocHost(&b->t0_host, sizeof(unsigned long long)), "pinned t0")))
        return bail(st, "");
    // queue: sized for the smallest work items the autotuner tries
    sisso_batch_tune small{1, 8, 1, 2, 256};
    long long cap = 0;
    for (auto& P : plans) cap += queue_items(P, rung, sis_size, max_dim, small);
    b->cap = cap + 16;
    if ((st = bcuda(b, cudaMalloc(&b->slots, sizeof(unsigned long long) * b->cap), "queue"))) return bail(st, "");
    // task records
    b->th.resize(n_tasks);
    std::vector<int2> tiles_all;
    tiles_all.reserve(n_tiles_all);
    std::vector<Space> sps(n_tasks);
    char* A = static_cast<char*>(b->arena);
    for (int i = 0; i < n_tasks; ++i) {
        const TaskPlan& P = plans[i];
        const Off& f = off[i];
        BTask& T = b->th[i];
        T = BTask{};
        T.N = b->Ns[i]; T.ldv = ((T.N + 31) / 32) * 32; T.d = b->ds[i]; T.rung = rung;
        T.P = P.P; T.Q = P.Q; T.n_feat = P.n_feat;
        T.n_low = P.n_low; T.n_un = P.n_un; T.n_tiles = P.n_tiles; T.n_units = P.n_low + P.n_un + P.n_tiles;
        int acc = 0;
        for (int l = 0; l <= kMaxRung; ++l) { T.lvl_first[l] = acc; acc += P.lvl_units[l]; }
        sps[i] = P.sp;
        T.sp = b->plans + i;
        T.pa = PairArgs{};
        T.pa.sp = b->plans + i;
        for (int o = 0; o < 4; ++o) T.pa.sec[o] = P.sec_bin[o];
        T.pa.P = P.P; T.pa.Q = P.Q;
        T.pa.nxp = P.sp.grammar == SISSO_GRAMMAR_NEW_X_PREV && rung >= 3;
        T.pa.N = T.N;
        T.pa.n_tiles = P.n_tiles;
        T.ua = P.ua;
        T.tiles = b->tiles_dev + tiles_all.size();
        T.pa.tiles = T.tiles;
        tiles_all.insert(tiles_all.end(), P.tiles.begin(), P.tiles.end());
        T.X = b->in_dev + b->in_off[i];
        T.y = T.X + (size_t)T.N * T.d;
        T.V = reinterpret_cast<double*>(A + f.V);
        T.cache = reinterpret_cast<float*>(A + f.cache);
        for (int l = 0; l < kMaxRung; ++l) T.vlvl[l] = reinterpret_cast<unsigned char*>(A + f.vlvl[l]);
        T.valid = reinterpret_cast<unsigned char*>(A + f.valid);
        T.yc = reinterpret_cast<double*>(A + f.yc);
        T.Z = reinterpret_cast<double*>(A + f.Z);
        T.zraw = reinterpret_cast<double*>(A + f.zraw);
        T.A1 = reinterpret_cast<double*>(A + f.A1);
        for (int t = 1; t <= max_dim; ++t) {
            BDim& D = T.dim[t];
            D.scores = reinterpret_cast<float*>(A + f.scores[t]);
            D.tc64 = reinterpret_cast<double*>(A + f.tc64[t]);
            D.tc32 = reinterpret_cast<float*>(A + f.tc32[t]);
            D.ts = reinterpret_cast<TargetStats*>(A + f.ts[t]);
            D.w_ids = reinterpret_cast<int64_t*>(A + f.w_ids[t]);
            D.w_score = reinterpret_cast<double*>(A + f.w_score[t]);
            D.w_mean = reinterpret_cast<double*>(A + f.w_mean[t]);
            D.w_sd = reinterpret_cast<double*>(A + f.w_sd[t]);
            D.w_valid = reinterpret_cast<int*>(A + f.w_valid[t]);
            D.w_probe = reinterpret_cast<double*>(A + f.w_probe[t]);
            D.gid = reinterpret_cast<int64_t*>(A + f.gid[t]);
            D.zmean = reinterpret_cast<double*>(A + f.zmean[t]);
            D.zsd = reinterpret_cast<double*>(A + f.zsd[t]);
            D.G64 = reinterpret_cast<double*>(A + f.G64[t]);
            D.b64 = reinterpret_cast<double*>(A + f.b64[t]);
            D.G32 = reinterpret_cast<float*>(A + f.G32[t]);
            D.b32 = reinterpret_cast<float*>(A + f.b32[t]);
            D.band = reinterpret_cast<uint64_t*>(A + f.band[t]);
            D.band_rss = reinterpret_cast<double*>(A + f.band_rss[t]);
            D.resid = reinterpret_cast<double*>(A + f.resid[t]);
            D.AR = reinterpret_cast<double*>(A + f.AR[t]);
        }
    }
    // longest first: estimated screening work |phi_L| x N
    std::vector<int> order(n_tasks);
    for (int i = 0; i < n_tasks; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (double)b->n_feat[a] * b->Ns[a] > (double)b->n_feat[c] * b->Ns[c];
    });
    cudaMemcpy(b->plans, sps.data(), sizeof(Space) * n_tasks, cudaMemcpyHostToDevice);
    cudaMemcpy(b->tasks_dev, b->th.data(), sizeof(BTask) * n_tasks, cudaMemcpyHostToDevice);
    cudaMemcpy(b->order_dev, order.data(), sizeof(int) * n_tasks, cudaMemcpyHostToDevice);
    if (!tiles_all.empty()) cudaMemcpy(b->tiles_dev, tiles_all.data(), sizeof(int2) * tiles_all.size(), cudaMemcpyHostToDevice);
    if ((st = bcuda(b, cudaGetLastError(), "upload"))) return bail(st, "");
    if ((st = sisso_batch_load(b, tasks, n_tasks))) return bail(st, "");
    cudaMemcpyAsync(b->in_dev, b->in_host, sizeof(double) * in_count, cudaMemcpyHostToDevice, b->stream);
    if ((st = bcuda(b, cudaStreamSynchronize(b->stream), "input copy"))) return bail(st, "");
    if ((st = bcuda(b, cudaFuncSetAttribute(k_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem),
                    "shared memory attribute")) ||
        (st = bcuda(b, cudaFuncSetAttribute(k_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem),
                    "shared memory attribute")))
        return bail(st, "");
    if ((st = rebuild(b))) return bail(st, "");
    *out = b;
    return SISSO_OK;
}

sisso_status sisso_batch_load(sisso_batch* b, const sisso_task* tasks, int n_tasks) {
    if (!b || !tasks || n_tasks != b->n_tasks) return SISSO_ERR_ARG;
    for (int i = 0; i < n_tasks; ++i) {
        if (tasks[i].N != b->Ns[i] || tasks[i].d != b->ds[i] || !tasks[i].X || !tasks[i].y)
            return bfail(b, SISSO_ERR_ARG, "task " + std::to_string(i) + ": shape differs from the batch");
        const size_t nx = (size_t)tasks[i].N * tasks[i].d;
        std::memcpy(b->in_host + b->in_off[i], tasks[i].X, sizeof(double) * nx);
        std::memcpy(b->in_host + b->in_off[i] + nx, tasks[i].y, sizeof(double) * tasks[i].N);
    }
    return SISSO_OK;
}

sisso_status sisso_batch_set_tune(sisso_batch* b, const sisso_batch_tune* tune) {
    if (!b || !tune) return SISSO_ERR_ARG;
    sisso_batch_tune t = b->tune;
    if (tune->score_units > 0) t.score_units = tune->score_units;
    if (tune->enum_items > 0) t.enum_items = tune->enum_items;
    if (tune->gram_rows > 0) t.gram_rows = tune->gram_rows;
    if (tune->ctas_per_sm > 0) t.ctas_per_sm = tune->ctas_per_sm;
    if (tune->window > 0) t.window = tune->window;
    if (t.ctas_per_sm > 2 || t.score_units > 4096 || t.enum_items > (1 << 20) || t.gram_rows > 512 ||
        t.window > kWinMax)
        return bfail(b, SISSO_ERR_ARG, "launch shape out of range");
    // the queue was sized for the smallest items
    if (t.score_units < 1 || t.enum_items < 8 || t.gram_rows < 1) return bfail(b, SISSO_ERR_ARG, "work items below the queue's sizing");
    cudaSetDevice(b->device);
    b->tune = t;
    return rebuild(b);
}

sisso_status sisso_batch_set_wait_limit(sisso_batch* b, int64_t ns) {
    if (!b || ns < 0) return SISSO_ERR_ARG;
    cudaSetDevice(b->device);
    b->idle_ns = (unsigned long long)ns;
    return rebuild(b);
}

sisso_status sisso_batch_get_tune(const sisso_batch* b, sisso_batch_tune* tune) {
    if (!b || !tune) return SISSO_ERR_ARG;
    *tune = b->tune;
    return SISSO_OK;
}

sisso_status sisso_batch_run(sisso_batch* b, int copies) {
    if (!b) return SISSO_ERR_ARG;
    cudaSetDevice(b->device);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
    sisso_status st = bcuda(b, cudaGraphLaunch(copies ? b->g_e2e : b->g_dev, b->stream), "graph launch");
    cudaEventRecord(e1, b->stream);
    if (!st) st = bcuda(b, cudaStreamSynchronize(b->stream), "batch run");
    float ms = 0.f;
    if (!st) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    if (st) return st;
    b->stats.ms_run = ms;
    b->ran = true;
    b->fetched = copies != 0;
    const int e = b->ctr_host[4];
    if (e & 4) return bfail(b, SISSO_ERR_CAPACITY, "work queue overflow");
    if (e) return bfail(b, SISSO_ERR_TIMEOUT, "a CTA found no work for the time limit");
    return SISSO_OK;
}

static sisso_status fetch(sisso_batch* b) {
    if (!b->ran) return bfail(b, SISSO_ERR_STATE, "no run yet");
    if (b->fetched) return SISSO_OK;
    cudaMemcpyAsync(b->res_host, b->res_dev, sizeof(sisso_task_result) * b->n_tasks, cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(b->state_host, b->state, sizeof(BState) * b->n_tasks, cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(b->t0_host, b->t0, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream);
    sisso_status st = bcuda(b, cudaStreamSynchronize(b->stream), "fetch");
    if (!st) b->fetched = true;
    return st;
}

sisso_status sisso_batch_results(sisso_batch* b, sisso_task_result* out, int n) {
    if (!b || !out || n < 0 || n > b->n_tasks) return SISSO_ERR_ARG;
    sisso_status st = fetch(b);
    if (st) return st;
    std::memcpy(out, b->res_host, sizeof(sisso_task_result) * n);
    return SISSO_OK;
}

sisso_status sisso_batch_timing(sisso_batch* b, double* start, double* end, int n) {
    if (!b || n < 0 || n > b->n_tasks) return SISSO_ERR_ARG;
    sisso_status st = fetch(b);
    if (st) return st;
    const unsigned long long t0 = *b->t0_host;
    for (int i = 0; i < n; ++i) {
        const BState& s = b->state_host[i];
        if (start) start[i] = s.t_start >= t0 ? (double)(s.t_start - t0) * 1e-6 : 0.0;
        if (end) end[i] = s.t_end >= t0 ? (double)(s.t_end - t0) * 1e-6 : 0.0;
    }
    return SISSO_OK;
}

sisso_status sisso_batch_get_stats(sisso_batch* b, sisso_batch_stats* out) {
    if (!b || !out) return SISSO_ERR_ARG;
    sisso_status st = fetch(b);
    if (st) return st;
    sisso_batch_stats s = b->stats;
    s.candidates_scored = 0; s.subsets_fit = 0; s.subsets_refit = 0;
    s.windows_grown = 0; s.windows_saturated = 0; s.tasks_failed = 0; s.walk_visits = 0; s.walk_checks = 0;
    for (int i = 0; i < b->n_tasks; ++i) {
        const BState& x = b->state_host[i];
        const int nd = b->res_host[i].n_dims;
        s.candidates_scored += b->n_feat[i] * (int64_t)std::max(nd, 1);
        for (int t = 1; t <= b->max_dim; ++t) {
            s.subsets_fit += (int64_t)x.examined[t];
            s.subsets_refit += x.band_count[t];
        }
        s.windows_grown += x.grown;
        s.walk_visits += x.visits;
        s.walk_checks += x.checks;
        s.windows_saturated += x.saturated;
        s.tasks_failed += b->res_host[i].status != SISSO_OK;
    }
    for (int q = 0; q < 16; ++q) {
        s.stage_ms[q] = (double)b->prof_host[q] * 1e-6;
        s.stage_count[q] = (int64_t)b->prof_host[16 + q];
        s.stage_max_ms[q] = (double)b->prof_host[32 + q] * 1e-6;
    }
    *out = s;
    return SISSO_OK;
}

const char* sisso_batch_last_error(const sisso_batch* b) { return b ? b->err.c_str() : "null batch"; }

void sisso_batch_destroy(sisso_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
}

sisso_status sisso_batch_autotune(sisso_batch* b, int reps, const char* cache_path, sisso_batch_tune* chosen) {
    if (!b) return SISSO_ERR_ARG;
    if (reps < 1) reps = 1;
    // signature of the batch's shape
    std::ostringstream sig;
    {
        int64_t sN = 0, sF = 0;
        for (int i = 0; i < b->n_tasks; ++i) { sN += b->Ns[i]; sF += b->n_feat[i]; }
        cudaDeviceProp prop{};
        cudaGetDeviceProperties(&prop, b->device);
        sig << "sms=" << b->sms << ";cc=" << prop.major << prop.minor << ";tasks=" << b->n_tasks << ";sumN=" << sN
            << ";sumF=" << sF << ";k=" << b->k << ";D=" << b->max_dim << ";rung=" << b->rung << ";ops=" << b->ops
            << ";g=" << b->grammar;
    }
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            const size_t sp = line.find(' ');
            if (sp == std::string::npos || line.substr(0, sp) != sig.str()) continue;
            sisso_batch_tune t{};
            std::istringstream vs(line.substr(sp + 1));
            if (vs >> t.score_units >> t.enum_items >> t.gram_rows >> t.ctas_per_sm >> t.window) {
                sisso_status st = sisso_batch_set_tune(b, &t);
                if (!st && chosen) *chosen = b->tune;
                return st;
            }
        }
    }
    auto time_it = [&](double& best_ms) -> sisso_status {
        double best = 1e30;
        for (int r = 0; r < reps; ++r) {
            sisso_status st = sisso_batch_run(b, 0);
            if (st) return st;
            best = std::min(best, (double)b->stats.ms_run);
        }
        best_ms = best;
        return SISSO_OK;
    };
    sisso_status st = sisso_batch_run(b, 0);   // warm-up
    if (st) return st;
    double cur_ms;
    if ((st = time_it(cur_ms))) return st;
    const std::vector<int> su = {1, 2, 4, 8};
    const std::vector<int> ei = {8, 32, 128, 512};
    const std::vector<int> gr = {1, 2, 4, 8};
    const std::vector<int> cp = {1, 2};
    const std::vector<int> wn = {std::max(b->k, 128), std::max(256, 4 * b->k), std::max(1024, 16 * b->k)};
    for (int param = 0; param < 5; ++param) {
        const std::vector<int>& vals = param == 0 ? su : param == 1 ? ei : param == 2 ? gr : param == 3 ? cp : wn;
        sisso_batch_tune best = b->tune;
        for (int v : vals) {
            sisso_batch_tune t = best;
            int* field = param == 0 ? &t.score_units : param == 1 ? &t.enum_items : param == 2 ? &t.gram_rows
                       : param == 3 ? &t.ctas_per_sm : &t.window;
            if (*field == v || v > kWinMax) continue;
            *field = v;
            if ((st = sisso_batch_set_tune(b, &t))) return st;
            double ms;
            if ((st = time_it(ms))) return st;
            if (ms < cur_ms) { cur_ms = ms; best = t; }
        }
        if ((st = sisso_batch_set_tune(b, &best))) return st;
    }
    if (cache_path) {
        std::ofstream outf(cache_path, std::ios::app);
        outf << sig.str() << ' ' << b->tune.score_units << ' ' << b->tune.enum_items << ' ' << b->tune.gram_rows << ' '
             << b->tune.ctas_per_sm << ' ' << b->tune.window << '\n';
    }
    if (chosen) *chosen = b->tune;
    return SISSO_OK;
}

sisso_status sisso_fit_batch(const sisso_task* tasks, int n_tasks, uint32_t op_set, int rung, int sis_size,
                             int max_dim, const sisso_opts* opts, sisso_task_result* results) {
    if (!results) return SISSO_ERR_ARG;
    sisso_batch* b = nullptr;
    sisso_status st = sisso_batch_create(tasks, n_tasks, op_set, rung, sis_size, max_dim, opts, &b);
    if (st) return st;
    st = sisso_batch_run(b, 1);
    if (!st) st = sisso_batch_results(b, results, n_tasks);
    sisso_batch_destroy(b);
    return st;
}

}  // extern "C"
