// pg_internal.cuh -- context, scratch, launch accounting and the device
// helpers shared by the kernels of libpg (GB300, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pg.h"

// ---------------------------------------------------------------- context
struct pg_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;  // 0 = unlimited
    size_t in_use = 0;
    std::string last_error;
    int *d_err = nullptr;                     // [4]: code, where, info lo, info hi
    unsigned long long *d_counters = nullptr;  // kernel statistics
    unsigned long long *h_pinned = nullptr;   // pinned host mirror for small reads
    int *h_err = nullptr;                      // pinned mirror of the error word
    int64_t launches = 0;
    int64_t connect_edges = 0;        // edges added by the connectivity step
    int64_t connect_full_rounds = 0;  // of those, rounds decided by a full scan
    int64_t connect_why_full = 0;     // batches cut short by a candidate that filled up
    int64_t connect_free = 0;         // nodes with a free slot when connectivity steps began
    int count_ties = 0;               // pruning counts near-tie decisions (pg_ctx_set_tie_count)
    int autotune = 0;                 // launch configurations chosen by timing (tune.cu)
    int last_derr = 0;                // device error code of the last failed synchronisation
    int64_t last_err_info = 0;        // ... and its info word (e.g. the refused node)
    // optional CUDA-event timing of named kernels
    int timing = 0;
    struct TimedPair {
        int slot;
        cudaEvent_t a, b;
    };
    std::vector<TimedPair> pending;
    std::vector<cudaEvent_t> event_pool;
    double timer_ms[16] = {0};
    int64_t timer_launches[16] = {0};
    double timer_work[16] = {0};  // algorithmic flops or bytes of the timed launches
};

// Data facts computed once per dataset: whether every FP32 distance the
// kernels form is exact (integer-valued rows small enough that all partial
// sums stay below 2^24), and the largest squared row norm.
struct DataFacts {
    int exact = 0;
    int bf16_exact = 0;  // integer rows with |x| <= 256: the BF16 copy is exact
    int u8_exact = 0;    // integer rows in [0, 255]: a byte copy is exact
    float max_norm2 = 0.f;
    float max_abs = 0.f;
    float min_v = 0.f, max_v = 0.f;  // value range of the rows
};

// ------------------------------------------------------------------ index
// One layer of an index and the index itself (built in build.cu, written
// and read by index_io.cu).
struct pg_layer {
    int64_t count = 0;
    int64_t cap = 0;  // rows allocated
    int R = 0;
    int32_t *gid = nullptr;   // [count] ascending point ids (null: identity)
    int32_t *nbr = nullptr;   // [count][R] point ids
    int32_t *deg = nullptr;   // [count]
    int32_t *rows = nullptr;  // [n] point id -> row, -1 if absent (null: identity)
};

struct pg_index {
    int64_t n = 0;
    int d = 0;
    pg_metric metric = PG_METRIC_L2SQ;
    const float *D = nullptr;
    std::vector<pg_layer> layers;
    int64_t ep_top = 0, ep_base = 0;
    double phase[6] = {0, 0, 0, 0, 0, 0};
    int32_t iters_run = 0;     // OptKCNA iterations of the last build (layer 0)
    int64_t quality_ns = 0;    // quality examination sample size (0: off)
    double quality_est[16] = {0};
    DataFacts facts{};         // of the points (kept up to date by insertion)
    int has_facts = 0;
    pg_build_params params{};  // of the build: levels, degrees, pruning angle
    float *owned = nullptr;    // private copy of the points once reserved
    int64_t capacity = 0;      // rows of `owned`
    // FP8 E4M3 copy of the points for screened queries: made on first use,
    // extended after insertions (rows [0, f8_rows) valid, f8_cap allocated)
    mutable std::mutex f8_mu;
    mutable uint8_t *f8 = nullptr;      // [f8_cap][d]
    mutable float *f8_scale = nullptr;  // [f8_cap] value of 1.0 in the FP8 row
    mutable int64_t f8_rows = 0, f8_cap = 0;
    // Published versions of the layers (serving): a search takes a snapshot
    // of `layers`, `n` and the entry points under ver_mu and counts as a
    // reader of `version` until it has synchronised; an insertion builds the
    // next version in copies of the layer arrays and publishes it; the arrays
    // of older versions are reused by a later insertion once no search pins
    // them (freed here at the end).
    mutable std::mutex ver_mu;
    uint64_t version = 0;
    mutable std::map<uint64_t, int> readers;
    // graph arrays (pointer, bytes) of earlier versions, kept for reuse by
    // the next insertion once no search pins them
    std::vector<std::pair<uint64_t, std::vector<std::pair<void *, size_t>>>> retired;
    ~pg_index() {
        cudaFree(owned);
        cudaFree(f8);
        cudaFree(f8_scale);
        for (auto &l : layers) {
            cudaFree(l.gid);
            cudaFree(l.nbr);
            cudaFree(l.deg);
            cudaFree(l.rows);
        }
        for (auto &r : retired)
            for (auto &b : r.second) cudaFree(b.first);
    }
};

// A search's view of an index: the published layers, point count and entry
// points of one version, held as a reader of that version while alive.
struct IndexSnap {
    const pg_index *idx;
    std::vector<pg_layer> layers;
    int64_t n = 0, ep_top = 0, ep_base = 0;
    uint64_t version = 0;
    DataFacts facts{};
    int has_facts = 0;
    explicit IndexSnap(const pg_index *index) : idx(index) {
        std::lock_guard<std::mutex> lk(idx->ver_mu);
        layers = idx->layers;
        n = idx->n;
        ep_top = idx->ep_top;
        ep_base = idx->ep_base;
        version = idx->version;
        facts = idx->facts;
        has_facts = idx->has_facts;
        idx->readers[version] += 1;
    }
    ~IndexSnap() {
        std::lock_guard<std::mutex> lk(idx->ver_mu);
        if (--idx->readers[version] == 0) idx->readers.erase(version);
    }
    IndexSnap(const IndexSnap &) = delete;
    IndexSnap &operator=(const IndexSnap &) = delete;
};

// pg_search on a pinned version of the index (the serving loop pins it when
// it dispatches a query group); synchronises the context's stream
pg_status pg_search_pinned(pg_ctx *ctx, const IndexSnap &sn, const float *Q, int64_t nq,
                           int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                           pg_precision precision, int32_t *out_ids, float *out_dist);

// FP8 rows of an index for screened queries (device pointers)
struct F8Rows {
    const uint8_t *q8;    // [n][d] E4M3 codes of x / scale
    const float *scale;   // [n]
};

// Batched beam search (Algorithm 1), one warp per query: self mode (Q null,
// query i is row i from start i) or queries Q from starts; D8 the byte rows
// (self mode, exact data), f8 the FP8 rows (screened queries); facts the
// data facts of D (nullptr: computed here, which synchronises the stream).
pg_status pg_search_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             const int32_t *nbr, const int32_t *deg, int32_t R,
                             const int32_t *rows, const float *Q, int64_t nq,
                             const int32_t *starts, int32_t k, int32_t L, int self,
                             int32_t *out_i, float *out_s, const uint8_t *D8 = nullptr,
                             const F8Rows *f8 = nullptr, const DataFacts *facts = nullptr);

// named kernel timers
enum {
    TM_KNN = 0, TM_PRUNE, TM_UNION, TM_CONNECT, TM_SEARCH, TM_MEDOID, TM_CSELECT, TM_CFAST,
    TM_CSCAN, TM_CCOMMIT, TM_SLOTS
};
extern const char *const pg_timer_names[TM_SLOTS];
// Record an event before / after a launch when timing is enabled.
void pg_timer_begin(pg_ctx *ctx, int slot);
void pg_timer_end(pg_ctx *ctx, int slot, double work = 0.0);
void pg_timer_resolve(pg_ctx *ctx);

enum { PG_CNT_SLOTS = 32 };
// counter slots
enum {
    CNT_ROWS = 0, CNT_CANDS, CNT_SCANNED, CNT_OCCL, CNT_RECHECK, CNT_FLIP, CNT_EDGES, CNT_LONG,
    CNT_LONG_LIST = 16, CNT_KNN_RECHECK = 17, CNT_KNN_UNRESOLVED = 18, CNT_SEARCH_EXP = 19,
    CNT_SEARCH_EVAL = 20, CNT_SEARCH_BYTES = 21, CNT_PRUNE_BYTES = 22, CNT_NEAR_TIE = 23,
    CNT_KNN_FALLBACK = 24
};

// device error codes (first one recorded wins)
enum {
    DERR_NONE = 0, DERR_BAD_ID = 1, DERR_CAPACITY = 2, DERR_NO_SLOT = 3, DERR_INTERNAL = 4,
    DERR_TIMEOUT = 5
};

pg_status pg_fail(pg_ctx *ctx, pg_status st, const char *fmt, ...);
pg_status pg_cuda_fail(pg_ctx *ctx, cudaError_t e, const char *what);

#define PG_TRY_CUDA(ctx, call)                                          \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return pg_cuda_fail((ctx), _e, #call);   \
    } while (0)

#define PG_TRY(call)                          \
    do {                                      \
        pg_status _s = (call);                \
        if (_s != PG_OK) return _s;           \
    } while (0)

// Count a kernel launch and check the launch error.
#define PG_LAUNCHED(ctx)                                                      \
    do {                                                                      \
        (ctx)->launches++;                                                    \
        cudaError_t _e = cudaGetLastError();                                  \
        if (_e != cudaSuccess) return pg_cuda_fail((ctx), _e, "kernel launch"); \
    } while (0)

// Stream-ordered scratch counted against the budget.
pg_status pg_alloc(pg_ctx *ctx, void **p, size_t bytes);
void pg_free(pg_ctx *ctx, void *p, size_t bytes);

template <class T>
struct Scratch {
    pg_ctx *ctx = nullptr;
    T *p = nullptr;
    size_t bytes = 0;
    Scratch() = default;
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    pg_status alloc(pg_ctx *c, size_t count) {
        release();
        ctx = c;
        bytes = count * sizeof(T);
        if (bytes == 0) bytes = sizeof(T);
        void *q = nullptr;
        pg_status s = pg_alloc(ctx, &q, bytes);
        p = static_cast<T *>(q);
        if (s != PG_OK) bytes = 0;
        return s;
    }
    void release() {
        if (p) pg_free(ctx, p, bytes);
        p = nullptr;
        bytes = 0;
    }
    ~Scratch() { release(); }
};

// Launch-configuration autotuner (tune.cu): a key names a kernel and the
// shape it runs on; configs are kernel-specific codes.
struct TuneKey {
    int device, kernel, d, p, form;
};
enum { TUNE_PRUNE = 1, TUNE_SEARCH = 2 };
bool pg_tune_lookup(const TuneKey &k, int *config);
void pg_tune_store(const TuneKey &k, int config, const std::vector<std::pair<int, float>> &tried,
                   const char *label);
// Time run(c) for every c (CUDA events on ctx's stream), *best = the fastest.
pg_status pg_tune_time(pg_ctx *ctx, const std::vector<int> &configs,
                       const std::function<pg_status(int)> &run, int *best,
                       std::vector<std::pair<int, float>> *tried);

// Dimension of the points of an index.
int pg_index_dim(const pg_index *index);

// Exclusive prefix sum of n int32 counts into n + 1 int64 offsets (async).
pg_status pg_scan_counts(pg_ctx *ctx, const int32_t *cnt, int64_t n, int64_t *off);

// Synchronise and translate the device error word.
pg_status pg_sync_check(pg_ctx *ctx, const char *where);
// Reset statistics counters (async).
pg_status pg_reset_counters(pg_ctx *ctx);
pg_status pg_read_counters(pg_ctx *ctx, unsigned long long *host32);

// ---------------------------------------------------------- arithmetic facts
// The facts of D [n][d] (one kernel pass; synchronises the stream).
pg_status pg_data_facts(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                        DataFacts *out);
// Extend the facts of D to the pairs (query row, row of D) of Q [nq][d]:
// exact only if both sides are and the combined range keeps every partial
// sum below 2^24; the norm and value bounds cover both.
pg_status pg_query_facts(pg_ctx *ctx, const float *Q, int64_t nq, int32_t d, pg_metric metric,
                         DataFacts *f);
// The facts from the per-block results of k_data_facts (host copy, `blocks`
// groups of {integral, min, max, max squared norm}); shared by every entry
// point so that all of them take the same exactness decisions.
DataFacts pg_reduce_facts(const float *blk, int blocks, int64_t n, int32_t d, pg_metric metric);

// Byte shadow of D for the screened (BF16) form: when every FP32 distance is
// exact and the rows are bytes, the gathers of prune / search read 16-byte
// chunks of a u8 copy and form the same integer distances with __dp4a.
// Leaves `out` empty (p == nullptr) when the data do not qualify.
bool pg_u8_usable(const DataFacts &f, pg_metric metric, int d, pg_precision precision);
pg_status pg_make_u8(pg_ctx *ctx, const float *D, int64_t n, int32_t d, Scratch<uint8_t> &out);
// FP8 E4M3 rows r0..r1-1 of D: codes of x / scale (scale = max|x| / 448,
// 1 for a zero row), queued on ctx's stream
pg_status pg_make_f8(pg_ctx *ctx, const float *D, int64_t r0, int64_t r1, int32_t d, uint8_t *q8,
                     float *scale);
// build-like entry points take FP32 or BF16 screening only
inline bool pg_build_precision(pg_precision p) {
    return p == PG_PREC_FP32 || p == PG_PREC_BF16_SCREEN;
}

// Split-column argmin on the tensor cores over the rows of D (BF16-exact
// integer data): best[i] = min over columns c with reached[c] != 0 and
// deg[c] < R of key(s(D[ids[i]], D[c]), c) for i < *count (device), where
// key = FP32 bits << 32 | c; best[] must hold ~0 beforehand.
struct TcArgmin {
    Scratch<__nv_bfloat16> xb;  // BF16 copy of the candidate rows of D, padded to dp
    Scratch<float> xn;          // their squared row norms
    Scratch<int> cid;           // candidate column -> point id (ascending)
    Scratch<__nv_bfloat16> qb;  // the <= 128 query rows
    Scratch<float> qn;
    alignas(64) unsigned char mapx[128];  // CUtensorMap of xb
    alignas(64) unsigned char mapq[128];  // CUtensorMap of qb
    int64_t n = 0;
    int d = 0, dp = 0;
};
bool pg_tc_argmin_supported(int d);
// The candidate columns are the points with deg < R when this is called
// (degrees only grow during the connectivity step, so no later candidate
// is missing); synchronises the stream once to size the copies.
pg_status pg_tc_argmin_init(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                            const int32_t *deg, int R, TcArgmin &t);
pg_status pg_tc_argmin(pg_ctx *ctx, TcArgmin &t, const float *D, const int *ids, const int *count,
                       const int *reached, const int32_t *deg, int R, unsigned long long *best);

// Error model of an FP32 distance s computed by the kernels (difference form
// sum of squares for L2, dot product for the chord).  Bounds the distance
// to the FP64 sequential value of the CPU reference.
struct ErrModel {
    int metric = 0;    // 0 = L2 (relative), else chord (absolute)
    float rel = 0.f;   // L2: |s32 - s64| <= rel * s32
    float abs_ = 0.f;  // chord: |s32 - s64| <= abs_
    __host__ __device__ inline float err(float s) const {
        return metric == 0 ? rel * s : abs_;
    }
};
ErrModel pg_err_model(pg_metric metric, int d, const DataFacts &f, bool gemm_form);

// --------------------------------------------------------- device helpers
#ifdef __CUDACC__

__device__ __forceinline__ void record_error(int *err, int code, long long info) {
    if (atomicCAS(err, 0, code) == 0) {
        err[2] = (int)(info & 0xffffffff);
        err[3] = (int)(info >> 32);
    }
}

// (s, id) ordering
__device__ __forceinline__ bool pair_less(float a, int ia, float b, int ib) {
    return a < b || (a == b && ia < ib);
}

// FP64 sequential distances, one rounding per operation (matches the CPU
// reference bit for bit).
static __device__ __noinline__ double dist64_rows(const float *x, const float *y, int d, int metric) {
    double s = 0.0;
    if (metric == 0) {
        for (int i = 0; i < d; ++i) {
            double t = __dsub_rn((double)x[i], (double)y[i]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        return s;
    }
    for (int i = 0; i < d; ++i) s = __dadd_rn(s, __dmul_rn((double)x[i], (double)y[i]));
    s = __dsub_rn(2.0, __dmul_rn(2.0, s));
    return s < 0.0 ? 0.0 : s;
}

// FP64 angle clause: (suw + svw) - suv < (2 cos a) * sqrt(suw * svw)
__device__ __forceinline__ bool angle_exceeds64(double suw, double svw, double suv, double ca) {
    double lhs = __dsub_rn(__dadd_rn(suw, svw), suv);
    double rhs = __dmul_rn(__dmul_rn(2.0, ca), __dsqrt_rn(__dmul_rn(suw, svw)));
    return lhs < rhs;
}

// Three-valued FP32 decision of a < b given error bounds: 1 true, 0 false,
// -1 undecided.
__device__ __forceinline__ int less_certain(float a, float ea, float b, float eb) {
    if (a + ea < b - eb) return 1;
    if (a - ea >= b + eb) return 0;
    return -1;
}

// Three-valued FP32 angle clause with interval arithmetic over the
// distance errors; FP32 rounding of the formula itself is covered by a
// relative slack of 8 ulps on every term.
__device__ __forceinline__ int angle_certain(float suw, float euw, float svw, float evw, float suv,
                                             float euv, float ca) {
    const float slack = 8.f * 5.9604645e-8f;
    float sum = suw + svw + suv;
    float lhs = (suw + svw) - suv;
    float elhs = euw + evw + euv + slack * sum;
    float lo_a = fmaxf(suw - euw, 0.f), hi_a = suw + euw;
    float lo_b = fmaxf(svw - evw, 0.f), hi_b = svw + evw;
    float sq_lo = sqrtf(lo_a * lo_b), sq_hi = sqrtf(hi_a * hi_b);
    float two_c = 2.f * ca;
    float r1 = two_c * sq_lo, r2 = two_c * sq_hi;
    float rlo = fminf(r1, r2), rhi = fmaxf(r1, r2);
    float erhs = slack * (fabsf(rhi) + sum);
    if (lhs + elhs < rlo - erhs) return 1;
    if (lhs - elhs >= rhi + erhs) return 0;
    return -1;
}

__device__ __forceinline__ float warp_sum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// Team-of-8 FP32 distance between a point held in registers/shared (q)
// and a row of D: lane li of the team owns float4 chunks li, li+8, ...
// Returns the full distance on every lane of the team.
__device__ __forceinline__ float team8_dist(const float4 *__restrict__ qrow,
                                            const float4 *__restrict__ xrow, int nch, int li,
                                            int metric) {
    float acc = 0.f;
    if (metric == 0) {
        for (int c = li; c < nch; c += 8) {
            float4 a = qrow[c];
            float4 b = __ldg(xrow + c);
            float t0 = a.x - b.x, t1 = a.y - b.y, t2 = a.z - b.z, t3 = a.w - b.w;
            acc = fmaf(t0, t0, acc);
            acc = fmaf(t1, t1, acc);
            acc = fmaf(t2, t2, acc);
            acc = fmaf(t3, t3, acc);
        }
        return warp_sum8(acc);
    }
    for (int c = li; c < nch; c += 8) {
        float4 a = qrow[c];
        float4 b = __ldg(xrow + c);
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        acc = fmaf(a.w, b.w, acc);
    }
    acc = warp_sum8(acc);
    return fmaxf(2.f - 2.f * acc, 0.f);
}

// Squared L2 distance of two byte rows held as 16-byte chunks, by a team of
// eight lanes (lane li takes chunks li, li+8, ...); exact integer arithmetic.
__device__ __forceinline__ unsigned sq_diff_u8(uint4 a, uint4 b, unsigned acc) {
    unsigned t = __vabsdiffu4(a.x, b.x);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.y, b.y);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.z, b.z);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.w, b.w);
    return __dp4a(t, t, acc);
}

__device__ __forceinline__ unsigned team8_sum_u(unsigned v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

__device__ __forceinline__ float team8_dist_u8(const uint4 *__restrict__ q, const uint4 *__restrict__ x,
                                               int nch16, int li) {
    unsigned acc = 0;
    for (int c = li; c < nch16; c += 8) acc = sq_diff_u8(q[c], __ldg(x + c), acc);
    return (float)team8_sum_u(acc);
}

// Distances of up to 32 byte rows ids[0..cnt) (ids < 0 give +inf) to the
// byte query q, written to out[0..cnt): four teams of eight lanes, and for
// rows of at most 128 bytes every row's chunk is requested before the first
// is used, so one expansion waits for one round trip to memory.
__device__ __forceinline__ void batch_dist_u8(const uint8_t *__restrict__ D8, int d,
                                              const uint4 *__restrict__ q, const int *ids, int cnt,
                                              float *out) {
    const int lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int nch16 = d >> 4;
    if (nch16 <= 8) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        const uint4 qa = li < nch16 ? q[li] : z;
        uint4 r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = k * 4 + team;
            const int v = i < cnt ? ids[i] : -1;
            r[k] = (v >= 0 && li < nch16)
                       ? __ldg(reinterpret_cast<const uint4 *>(D8 + (int64_t)v * d) + li)
                       : z;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = k * 4 + team;
            const unsigned acc = team8_sum_u(sq_diff_u8(qa, r[k], 0u));
            if (li == 0 && i < cnt) out[i] = ids[i] >= 0 ? (float)acc : INFINITY;
        }
        return;
    }
    for (int b0 = 0; b0 < cnt; b0 += 4) {
        const int i = b0 + team;
        const int v = i < cnt ? ids[i] : -1;
        const float s = team8_dist_u8(q, reinterpret_cast<const uint4 *>(D8 + (int64_t)max(v, 0) * d),
                                      nch16, li);
        if (li == 0 && i < cnt) out[i] = v >= 0 ? s : INFINITY;
    }
}

// In-shared-memory bitonic sort of n (power of two) (key, id) pairs by one
// warp, ascending by (key, id).
__device__ __forceinline__ void warp_bitonic_sort(float *key, int *id, int n) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                int p = i ^ j;
                if (p > i) {
                    bool up = (i & k) == 0;
                    float a = key[i], b = key[p];
                    int ia = id[i], ib = id[p];
                    bool swap = up ? pair_less(b, ib, a, ia) : pair_less(a, ia, b, ib);
                    if (swap) {
                        key[i] = b; key[p] = a;
                        id[i] = ib; id[p] = ia;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Register bitonic sort of one (key, id) per lane across the warp.
__device__ __forceinline__ void warp_sort32(float &key, int &id) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= 32; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            float ok = __shfl_xor_sync(0xffffffffu, key, j);
            int oi = __shfl_xor_sync(0xffffffffu, id, j);
            bool lower = (lane & j) == 0;
            bool up = (lane & k) == 0;
            bool other_less = pair_less(ok, oi, key, id);
            bool take_other = (lower == up) ? other_less : pair_less(key, id, ok, oi);
            if (take_other) {
                key = ok;
                id = oi;
            }
        }
    }
}

#endif  // __CUDACC__
