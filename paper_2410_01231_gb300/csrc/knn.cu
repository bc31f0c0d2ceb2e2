// knn.cu -- exact K-nearest-neighbour graph (the KNNG G_k0 of the
// initialization phase, Section 3.1 / Algorithm 6) by brute-force
// distance tiles with a fused top-K.
//
// FP32 form: a CTA owns 64 query rows and streams every candidate column in
// tiles of 128, computing s = |q|^2 + |x|^2 - 2<q,x> (chord: 2 - 2<q,x>)
// with a 4x8 register tile per thread.  Each tile's values are filtered
// against the row's current K-th distance and survivors are appended to a
// per-row shared buffer; a buffer that could overflow is merged into the
// row's sorted top-K list (kept in the output arrays) by one warp.
// A post pass re-orders near-tie runs by their FP64 distance when the data
// is not exactly representable (integer data below 2^24 is exact).
#include <cfloat>
#include <climits>

#include "pg_internal.cuh"

namespace {

constexpr int BM = 64, BN = 128, BK = 32, NT = 256;
constexpr int BUF = 128;       // per-row survivor buffer (>= BN)
constexpr int APAD = BM + 4, BPAD = BN + 4;
constexpr int KMAX = 256;

struct KnnSmem {
    float As[BK][APAD];
    float Bs[BK][BPAD];
    float buf_s[BM][BUF];
    int buf_i[BM][BUF];
    float tmp_s[8][KMAX];
    int tmp_i[8][KMAX];
    float thr[BM];
    int cnt[BM];
    int pend[BM];
    float qn[BM];
};

__global__ void k_row_norms(const float *__restrict__ X, int64_t n, int d, float *out) {
    int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *row = X + r * d;
    float acc = 0.f;
    for (int c = lane; c < d; c += 32) acc = fmaf(row[c], row[c], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = acc;
}

__device__ __forceinline__ int lower_bound_pairs(const float *s, const int *id, int len, float key,
                                                 int kid) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (pair_less(s[mid], id[mid], key, kid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Merge row r's buffer into its global top-K list; one warp.
__device__ void merge_row(KnnSmem &sm, int r, int wid, int K, float *top_s, int *top_i) {
    const int lane = threadIdx.x & 31;
    int c = sm.cnt[r];
    if (c == 0) return;
    float *bs = sm.buf_s[r];
    int *bi = sm.buf_i[r];
    for (int j = c + lane; j < BUF; j += 32) {
        bs[j] = INFINITY;
        bi[j] = INT_MAX;
    }
    float *ts = sm.tmp_s[wid];
    int *ti = sm.tmp_i[wid];
    for (int j = lane; j < K; j += 32) {
        ts[j] = top_s[j];
        ti[j] = top_i[j];
    }
    __syncwarp();
    int len = BUF;
    while (len > 32 && bs[len / 2 - 1] == INFINITY && len / 2 >= c) len /= 2;
    if (len < 32) len = 32;
    warp_bitonic_sort(bs, bi, len);
    // top entries that are real (id >= 0) keep rank i + #buf before them
    for (int j = lane; j < K; j += 32) {
        float s = ts[j];
        int id = ti[j];
        if (id < 0) continue;
        int rank = j + lower_bound_pairs(bs, bi, c, s, id);
        if (rank < K) {
            top_s[rank] = s;
            top_i[rank] = id;
        }
    }
    // number of real entries in the old list
    int real = 0;
    for (int j = lane; j < K; j += 32) real += ti[j] >= 0;
    for (int o = 16; o; o >>= 1) real += __shfl_xor_sync(0xffffffffu, real, o);
    for (int j = lane; j < c; j += 32) {
        float s = bs[j];
        int id = bi[j];
        int rank = j + lower_bound_pairs(ts, ti, real, s, id);
        if (rank < K) {
            top_s[rank] = s;
            top_i[rank] = id;
        }
    }
    __syncwarp();
    __threadfence_block();
    if (lane == 0) {
        sm.cnt[r] = 0;
        sm.thr[r] = (real + c >= K) ? top_s[K - 1] : INFINITY;
    }
    __syncwarp();
}

// self_exclude: column id == query row id is skipped (Q == D).
__global__ void __launch_bounds__(NT, 2)
k_knn_fp32(const float *__restrict__ Q, int64_t nq, const float *__restrict__ X, int64_t n, int d,
           const float *__restrict__ qnorm, const float *__restrict__ xnorm, int metric, int K,
           int self_exclude, int32_t *__restrict__ out_i, float *__restrict__ out_s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KnnSmem &sm = *reinterpret_cast<KnnSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
    const int64_t row0 = (int64_t)blockIdx.x * BM;

    for (int r = tid; r < BM; r += NT) {
        sm.thr[r] = INFINITY;
        sm.cnt[r] = 0;
        sm.pend[r] = 0;
        int64_t g = row0 + r;
        sm.qn[r] = (g < nq) ? qnorm[g] : 0.f;
    }
    for (int64_t e = tid; e < (int64_t)BM * K; e += NT) {
        int64_t g = row0 + e / K;
        if (g < nq) {
            out_s[g * K + e % K] = INFINITY;
            out_i[g * K + e % K] = -1;
        }
    }
    __syncthreads();

    const int nkb = (d + BK - 1) / BK;
    for (int64_t col0 = 0; col0 < n; col0 += BN) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        for (int kb = 0; kb < nkb; ++kb) {
            const int k0 = kb * BK;
            // A tile: 64 rows x 32 k, 4 threads per row, 2 float4 each
            {
                int r = tid >> 2, kq = tid & 3;
                int64_t g = row0 + r;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int kk = kq * 4 + h * 16;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (g < nq && k0 + kk < d)
                        v = *reinterpret_cast<const float4 *>(Q + g * d + k0 + kk);
                    sm.As[kk + 0][r] = v.x;
                    sm.As[kk + 1][r] = v.y;
                    sm.As[kk + 2][r] = v.z;
                    sm.As[kk + 3][r] = v.w;
                }
            }
            // B tile: 128 cols x 32 k
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int r = (tid >> 2) + h * 64, kq = tid & 3;
                int64_t g = col0 + r;
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    int kk = kq * 4 + h2 * 16;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (g < n && k0 + kk < d)
                        v = __ldg(reinterpret_cast<const float4 *>(X + g * d + k0 + kk));
                    sm.Bs[kk + 0][r] = v.x;
                    sm.Bs[kk + 1][r] = v.y;
                    sm.Bs[kk + 2][r] = v.z;
                    sm.Bs[kk + 3][r] = v.w;
                }
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < BK; ++k) {
                float4 a = *reinterpret_cast<const float4 *>(&sm.As[k][ty * 4]);
                float4 b0 = *reinterpret_cast<const float4 *>(&sm.Bs[k][tx * 4]);
                float4 b1 = *reinterpret_cast<const float4 *>(&sm.Bs[k][64 + tx * 4]);
                float av[4] = {a.x, a.y, a.z, a.w};
                float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }

        // distances and filter count
        float dv[4][8];
        int pass_mask[4] = {0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = ty * 4 + i;
            int64_t g = row0 + r;
            float thr = sm.thr[r];
            int np = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int cl = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                int64_t gc = col0 + cl;
                float s;
                if (metric == 0) s = fmaxf(sm.qn[r] + xnorm[gc < n ? gc : 0] - 2.f * acc[i][j], 0.f);
                else s = fmaxf(2.f - 2.f * acc[i][j], 0.f);
                dv[i][j] = s;
                bool ok = g < nq && gc < n && !(self_exclude && gc == g) && s <= thr;
                if (ok) {
                    pass_mask[i] |= 1 << j;
                    ++np;
                }
            }
            if (np) atomicAdd(&sm.pend[r], np);
        }
        __syncthreads();
        // merge rows that could overflow
        for (int r = wid; r < BM; r += NT / 32) {
            if (sm.cnt[r] + sm.pend[r] > BUF) {
                int64_t g = row0 + r;
                merge_row(sm, r, wid, K, out_s + g * K, out_i + g * K);
            }
        }
        __syncthreads();
        // append survivors (re-test: a merge may have lowered the threshold)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (!pass_mask[i]) continue;
            int r = ty * 4 + i;
            float thr = sm.thr[r];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!((pass_mask[i] >> j) & 1)) continue;
                if (!(dv[i][j] <= thr)) continue;
                int cl = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                int slot = atomicAdd(&sm.cnt[r], 1);
                sm.buf_s[r][slot] = dv[i][j];
                sm.buf_i[r][slot] = (int)(col0 + cl);
            }
        }
        __syncthreads();
        for (int r = tid; r < BM; r += NT) sm.pend[r] = 0;
    }
    __syncthreads();
    for (int r = wid; r < BM; r += NT / 32) {
        int64_t g = row0 + r;
        if (g < nq) merge_row(sm, r, wid, K, out_s + g * K, out_i + g * K);
    }
    (void)lane;
}

// Re-order near-tie runs of each sorted row by FP64 distance (one warp per
// row).  Rows hold Kx entries; ties are judged with the per-pair error
// bound of the norm form.  The first K entries are written to the output.
// A run that reaches the last stored entry cannot be closed: counted.
__global__ void k_knn_fix(const float *__restrict__ Q, const float *__restrict__ X, int64_t nq,
                          int d, int metric, const float *__restrict__ qnorm,
                          const float *__restrict__ xnorm, float rel, float abs_err, int Kx, int K,
                          int32_t *__restrict__ ids, float *__restrict__ ds,
                          int32_t *__restrict__ out_i, float *__restrict__ out_s,
                          unsigned long long *counters) {
    int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (q >= nq) return;
    int32_t *ri = ids + q * Kx;
    float *rs = ds + q * Kx;
    const float *qrow = Q + q * d;
    auto err = [&](int j) -> float {
        int id = ri[j];
        if (id < 0) return 0.f;
        if (metric == 0) return rel * (qnorm[q] + xnorm[id] + fabsf(qnorm[q] + xnorm[id] - rs[j]));
        return abs_err;
    };
    // lane 0 walks the row; runs are rare
    if (lane == 0) {
        int j = 0;
        unsigned long long rechecked = 0, unresolved = 0;
        while (j < Kx && ri[j] >= 0) {
            int e = j;
            while (e + 1 < Kx && ri[e + 1] >= 0 && rs[e + 1] - rs[e] <= err(e) + err(e + 1)) ++e;
            if (e > j && j < K) {
                // FP64 distances and insertion sort of the run
                double tmp_d[64];
                int tmp_i[64];
                int m = e - j + 1;
                if (m > 64) m = 64;
                for (int t = 0; t < m; ++t) {
                    tmp_i[t] = ri[j + t];
                    tmp_d[t] = dist64_rows(qrow, X + (int64_t)tmp_i[t] * d, d, metric);
                }
                for (int a = 1; a < m; ++a) {
                    double kd = tmp_d[a];
                    int ki = tmp_i[a];
                    int b = a - 1;
                    while (b >= 0 && (tmp_d[b] > kd || (tmp_d[b] == kd && tmp_i[b] > ki))) {
                        tmp_d[b + 1] = tmp_d[b];
                        tmp_i[b + 1] = tmp_i[b];
                        --b;
                    }
                    tmp_d[b + 1] = kd;
                    tmp_i[b + 1] = ki;
                }
                for (int t = 0; t < m; ++t) {
                    ri[j + t] = tmp_i[t];
                    rs[j + t] = (float)tmp_d[t];
                }
                rechecked += m;
                if (e == Kx - 1 && K < Kx) ++unresolved;
            }
            j = e + 1;
        }
        if (rechecked) atomicAdd(counters + CNT_KNN_RECHECK, rechecked);
        if (unresolved) atomicAdd(counters + CNT_KNN_UNRESOLVED, unresolved);
    }
    __syncwarp();
    // the norm form loses relative accuracy to cancellation: report every
    // kept distance as the rounded FP64 value
    for (int t = lane; t < K; t += 32) {
        int id = ri[t];
        out_i[q * K + t] = id;
        out_s[q * K + t] = id >= 0 ? (float)dist64_rows(qrow, X + (int64_t)id * d, d, metric)
                                   : INFINITY;
    }
}

// Screened form on non-integer data: the Kx BF16-nearest candidates of a
// row re-measured in FP32 (difference form / chord, the same arithmetic as
// the FP32 gathers) and the K best by (s, id) kept.  One warp per row.
__global__ void k_knn_rerank(const float *__restrict__ Q, const float *__restrict__ X, int64_t nq,
                             int d, int metric, int Kx, int K, const int32_t *__restrict__ ci,
                             int32_t *__restrict__ out_i, float *__restrict__ out_s) {
    __shared__ float ks[8][128];
    __shared__ int kid[8][128];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int64_t row = (int64_t)blockIdx.x * 8 + w;
    if (row >= nq) return;
    for (int j = lane; j < 128; j += 32) {
        ks[w][j] = INFINITY;
        kid[w][j] = INT_MAX;
    }
    __syncwarp();
    const float4 *q4 = reinterpret_cast<const float4 *>(Q + row * d);
    for (int b0 = 0; b0 < Kx; b0 += 4) {
        const int j = b0 + team;
        const int id = j < Kx ? ci[row * Kx + j] : -1;
        const float sv = team8_dist(q4, reinterpret_cast<const float4 *>(X + (int64_t)(id >= 0 ? id : 0) * d),
                                    d / 4, li, metric);
        if (li == 0 && id >= 0) {
            ks[w][j] = sv;
            kid[w][j] = id;
        }
    }
    __syncwarp();
    warp_bitonic_sort(ks[w], kid[w], 128);
    for (int t = lane; t < K; t += 32) {
        const bool ok = kid[w][t] != INT_MAX;
        out_i[row * K + t] = ok ? kid[w][t] : -1;
        out_s[row * K + t] = ok ? ks[w][t] : INFINITY;
    }
}

}  // namespace

bool pg_knn_tc_supported(int d, int K);
int pg_knn_tc_max_k();
pg_status pg_knn_tc(pg_ctx *ctx, const float *D, int64_t n, int32_t d, const float *Q, int64_t nq,
                    int self, int32_t K, const float *xnorm, const float *qnorm, int32_t *ids,
                    float *dist);

namespace {

pg_status knn_core(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                   const float *Q, int64_t nq, int self, int32_t K, pg_precision precision,
                   int32_t *ids, float *dist) {
    if (!D || !ids || !dist || (!Q && !self)) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || nq < 0 || d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "knn: need n >= 1, d % 4 == 0, 4 <= d <= 8192");
    if (K < 1 || K > KMAX) return pg_fail(ctx, PG_ERR_INVALID_ARG, "knn: need 1 <= K <= %d", KMAX);
    if (!pg_build_precision(precision))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "knn takes FP32 or BF16 screening");
    if (nq == 0) return PG_OK;
    const float *Qp = self ? D : Q;
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, D, n, d, metric, &facts));
    if (!self) {
        DataFacts fq;
        PG_TRY(pg_data_facts(ctx, Q, nq, d, metric, &fq));
        facts.exact = facts.exact && fq.exact;
        facts.max_norm2 = fmaxf(facts.max_norm2, fq.max_norm2);
    }
    Scratch<float> xn, qn;
    PG_TRY(xn.alloc(ctx, (size_t)n));
    k_row_norms<<<(unsigned)((n + 7) / 8), 256, 0, ctx->stream>>>(D, n, d, xn.p);
    PG_LAUNCHED(ctx);
    const float *qnp = xn.p;
    if (!self) {
        PG_TRY(qn.alloc(ctx, (size_t)nq));
        k_row_norms<<<(unsigned)((nq + 7) / 8), 256, 0, ctx->stream>>>(Q, nq, d, qn.p);
        PG_LAUNCHED(ctx);
        qnp = qn.p;
    }
    // BF16 tiles on the tensor cores when the BF16 copy and every partial
    // sum are exact (integer data): the result equals the FP32 form's
    if (precision == PG_PREC_BF16_SCREEN && metric == PG_METRIC_L2SQ && facts.exact &&
        facts.bf16_exact && pg_knn_tc_supported(d, K))
        return pg_knn_tc(ctx, D, n, d, self ? nullptr : Q, nq, self, K, xn.p, qnp, ids, dist);
    // Other data in the screened form: the Ks = min(128, max(2K, K + 8))
    // nearest by BF16 tiles (the BF16 rounding moves distances by up to
    // ~2^-8 (|x| + |y|) sqrt(s)), re-measured in FP32 and cut to K.
    // Membership at the K-th place can differ from the exact kNN; the
    // candidate order and distances are FP32.
    const int Ks = std::min(pg_knn_tc_max_k(), std::max(2 * K, K + 8));
    if (precision == PG_PREC_BF16_SCREEN && !(facts.exact && facts.bf16_exact) && Ks >= K + 8 &&
        pg_knn_tc_supported(d, Ks)) {
        Scratch<int32_t> wi;
        Scratch<float> ws;
        PG_TRY(wi.alloc(ctx, (size_t)nq * Ks));
        PG_TRY(ws.alloc(ctx, (size_t)nq * Ks));
        PG_TRY(pg_knn_tc(ctx, D, n, d, self ? nullptr : Q, nq, self, Ks, xn.p, qnp, wi.p, ws.p));
        k_knn_rerank<<<(unsigned)((nq + 7) / 8), 256, 0, ctx->stream>>>(
            Qp, D, nq, d, metric == PG_METRIC_L2SQ ? 0 : 1, Ks, K, wi.p, ids, dist);
        PG_LAUNCHED(ctx);
        return PG_OK;
    }
    // rows hold Kx entries when ties must be resolved in FP64 afterwards
    int Kx = facts.exact ? K : (int)std::min<int64_t>((int64_t)K + 8, KMAX);
    Scratch<int32_t> wi;
    Scratch<float> ws;
    int32_t *ti = ids;
    float *ts = dist;
    if (Kx != K) {
        PG_TRY(wi.alloc(ctx, (size_t)nq * Kx));
        PG_TRY(ws.alloc(ctx, (size_t)nq * Kx));
        ti = wi.p;
        ts = ws.p;
    }
    size_t smem = sizeof(KnnSmem);
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(k_knn_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    unsigned blocks = (unsigned)((nq + BM - 1) / BM);
    pg_timer_begin(ctx, TM_KNN);
    k_knn_fp32<<<blocks, NT, smem, ctx->stream>>>(Qp, nq, D, n, d, qnp, xn.p,
                                                  metric == PG_METRIC_L2SQ ? 0 : 1, Kx, self, ti,
                                                  ts);
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_KNN, 2.0 * (double)nq * (double)n * (double)d);
    if (Kx != K) {
        ErrModel em = pg_err_model(metric, d, facts, true);
        k_knn_fix<<<(unsigned)((nq + 7) / 8), 256, 0, ctx->stream>>>(
            Qp, D, nq, d, metric == PG_METRIC_L2SQ ? 0 : 1, qnp, xn.p, em.rel, em.abs_, Kx, K, ti,
            ts, ids, dist, ctx->d_counters);
        PG_LAUNCHED(ctx);
    }
    return PG_OK;
}

}  // namespace

pg_status pg_knn_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                          int32_t K, pg_precision precision, int32_t *ids, float *dist) {
    return knn_core(ctx, D, n, d, metric, nullptr, n, 1, K, precision, ids, dist);
}

pg_status pg_knn_query_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                pg_metric metric, const float *Q, int64_t nq, int32_t k,
                                pg_precision precision, int32_t *ids, float *dist) {
    return knn_core(ctx, D, n, d, metric, Q, nq, 0, k, precision, ids, dist);
}

extern "C" pg_status pg_build_knn(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  pg_metric metric, int32_t K, pg_precision precision,
                                  int32_t *ids, float *dist) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    PG_TRY(knn_core(ctx, D, n, d, metric, nullptr, n, 1, K, precision, ids, dist));
    return pg_sync_check(ctx, "pg_build_knn");
}

extern "C" pg_status pg_knn_query(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  pg_metric metric, const float *Q, int64_t nq, int32_t k,
                                  pg_precision precision, int32_t *ids, float *dist) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!Q) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null Q");
    PG_TRY(knn_core(ctx, D, n, d, metric, Q, nq, 0, k, precision, ids, dist));
    return pg_sync_check(ctx, "pg_knn_query");
}
