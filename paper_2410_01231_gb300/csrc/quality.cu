// quality.cu -- quality examination of the k-CNA lists (Section 5.2):
// the recall r(u) of the first k entries of C(u) against the exact k
// nearest neighbours of u, on a uniform sample of points whose size meets
// Theorem 3, and the sampled mean that ends Algorithm 6's loop.
//
// The exact neighbours of the sampled points come from the FP32 distance
// tiles with FP64 near-tie fixes (exact by (s, id)); the k-th distance and
// every candidate's distance are then taken in FP64 with the sequential
// coordinate order, so "an entry counts when its distance is at most the
// exact k-th distance" is decided exactly.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "pg_internal.cuh"

pg_status pg_knn_query_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                pg_metric metric, const float *Q, int64_t nq, int32_t k,
                                pg_precision precision, int32_t *ids, float *dist);

namespace {

__global__ void k_gather_sample(const float *__restrict__ D, int64_t n, int d,
                                const int32_t *sample, int64_t ns, float *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nch = d / 4;
    if (t >= ns * nch) return;
    const int64_t r = t / nch, c = t % nch;
    const int64_t u = sample[r];
    if (u < 0 || u >= n) return;  // reported by k_kcna_recall
    reinterpret_cast<float4 *>(out)[r * nch + c] =
        reinterpret_cast<const float4 *>(D + u * d)[c];
}

// One warp per sampled point u.  gt [ns][k + 1] holds the k + 1 nearest
// points of u by (s, id), u itself included; since s(u, u) = 0 is the
// smallest distance, the k-th nearest point other than u has the distance
// of entry k of that list.  r(u) = |{distinct v in C(u)[0..k) \ {u}, v >= 0,
// s(u, v) <= kth}| / k (capped at k).
__global__ void k_kcna_recall(const float *__restrict__ D, int64_t n, int d, int metric,
                              const int32_t *__restrict__ cand, int L, int k,
                              const int32_t *__restrict__ sample, int64_t ns,
                              const int32_t *__restrict__ gt, double *recall, int *err) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= ns) return;
    const int64_t u = sample[i];
    if (u < 0 || u >= n) {
        if (lane == 0) {
            record_error(err, DERR_BAD_ID, u);
            recall[i] = 0.0;
        }
        return;
    }
    const float *xu = D + u * d;
    const int g = gt[i * (k + 1) + k];
    if (g < 0 || g >= n) {
        if (lane == 0) record_error(err, DERR_INTERNAL, u);
        return;
    }
    const double kth = dist64_rows(xu, D + (int64_t)g * d, d, metric);
    const int32_t *row = cand + u * L;
    int hits = 0;
    for (int j = lane; j < k; j += 32) {
        const int v = row[j];
        bool count = v >= 0 && v < n && v != u;
        for (int e = 0; e < j && count; ++e) count = row[e] != v;  // repeated ids count once
        if (count && dist64_rows(xu, D + (int64_t)v * d, d, metric) <= kth) ++hits;
    }
    for (int o = 16; o; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
    if (lane == 0) recall[i] = (double)min(hits, k) / (double)k;
}

uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" int64_t pg_quality_sample_size(int64_t n, double eps, double l) {
    if (n < 2 || !(eps > 0.0) || !(l > 0.0)) return -1;
    return (int64_t)std::ceil((8.0 + 2.0 * eps) * l * std::log((double)n) / (eps * eps));
}

extern "C" pg_status pg_quality_sample(int64_t n, int64_t ns, uint64_t seed, int32_t *host_ids) {
    if (n < 1 || n >= INT_MAX || ns < 0 || ns > n || (ns > 0 && !host_ids))
        return PG_ERR_INVALID_ARG;
    // ns distinct ids: SplitMix64 draws mapped to [0, n) by the high 64 bits of
    // a 64 x 64-bit product, repeats skipped; then sorted ascending
    std::vector<uint8_t> taken((size_t)n, 0);
    int64_t got = 0;
    for (uint64_t c = 0; got < ns; ++c) {
        const uint64_t z = splitmix64(seed ^ (0x51a3c0ffee000000ULL + c));
        const int64_t v = (int64_t)(((unsigned __int128)z * (uint64_t)n) >> 64);
        if (!taken[(size_t)v]) {
            taken[(size_t)v] = 1;
            ++got;
        }
    }
    int64_t w = 0;
    for (int64_t v = 0; v < n && w < ns; ++v)
        if (taken[(size_t)v]) host_ids[w++] = (int32_t)v;
    return PG_OK;
}

// r(u) for every sampled point (device sample [ns], device recall [ns]) and
// their mean (host).
pg_status pg_kcna_recall_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  pg_metric metric, const int32_t *cand, int32_t L, int32_t k,
                                  const int32_t *sample, int64_t ns, double *recall,
                                  double *host_mean) {
    if (ns == 0) {
        if (host_mean) *host_mean = 0.0;
        return PG_OK;
    }
    Scratch<float> Q;
    Scratch<int32_t> gi;
    Scratch<float> gs;
    PG_TRY(Q.alloc(ctx, (size_t)(ns * d)));
    PG_TRY(gi.alloc(ctx, (size_t)(ns * (k + 1))));
    PG_TRY(gs.alloc(ctx, (size_t)(ns * (k + 1))));
    const int64_t tot = ns * (d / 4);
    PG_TRY_CUDA(ctx, cudaMemsetAsync(Q.p, 0, (size_t)(ns * d) * sizeof(float), ctx->stream));
    k_gather_sample<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(D, n, d, sample, ns,
                                                                            Q.p);
    PG_LAUNCHED(ctx);
    PG_TRY(pg_knn_query_internal(ctx, D, n, d, metric, Q.p, ns, k + 1, PG_PREC_FP32, gi.p, gs.p));
    k_kcna_recall<<<(unsigned)((ns + 7) / 8), 256, 0, ctx->stream>>>(
        D, n, d, metric == PG_METRIC_L2SQ ? 0 : 1, cand, L, k, sample, ns, gi.p, recall,
        ctx->d_err);
    PG_LAUNCHED(ctx);
    if (host_mean) {
        std::vector<double> h((size_t)ns);
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(h.data(), recall, (size_t)ns * sizeof(double),
                                         cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY(pg_sync_check(ctx, "quality examination"));
        double s = 0.0;
        for (double v : h) s += v;  // in sample order
        *host_mean = s / (double)ns;
    }
    return PG_OK;
}

// The estimator of one iteration of Algorithm 6: n_s = Theorem 3's size for
// eps (l = 1), a SplitMix64 sample, the mean of r(u).
pg_status pg_quality_estimate(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              const int32_t *cand, int32_t L, int32_t k, double eps, uint64_t seed,
                              double *est, int64_t *ns_out) {
    int64_t ns = pg_quality_sample_size(n, eps, 1.0);
    if (ns < 0) return pg_fail(ctx, PG_ERR_INVALID_ARG, "quality examination: bad eps or n");
    ns = std::min(ns, n);
    std::vector<int32_t> hs((size_t)ns);
    PG_TRY(pg_quality_sample(n, ns, seed, hs.data()));
    Scratch<int32_t> sd;
    Scratch<double> rec;
    PG_TRY(sd.alloc(ctx, (size_t)ns));
    PG_TRY(rec.alloc(ctx, (size_t)ns));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(sd.p, hs.data(), (size_t)ns * 4, cudaMemcpyHostToDevice,
                                     ctx->stream));
    if (ns_out) *ns_out = ns;
    return pg_kcna_recall_internal(ctx, D, n, d, metric, cand, L, k, sd.p, ns, rec.p, est);
}

extern "C" pg_status pg_kcna_recall(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                    pg_metric metric, const int32_t *cand, int32_t L, int32_t k,
                                    const int32_t *sample, int64_t ns, double *recall,
                                    double *host_mean) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !cand || (ns > 0 && (!sample || !recall)))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 2 || n >= INT_MAX || d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 2 <= n < 2^31, d % 4 == 0, 4 <= d <= 8192");
    if (k < 1 || k > 255 || k > L || k >= n || ns < 0)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= k <= min(L, 255), k < n, ns >= 0");
    PG_TRY(pg_kcna_recall_internal(ctx, D, n, d, metric, cand, L, k, sample, ns, recall,
                                   host_mean));
    return pg_sync_check(ctx, "pg_kcna_recall");
}
