// build.cu -- the construction pipelines and the index object.
//
// pg_build_rng: IterNSG with a fixed number of iterations (Algorithm 6),
// each iteration one OptKCNA (Algorithm 5): alpha-prune C -> reverse-edge
// union -> alpha-prune -> connect -> self-search for new C; then the final
// refinement steps of Algorithm 2 at alpha_final.  The graph,
// vectors and candidate lists stay on the device for the whole build; the
// host only reads scalars (the medoid id, connectivity progress).
//
// pg_build_nswg: OptHNSW (Algorithm 7): levels drawn up front, each layer
// built independently (complete graph when small, otherwise IterNSG on the
// gathered layer without the final connectivity step).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>

#include "pg_internal.cuh"

pg_status pg_knn_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                          int32_t K, pg_precision precision, int32_t *ids, float *dist);
pg_status pg_prune_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                            const int64_t *off, const int32_t *cand, int32_t R, double alpha_deg,
                            const DataFacts &facts, int32_t *nbr, int32_t *deg,
                            const uint8_t *D8 = nullptr, int64_t rows = 0,
                            const int32_t *self_ids = nullptr, const int32_t *prev_nbr = nullptr,
                            const int32_t *prev_deg = nullptr, int32_t prev_R = 0);
pg_status pg_reverse_union_internal(pg_ctx *ctx, const int32_t *nbr, const int32_t *deg, int64_t n,
                                    int32_t R, int64_t *off, int32_t *ids);
pg_status pg_medoid_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             int64_t *host_ep);
pg_status pg_connect_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              int32_t *nbr, int32_t *deg, int32_t R, int64_t ep,
                              const DataFacts &facts, const int32_t *knn, int32_t K,
                              int64_t *host_added);
pg_status pg_connect_replace_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                      pg_metric metric, int32_t *nbr, int32_t *deg, int32_t R,
                                      int64_t ep, const DataFacts &facts, const int32_t *knn,
                                      int32_t K, int64_t *host_added, int64_t *host_replaced);
pg_status pg_knn_descent_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  pg_metric metric, int32_t K, int32_t iters,
                                  const int32_t *init, uint64_t seed, int32_t *ids, float *dist,
                                  int64_t *host_updates);
pg_status pg_quality_estimate(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              const int32_t *cand, int32_t L, int32_t k, double eps, uint64_t seed,
                              double *est, int64_t *ns_out);

namespace {

enum { PH_KNN = 0, PH_PRUNE, PH_UNION, PH_CONNECT, PH_ACQUIRE, PH_LAYERS };

struct PhaseClock {
    pg_ctx *ctx;
    double *acc;
    std::chrono::steady_clock::time_point t0;
    int cur = -1;
    void start(int ph) {
        stop();
        cudaStreamSynchronize(ctx->stream);
        t0 = std::chrono::steady_clock::now();
        cur = ph;
    }
    void stop() {
        if (cur < 0) return;
        cudaStreamSynchronize(ctx->stream);
        acc[cur] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        cur = -1;
    }
};

__global__ void k_fill_off(int64_t *off, int64_t n, int64_t stride) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) off[i] = i * stride;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_gather_rows(const float *D, int d, const int32_t *gid, int64_t m, float *out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nch = d / 4;
    if (t >= m * nch) return;
    int64_t r = t / nch, c = t % nch;
    reinterpret_cast<float4 *>(out)[r * nch + c] =
        reinterpret_cast<const float4 *>(D + (int64_t)gid[r] * d)[c];
}

__global__ void k_map_ids(int32_t *nbr, int64_t total, const int32_t *gid) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int v = nbr[t];
    if (v >= 0) nbr[t] = gid[v];
}

__global__ void k_rows_map(const int32_t *gid, int64_t m, int32_t *rows) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) rows[gid[t]] = (int32_t)t;
}

// complete layer: row a = every other member by FP64 (s, id); one warp/row
__global__ void k_complete_layer(const float *D, int d, int metric, const int32_t *gid, int m,
                                 int R, int32_t *nbr, int32_t *deg) {
    int a = blockIdx.x;
    if (a >= m || threadIdx.x != 0) return;
    double ds[64];
    int id[64];
    int c = 0;
    const float *xa = D + (int64_t)gid[a] * d;
    for (int b = 0; b < m && c < 64; ++b) {
        if (b == a) continue;
        ds[c] = dist64_rows(xa, D + (int64_t)gid[b] * d, d, metric);
        id[c] = gid[b];
        ++c;
    }
    for (int i = 1; i < c; ++i) {
        double kd = ds[i];
        int ki = id[i];
        int j = i - 1;
        while (j >= 0 && (ds[j] > kd || (ds[j] == kd && id[j] > ki))) {
            ds[j + 1] = ds[j];
            id[j + 1] = id[j];
            --j;
        }
        ds[j + 1] = kd;
        id[j + 1] = ki;
    }
    for (int j = 0; j < R; ++j) nbr[(int64_t)a * R + j] = j < c ? id[j] : -1;
    deg[a] = c < R ? c : R;
}

uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Level of a point: floor(-ln U / ln M), U = ((z >> 11) + 1) 2^-53 with
// z = SplitMix64(seed XOR id) -- the exponentially decaying level draw of
// Algorithm 4 / Algorithm 7.
int level_of(int64_t id, uint64_t seed, int M) {
    const uint64_t z = splitmix64(seed ^ (uint64_t)id);
    const double U = (double)((z >> 11) + 1) * (1.0 / 9007199254740992.0);
    return (int)std::floor(-std::log(U) / std::log((double)M));
}

std::vector<int> draw_levels(int64_t n, uint64_t seed, int M) {
    std::vector<int> lev((size_t)n);
    for (int64_t i = 0; i < n; ++i) lev[(size_t)i] = level_of(i, seed, M);
    return lev;
}

pg_status check_params(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                       const pg_build_params *p) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !p) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 2 || n >= INT_MAX) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 2 <= n < 2^31");
    if (d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need d % 4 == 0 and 4 <= d <= 8192");
    if (p->K < 1 || p->K > 256) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= K <= 256");
    if (p->L < 1 || p->L > 256) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= L <= 256");
    if (p->R < 1 || p->R > 64) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= R <= 64");
    if (p->M < 2 || p->M > 64) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 2 <= M <= 64");
    if (p->iters < 0 || p->iters > 16) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 0 <= I <= 16");
    if (!(p->alpha_deg >= 0 && p->alpha_deg <= 180 && p->alpha_final_deg >= 0 &&
          p->alpha_final_deg <= 180))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 0 <= alpha <= 180");
    if (p->metric < PG_METRIC_L2SQ || p->metric > PG_METRIC_IP)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "bad metric");
    if (!pg_build_precision(p->precision))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "builds take FP32 or BF16 screening");
    if (p->knn_descent_iters > 64 || (p->knn_descent_iters >= 0 && p->K > 64))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "kNN descent: need iterations <= 64 and K <= 64");
    if (!(p->quality_target >= 0.0 && p->quality_target <= 1.0) ||
        (p->quality_target > 0.0 && !(p->quality_eps > 0.0)) || p->quality_k < 0 ||
        p->quality_k > 255)
        return pg_fail(ctx, PG_ERR_INVALID_ARG,
                       "need 0 <= quality_target <= 1, quality_eps > 0, 0 <= quality_k <= 255");
    return PG_OK;
}

// IterNSG on a dense dataset X [m][d]: writes nbr [m][R] / deg [m] (local ids)
// Quality examination record of one IterNSG run.
struct QualityRecord {
    int32_t iters = 0;
    int64_t ns = 0;
    double est[16] = {0};
};

pg_status iter_nsg(pg_ctx *ctx, const float *X, int64_t m, int32_t d, const pg_build_params *p,
                   int R, int connect_final, int32_t *nbr, int32_t *deg, int64_t *ep_out,
                   double *phase, QualityRecord *qrec = nullptr) {
    PhaseClock clk{ctx, phase};
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, X, m, d, p->metric, &facts));
    int64_t ep = 0;
    PG_TRY(pg_medoid_internal(ctx, X, m, d, p->metric, &ep));
    *ep_out = ep;
    const int K = (int)std::min<int64_t>(p->K, m - 1);
    const int L = p->L;
    Scratch<int32_t> knn_i, cand, nbr1, deg1, uids, pv1n, pv1d, pv2n, pv2d;
    Scratch<float> knn_s;
    Scratch<int64_t> off, uoff;
    PG_TRY(knn_i.alloc(ctx, (size_t)(m * K)));
    PG_TRY(knn_s.alloc(ctx, (size_t)(m * K)));
    PG_TRY(off.alloc(ctx, (size_t)m + 1));
    PG_TRY(uoff.alloc(ctx, (size_t)m + 1));
    PG_TRY(nbr1.alloc(ctx, (size_t)(m * R)));
    PG_TRY(deg1.alloc(ctx, (size_t)m));
    PG_TRY(uids.alloc(ctx, (size_t)(2 * m * R)));
    clk.start(PH_KNN);
    if (p->knn_descent_iters >= 0)  // approximate initial KNNG (Section 3.1, Exp. 12)
        PG_TRY(pg_knn_descent_internal(ctx, X, m, d, p->metric, K, p->knn_descent_iters, nullptr,
                                       p->seed, knn_i.p, knn_s.p, nullptr));
    else
        PG_TRY(pg_knn_internal(ctx, X, m, d, p->metric, K, p->precision, knn_i.p, knn_s.p));
    knn_s.release();
    const unsigned g1 = (unsigned)((m + 256) / 256);
    k_fill_off<<<g1, 256, 0, ctx->stream>>>(off.p, m, K);
    PG_LAUNCHED(ctx);
    const int32_t *cur = knn_i.p;
    // the screened form gathers byte rows when the data are exact bytes
    Scratch<uint8_t> x8;
    if (pg_u8_usable(facts, p->metric, d, p->precision)) PG_TRY(pg_make_u8(ctx, X, m, d, x8));
    // K2P (Section 5.4): each pass may reuse the previous refinement's
    // pass of the same kind (pass 1 on C(u), pass 2 on the union rows before
    // connectivity) when its angle is at least the previous one
    const bool k2p = p->reuse_pruning &&
                     (p->iters >= 2 || (p->iters >= 1 && p->alpha_final_deg >= p->alpha_deg));
    if (k2p) {
        PG_TRY(pv1n.alloc(ctx, (size_t)(m * R)));
        PG_TRY(pv1d.alloc(ctx, (size_t)m));
        PG_TRY(pv2n.alloc(ctx, (size_t)(m * R)));
        PG_TRY(pv2d.alloc(ctx, (size_t)m));
    }
    int refines = 0;
    double prev_alpha = 0.0;
    auto refine = [&](double alpha, int do_connect, bool last) -> pg_status {
        const bool reuse = k2p && refines > 0 && alpha >= prev_alpha;
        clk.start(PH_PRUNE);
        if (reuse) {
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(pv1n.p, nbr1.p, (size_t)(m * R) * 4,
                                             cudaMemcpyDeviceToDevice, ctx->stream));
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(pv1d.p, deg1.p, (size_t)m * 4,
                                             cudaMemcpyDeviceToDevice, ctx->stream));
        }
        PG_TRY(pg_prune_internal(ctx, X, m, d, p->metric, off.p, cur, R, alpha, facts, nbr1.p,
                                 deg1.p, x8.p, 0, nullptr, reuse ? pv1n.p : nullptr,
                                 reuse ? pv1d.p : nullptr, R));
        clk.start(PH_UNION);
        PG_TRY(pg_reverse_union_internal(ctx, nbr1.p, deg1.p, m, R, uoff.p, uids.p));
        clk.start(PH_PRUNE);
        PG_TRY(pg_prune_internal(ctx, X, m, d, p->metric, uoff.p, uids.p, R, alpha, facts, nbr,
                                 deg, x8.p, 0, nullptr, reuse ? pv2n.p : nullptr,
                                 reuse ? pv2d.p : nullptr, R));
        if (k2p && !last) {  // pass-2 lists before connectivity, for the next refinement
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(pv2n.p, nbr, (size_t)(m * R) * 4,
                                             cudaMemcpyDeviceToDevice, ctx->stream));
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(pv2d.p, deg, (size_t)m * 4,
                                             cudaMemcpyDeviceToDevice, ctx->stream));
        }
        ++refines;
        prev_alpha = alpha;
        if (do_connect) {
            clk.start(PH_CONNECT);
            if (p->connect_replace)
                PG_TRY(pg_connect_replace_internal(ctx, X, m, d, p->metric, nbr, deg, R, ep, facts,
                                                   knn_i.p, K, nullptr, nullptr));
            else
                PG_TRY(pg_connect_internal(ctx, X, m, d, p->metric, nbr, deg, R, ep, facts,
                                           knn_i.p, K, nullptr));
        }
        return PG_OK;
    };
    // Algorithm 6: OptKCNA iterations until the quality examination
    // (Section 5.2) accepts the k-CNA lists, at most `iters` of them; with
    // the examination off, exactly `iters`
    const bool qexam = p->quality_target > 0.0;
    const int qk = std::min(p->quality_k > 0 ? p->quality_k : K, std::min(L, 255));
    QualityRecord q;
    for (int it = 0; it < p->iters; ++it) {
        PG_TRY(refine(p->alpha_deg, 1, false));
        if (!cand.p) PG_TRY(cand.alloc(ctx, (size_t)(m * L)));
        clk.start(PH_ACQUIRE);
        PG_TRY(pg_search_internal(ctx, X, m, d, p->metric, nbr, deg, R, nullptr, nullptr, m,
                                  nullptr, L, L, 1, cand.p, nullptr, x8.p, nullptr, &facts));
        k_fill_off<<<g1, 256, 0, ctx->stream>>>(off.p, m, L);
        PG_LAUNCHED(ctx);
        cur = cand.p;
        q.iters = it + 1;
        if (qexam && qk < m) {
            clk.stop();
            double est = 0.0;
            PG_TRY(pg_quality_estimate(ctx, X, m, d, p->metric, cand.p, L, qk, p->quality_eps,
                                       p->seed + (uint64_t)it, &est, &q.ns));
            if (it < 16) q.est[it] = est;
            if (est >= p->quality_target) break;
        }
    }
    if (qrec) *qrec = q;
    PG_TRY(refine(p->alpha_final_deg, connect_final, true));
    clk.stop();
    return pg_sync_check(ctx, "build");
}

pg_status alloc_layer(pg_ctx *ctx, pg_layer &l, int64_t count, int R, int64_t n, bool ident) {
    l.count = count;
    l.cap = count;
    l.R = R;
    PG_TRY_CUDA(ctx, cudaMalloc(&l.nbr, (size_t)(count * R) * sizeof(int32_t)));
    PG_TRY_CUDA(ctx, cudaMalloc(&l.deg, (size_t)count * sizeof(int32_t)));
    if (!ident) {
        PG_TRY_CUDA(ctx, cudaMalloc(&l.gid, (size_t)count * sizeof(int32_t)));
        PG_TRY_CUDA(ctx, cudaMalloc(&l.rows, (size_t)n * sizeof(int32_t)));
    }
    return PG_OK;
}

// Upper layers i >= first of Algorithm 7 (layer 0 handled by the caller).
pg_status build_layers(pg_ctx *ctx, pg_index *idx, const float *D, int64_t n, int32_t d,
                       const pg_build_params *p, int first) {
    std::vector<int> lev = draw_levels(n, p->seed, p->M);
    int top = 0;
    for (int v : lev) top = std::max(top, v);
    idx->layers.resize((size_t)std::max(top + 1, 1));
    for (int i = std::max(first, 1); i <= top; ++i) {
        std::vector<int32_t> gid;
        for (int64_t u = 0; u < n; ++u)
            if (lev[(size_t)u] >= i) gid.push_back((int32_t)u);
        const int64_t m = (int64_t)gid.size();
        const int Ri = p->M;
        pg_layer &lay = idx->layers[(size_t)i];
        PG_TRY(alloc_layer(ctx, lay, m, Ri, n, false));
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(lay.gid, gid.data(), (size_t)m * 4, cudaMemcpyHostToDevice,
                                         ctx->stream));
        k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(lay.rows, n, -1);
        PG_LAUNCHED(ctx);
        k_rows_map<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(lay.gid, m, lay.rows);
        PG_LAUNCHED(ctx);
        if (m <= Ri) {
            k_complete_layer<<<(unsigned)m, 32, 0, ctx->stream>>>(
                D, d, p->metric == PG_METRIC_L2SQ ? 0 : 1, lay.gid, (int)m, Ri, lay.nbr, lay.deg);
            PG_LAUNCHED(ctx);
        } else {
            Scratch<float> X;
            PG_TRY(X.alloc(ctx, (size_t)(m * d)));
            int64_t tot = m * (d / 4);
            k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(D, d, lay.gid, m,
                                                                                  X.p);
            PG_LAUNCHED(ctx);
            int64_t ep_local = 0;
            double ph[6] = {0, 0, 0, 0, 0, 0};
            PG_TRY(iter_nsg(ctx, X.p, m, d, p, Ri, 0, lay.nbr, lay.deg, &ep_local, ph));
            int64_t tn = m * Ri;
            k_map_ids<<<(unsigned)((tn + 255) / 256), 256, 0, ctx->stream>>>(lay.nbr, tn, lay.gid);
            PG_LAUNCHED(ctx);
        }
        if (i == top) idx->ep_top = gid[0];
    }
    if (top == 0) idx->ep_top = idx->ep_base;
    return pg_sync_check(ctx, "layers");
}

pg_status build_common(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                       const pg_build_params *p, bool rng, pg_index **out) {
    PG_TRY(check_params(ctx, D, n, d, p));
    if (!out) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    pg_index *idx = new (std::nothrow) pg_index();
    if (!idx) return pg_fail(ctx, PG_ERR_OOM, "host allocation");
    idx->n = n;
    idx->d = d;
    idx->metric = p->metric;
    idx->D = D;
    idx->params = *p;
    idx->layers.resize(1);
    pg_status st = alloc_layer(ctx, idx->layers[0], n, p->R, n, true);
    int64_t ep = 0;
    QualityRecord q;
    if (st == PG_OK)
        st = iter_nsg(ctx, D, n, d, p, p->R, rng ? p->connect_final : 0, idx->layers[0].nbr,
                      idx->layers[0].deg, &ep, idx->phase, &q);
    if (st == PG_OK) {
        st = pg_data_facts(ctx, D, n, d, p->metric, &idx->facts);
        idx->has_facts = st == PG_OK;
    }
    idx->iters_run = q.iters;
    idx->quality_ns = q.ns;
    memcpy(idx->quality_est, q.est, sizeof q.est);
    idx->ep_base = ep;
    idx->ep_top = ep;
    if (st == PG_OK && (!rng || p->route_layers)) {
        auto t0 = std::chrono::steady_clock::now();
        st = build_layers(ctx, idx, D, n, d, p, 1);
        idx->phase[PH_LAYERS] +=
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (st != PG_OK) {
        delete idx;
        return st;
    }
    *out = idx;
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_build_rng(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  const pg_build_params *params, pg_index **out) {
    return build_common(ctx, D, n, d, params, true, out);
}

extern "C" pg_status pg_build_rng_host(pg_ctx *ctx, const float *D_host, int64_t n, int32_t d,
                                       const pg_build_params *params, int32_t *nbr_host,
                                       int32_t *deg_host, pg_index **out) {
    PG_TRY(check_params(ctx, D_host, n, d, params));
    if (!nbr_host || !deg_host) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (out) *out = nullptr;
    float *Dd = nullptr;
    PG_TRY_CUDA(ctx, cudaMalloc(&Dd, (size_t)(n * d) * sizeof(float)));
    cudaError_t e = cudaMemcpyAsync(Dd, D_host, (size_t)(n * d) * sizeof(float),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(Dd);
        return pg_cuda_fail(ctx, e, "pg_build_rng_host upload");
    }
    pg_index *idx = nullptr;
    pg_status st = build_common(ctx, Dd, n, d, params, true, &idx);
    if (st != PG_OK) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(Dd);
        return st;
    }
    idx->owned = Dd;  // the index owns the uploaded points from here on
    idx->capacity = n;
    const pg_layer &b = idx->layers[0];
    e = cudaMemcpyAsync(nbr_host, b.nbr, (size_t)(n * b.R) * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(deg_host, b.deg, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e != cudaSuccess) {
        delete idx;
        return pg_cuda_fail(ctx, e, "pg_build_rng_host download");
    }
    st = pg_sync_check(ctx, "pg_build_rng_host");
    if (st != PG_OK || !out) {
        delete idx;
        return st;
    }
    *out = idx;
    return PG_OK;
}

extern "C" pg_status pg_build_nswg(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                   const pg_build_params *params, pg_index **out) {
    return build_common(ctx, D, n, d, params, false, out);
}

extern "C" pg_status pg_levels(int64_t n, uint64_t seed, int32_t M, int32_t *host_levels) {
    if (n < 0 || M < 2 || (n > 0 && !host_levels)) return PG_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i) host_levels[i] = level_of(i, seed, M);
    return PG_OK;
}

extern "C" void pg_index_destroy(pg_index *index) { delete index; }

int pg_index_dim(const pg_index *index) { return index->d; }

extern "C" pg_status pg_index_info(const pg_index *idx, int32_t *n_layers, int64_t *n,
                                   int64_t *ep_top, int64_t *ep_base) {
    if (!idx) return PG_ERR_INVALID_ARG;
    if (n_layers) *n_layers = (int32_t)idx->layers.size();
    if (n) *n = idx->n;
    if (ep_top) *ep_top = idx->ep_top;
    if (ep_base) *ep_base = idx->ep_base;
    return PG_OK;
}

extern "C" pg_status pg_index_layer(const pg_index *idx, int32_t layer, int64_t *count, int32_t *R,
                                    const int32_t **gid, const int32_t **nbr,
                                    const int32_t **deg) {
    if (!idx || layer < 0 || layer >= (int32_t)idx->layers.size()) return PG_ERR_INVALID_ARG;
    const pg_layer &l = idx->layers[(size_t)layer];
    if (count) *count = l.count;
    if (R) *R = l.R;
    if (gid) *gid = l.gid;
    if (nbr) *nbr = l.nbr;
    if (deg) *deg = l.deg;
    return PG_OK;
}

__global__ void k_iota(int32_t *p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

extern "C" pg_status pg_index_export_layer(pg_ctx *ctx, const pg_index *idx, int32_t layer,
                                           int32_t *gid, int32_t *nbr, int32_t *deg) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!idx || layer < 0 || layer >= (int32_t)idx->layers.size())
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "bad index or layer");
    const pg_layer &l = idx->layers[(size_t)layer];
    if (nbr)
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(nbr, l.nbr, (size_t)(l.count * l.R) * 4,
                                         cudaMemcpyDeviceToDevice, ctx->stream));
    if (deg)
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(deg, l.deg, (size_t)l.count * 4, cudaMemcpyDeviceToDevice,
                                         ctx->stream));
    if (gid) {
        if (l.gid) {
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(gid, l.gid, (size_t)l.count * 4,
                                             cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            k_iota<<<(unsigned)((l.count + 255) / 256), 256, 0, ctx->stream>>>(gid, l.count);
            PG_LAUNCHED(ctx);
        }
    }
    return pg_sync_check(ctx, "pg_index_export_layer");
}

extern "C" pg_status pg_index_quality(const pg_index *idx, int32_t *iters_run,
                                      int64_t *sample_size, double *host_estimates) {
    if (!idx) return PG_ERR_INVALID_ARG;
    if (iters_run) *iters_run = idx->iters_run;
    if (sample_size) *sample_size = idx->quality_ns;
    if (host_estimates)
        for (int i = 0; i < std::min(idx->iters_run, 16); ++i) host_estimates[i] = idx->quality_est[i];
    return PG_OK;
}

extern "C" pg_status pg_index_phase_seconds(const pg_index *idx, double *host_seconds6) {
    if (!idx || !host_seconds6) return PG_ERR_INVALID_ARG;
    memcpy(host_seconds6, idx->phase, sizeof idx->phase);
    return PG_OK;
}

// The FP8 rows of the index for screened queries, made or extended on this
// context's stream (rows added by insertions are encoded on first use).
// Serialised per index: concurrent searches of a serving loop wait for one
// encoding, which completes before the lock is released.
static pg_status index_f8(pg_ctx *ctx, const pg_index *idx, int64_t n, F8Rows *out) {
    std::lock_guard<std::mutex> lk(idx->f8_mu);
    const int64_t cap = std::max(n, idx->capacity);
    if (idx->f8_cap < cap) {
        cudaFree(idx->f8);
        cudaFree(idx->f8_scale);
        idx->f8 = nullptr;
        idx->f8_scale = nullptr;
        idx->f8_rows = idx->f8_cap = 0;
        PG_TRY_CUDA(ctx, cudaMalloc(&idx->f8, (size_t)(cap * idx->d)));
        PG_TRY_CUDA(ctx, cudaMalloc(&idx->f8_scale, (size_t)cap * 4));
        idx->f8_cap = cap;
    }
    if (idx->f8_rows < n) {
        PG_TRY(pg_make_f8(ctx, idx->D, idx->f8_rows, n, idx->d, idx->f8, idx->f8_scale));
        PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        idx->f8_rows = n;
    }
    *out = F8Rows{idx->f8, idx->f8_scale};
    return PG_OK;
}

// Queries on one published version of the index (the snapshot sn).
static pg_status search_index(pg_ctx *ctx, const IndexSnap &sn, const float *Q, int64_t nq,
                              int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                              pg_precision precision, int32_t *out_ids, float *out_dist) {
    if (nq == 0) return PG_OK;
    const pg_index *idx = sn.idx;
    F8Rows f8{};
    if (precision == PG_PREC_FP8_SCREEN) PG_TRY(index_f8(ctx, idx, sn.n, &f8));
    // exactness of every (query, point) distance, for the search's comparator
    DataFacts facts;
    if (sn.has_facts) facts = sn.facts;
    else PG_TRY(pg_data_facts(ctx, idx->D, sn.n, idx->d, idx->metric, &facts));
    PG_TRY(pg_query_facts(ctx, Q, nq, idx->d, idx->metric, &facts));
    Scratch<int32_t> w, w2;
    Scratch<float> s2;
    PG_TRY(w.alloc(ctx, (size_t)nq));
    const bool layered = sn.layers.size() > 1 && !(flags & PG_SEARCH_FLAT);
    k_fill_i32<<<(unsigned)((nq + 255) / 256), 256, 0, ctx->stream>>>(
        w.p, nq, (int32_t)(layered ? sn.ep_top : sn.ep_base));
    PG_LAUNCHED(ctx);
    if (layered) {
        PG_TRY(w2.alloc(ctx, (size_t)nq));
        PG_TRY(s2.alloc(ctx, (size_t)nq));
        for (int i = (int)sn.layers.size() - 1; i >= 1; --i) {
            const pg_layer &l = sn.layers[(size_t)i];
            PG_TRY(pg_search_internal(ctx, idx->D, sn.n, idx->d, idx->metric, l.nbr, l.deg, l.R,
                                      l.rows, Q, nq, w.p, 1, upper_beam, 0, w2.p, s2.p, nullptr,
                                      nullptr, &facts));
            std::swap(w.p, w2.p);
        }
    }
    const pg_layer &b = sn.layers[0];
    return pg_search_internal(ctx, idx->D, sn.n, idx->d, idx->metric, b.nbr, b.deg, b.R, nullptr,
                              Q, nq, w.p, k, beam, 0, out_ids, out_dist, nullptr,
                              precision == PG_PREC_FP8_SCREEN ? &f8 : nullptr, &facts);
}

static pg_status check_search(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                              int32_t k, int32_t beam, int32_t upper_beam, pg_precision precision,
                              const void *a, const void *b) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!idx || !Q || !a || !b) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (nq < 0 || k < 1 || beam < k || beam > 256 || upper_beam < 1 || upper_beam > 256)
        return pg_fail(ctx, PG_ERR_INVALID_ARG,
                       "need 1 <= k <= beam <= 256 and 1 <= upper_beam <= 256");
    if (precision != PG_PREC_FP32 && precision != PG_PREC_BF16_SCREEN &&
        precision != PG_PREC_FP8_SCREEN)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "bad precision");
    return PG_OK;
}

extern "C" pg_status pg_search(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                               int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                               pg_precision precision, int32_t *out_ids, float *out_dist) {
    PG_TRY(check_search(ctx, idx, Q, nq, k, beam, upper_beam, precision, out_ids, out_dist));
    const IndexSnap sn(idx);  // a reader of this version until the work has synchronised
    PG_TRY(search_index(ctx, sn, Q, nq, k, beam, upper_beam, flags, precision, out_ids,
                        out_dist));
    return pg_sync_check(ctx, "pg_search");
}

pg_status pg_search_pinned(pg_ctx *ctx, const IndexSnap &sn, const float *Q, int64_t nq,
                           int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                           pg_precision precision, int32_t *out_ids, float *out_dist) {
    PG_TRY(check_search(ctx, sn.idx, Q, nq, k, beam, upper_beam, precision, out_ids, out_dist));
    PG_TRY(search_index(ctx, sn, Q, nq, k, beam, upper_beam, flags, precision, out_ids,
                        out_dist));
    return pg_sync_check(ctx, "pg_search");
}

extern "C" pg_status pg_search_host(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                                    int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                                    pg_precision precision, int32_t *out_ids, float *out_dist) {
    PG_TRY(check_search(ctx, idx, Q, nq, k, beam, upper_beam, precision, out_ids, out_dist));
    if (nq == 0) return PG_OK;
    const IndexSnap sn(idx);  // a reader of this version until the work has synchronised
    Scratch<float> dq, ds;
    Scratch<int32_t> di;
    PG_TRY(dq.alloc(ctx, (size_t)(nq * idx->d)));
    PG_TRY(ds.alloc(ctx, (size_t)(nq * k)));
    PG_TRY(di.alloc(ctx, (size_t)(nq * k)));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(dq.p, Q, (size_t)(nq * idx->d) * 4, cudaMemcpyHostToDevice,
                                     ctx->stream));
    PG_TRY(search_index(ctx, sn, dq.p, nq, k, beam, upper_beam, flags, precision, di.p, ds.p));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(out_ids, di.p, (size_t)(nq * k) * 4, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(out_dist, ds.p, (size_t)(nq * k) * 4, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    return pg_sync_check(ctx, "pg_search_host");
}

// ---------------------------------------------------------------- insertion
namespace {

__global__ void k_gather_i32(const int32_t *src, const int32_t *idx, int64_t m, int32_t *dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) dst[t] = src[idx[t]];
}

// dst[idx[k]] = W[k * stride]
__global__ void k_scatter_first(int32_t *dst, const int32_t *idx, int64_t m, const int32_t *W,
                                int stride) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) dst[idx[t]] = W[t * stride];
}

// in-edge counts per layer row from the new nodes' lists
__global__ void k_in_count(const int32_t *nb, const int32_t *dg, int64_t ns, int R,
                           const int32_t *rows, int32_t *cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * R) return;
    const int64_t k = t / R;
    if ((int)(t % R) >= dg[k]) return;
    const int v = nb[t];
    atomicAdd(&cnt[rows ? rows[v] : v], 1);
}

__global__ void k_in_fill(const int32_t *nb, const int32_t *dg, int64_t ns, int R,
                          const int32_t *rows, const int32_t *sglob, unsigned long long *cursor,
                          int32_t *inlist) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * R) return;
    const int64_t k = t / R;
    if ((int)(t % R) >= dg[k]) return;
    const int v = nb[t];
    inlist[atomicAdd(&cursor[rows ? rows[v] : v], 1ull)] = sglob[k];
}

__global__ void k_flag_pos(const int32_t *cnt, int64_t m, int32_t *flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) flag[t] = cnt[t] > 0;
}

__global__ void k_compact(const int32_t *cnt, int64_t m, const int64_t *pos, int32_t *A) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m && cnt[t] > 0) A[pos[t]] = (int32_t)t;
}

__global__ void k_union_sizes(const int32_t *A, int64_t na, const int32_t *deg, int R,
                              const int32_t *cnt, int32_t *sz) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < na) sz[t] = min(deg[A[t]], R) + cnt[A[t]];
}

// row a of the union CSR: the old list of layer row A[a], then its in-edges
__global__ void k_union_fill(const int32_t *A, int64_t na, const int32_t *nbr, const int32_t *deg,
                             int R, const int64_t *in_off, const int32_t *inlist,
                             const int64_t *uoff, int32_t *ucand) {
    const int64_t a = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (a >= na) return;
    const int r = A[a];
    const int dr = min(deg[r], R);
    int32_t *out = ucand + uoff[a];
    for (int j = lane; j < dr; j += 32) out[j] = nbr[(int64_t)r * R + j];
    const int64_t b0 = in_off[r], b1 = in_off[r + 1];
    for (int64_t j = b0 + lane; j < b1; j += 32) out[dr + (j - b0)] = inlist[j];
}

__global__ void k_scatter_rows(const int32_t *A, int64_t na, const int32_t *tn, const int32_t *td,
                               int R, int32_t *nbr, int32_t *deg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na * R) return;
    const int64_t a = t / R;
    const int j = (int)(t % R);
    nbr[(int64_t)A[a] * R + j] = tn[t];
    if (j == 0) deg[A[a]] = td[a];
}

// new members of an upper layer: gid entries and the point -> row map
__global__ void k_append_members(const int32_t *sglob, int64_t ns, int64_t base, int32_t *gid,
                                 int32_t *rows) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns) return;
    gid[base + t] = sglob[t];
    rows[sglob[t]] = (int32_t)(base + t);
}

unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

template <typename T>
pg_status grow(pg_ctx *ctx, T *&p, int64_t keep, int64_t cap) {
    T *q = nullptr;
    PG_TRY_CUDA(ctx, cudaMalloc(&q, (size_t)std::max<int64_t>(cap, 1) * sizeof(T)));
    if (p && keep > 0)
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(q, p, (size_t)keep * sizeof(T), cudaMemcpyDeviceToDevice,
                                         ctx->stream));
    PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(p);
    p = q;
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_index_reserve(pg_ctx *ctx, pg_index *idx, int64_t capacity) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!idx) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null index");
    if (capacity < idx->n || capacity >= INT_MAX)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need n <= capacity < 2^31");
    if (capacity <= idx->capacity) return PG_OK;
    const int64_t n = idx->n, d = idx->d;
    float *pts = nullptr;
    PG_TRY_CUDA(ctx, cudaMalloc(&pts, (size_t)(capacity * d) * 4));
    cudaError_t e = cudaMemcpyAsync(pts, idx->D, (size_t)(n * d) * 4, cudaMemcpyDeviceToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(pts);
        return pg_cuda_fail(ctx, e, "pg_index_reserve copy");
    }
    cudaFree(idx->owned);
    idx->owned = pts;
    idx->D = pts;
    for (size_t i = 0; i < idx->layers.size(); ++i) {
        pg_layer &l = idx->layers[i];
        const int64_t cap = i == 0 ? capacity : l.count + (capacity - n);
        PG_TRY(grow(ctx, l.nbr, l.count * l.R, cap * l.R));
        PG_TRY(grow(ctx, l.deg, l.count, cap));
        if (l.gid) {
            PG_TRY(grow(ctx, l.gid, l.count, cap));
            PG_TRY(grow(ctx, l.rows, n, capacity));
            k_fill_i32<<<blocks(capacity - n), 256, 0, ctx->stream>>>(l.rows + n, capacity - n, -1);
            PG_LAUNCHED(ctx);
        }
        l.cap = cap;
    }
    idx->capacity = capacity;
    return pg_sync_check(ctx, "pg_index_reserve");
}

// Algorithm 4 on a snapshot, applied to the working copy L of the layers
// (n0 points before the batch); facts_out receives the facts of all N rows.
static pg_status insert_into(pg_ctx *ctx, pg_index *idx, std::vector<pg_layer> &L, int64_t n0,
                             const float *X, int64_t m, int32_t ef, int32_t upper_beam,
                             DataFacts *facts_out) {
    const int64_t N = n0 + m, d = idx->d;
    const pg_build_params &p = idx->params;
    float *Dall = idx->owned;
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(Dall + n0 * d, X, (size_t)(m * d) * 4,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, Dall, N, (int32_t)d, idx->metric, &facts));
    const int top = (int)L.size() - 1;
    std::vector<int> lev((size_t)m);
    for (int64_t k = 0; k < m; ++k)
        lev[(size_t)k] = std::min(level_of(n0 + k, p.seed, p.M), top);
    Scratch<int32_t> w, sel, sglob, starts, out1, W, nnb, ndg, cnt, flag, A, sz, ucand, self, tn, td,
        inl;
    Scratch<float> Q, out1s, Ws;
    Scratch<int64_t> off, in_off, pos, uoff;
    Scratch<unsigned long long> cur;
    PG_TRY(w.alloc(ctx, (size_t)m));
    k_fill_i32<<<blocks(m), 256, 0, ctx->stream>>>(w.p, m, (int32_t)idx->ep_top);
    PG_LAUNCHED(ctx);
    std::vector<int32_t> hs, hb, hg;
    for (int i = top; i >= 0; --i) {
        pg_layer &l = L[(size_t)i];
        const int Ri = l.R;
        hs.clear();
        hb.clear();
        for (int64_t k = 0; k < m; ++k) (lev[(size_t)k] >= i ? hs : hb).push_back((int32_t)k);
        // routing through a layer above the point's level: pool upper_beam, keep the best
        if (i >= 1 && !hb.empty()) {
            const int64_t nb = (int64_t)hb.size();
            PG_TRY(sel.alloc(ctx, (size_t)nb));
            PG_TRY(sglob.alloc(ctx, (size_t)nb));
            hg.resize(hb.size());
            for (size_t a = 0; a < hb.size(); ++a) hg[a] = (int32_t)(n0 + hb[a]);
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(sel.p, hb.data(), (size_t)nb * 4,
                                             cudaMemcpyHostToDevice, ctx->stream));
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(sglob.p, hg.data(), (size_t)nb * 4,
                                             cudaMemcpyHostToDevice, ctx->stream));
            PG_TRY(Q.alloc(ctx, (size_t)(nb * d)));
            PG_TRY(starts.alloc(ctx, (size_t)nb));
            PG_TRY(out1.alloc(ctx, (size_t)nb));
            PG_TRY(out1s.alloc(ctx, (size_t)nb));
            k_gather_rows<<<blocks(nb * (d / 4)), 256, 0, ctx->stream>>>(Dall, (int)d, sglob.p, nb,
                                                                         Q.p);
            PG_LAUNCHED(ctx);
            k_gather_i32<<<blocks(nb), 256, 0, ctx->stream>>>(w.p, sel.p, nb, starts.p);
            PG_LAUNCHED(ctx);
            PG_TRY(pg_search_internal(ctx, Dall, n0, (int32_t)d, idx->metric, l.nbr, l.deg, Ri,
                                      l.rows, Q.p, nb, starts.p, 1, upper_beam, 0, out1.p,
                                      out1s.p, nullptr, nullptr, &facts));
            k_scatter_first<<<blocks(nb), 256, 0, ctx->stream>>>(w.p, sel.p, nb, out1.p, 1);
            PG_LAUNCHED(ctx);
        }
        if (hs.empty()) continue;
        const int64_t ns = (int64_t)hs.size();
        PG_TRY(sel.alloc(ctx, (size_t)ns));
        PG_TRY(sglob.alloc(ctx, (size_t)ns));
        hg.resize(hs.size());
        for (size_t a = 0; a < hs.size(); ++a) hg[a] = (int32_t)(n0 + hs[a]);
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(sel.p, hs.data(), (size_t)ns * 4, cudaMemcpyHostToDevice,
                                         ctx->stream));
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(sglob.p, hg.data(), (size_t)ns * 4,
                                         cudaMemcpyHostToDevice, ctx->stream));
        // W_i: pool ef on this layer, from the entry found above
        PG_TRY(Q.alloc(ctx, (size_t)(ns * d)));
        PG_TRY(starts.alloc(ctx, (size_t)ns));
        PG_TRY(W.alloc(ctx, (size_t)(ns * ef)));
        PG_TRY(Ws.alloc(ctx, (size_t)(ns * ef)));
        k_gather_rows<<<blocks(ns * (d / 4)), 256, 0, ctx->stream>>>(Dall, (int)d, sglob.p, ns,
                                                                     Q.p);
        PG_LAUNCHED(ctx);
        k_gather_i32<<<blocks(ns), 256, 0, ctx->stream>>>(w.p, sel.p, ns, starts.p);
        PG_LAUNCHED(ctx);
        PG_TRY(pg_search_internal(ctx, Dall, n0, (int32_t)d, idx->metric, l.nbr, l.deg, Ri, l.rows,
                                  Q.p, ns, starts.p, ef, ef, 0, W.p, Ws.p, nullptr, nullptr,
                                  &facts));
        k_scatter_first<<<blocks(ns), 256, 0, ctx->stream>>>(w.p, sel.p, ns, W.p, ef);
        PG_LAUNCHED(ctx);
        // N_i(u) = Prune(u, W_i)
        PG_TRY(off.alloc(ctx, (size_t)ns + 1));
        PG_TRY(nnb.alloc(ctx, (size_t)(ns * Ri)));
        PG_TRY(ndg.alloc(ctx, (size_t)ns));
        k_fill_off<<<blocks(ns + 1), 256, 0, ctx->stream>>>(off.p, ns, ef);
        PG_LAUNCHED(ctx);
        PG_TRY(pg_prune_internal(ctx, Dall, N, (int32_t)d, idx->metric, off.p, W.p, Ri,
                                 p.alpha_final_deg, facts, nnb.p, ndg.p, nullptr, ns, sglob.p));
        // reverse step: old rows that gained in-edges re-prune their list plus the in-edges
        const int64_t cnt_rows = l.count;
        PG_TRY(cnt.alloc(ctx, (size_t)cnt_rows));
        PG_TRY(in_off.alloc(ctx, (size_t)cnt_rows + 1));
        PG_TRY(cur.alloc(ctx, (size_t)cnt_rows + 1));
        PG_TRY(inl.alloc(ctx, (size_t)(ns * Ri)));
        PG_TRY_CUDA(ctx, cudaMemsetAsync(cnt.p, 0, (size_t)cnt_rows * 4, ctx->stream));
        k_in_count<<<blocks(ns * Ri), 256, 0, ctx->stream>>>(nnb.p, ndg.p, ns, Ri, l.rows, cnt.p);
        PG_LAUNCHED(ctx);
        PG_TRY(pg_scan_counts(ctx, cnt.p, cnt_rows, in_off.p));
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(cur.p, in_off.p, (size_t)(cnt_rows + 1) * 8,
                                         cudaMemcpyDeviceToDevice, ctx->stream));
        k_in_fill<<<blocks(ns * Ri), 256, 0, ctx->stream>>>(nnb.p, ndg.p, ns, Ri, l.rows, sglob.p,
                                                            cur.p, inl.p);
        PG_LAUNCHED(ctx);
        PG_TRY(flag.alloc(ctx, (size_t)cnt_rows));
        PG_TRY(pos.alloc(ctx, (size_t)cnt_rows + 1));
        k_flag_pos<<<blocks(cnt_rows), 256, 0, ctx->stream>>>(cnt.p, cnt_rows, flag.p);
        PG_LAUNCHED(ctx);
        PG_TRY(pg_scan_counts(ctx, flag.p, cnt_rows, pos.p));
        int64_t na = 0;
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, pos.p + cnt_rows, 8, cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PG_TRY(pg_sync_check(ctx, "insert"));
        memcpy(&na, ctx->h_pinned, 8);
        if (na > 0) {
            PG_TRY(A.alloc(ctx, (size_t)na));
            PG_TRY(sz.alloc(ctx, (size_t)na));
            PG_TRY(uoff.alloc(ctx, (size_t)na + 1));
            k_compact<<<blocks(cnt_rows), 256, 0, ctx->stream>>>(cnt.p, cnt_rows, pos.p, A.p);
            PG_LAUNCHED(ctx);
            k_union_sizes<<<blocks(na), 256, 0, ctx->stream>>>(A.p, na, l.deg, Ri, cnt.p, sz.p);
            PG_LAUNCHED(ctx);
            PG_TRY(pg_scan_counts(ctx, sz.p, na, uoff.p));
            PG_TRY(ucand.alloc(ctx, (size_t)(na * Ri + ns * Ri)));
            k_union_fill<<<(unsigned)((na + 7) / 8), 256, 0, ctx->stream>>>(
                A.p, na, l.nbr, l.deg, Ri, in_off.p, inl.p, uoff.p, ucand.p);
            PG_LAUNCHED(ctx);
            const int32_t *selfp = A.p;
            if (l.gid) {
                PG_TRY(self.alloc(ctx, (size_t)na));
                k_gather_i32<<<blocks(na), 256, 0, ctx->stream>>>(l.gid, A.p, na, self.p);
                PG_LAUNCHED(ctx);
                selfp = self.p;
            }
            PG_TRY(tn.alloc(ctx, (size_t)(na * Ri)));
            PG_TRY(td.alloc(ctx, (size_t)na));
            PG_TRY(pg_prune_internal(ctx, Dall, N, (int32_t)d, idx->metric, uoff.p, ucand.p, Ri,
                                     p.alpha_final_deg, facts, tn.p, td.p, nullptr, na, selfp));
            k_scatter_rows<<<blocks(na * Ri), 256, 0, ctx->stream>>>(A.p, na, tn.p, td.p, Ri,
                                                                    l.nbr, l.deg);
            PG_LAUNCHED(ctx);
        }
        // append the new members
        if (l.count + ns > l.cap) return pg_fail(ctx, PG_ERR_INTERNAL, "insert: layer capacity");
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(l.nbr + l.count * Ri, nnb.p, (size_t)(ns * Ri) * 4,
                                         cudaMemcpyDeviceToDevice, ctx->stream));
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(l.deg + l.count, ndg.p, (size_t)ns * 4,
                                         cudaMemcpyDeviceToDevice, ctx->stream));
        if (l.gid) {
            k_append_members<<<blocks(ns), 256, 0, ctx->stream>>>(sglob.p, ns, l.count, l.gid,
                                                                  l.rows);
            PG_LAUNCHED(ctx);
        }
        l.count += ns;
        PG_TRY(pg_sync_check(ctx, "insert"));
    }
    *facts_out = facts;
    return pg_sync_check(ctx, "pg_index_insert");
}

extern "C" pg_status pg_index_insert(pg_ctx *ctx, pg_index *idx, const float *X, int64_t m,
                                     int32_t ef, int32_t upper_beam) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!idx || (!X && m > 0)) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (m < 0 || ef < 1 || ef > 256 || upper_beam < 1 || upper_beam > 256)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need m >= 0, 1 <= ef, upper_beam <= 256");
    if (m == 0) return PG_OK;
    std::vector<pg_layer> L;
    int64_t n0 = 0;
    {
        std::lock_guard<std::mutex> lk(idx->ver_mu);
        L = idx->layers;
        n0 = idx->n;
    }
    if (!idx->owned || n0 + m > idx->capacity)
        return pg_fail(ctx, PG_ERR_CAPACITY, "insert: %lld points exceed the reserved capacity",
                       (long long)m);
    // the next version in copies of every layer's arrays: searches keep
    // reading the published version meanwhile.  The arrays of an earlier
    // version that no search pins any more are reused (same layer sizes), so
    // an insertion allocates (and synchronises the device) only when there
    // is none, e.g. the first time.
    auto bytes_of = [](int64_t count) { return (size_t)std::max<int64_t>(count, 1) * 4; };
    std::vector<std::pair<void *, size_t>> spare, fresh, extra;
    {
        // one unpinned earlier version is reused, any other unpinned one freed
        std::lock_guard<std::mutex> lk(idx->ver_mu);
        for (auto it = idx->retired.begin(); it != idx->retired.end();) {
            if (idx->readers.count(it->first) != 0) {
                ++it;
                continue;
            }
            auto &dst = spare.empty() ? spare : extra;
            dst.insert(dst.end(), it->second.begin(), it->second.end());
            it = idx->retired.erase(it);
        }
    }
    for (auto &b : extra) cudaFree(b.first);
    size_t next_spare = 0;
    auto copy_of = [&](int32_t *&ptr, int64_t count, int64_t keep) -> pg_status {
        const size_t bytes = bytes_of(count);
        int32_t *q = nullptr;
        if (next_spare < spare.size() && spare[next_spare].second == bytes) {
            q = static_cast<int32_t *>(spare[next_spare].first);
            spare[next_spare++].first = nullptr;
        } else {
            PG_TRY_CUDA(ctx, cudaMalloc(&q, bytes));
        }
        fresh.push_back({q, bytes});
        if (keep > 0)
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(q, ptr, (size_t)keep * 4, cudaMemcpyDeviceToDevice,
                                             ctx->stream));
        ptr = q;
        return PG_OK;
    };
    pg_status st = PG_OK;
    for (auto &l : L) {
        if (st == PG_OK) st = copy_of(l.nbr, l.cap * l.R, l.count * l.R);
        if (st == PG_OK) st = copy_of(l.deg, l.cap, l.count);
        if (st == PG_OK && l.gid) st = copy_of(l.gid, l.cap, l.count);
        if (st == PG_OK && l.rows) st = copy_of(l.rows, idx->capacity, idx->capacity);
    }
    for (auto &b : spare) cudaFree(b.first);  // sizes that no longer match (cudaFree(NULL): no-op)
    DataFacts facts;
    if (st == PG_OK) st = insert_into(ctx, idx, L, n0, X, m, ef, upper_beam, &facts);
    if (st != PG_OK) {
        cudaStreamSynchronize(ctx->stream);
        for (auto &b : fresh) cudaFree(b.first);
        return st;
    }
    // publish; the old arrays wait for reuse until no search pins their version
    std::lock_guard<std::mutex> lk(idx->ver_mu);
    std::vector<std::pair<void *, size_t>> old;
    for (auto &l : idx->layers) {
        old.push_back({l.nbr, bytes_of(l.cap * l.R)});
        old.push_back({l.deg, bytes_of(l.cap)});
        if (l.gid) old.push_back({l.gid, bytes_of(l.cap)});
        if (l.rows) old.push_back({l.rows, bytes_of(idx->capacity)});
    }
    idx->retired.push_back({idx->version, std::move(old)});
    idx->layers = L;
    idx->n = n0 + m;
    idx->facts = facts;
    idx->has_facts = 1;
    idx->version += 1;
    return PG_OK;
}
