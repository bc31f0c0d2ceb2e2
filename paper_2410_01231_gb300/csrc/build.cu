// build.cu -- the construction pipelines and the index object.
//
// pg_build_rng: IterNSG with a fixed number of iterations (Algorithm 6),
// each iteration one OptKCNA (Algorithm 5): alpha-prune C -> reverse-edge
// union -> alpha-prune -> connect -> self-search for new C; then the final
// refinement of Algorithm 2 (lines 5-11) at alpha_final.  The graph,
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
                            const int32_t *self_ids = nullptr);
pg_status pg_reverse_union_internal(pg_ctx *ctx, const int32_t *nbr, const int32_t *deg, int64_t n,
                                    int32_t R, int64_t *off, int32_t *ids);
pg_status pg_medoid_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             int64_t *host_ep);
pg_status pg_connect_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              int32_t *nbr, int32_t *deg, int32_t R, int64_t ep,
                              const DataFacts &facts, const int32_t *knn, int32_t K,
                              int64_t *host_added);
pg_status pg_search_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             const int32_t *nbr, const int32_t *deg, int32_t R,
                             const int32_t *rows, const float *Q, int64_t nq,
                             const int32_t *starts, int32_t k, int32_t L, int self,
                             int32_t *out_i, float *out_s, const uint8_t *D8 = nullptr);

struct pg_layer {
    int64_t count = 0;
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
    ~pg_index() {
        for (auto &l : layers) {
            cudaFree(l.gid);
            cudaFree(l.nbr);
            cudaFree(l.deg);
            cudaFree(l.rows);
        }
    }
};

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

// Level of every point: floor(-ln U / ln M), U = ((z >> 11) + 1) 2^-53 with
// z = SplitMix64(seed XOR id) -- the exponentially decaying level draw of
// Algorithm 4 line 4 / Algorithm 7 line 2.
std::vector<int> draw_levels(int64_t n, uint64_t seed, int M) {
    std::vector<int> lev((size_t)n);
    const double lnM = std::log((double)M);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t z = splitmix64(seed ^ (uint64_t)i);
        double U = (double)((z >> 11) + 1) * (1.0 / 9007199254740992.0);
        lev[(size_t)i] = (int)std::floor(-std::log(U) / lnM);
    }
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
    return PG_OK;
}

// IterNSG on a dense dataset X [m][d]: writes nbr [m][R] / deg [m] (local ids)
pg_status iter_nsg(pg_ctx *ctx, const float *X, int64_t m, int32_t d, const pg_build_params *p,
                   int R, int connect_final, int32_t *nbr, int32_t *deg, int64_t *ep_out,
                   double *phase) {
    PhaseClock clk{ctx, phase};
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, X, m, d, p->metric, &facts));
    int64_t ep = 0;
    PG_TRY(pg_medoid_internal(ctx, X, m, d, p->metric, &ep));
    *ep_out = ep;
    const int K = (int)std::min<int64_t>(p->K, m - 1);
    const int L = p->L;
    Scratch<int32_t> knn_i, cand, nbr1, deg1, uids;
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
    PG_TRY(pg_knn_internal(ctx, X, m, d, p->metric, K, p->precision, knn_i.p, knn_s.p));
    knn_s.release();
    const unsigned g1 = (unsigned)((m + 256) / 256);
    k_fill_off<<<g1, 256, 0, ctx->stream>>>(off.p, m, K);
    PG_LAUNCHED(ctx);
    const int32_t *cur = knn_i.p;
    // the screened form gathers byte rows when the data are exact bytes
    Scratch<uint8_t> x8;
    if (pg_u8_usable(facts, p->metric, d, p->precision)) PG_TRY(pg_make_u8(ctx, X, m, d, x8));
    auto refine = [&](double alpha, int do_connect) -> pg_status {
        clk.start(PH_PRUNE);
        PG_TRY(pg_prune_internal(ctx, X, m, d, p->metric, off.p, cur, R, alpha, facts, nbr1.p,
                                 deg1.p, x8.p));
        clk.start(PH_UNION);
        PG_TRY(pg_reverse_union_internal(ctx, nbr1.p, deg1.p, m, R, uoff.p, uids.p));
        clk.start(PH_PRUNE);
        PG_TRY(pg_prune_internal(ctx, X, m, d, p->metric, uoff.p, uids.p, R, alpha, facts, nbr,
                                 deg, x8.p));
        if (do_connect) {
            clk.start(PH_CONNECT);
            PG_TRY(pg_connect_internal(ctx, X, m, d, p->metric, nbr, deg, R, ep, facts, knn_i.p, K,
                                       nullptr));
        }
        return PG_OK;
    };
    for (int it = 0; it < p->iters; ++it) {
        PG_TRY(refine(p->alpha_deg, 1));
        if (!cand.p) PG_TRY(cand.alloc(ctx, (size_t)(m * L)));
        clk.start(PH_ACQUIRE);
        PG_TRY(pg_search_internal(ctx, X, m, d, p->metric, nbr, deg, R, nullptr, nullptr, m,
                                  nullptr, L, L, 1, cand.p, nullptr, x8.p));
        k_fill_off<<<g1, 256, 0, ctx->stream>>>(off.p, m, L);
        PG_LAUNCHED(ctx);
        cur = cand.p;
    }
    PG_TRY(refine(p->alpha_final_deg, connect_final));
    clk.stop();
    return pg_sync_check(ctx, "build");
}

pg_status alloc_layer(pg_ctx *ctx, pg_layer &l, int64_t count, int R, int64_t n, bool ident) {
    l.count = count;
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
    idx->layers.resize(1);
    pg_status st = alloc_layer(ctx, idx->layers[0], n, p->R, n, true);
    int64_t ep = 0;
    if (st == PG_OK)
        st = iter_nsg(ctx, D, n, d, p, p->R, rng ? p->connect_final : 0, idx->layers[0].nbr,
                      idx->layers[0].deg, &ep, idx->phase);
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

extern "C" pg_status pg_build_nswg(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                   const pg_build_params *params, pg_index **out) {
    return build_common(ctx, D, n, d, params, false, out);
}

extern "C" void pg_index_destroy(pg_index *index) { delete index; }

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

extern "C" pg_status pg_index_phase_seconds(const pg_index *idx, double *host_seconds6) {
    if (!idx || !host_seconds6) return PG_ERR_INVALID_ARG;
    memcpy(host_seconds6, idx->phase, sizeof idx->phase);
    return PG_OK;
}

static pg_status search_index(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                              int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                              int32_t *out_ids, float *out_dist) {
    if (nq == 0) return PG_OK;
    Scratch<int32_t> w, w2;
    Scratch<float> s2;
    PG_TRY(w.alloc(ctx, (size_t)nq));
    const bool layered = idx->layers.size() > 1 && !(flags & PG_SEARCH_FLAT);
    k_fill_i32<<<(unsigned)((nq + 255) / 256), 256, 0, ctx->stream>>>(
        w.p, nq, (int32_t)(layered ? idx->ep_top : idx->ep_base));
    PG_LAUNCHED(ctx);
    if (layered) {
        PG_TRY(w2.alloc(ctx, (size_t)nq));
        PG_TRY(s2.alloc(ctx, (size_t)nq));
        for (int i = (int)idx->layers.size() - 1; i >= 1; --i) {
            const pg_layer &l = idx->layers[(size_t)i];
            PG_TRY(pg_search_internal(ctx, idx->D, idx->n, idx->d, idx->metric, l.nbr, l.deg, l.R,
                                      l.rows, Q, nq, w.p, 1, upper_beam, 0, w2.p, s2.p));
            std::swap(w.p, w2.p);
        }
    }
    const pg_layer &b = idx->layers[0];
    return pg_search_internal(ctx, idx->D, idx->n, idx->d, idx->metric, b.nbr, b.deg, b.R, nullptr,
                              Q, nq, w.p, k, beam, 0, out_ids, out_dist);
}

static pg_status check_search(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                              int32_t k, int32_t beam, int32_t upper_beam, const void *a,
                              const void *b) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!idx || !Q || !a || !b) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (nq < 0 || k < 1 || beam < k || beam > 256 || upper_beam < 1 || upper_beam > 256)
        return pg_fail(ctx, PG_ERR_INVALID_ARG,
                       "need 1 <= k <= beam <= 256 and 1 <= upper_beam <= 256");
    return PG_OK;
}

extern "C" pg_status pg_search(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                               int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                               pg_precision precision, int32_t *out_ids, float *out_dist) {
    (void)precision;
    PG_TRY(check_search(ctx, idx, Q, nq, k, beam, upper_beam, out_ids, out_dist));
    PG_TRY(search_index(ctx, idx, Q, nq, k, beam, upper_beam, flags, out_ids, out_dist));
    return pg_sync_check(ctx, "pg_search");
}

extern "C" pg_status pg_search_host(pg_ctx *ctx, const pg_index *idx, const float *Q, int64_t nq,
                                    int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                                    pg_precision precision, int32_t *out_ids, float *out_dist) {
    (void)precision;
    PG_TRY(check_search(ctx, idx, Q, nq, k, beam, upper_beam, out_ids, out_dist));
    if (nq == 0) return PG_OK;
    Scratch<float> dq, ds;
    Scratch<int32_t> di;
    PG_TRY(dq.alloc(ctx, (size_t)(nq * idx->d)));
    PG_TRY(ds.alloc(ctx, (size_t)(nq * k)));
    PG_TRY(di.alloc(ctx, (size_t)(nq * k)));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(dq.p, Q, (size_t)(nq * idx->d) * 4, cudaMemcpyHostToDevice,
                                     ctx->stream));
    PG_TRY(search_index(ctx, idx, dq.p, nq, k, beam, upper_beam, flags, di.p, ds.p));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(out_ids, di.p, (size_t)(nq * k) * 4, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(out_dist, ds.p, (size_t)(nq * k) * 4, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    return pg_sync_check(ctx, "pg_search_host");
}
