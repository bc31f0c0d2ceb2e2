// descent.cu -- approximate kNN graph by 2-hop refinement (the KGraph /
// NN-descent iteration of the initialization phase, Section 3.1, as Exp. 12
// describes it): start from K neighbours per point drawn at random; every
// iteration each point u takes the K best by (s, id) of its neighbours and
// their neighbours (u excluded).
//
// One warp per point u reads the iteration's snapshot of the lists (so the
// result does not depend on the order of the points) and keeps u's list as a
// sorted pool of K (s, id) entries in shared memory.  Every entry carries a
// "new" bit: set when it entered the list in the previous iteration.  A pair
// (v in N(u), w in N(v)) whose both entries are old was already compared in
// the previous iteration, and w was not kept then; since the K-th distance
// of a list never grows, it cannot be kept now either, so such pairs are
// skipped (NN-descent's incremental search) without changing the result.
// Candidates are filtered by a lossy visited table, measured by four teams
// of eight lanes, sorted in registers and merged into the pool; a candidate
// already in the pool is found by an exact (s, id) binary search.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "pg_internal.cuh"

namespace {

constexpr unsigned NEW_BIT = 0x80000000u;
constexpr int IDM = 0x7fffffff;
constexpr int DK = 64;     // largest K
constexpr int DW = 4;      // warps per CTA
constexpr int HB = 10;     // visited-table slots 1 << HB

__host__ __device__ inline size_t descent_warp_smem(int d) {
    return (size_t)DK * 8 * 2 + ((size_t)4 << HB) + 32 * 8 + (size_t)d * 4;
}

__device__ __forceinline__ unsigned dslot(int v) { return ((unsigned)v * 2654435761u) >> (32 - HB); }

__device__ __forceinline__ int lower_bound_pool(const float *ps, const int *pi, int size, float s,
                                                int id) {
    int lo = 0, hi = size;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pair_less(ps[mid], pi[mid] & IDM, s, id)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct DescentParams {
    const float *D;
    int64_t n;
    int d;
    int metric;
    int K;
    const int32_t *cur_i;  // [n][K] ids | NEW_BIT, -1 empty
    const float *cur_s;    // [n][K]
    int32_t *nxt_i;
    float *nxt_s;
    const int32_t *init;   // first pass only: [n][K] initial ids (any order, any repeats)
    unsigned long long *updates;
    int *err;
};

// Initial lists: the distinct valid ids of init[u] other than u, sorted by
// (s, id), every entry new.
__global__ void __launch_bounds__(DW * 32) k_descent_init(DescentParams P) {
    __shared__ float ks[DW][DK];
    __shared__ int ki[DW][DK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int64_t u = (int64_t)blockIdx.x * DW + w;
    if (u >= P.n) return;
    const int K = P.K;
    for (int j = lane; j < DK; j += 32) {
        ks[w][j] = INFINITY;
        ki[w][j] = INT_MAX;
    }
    __syncwarp();
    const float4 *q4 = reinterpret_cast<const float4 *>(P.D + u * P.d);
    for (int b0 = 0; b0 < K; b0 += 4) {
        const int j = b0 + team;
        int v = j < K ? P.init[u * K + j] : -1;
        if (v >= P.n || v < -1) {
            if (li == 0) record_error(P.err, DERR_BAD_ID, u);
            v = -1;
        }
        bool ok = v >= 0 && v != (int)u;
        for (int e = 0; e < j && ok; ++e) ok = P.init[u * K + e] != v;  // first occurrence only
        const float s = team8_dist(q4, reinterpret_cast<const float4 *>(P.D + (int64_t)(ok ? v : 0) * P.d),
                                   P.d / 4, li, P.metric);
        if (li == 0 && j < K && ok) {
            ks[w][j] = s;
            ki[w][j] = v;
        }
    }
    __syncwarp();
    warp_bitonic_sort(ks[w], ki[w], DK);
    for (int j = lane; j < K; j += 32) {
        const bool ok = ki[w][j] != INT_MAX;
        P.nxt_i[u * K + j] = ok ? (int)((unsigned)ki[w][j] | NEW_BIT) : -1;
        P.nxt_s[u * K + j] = ok ? ks[w][j] : INFINITY;
    }
}

__global__ void __launch_bounds__(DW * 32) k_descent_iter(DescentParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int64_t u = (int64_t)blockIdx.x * DW + w;
    if (u >= P.n) return;
    const int K = P.K, d = P.d;
    unsigned char *ws = smem + (size_t)w * descent_warp_smem(d);
    float *psA = reinterpret_cast<float *>(ws);
    int *piA = reinterpret_cast<int *>(psA + DK);
    float *psB = reinterpret_cast<float *>(piA + DK);
    int *piB = reinterpret_cast<int *>(psB + DK);
    int *htab = piB + DK;
    float *nd = reinterpret_cast<float *>(htab + (1 << HB));
    int *ni = reinterpret_cast<int *>(nd + 32);
    float *q = reinterpret_cast<float *>(ni + 32);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    for (int c = lane; c < d / 4; c += 32)
        reinterpret_cast<float4 *>(q)[c] = __ldg(reinterpret_cast<const float4 *>(P.D + u * d) + c);
    for (int h = lane; h < (1 << HB); h += 32) htab[h] = -1;
    __syncwarp();
    // the pool starts as u's list (entries old for the next iteration)
    int size = 0;
    for (int b0 = 0; b0 < K; b0 += 32) {
        const int j = b0 + lane;
        const int e = j < K ? P.cur_i[u * K + j] : -1;
        const bool ok = e != -1;
        if (j < K) {
            psA[j] = ok ? P.cur_s[u * K + j] : INFINITY;
            piA[j] = ok ? (e & IDM) : INT_MAX;
        }
        size += __popc(__ballot_sync(0xffffffffu, ok));
    }
    __syncwarp();
    if (lane == 0) htab[dslot((int)u)] = (int)u;
    for (int j = lane; j < size; j += 32) htab[dslot(piA[j])] = piA[j];
    __syncwarp();
    float *ps = psA, *ps2 = psB;
    int *pi = piA, *pi2 = piB;
    unsigned long long inserted = 0;
    for (int a = 0; a < K; ++a) {
        const int ev = P.cur_i[u * K + a];
        if (ev == -1) continue;
        const int v = ev & IDM;
        const bool vnew = (ev & (int)NEW_BIT) != 0;
        if (v >= P.n) {
            if (lane == 0) record_error(P.err, DERR_BAD_ID, u);
            continue;
        }
        for (int c0 = 0; c0 < K; c0 += 32) {
            const int j = c0 + lane;
            const int ew = j < K ? P.cur_i[(int64_t)v * K + j] : -1;
            int x = ew == -1 ? -1 : (ew & IDM);
            if (x >= P.n) {
                record_error(P.err, DERR_BAD_ID, v);
                x = -1;
            }
            bool fresh = x >= 0 && x != (int)u && (vnew || (ew & (int)NEW_BIT));
            if (fresh) {
                const unsigned h = dslot(x);
                if (htab[h] == x) fresh = false;
                else htab[h] = x;
            }
            const unsigned fb = __ballot_sync(0xffffffffu, fresh);
            const int cnt = __popc(fb);
            if (fresh) ni[__popc(fb & ((1u << lane) - 1))] = x;
            __syncwarp();
            for (int b0 = 0; b0 < cnt; b0 += 4) {
                const int i = b0 + team;
                const int xx = ni[i < cnt ? i : 0];
                const float s = team8_dist(q4, reinterpret_cast<const float4 *>(P.D + (int64_t)xx * d),
                                           d / 4, li, P.metric);
                if (li == 0 && i < cnt) nd[i] = s;
            }
            __syncwarp();
            float s = INFINITY;
            int id = INT_MAX;
            if (lane < cnt) {
                s = nd[lane];
                id = ni[lane];
                if (size == K && !pair_less(s, id, ps[K - 1], pi[K - 1] & IDM)) {
                    id = INT_MAX;
                } else {
                    const int pos = lower_bound_pool(ps, pi, size, s, id);
                    if (pos < size && ps[pos] == s && (pi[pos] & IDM) == id) id = INT_MAX;
                }
                if (id == INT_MAX) s = INFINITY;
            }
            const int m2 = __popc(__ballot_sync(0xffffffffu, id != INT_MAX));
            if (m2 == 0) continue;
            warp_sort32(s, id);  // survivors first, ascending
            __syncwarp();
            if (lane < m2) {
                nd[lane] = s;
                ni[lane] = id;
            }
            __syncwarp();
            // merge pool and survivors into the other buffer, keep K
            for (int b0 = 0; b0 < size; b0 += 32) {
                const int i = b0 + lane;
                if (i < size) {
                    const float es = ps[i];
                    const int eid = pi[i];
                    int lo = 0, hi = m2;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (pair_less(nd[mid], ni[mid], es, eid & IDM)) lo = mid + 1;
                        else hi = mid;
                    }
                    const int dst = i + lo;
                    if (dst < K) {
                        ps2[dst] = es;
                        pi2[dst] = eid;
                    }
                }
            }
            if (lane < m2) {
                const int dst = lane + lower_bound_pool(ps, pi, size, s, id);
                if (dst < K) {
                    ps2[dst] = s;
                    pi2[dst] = (int)((unsigned)id | NEW_BIT);
                }
            }
            __syncwarp();
            size = min(K, size + m2);
            float *tf = ps;
            ps = ps2;
            ps2 = tf;
            int *ti = pi;
            pi = pi2;
            pi2 = ti;
        }
    }
    for (int j = lane; j < K; j += 32) {
        const bool ok = j < size;
        const int e = ok ? pi[j] : -1;
        P.nxt_i[u * K + j] = e;
        P.nxt_s[u * K + j] = ok ? ps[j] : INFINITY;
        if (ok && (e & (int)NEW_BIT)) ++inserted;
    }
    for (int o = 16; o; o >>= 1) inserted += __shfl_xor_sync(0xffffffffu, inserted, o);
    if (lane == 0 && inserted) atomicAdd(P.updates, inserted);
}

__global__ void k_descent_strip(const int32_t *src, const float *ss, int64_t total, int32_t *ids,
                                float *dist) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int e = src[t];
    ids[t] = e == -1 ? -1 : (e & IDM);
    dist[t] = ss[t];
}

// initial ids of the random draw: splitmix64(seed XOR (u K + j)) mapped to
// [0, n) by the high 64 bits of its product with n
__global__ void k_descent_draw(int64_t n, int K, uint64_t seed, int32_t *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * K) return;
    uint64_t z = (uint64_t)t ^ seed;
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    out[t] = (int32_t)__umul64hi(z, (uint64_t)n);
}

}  // namespace

pg_status pg_knn_descent_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  pg_metric metric, int32_t K, int32_t iters,
                                  const int32_t *init, uint64_t seed, int32_t *ids, float *dist,
                                  int64_t *host_updates) {
    Scratch<int32_t> drawn, ai, bi;
    Scratch<float> as, bs;
    Scratch<unsigned long long> upd;
    const int64_t total = n * K;
    if (!init) {
        PG_TRY(drawn.alloc(ctx, (size_t)total));
        k_descent_draw<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(n, K, seed,
                                                                                 drawn.p);
        PG_LAUNCHED(ctx);
        init = drawn.p;
    }
    PG_TRY(ai.alloc(ctx, (size_t)total));
    PG_TRY(bi.alloc(ctx, (size_t)total));
    PG_TRY(as.alloc(ctx, (size_t)total));
    PG_TRY(bs.alloc(ctx, (size_t)total));
    PG_TRY(upd.alloc(ctx, (size_t)std::max(iters, 1)));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(upd.p, 0, (size_t)std::max(iters, 1) * 8, ctx->stream));
    DescentParams P;
    P.D = D;
    P.n = n;
    P.d = d;
    P.metric = metric == PG_METRIC_L2SQ ? 0 : 1;
    P.K = K;
    P.init = init;
    P.err = ctx->d_err;
    P.cur_i = nullptr;
    P.cur_s = nullptr;
    P.nxt_i = ai.p;
    P.nxt_s = as.p;
    P.updates = upd.p;
    const unsigned grid = (unsigned)((n + DW - 1) / DW);
    k_descent_init<<<grid, DW * 32, 0, ctx->stream>>>(P);
    PG_LAUNCHED(ctx);
    const size_t smem = descent_warp_smem(d) * DW;
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(k_descent_iter,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int32_t *ci = ai.p, *ni = bi.p;
    float *cs = as.p, *ns = bs.p;
    for (int it = 0; it < iters; ++it) {
        P.cur_i = ci;
        P.cur_s = cs;
        P.nxt_i = ni;
        P.nxt_s = ns;
        P.updates = upd.p + it;
        pg_timer_begin(ctx, TM_KNN);
        k_descent_iter<<<grid, DW * 32, smem, ctx->stream>>>(P);
        PG_LAUNCHED(ctx);
        pg_timer_end(ctx, TM_KNN);
        std::swap(ci, ni);
        std::swap(cs, ns);
    }
    k_descent_strip<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(ci, cs, total, ids,
                                                                              dist);
    PG_LAUNCHED(ctx);
    if (host_updates && iters > 0) {
        std::vector<unsigned long long> h((size_t)iters);
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(h.data(), upd.p, (size_t)iters * 8, cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PG_TRY(pg_sync_check(ctx, "pg_knn_descent"));
        for (int it = 0; it < iters; ++it) host_updates[it] = (int64_t)h[(size_t)it];
    }
    return PG_OK;
}

extern "C" pg_status pg_knn_descent(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                    pg_metric metric, int32_t K, int32_t iters,
                                    const int32_t *init, uint64_t seed, int32_t *ids, float *dist,
                                    int64_t *host_updates) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !ids || !dist) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 2 || n >= INT_MAX || d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 2 <= n < 2^31, d % 4 == 0, 4 <= d <= 8192");
    if (K < 1 || K > DK || iters < 0 || iters > 64)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= K <= %d and 0 <= iters <= 64", DK);
    if (metric < PG_METRIC_L2SQ || metric > PG_METRIC_IP)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "bad metric");
    if (descent_warp_smem(d) * DW > 227 * 1024)
        return pg_fail(ctx, PG_ERR_CAPACITY, "kNN descent: rows too wide for shared memory");
    PG_TRY(pg_knn_descent_internal(ctx, D, n, d, metric, K, iters, init, seed, ids, dist,
                                   host_updates));
    return pg_sync_check(ctx, "pg_knn_descent");
}
