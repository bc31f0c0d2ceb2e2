// graph.cu -- entry point (medoid) and the connectivity step.
//
// Medoid (Section 3.1, search phase: ep is the point of D closest to the
// centroid).  The centroid is summed in FP64 per coordinate over blocks of
// 1024 consecutive points (one thread per (block, coordinate), index order
// inside the block), the block sums are added in block order and divided
// by n; ep is the exact FP64 argmin of s(x, centroid), ties by id.
//
// Connectivity (Algorithm 2 lines 10-11, Algorithm 5 lines 5-6): nodes
// reachable from ep are marked by a breadth-first pass; then, one round per
// unreached component, the smallest unreached id r is linked from the
// nearest reached node with a free adjacency slot (FP32 argmin, re-decided
// in FP64 among the candidates inside the error bound), and everything
// reachable from r is marked.  Rounds run on the device in batches; the
// host only checks between batches whether any node is still unreached.
#include <climits>
#include <cmath>

#include "pg_internal.cuh"

namespace {

constexpr int CB = 1024;  // centroid block

__global__ void k_centroid_partial(const float *__restrict__ D, int64_t n, int d, double *part) {
    int64_t nb = (n + CB - 1) / CB;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * d) return;
    int64_t b = t / d;
    int i = (int)(t % d);
    int64_t e = min(n, (b + 1) * CB);
    double s = 0.0;
    for (int64_t v = b * CB; v < e; ++v) s = __dadd_rn(s, (double)D[v * d + i]);
    part[b * d + i] = s;
}

__global__ void k_centroid_final(const double *part, int64_t nb, int d, int64_t n, double *c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double t = 0.0;
    for (int64_t b = 0; b < nb; ++b) t = __dadd_rn(t, part[b * d + i]);
    c[i] = __ddiv_rn(t, (double)n);
}

__device__ __forceinline__ void better64(double &bs, int &bi, double s, int i) {
    if (s < bs || (s == bs && i < bi)) {
        bs = s;
        bi = i;
    }
}

__global__ void k_medoid_argmin(const float *__restrict__ D, int64_t n, int d, int metric,
                                const double *__restrict__ c, double *blk_s, int *blk_i) {
    __shared__ double ss[256];
    __shared__ int si[256];
    double bs = INFINITY;
    int bi = INT_MAX;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const float *row = D + x * d;
        double s = 0.0;
        if (metric == 0) {
            for (int i = 0; i < d; ++i) {
                double t = __dsub_rn((double)row[i], c[i]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
        } else {
            for (int i = 0; i < d; ++i) s = __dadd_rn(s, __dmul_rn((double)row[i], c[i]));
            s = __dsub_rn(2.0, __dmul_rn(2.0, s));
            if (s < 0.0) s = 0.0;
        }
        better64(bs, bi, s, (int)x);
    }
    ss[threadIdx.x] = bs;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) {
            double s2 = ss[threadIdx.x + o];
            int i2 = si[threadIdx.x + o];
            if (s2 < ss[threadIdx.x] || (s2 == ss[threadIdx.x] && i2 < si[threadIdx.x])) {
                ss[threadIdx.x] = s2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        blk_s[blockIdx.x] = ss[0];
        blk_i[blockIdx.x] = si[0];
    }
}

__global__ void k_medoid_final(const double *blk_s, const int *blk_i, int nb, int *out) {
    if (threadIdx.x != 0) return;
    double bs = INFINITY;
    int bi = INT_MAX;
    for (int b = 0; b < nb; ++b) better64(bs, bi, blk_s[b], blk_i[b]);
    *out = bi;
}

// ------------------------------------------------------------ connect
struct ConnState {
    int cursor;        // smallest unreached id (n when none)
    int added;         // edges added
    int need_full;     // the round of `cursor` needs the grid-wide argmin
    int full_rounds;   // rounds decided by the grid-wide argmin
    int fast_rounds;   // rounds decided from the kNN list of r
    int pad;
    unsigned long long best;    // packed (float bits << 32 | id)
    unsigned long long best64;  // FP64 bits of the best distance (recheck)
    int best_id;
};

// grid-wide BFS level from a frontier
__global__ void k_bfs_level(const int32_t *nbr, const int32_t *deg, int R, int64_t n, int *reached,
                            const int *fin, int fcount, int *fout, int *fout_count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= fcount) return;
    int x = fin[i];
    int dx = min(deg[x], R);
    for (int j = 0; j < dx; ++j) {
        int y = nbr[(int64_t)x * R + j];
        if (y < 0 || y >= n) continue;
        if (atomicCAS(&reached[y], 0, 1) == 0) fout[atomicAdd(fout_count, 1)] = y;
    }
}

// single block: BFS from one source over unreached nodes
__device__ void block_bfs(const int32_t *nbr, const int32_t *deg, int R, int64_t n, int *reached,
                          int *queue, int src, int *s_tail) {
    if (threadIdx.x == 0) {
        *s_tail = 0;
        if (atomicCAS(&reached[src], 0, 1) == 0) {
            queue[0] = src;
            *s_tail = 1;
        }
    }
    __syncthreads();
    int head = 0;
    int tail = *s_tail;
    while (head < tail) {
        for (int i = head + threadIdx.x; i < tail; i += blockDim.x) {
            int x = queue[i];
            int dx = min(deg[x], R);
            for (int j = 0; j < dx; ++j) {
                int y = nbr[(int64_t)x * R + j];
                if (y < 0 || y >= n) continue;
                if (atomicCAS(&reached[y], 0, 1) == 0) queue[atomicAdd(s_tail, 1)] = y;
            }
        }
        __syncthreads();
        head = tail;
        tail = *s_tail;
        __syncthreads();
    }
}

// single block: smallest unreached id at or after st->cursor
__device__ void block_next_unreached(const int *reached, int64_t n, ConnState *st, int *s_min) {
    int from = st->cursor;
    __syncthreads();
    for (int64_t base = from; base < n; base += blockDim.x) {
        if (threadIdx.x == 0) *s_min = INT_MAX;
        __syncthreads();
        int64_t x = base + threadIdx.x;
        if (x < n && !reached[x]) atomicMin(s_min, (int)x);
        __syncthreads();
        int m = *s_min;
        __syncthreads();
        if (m != INT_MAX) {
            if (threadIdx.x == 0) st->cursor = m;
            __syncthreads();
            return;
        }
    }
    if (threadIdx.x == 0) st->cursor = (int)n;
    __syncthreads();
}

__global__ void k_connect_init(int64_t n, int *reached, ConnState *st) {
    __shared__ int s_min;
    if (threadIdx.x == 0) {
        st->cursor = 0;
        st->need_full = 0;
        st->best = ~0ull;
        st->best64 = ~0ull;
        st->best_id = INT_MAX;
    }
    __syncthreads();
    block_next_unreached(reached, n, st, &s_min);
}

// link r from p, mark what r reaches, advance to the next unreached id
__device__ void block_link_advance(int32_t *nbr, int32_t *deg, int R, int64_t n, int *reached,
                                   int *queue, ConnState *st, int r, int p, int *s_tail,
                                   int *s_min) {
    if (threadIdx.x == 0) {
        int dp = deg[p];
        nbr[(int64_t)p * R + dp] = r;
        deg[p] = dp + 1;
        st->added += 1;
    }
    __syncthreads();
    block_bfs(nbr, deg, R, n, reached, queue, r, s_tail);
    block_next_unreached(reached, n, st, s_min);
}

// Rounds decided from the exact kNN list of r: the list holds the K
// smallest (s, id) over all points, so when some member is reached and has
// a free slot, the best such member is the global argmin (an outside point
// at equal distance has a larger id).  Otherwise the round is left to the
// grid-wide argmin (need_full).  One block of 1024 threads, teams of 16
// threads per candidate; FP64 re-decision of near ties unless exact.
constexpr int CT = 1024, TEAM = 16, NTEAM = CT / TEAM;

__global__ void __launch_bounds__(CT)
k_connect_rounds(const float *__restrict__ D, int64_t n, int d, int metric, int32_t *nbr,
                 int32_t *deg, int R, int *reached, int *queue, ConnState *st,
                 const int32_t *__restrict__ knn, int K, ErrModel em, int exact, int max_rounds) {
    extern __shared__ __align__(16) float rq[];  // r's vector [d]
    __shared__ unsigned long long s_best;
    __shared__ unsigned long long s_best64;
    __shared__ int s_best_id, s_tail, s_min;
    __shared__ float s_cand[256];
    __shared__ int s_cid[256];
    if (st->need_full) return;
    const int tid = threadIdx.x, team = tid / TEAM, li = tid % TEAM;
    const int nch = d / 4;
    for (int round = 0; round < max_rounds; ++round) {
        const int r = st->cursor;
        if (r >= n) return;
        for (int c = tid; c < nch; c += CT)
            reinterpret_cast<float4 *>(rq)[c] = reinterpret_cast<const float4 *>(D + (int64_t)r * d)[c];
        if (tid == 0) {
            s_best = ~0ull;
            s_best64 = ~0ull;
            s_best_id = INT_MAX;
        }
        __syncthreads();
        for (int base = 0; base < K; base += NTEAM) {
            const int j = base + team;
            int x = j < K ? knn[(int64_t)r * K + j] : -1;
            bool ok = x >= 0 && x < n && reached[x] && deg[x] < R;
            const float4 *xr = reinterpret_cast<const float4 *>(D + (int64_t)(ok ? x : r) * d);
            float acc = 0.f;
            for (int c = li; c < nch; c += TEAM) {
                float4 a = reinterpret_cast<const float4 *>(rq)[c];
                float4 b = xr[c];
                if (metric == 0) {
                    float t0 = a.x - b.x, t1 = a.y - b.y, t2 = a.z - b.z, t3 = a.w - b.w;
                    acc = fmaf(t0, t0, acc);
                    acc = fmaf(t1, t1, acc);
                    acc = fmaf(t2, t2, acc);
                    acc = fmaf(t3, t3, acc);
                } else {
                    acc = fmaf(a.x, b.x, acc);
                    acc = fmaf(a.y, b.y, acc);
                    acc = fmaf(a.z, b.z, acc);
                    acc = fmaf(a.w, b.w, acc);
                }
            }
            for (int o = TEAM / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            float s = metric == 0 ? acc : fmaxf(2.f - 2.f * acc, 0.f);
            if (li == 0 && j < K) {
                s_cand[j] = ok ? s : INFINITY;
                s_cid[j] = ok ? x : -1;
                if (ok) {
                    unsigned long long pk = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)x;
                    atomicMin(&s_best, pk);
                }
            }
        }
        __syncthreads();
        if (s_best == ~0ull) {  // no list member qualifies: grid-wide round
            if (tid == 0) st->need_full = 1;
            __syncthreads();
            return;
        }
        int p = (int)(s_best & 0xffffffffu);
        if (!exact) {
            const float bmin = __uint_as_float((unsigned)(s_best >> 32));
            for (int j = tid; j < K; j += CT) {
                if (s_cid[j] < 0) continue;
                float s = s_cand[j];
                if (s - 2.f * em.err(s) > bmin + 2.f * em.err(bmin)) continue;
                double s64 = dist64_rows(rq, D + (int64_t)s_cid[j] * d, d, metric);
                atomicMin(&s_best64, (unsigned long long)__double_as_longlong(s64));
            }
            __syncthreads();
            for (int j = tid; j < K; j += CT) {
                if (s_cid[j] < 0) continue;
                float s = s_cand[j];
                if (s - 2.f * em.err(s) > bmin + 2.f * em.err(bmin)) continue;
                double s64 = dist64_rows(rq, D + (int64_t)s_cid[j] * d, d, metric);
                if ((unsigned long long)__double_as_longlong(s64) == s_best64)
                    atomicMin(&s_best_id, s_cid[j]);
            }
            __syncthreads();
            p = s_best_id;
        }
        if (tid == 0) st->fast_rounds += 1;
        block_link_advance(nbr, deg, R, n, reached, queue, st, r, p, &s_tail, &s_min);
    }
}

// without kNN lists every round is a grid-wide round
__global__ void k_connect_request_full(int64_t n, ConnState *st) {
    if (threadIdx.x == 0 && st->cursor < n) st->need_full = 1;
}

// FP32 argmin over reached nodes with a free slot of (s(x, r), x); runs
// only when the round of `cursor` needs it.
__global__ void k_connect_argmin(const float *__restrict__ D, int64_t n, int d, int metric,
                                 const int *reached, const int32_t *deg, int R, ConnState *st) {
    extern __shared__ __align__(16) float rq[];
    int r = st->cursor;
    if (r >= n || !st->need_full) return;
    const int nch = d / 4;
    for (int c = threadIdx.x; c < nch; c += blockDim.x)
        reinterpret_cast<float4 *>(rq)[c] = reinterpret_cast<const float4 *>(D + (int64_t)r * d)[c];
    __syncthreads();
    const int lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int64_t teams = (int64_t)gridDim.x * (blockDim.x / 8);
    unsigned long long best = ~0ull;
    for (int64_t base = (int64_t)blockIdx.x * (blockDim.x / 8) + (threadIdx.x >> 5) * 4;
         base < n; base += teams) {
        int64_t x = base + team;
        bool ok = x < n && reached[x] && deg[x] < R;
        int64_t row = ok ? x : r;
        float s = team8_dist(reinterpret_cast<const float4 *>(rq),
                             reinterpret_cast<const float4 *>(D + row * d), nch, li, metric);
        if (ok && li == 0) {
            unsigned long long p = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)x;
            if (p < best) best = p;
        }
    }
    for (int o = 16; o; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
        if (t < best) best = t;
    }
    if (lane == 0 && best != ~0ull) atomicMin(&st->best, best);
}

// FP64 re-decision among candidates inside the FP32 error bound of the min
__global__ void k_connect_recheck(const float *__restrict__ D, int64_t n, int d, int metric,
                                  const int *reached, const int32_t *deg, int R, ConnState *st,
                                  ErrModel em, int pass) {
    int r = st->cursor;
    if (r >= n || !st->need_full || st->best == ~0ull) return;
    float bmin = __uint_as_float((unsigned)(st->best >> 32));
    const float *xr = D + (int64_t)r * d;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (!reached[x] || deg[x] >= R) continue;
        // conservative FP32 screen (sequential order; any order is within the bound)
        float s = 0.f;
        const float *xx = D + x * d;
        if (metric == 0) {
            for (int i = 0; i < d; ++i) {
                float t = xx[i] - xr[i];
                s = fmaf(t, t, s);
            }
        } else {
            for (int i = 0; i < d; ++i) s = fmaf(xx[i], xr[i], s);
            s = fmaxf(2.f - 2.f * s, 0.f);
        }
        if (s - 2.f * em.err(s) > bmin + 2.f * em.err(bmin)) continue;
        double s64 = dist64_rows(xx, xr, d, metric);
        if (pass == 0) {
            atomicMin(&st->best64, (unsigned long long)__double_as_longlong(s64));
        } else if ((unsigned long long)__double_as_longlong(s64) == st->best64) {
            atomicMin(&st->best_id, (int)x);
        }
    }
}

// finish a grid-wide round: link, mark, advance, clear the request
__global__ void k_connect_link(int32_t *nbr, int32_t *deg, int R, int64_t n, int *reached,
                               int *queue, ConnState *st, int use64, int *err) {
    __shared__ int s_tail, s_min, s_p;
    const int r = st->cursor;
    if (r >= n || !st->need_full) return;
    if (threadIdx.x == 0) {
        int p = use64 ? st->best_id : (int)(st->best & 0xffffffffu);
        if (st->best == ~0ull || p == INT_MAX) {
            record_error(err, DERR_NO_SLOT, r);
            st->cursor = (int)n;
            p = -1;
        }
        s_p = p;
        st->best = ~0ull;
        st->best64 = ~0ull;
        st->best_id = INT_MAX;
        st->need_full = 0;
        st->full_rounds += 1;
    }
    __syncthreads();
    if (s_p < 0) return;
    block_link_advance(nbr, deg, R, n, reached, queue, st, r, s_p, &s_tail, &s_min);
}

}  // namespace

pg_status pg_medoid_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             int64_t *host_ep) {
    int64_t nb = (n + CB - 1) / CB;
    Scratch<double> part, cen, bs;
    Scratch<int> bi;
    PG_TRY(part.alloc(ctx, (size_t)(nb * d)));
    PG_TRY(cen.alloc(ctx, (size_t)d));
    int blocks = ctx->num_sms * 4;
    PG_TRY(bs.alloc(ctx, (size_t)blocks));
    PG_TRY(bi.alloc(ctx, (size_t)blocks + 1));
    k_centroid_partial<<<(unsigned)((nb * d + 255) / 256), 256, 0, ctx->stream>>>(D, n, d, part.p);
    PG_LAUNCHED(ctx);
    k_centroid_final<<<(d + 127) / 128, 128, 0, ctx->stream>>>(part.p, nb, d, n, cen.p);
    PG_LAUNCHED(ctx);
    pg_timer_begin(ctx, TM_MEDOID);
    k_medoid_argmin<<<blocks, 256, 0, ctx->stream>>>(D, n, d, metric == PG_METRIC_L2SQ ? 0 : 1,
                                                     cen.p, bs.p, bi.p);
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_MEDOID);
    k_medoid_final<<<1, 32, 0, ctx->stream>>>(bs.p, bi.p, blocks, bi.p + blocks);
    PG_LAUNCHED(ctx);
    int h = -1;
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(&h, bi.p + blocks, sizeof(int), cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PG_TRY(pg_sync_check(ctx, "medoid"));
    *host_ep = h;
    return PG_OK;
}

pg_status pg_connect_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              int32_t *nbr, int32_t *deg, int32_t R, int64_t ep,
                              const DataFacts &facts, const int32_t *knn, int32_t K,
                              int64_t *host_added) {
    Scratch<int> reached, queue, fcnt;
    Scratch<ConnState> st;
    PG_TRY(reached.alloc(ctx, (size_t)n));
    PG_TRY(queue.alloc(ctx, (size_t)n * 2));
    PG_TRY(fcnt.alloc(ctx, 2));
    PG_TRY(st.alloc(ctx, 1));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(reached.p, 0, (size_t)n * 4, ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(st.p, 0, sizeof(ConnState), ctx->stream));
    pg_timer_begin(ctx, TM_CONNECT);
    // reachability from ep: level-synchronous passes over the whole grid
    int one = 1;
    int epi = (int)ep;
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(reached.p + ep, &one, sizeof(int), cudaMemcpyHostToDevice,
                                     ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(queue.p, &epi, sizeof(int), cudaMemcpyHostToDevice,
                                     ctx->stream));
    int *fa = queue.p, *fb = queue.p + n;
    int fcount = 1;
    while (fcount > 0) {
        PG_TRY_CUDA(ctx, cudaMemsetAsync(fcnt.p, 0, sizeof(int), ctx->stream));
        k_bfs_level<<<(fcount + 255) / 256, 256, 0, ctx->stream>>>(nbr, deg, R, n, reached.p, fa,
                                                                   fcount, fb, fcnt.p);
        PG_LAUNCHED(ctx);
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, fcnt.p, sizeof(int),
                                         cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        memcpy(&fcount, ctx->h_pinned, sizeof(int));
        std::swap(fa, fb);
    }
    k_connect_init<<<1, CT, 0, ctx->stream>>>(n, reached.p, st.p);
    PG_LAUNCHED(ctx);
    const ErrModel em = pg_err_model(metric, d, facts, false);
    const int m = metric == PG_METRIC_L2SQ ? 0 : 1;
    const bool recheck = !facts.exact;
    const size_t smem = (size_t)d * 4;
    const int grid = ctx->num_sms * 8;
    // each queued group runs kNN-decided rounds until one needs the grid-wide
    // argmin, then that round; a group makes progress on at least one round
    const int64_t max_batches = n / 8 + 2;
    for (int64_t batch = 0;; ++batch) {
        if (batch > max_batches)
            return pg_fail(ctx, PG_ERR_INTERNAL, "connect: no progress after %lld batches",
                           (long long)batch);
        for (int g = 0; g < 8; ++g) {
            if (knn) {
                k_connect_rounds<<<1, CT, smem, ctx->stream>>>(D, n, d, m, nbr, deg, R, reached.p,
                                                               queue.p, st.p, knn, K, em,
                                                               facts.exact, 1 << 20);
                PG_LAUNCHED(ctx);
            } else {
                k_connect_request_full<<<1, 32, 0, ctx->stream>>>(n, st.p);
                PG_LAUNCHED(ctx);
            }
            k_connect_argmin<<<grid, 256, smem, ctx->stream>>>(D, n, d, m, reached.p, deg, R, st.p);
            PG_LAUNCHED(ctx);
            if (recheck) {
                for (int pass = 0; pass < 2; ++pass) {
                    k_connect_recheck<<<grid, 256, 0, ctx->stream>>>(D, n, d, m, reached.p, deg, R,
                                                                     st.p, em, pass);
                    PG_LAUNCHED(ctx);
                }
            }
            k_connect_link<<<1, CT, 0, ctx->stream>>>(nbr, deg, R, n, reached.p, queue.p, st.p,
                                                      recheck ? 1 : 0, ctx->d_err);
            PG_LAUNCHED(ctx);
        }
        ConnState h;
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, st.p, sizeof(ConnState),
                                         cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY(pg_sync_check(ctx, "connect"));
        memcpy(&h, ctx->h_pinned, sizeof(ConnState));
        if (h.cursor >= n) {
            if (host_added) *host_added = h.added;
            ctx->connect_edges += h.added;
            ctx->connect_full_rounds += h.full_rounds;
            break;
        }
    }
    pg_timer_end(ctx, TM_CONNECT);
    return PG_OK;
}

extern "C" pg_status pg_medoid(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                               pg_metric metric, int64_t *host_ep) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !host_ep) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n >= INT_MAX || d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= n < 2^31, d % 4 == 0, 4 <= d <= 8192");
    return pg_medoid_internal(ctx, D, n, d, metric, host_ep);
}

extern "C" pg_status pg_connect(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                pg_metric metric, int32_t *nbr, int32_t *deg, int32_t R,
                                int64_t ep, int64_t *host_added) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !nbr || !deg) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n >= INT_MAX || d < 4 || d % 4 || d > 8192 || R < 1 || R > 64)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "bad n / d / R");
    if (ep < 0 || ep >= n) return pg_fail(ctx, PG_ERR_INVALID_ARG, "ep out of range");
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, D, n, d, metric, &facts));
    return pg_connect_internal(ctx, D, n, d, metric, nbr, deg, R, ep, facts, nullptr, 0,
                               host_added);
}
