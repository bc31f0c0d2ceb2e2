// search.cu -- batched beam search, KANNSearch(G, q, k, L, ep) of
// Algorithm 1, one warp per query; used for the k-CNA acquisition of
// Algorithm 5 (every point searches for itself from itself) and for k-ANN
// queries.
//
// Per warp, in shared memory: the pool (<= L entries sorted by (s, id), the
// expanded flag in bit 31 of the id), a lossy
// visited table (a node id per slot, last writer wins: it never reports an
// unvisited node as visited, it may forget a visited one), the query vector
// and a 32-entry staging area.  One expansion: find the first unexpanded
// entry, read its adjacency row (one id per lane), drop ids the table
// remembers, compute the survivors' distances with four teams of eight
// lanes, drop those that cannot enter the pool (worse than the last entry
// of a full pool, or already present -- found by an exact (s, id) binary
// search, which covers what the table forgot), sort the rest in registers
// and merge them into the pool in place: only the entries behind the first
// insertion point move (read into registers chunk by chunk from the back,
// then written to their shifted slots), truncating at L.
//
// Because the pool is always the L best of everything inserted so far, a
// node that was evaluated and left the pool can never re-enter it; the
// lossy table therefore changes the work done, never the result.
#include <climits>
#include <mutex>

#include "pg_internal.cuh"

namespace {

constexpr unsigned EXP_BIT = 0x80000000u;
constexpr int ID_MASK = 0x7fffffff;
constexpr int SW = 4;  // warps per CTA

struct SearchParams {
    const float *D;
    const uint8_t *D8;  // byte shadow of D (exact data, self mode) or nullptr
    int64_t n;
    int d;
    int metric;
    const int32_t *nbr;
    const int32_t *deg;
    int R;
    const int32_t *rows;
    const float *Q;  // nullptr: self mode (query i is D row i, start i)
    int64_t nq;
    const int32_t *starts;
    int k;
    int L;
    int self;
    int hbits;
    int32_t *out_i;
    float *out_s;
    int *err;
    unsigned long long *counters;
    int *qcounter;
};

// the pool arrays hold an even number of slots, so that the query row that
// follows the table and the staging area starts on a 16-byte boundary
__host__ __device__ inline int pool_slots(int L) { return (L + 1) & ~1; }

__host__ __device__ inline size_t search_warp_smem(int L, int hbits, int d) {
    size_t b = (size_t)pool_slots(L) * 8 + ((size_t)4 << hbits) + 32 * 8 + (size_t)d * 4;
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ int pool_lower_bound(const float *pd, const int *pi, int size, float s,
                                                int id) {
    int lo = 0, hi = size;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (pair_less(pd[mid], pi[mid] & ID_MASK, s, id)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned hslot(int v, int hbits) {
    return ((unsigned)v * 2654435761u) >> (32 - hbits);
}

__device__ void search_one(const SearchParams &P, int64_t qi, unsigned char *ws,
                           unsigned long long &n_exp, unsigned long long &n_eval) {
    const int lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int L = P.L, d = P.d, nch = d / 4;
    const int Lp = pool_slots(L);
    float *pdA = reinterpret_cast<float *>(ws);
    int *piA = reinterpret_cast<int *>(pdA + Lp);
    int *htab = piA + Lp;
    const int H = 1 << P.hbits;
    float *nd = reinterpret_cast<float *>(htab + H);
    int *ni = reinterpret_cast<int *>(nd + 32);
    float *q = reinterpret_cast<float *>(ni + 32);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);

    const uint8_t *D8 = P.D8;
    const uint4 *q16 = reinterpret_cast<const uint4 *>(q);
    if (D8) {  // self mode: the query is row qi of the byte shadow
        for (int c = lane; c < (d >> 4); c += 32)
            reinterpret_cast<uint4 *>(q)[c] = __ldg(reinterpret_cast<const uint4 *>(D8 + qi * d) + c);
    } else {
        const float *qsrc = P.self ? P.D + qi * d : P.Q + qi * d;
        for (int c = lane; c < nch; c += 32)
            reinterpret_cast<float4 *>(q)[c] = __ldg(reinterpret_cast<const float4 *>(qsrc) + c);
    }
    for (int h = lane; h < H; h += 32) htab[h] = -1;
    int start = P.self ? (int)qi : P.starts[qi];
    bool bad = start < 0 || start >= P.n;
    if (bad) {
        if (lane == 0) record_error(P.err, DERR_BAD_ID, qi);
        start = 0;
    }
    __syncwarp();
    float s0;
    if (D8) {
        s0 = team8_dist_u8(q16, reinterpret_cast<const uint4 *>(D8 + (int64_t)start * d), d >> 4, li);
    } else {
        s0 = team8_dist(q4, reinterpret_cast<const float4 *>(P.D + (int64_t)start * d), nch, li,
                        P.metric);
    }
    int size = 1, cursor = 0;
    if (lane == 0) {
        pdA[0] = s0;
        piA[0] = start;
        htab[hslot(start, P.hbits)] = start;
    }
    __syncwarp();
    unsigned long long ev = 1, ex = 0;
    while (!bad) {
        // first unexpanded entry at or after the cursor
        while (cursor < size) {
            int idx = cursor + lane;
            bool unexp = idx < size && !(piA[idx] & EXP_BIT);
            unsigned b = __ballot_sync(0xffffffffu, unexp);
            if (b) {
                cursor += __ffs(b) - 1;
                break;
            }
            cursor += 32;
        }
        if (cursor >= size) break;
        // a node is expanded at most once, so n expansions bound any search
        if (ex > (unsigned long long)P.n) {
            if (lane == 0) record_error(P.err, DERR_INTERNAL, qi);
            break;
        }
        const int u = piA[cursor] & ID_MASK;
        __syncwarp();
        if (lane == 0) piA[cursor] |= EXP_BIT;
        __syncwarp();
        ++ex;
        int row = u;
        if (P.rows) row = P.rows[u];
        if (row < 0) {
            if (lane == 0) record_error(P.err, DERR_BAD_ID, u);
            __syncwarp();
            continue;
        }
        const int du = min(P.deg[row], P.R);
        for (int c0 = 0; c0 < du; c0 += 32) {
            int j = c0 + lane;
            int v = j < du ? P.nbr[(int64_t)row * P.R + j] : -1;
            if (v >= P.n) {
                record_error(P.err, DERR_BAD_ID, u);
                v = -1;
            }
            bool fresh = false;
            if (v >= 0) {
                unsigned h = hslot(v, P.hbits);
                if (htab[h] != v) {
                    htab[h] = v;
                    fresh = true;
                }
            }
            unsigned fb = __ballot_sync(0xffffffffu, fresh);
            int cnt = __popc(fb);
            if (fresh) ni[__popc(fb & ((1u << lane) - 1))] = v;
            __syncwarp();
            if (D8) {
                batch_dist_u8(D8, d, q16, ni, cnt, nd);
            } else {
                for (int b0 = 0; b0 < cnt; b0 += 4) {
                    int i = b0 + team;
                    int vv = ni[i < cnt ? i : 0];
                    float s = team8_dist(q4, reinterpret_cast<const float4 *>(P.D + (int64_t)vv * d),
                                         nch, li, P.metric);
                    if (li == 0 && i < cnt) nd[i] = s;
                }
            }
            ev += cnt;
            __syncwarp();
            float s = INFINITY;
            int id = INT_MAX;
            if (lane < cnt) {
                s = nd[lane];
                id = ni[lane];
                if (size == L && !pair_less(s, id, pdA[L - 1], piA[L - 1] & ID_MASK)) {
                    id = INT_MAX;
                } else {
                    int pos = pool_lower_bound(pdA, piA, size, s, id);
                    if (pos < size && pdA[pos] == s && (piA[pos] & ID_MASK) == id) id = INT_MAX;
                }
                if (id == INT_MAX) s = INFINITY;
            }
            const unsigned live = __ballot_sync(0xffffffffu, id != INT_MAX);
            const int m2 = __popc(live);
            if (m2 == 0) continue;
            if (m2 > 1) {
                warp_sort32(s, id);  // survivors first, ascending
            } else {
                const int src = __ffs(live) - 1;
                s = __shfl_sync(0xffffffffu, s, src);
                id = __shfl_sync(0xffffffffu, id, src);
                if (lane != 0) {
                    s = INFINITY;
                    id = INT_MAX;
                }
            }
            __syncwarp();
            if (lane < m2) {
                nd[lane] = s;
                ni[lane] = id;
            }
            // final slots of the new entries, against the pool before the merge
            int mydst = L;
            if (lane < m2) mydst = lane + pool_lower_bound(pdA, piA, size, s, id);
            const int first = __shfl_sync(0xffffffffu, mydst, 0);
            __syncwarp();
            // entries at or after `first` move right by the number of new
            // entries below them; chunks from the back, so every slot is read
            // before it is overwritten
            const int moved = size - first;
            for (int c0 = first + ((moved - 1) & ~31); moved > 0 && c0 >= first; c0 -= 32) {
                const int i = c0 + lane;
                float es = 0.f;
                int eid = 0, dst = L;
                if (i < size) {
                    es = pdA[i];
                    eid = piA[i];
                    const int key = eid & ID_MASK;
                    int lo = 0, hi = m2;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (pair_less(nd[mid], ni[mid], es, key)) lo = mid + 1;
                        else hi = mid;
                    }
                    dst = i + lo;
                }
                __syncwarp();
                if (dst < L) {
                    pdA[dst] = es;
                    piA[dst] = eid;
                }
                __syncwarp();
            }
            if (mydst < L) {
                pdA[mydst] = s;
                piA[mydst] = id;
            }
            size = min(L, size + m2);
            if (first < cursor) cursor = first;
            __syncwarp();
        }
    }
    n_exp += ex;
    n_eval += ev;
    // output
    if (P.self) {
        int w = 0;
        for (int base = 0; base < L; base += 32) {
            int i = base + lane;
            int id = i < size ? (piA[i] & ID_MASK) : -1;
            float s = i < size ? pdA[i] : INFINITY;
            bool keep = i < size && id != (int)qi;
            unsigned b = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                int dst = w + __popc(b & ((1u << lane) - 1));
                P.out_i[qi * L + dst] = id;
                if (P.out_s) P.out_s[qi * L + dst] = s;
            }
            w += __popc(b);
        }
        for (int t = w + lane; t < L; t += 32) {
            P.out_i[qi * L + t] = -1;
            if (P.out_s) P.out_s[qi * L + t] = INFINITY;
        }
    } else {
        for (int t = lane; t < P.k; t += 32) {
            bool ok = t < size && !bad;
            P.out_i[qi * P.k + t] = ok ? (piA[t] & ID_MASK) : -1;
            P.out_s[qi * P.k + t] = ok ? pdA[t] : INFINITY;
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(SW * 32, 8) k_search(SearchParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *ws = smem + (size_t)wid * search_warp_smem(P.L, P.hbits, P.d);
    unsigned long long n_exp = 0, n_eval = 0;
    for (;;) {
        int64_t qi = 0;
        if (lane == 0) qi = atomicAdd(P.qcounter, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= P.nq) break;
        search_one(P, qi, ws, n_exp, n_eval);
    }
    if (lane == 0) {
        // algorithmic bytes: one row per evaluation, one adjacency row per expansion
        const unsigned long long row = P.D8 ? (unsigned long long)P.d : 4ull * P.d;
        atomicAdd(P.counters + CNT_SEARCH_EXP, n_exp);
        atomicAdd(P.counters + CNT_SEARCH_EVAL, n_eval);
        atomicAdd(P.counters + CNT_SEARCH_BYTES, n_eval * row + n_exp * 4ull * P.R);
    }
}

std::mutex search_launch_mu;

}  // namespace

pg_status pg_search_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             const int32_t *nbr, const int32_t *deg, int32_t R,
                             const int32_t *rows, const float *Q, int64_t nq,
                             const int32_t *starts, int32_t k, int32_t L, int self,
                             int32_t *out_i, float *out_s, const uint8_t *D8) {
    if (nq == 0) return PG_OK;
    SearchParams P;
    P.D = D;
    P.D8 = self ? D8 : nullptr;
    P.n = n;
    P.d = d;
    P.metric = metric == PG_METRIC_L2SQ ? 0 : 1;
    P.nbr = nbr;
    P.deg = deg;
    P.R = R;
    P.rows = rows;
    P.Q = Q;
    P.nq = nq;
    P.starts = starts;
    P.k = k;
    P.L = L;
    P.self = self;
    // visited-table slots: with byte rows the distances of one expansion
    // cost one round trip whatever their number, so a smaller table (more
    // re-evaluations of forgotten nodes, more resident warps) pays off
    int hb = 9;
    while ((1 << hb) < (D8 && self ? 4 : 8) * L && hb < 12) ++hb;
    P.hbits = hb;
    P.out_i = out_i;
    P.out_s = out_s;
    P.err = ctx->d_err;
    P.counters = ctx->d_counters;
    Scratch<int> qc;
    PG_TRY(qc.alloc(ctx, 1));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(qc.p, 0, sizeof(int), ctx->stream));
    P.qcounter = qc.p;
    size_t smem = search_warp_smem(L, hb, d) * SW;
    if (smem > 227 * 1024)
        return pg_fail(ctx, PG_ERR_CAPACITY, "search: pool/table do not fit shared memory");
    // the shared-memory attribute is per kernel, not per launch: searches
    // of other contexts on other threads (the serving workers) may set a
    // different size, so setting it and launching are one critical section
    std::lock_guard<std::mutex> lk(search_launch_mu);
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(k_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    int bps = 0;
    PG_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_search, SW * 32, smem));
    if (bps < 1) bps = 1;
    int64_t want = (nq + SW - 1) / SW;
    int64_t grid = std::min<int64_t>((int64_t)ctx->num_sms * bps, want);
    pg_timer_begin(ctx, TM_SEARCH);
    k_search<<<(unsigned)grid, SW * 32, smem, ctx->stream>>>(P);
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_SEARCH);
    return PG_OK;
}

static pg_status check_graph_args(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  const int32_t *nbr, const int32_t *deg, int32_t R, int32_t L) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !nbr || !deg) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n >= INT_MAX) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= n < 2^31");
    if (d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need d % 4 == 0 and 4 <= d <= 8192");
    if (R < 1 || R > 64) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= R <= 64");
    if (L < 1 || L > 256) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= L <= 256");
    return PG_OK;
}

extern "C" pg_status pg_acquire_candidates(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                           pg_metric metric, const int32_t *nbr,
                                           const int32_t *deg, int32_t R, int32_t L,
                                           pg_precision precision, int32_t *cand) {
    PG_TRY(check_graph_args(ctx, D, n, d, nbr, deg, R, L));
    if (!cand) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null cand");
    Scratch<uint8_t> d8;
    if (precision == PG_PREC_BF16_SCREEN) {
        DataFacts facts;
        PG_TRY(pg_data_facts(ctx, D, n, d, metric, &facts));
        if (pg_u8_usable(facts, metric, d, precision)) PG_TRY(pg_make_u8(ctx, D, n, d, d8));
    }
    PG_TRY(pg_search_internal(ctx, D, n, d, metric, nbr, deg, R, nullptr, nullptr, n, nullptr, L,
                              L, 1, cand, nullptr, d8.p));
    return pg_sync_check(ctx, "pg_acquire_candidates");
}

extern "C" pg_status pg_search_graph(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                     pg_metric metric, const int32_t *nbr, const int32_t *deg,
                                     int32_t R, const int32_t *rows, const float *Q, int64_t nq,
                                     const int32_t *starts, int32_t k, int32_t L,
                                     pg_precision precision, int32_t *out_ids, float *out_dist) {
    PG_TRY(check_graph_args(ctx, D, n, d, nbr, deg, R, L));
    (void)precision;
    if (!Q || !starts || !out_ids || !out_dist)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (nq < 0 || k < 1 || k > L) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= k <= L");
    PG_TRY(pg_search_internal(ctx, D, n, d, metric, nbr, deg, R, rows, Q, nq, starts, k, L, 0,
                              out_ids, out_dist, nullptr));
    return pg_sync_check(ctx, "pg_search_graph");
}
