// graph.cu -- entry point (medoid) and the connectivity step.
//
// Medoid (Section 3.1, search phase: ep is the point of D closest to the
// centroid).  The centroid is summed in FP64 per coordinate over blocks of
// 1024 consecutive points (one thread per (block, coordinate), index order
// inside the block), the block sums are added in block order and divided
// by n; ep is the exact FP64 argmin of s(x, centroid), ties by id.
//
// Connectivity (Algorithm 2, Algorithm 5): nodes
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
// Rounds are processed in batches that reproduce the sequential order
// exactly.  A batch takes the next B unreached ids r_1 < ... < r_B (no
// unreached id lies between them).  Every round's candidate is computed in
// parallel against the reached set S of the batch start: from r's exact
// kNN list when one of its members is reached with a free slot (the list
// holds the K smallest (s, id), so its best qualifying member is the global
// argmin), otherwise by a scan over the nodes that had a free slot when the
// step began (degrees only grow, so that list covers every candidate).
// A single CTA then commits the rounds in id order; a round whose r was
// reached meanwhile is skipped, a round whose candidate filled up ends the
// batch (it is redone by the next one), and the nodes reached by earlier
// commits of the batch are compared explicitly.  The result is the same as
// deciding the rounds one at a time.
constexpr int CB_B = 128;  // rounds per batch
constexpr int CT = 1024;

struct ConnState {
    int cursor;       // smallest id that may be unreached (n: done)
    int added;        // edges added
    int full_rounds;  // rounds whose candidate came from the scan
    int fast_rounds;  // rounds decided from the kNN list
    int conflicts;    // batches cut short by a candidate that filled up
    int b;            // rounds in the current batch
    int nneed;        // rounds of the batch that need the scan
    int nfree;        // length of the free list
    int ns_cap;       // rounds of this batch the scan serves
    int cut;          // the previous batch ended after a large reached set
    int r[CB_B];
    int flag[CB_B];   // 1: the round's kNN list had no qualifier at the batch start
    int need[CB_B];   // the first ns_cap flagged rounds, ascending
    unsigned long long best[CB_B];    // packed (FP32 bits << 32 | id)
    unsigned long long best64[CB_B];  // FP64 bits of the minimum (non-exact data)
    int best_id[CB_B];                // FP64-resolved argmin (non-exact data)
};

__device__ __forceinline__ unsigned long long pack_sid(float s, int id) {
    return ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)id;
}

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

// nodes that have a free slot when the step begins
__global__ void k_free_list(const int32_t *deg, int64_t n, int R, int *list, ConnState *st) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n && deg[x] < R) list[atomicAdd(&st->nfree, 1)] = (int)x;
}

// single block: BFS from src over unreached nodes, appending to queue[*s_tail..]
__device__ void block_bfs_append(const int32_t *nbr, const int32_t *deg, int R, int64_t n,
                                 int *reached, int *queue, int src, int *s_tail) {
    int head = *s_tail;
    __syncthreads();
    if (threadIdx.x == 0 && atomicCAS(&reached[src], 0, 1) == 0) queue[(*s_tail)++] = src;
    __syncthreads();
    int tail = *s_tail;
    while (head < tail) {
        // one (node, edge) pair per thread, so a frontier of one node still
        // spreads its R edges over R threads
        const int pairs = (tail - head) * R;
        for (int t = threadIdx.x; t < pairs; t += blockDim.x) {
            const int x = queue[head + t / R];
            const int j = t % R;
            if (j >= min(deg[x], R)) continue;
            const int y = nbr[(int64_t)x * R + j];
            if (y < 0 || y >= n || reached[y]) continue;
            if (atomicCAS(&reached[y], 0, 1) == 0) queue[atomicAdd(s_tail, 1)] = y;
        }
        __syncthreads();
        head = tail;
        tail = *s_tail;
        __syncthreads();
    }
}

__global__ void k_connect_init(int64_t n, const int *reached, ConnState *st) {
    __shared__ int s_min;
    if (threadIdx.x == 0) s_min = INT_MAX;
    __syncthreads();
    for (int64_t x = threadIdx.x; x < n; x += blockDim.x)
        if (!reached[x]) {
            atomicMin(&s_min, (int)x);
            break;
        }
    __syncthreads();
    if (threadIdx.x == 0) st->cursor = s_min == INT_MAX ? (int)n : s_min;
}

// the next B unreached ids at or after the cursor, ascending
__global__ void __launch_bounds__(CT) k_cb_select(const int *reached, int64_t n, ConnState *st) {
    __shared__ int s_wcnt[CT / 32];
    __shared__ int s_b;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int from = st->cursor;
    if (tid == 0) {
        s_b = 0;
        st->nneed = 0;
        // one scan covers at most ~8M (point, round) pairs; right after a
        // batch was cut short only a few rounds are likely to be used
        int cap = st->nfree > 0 ? (int)min(128ll, max(4ll, 8000000ll / st->nfree)) : 128;
        st->ns_cap = st->cut ? 4 : cap;
        st->cut = 0;
    }
    for (int i = tid; i < CB_B; i += CT) {
        st->best[i] = ~0ull;
        st->best64[i] = ~0ull;
        st->best_id[i] = INT_MAX;
    }
    __syncthreads();
    for (int64_t base = from; base < n; base += CT) {
        if (s_b >= CB_B) break;
        int64_t x = base + tid;
        bool un = x < n && !reached[x];
        unsigned bal = __ballot_sync(0xffffffffu, un);
        if (lane == 0) s_wcnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < CT / 32; ++w) {
            int c = s_wcnt[w];
            if (w < wid) before += c;
            total += c;
        }
        int pos = s_b + before + __popc(bal & ((1u << lane) - 1));
        if (un && pos < CB_B) st->r[pos] = (int)x;
        __syncthreads();
        if (tid == 0) s_b = min(CB_B, s_b + total);
        __syncthreads();
    }
    if (tid == 0) {
        st->b = s_b;
        if (s_b == 0) st->cursor = (int)n;
    }
}

// rounds whose kNN list has no reached member with a free slot at the batch
// start need the scan (one warp per round)
__global__ void k_cb_fast(int64_t n, const int *reached, const int32_t *deg, int R,
                          const int32_t *__restrict__ knn, int K, ConnState *st) {
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= st->b) return;
    const int r = st->r[i];
    bool any = false;
    for (int j = lane; j < K; j += 32) {
        int x = knn[(int64_t)r * K + j];
        any |= x >= 0 && x < n && reached[x] && deg[x] < R;
    }
    bool none = !__any_sync(0xffffffffu, any);
    if (lane == 0) st->flag[i] = none ? 1 : 0;
}

// Scan of the free list for the rounds that need it.  pass 0: FP32 argmin;
// passes 1 and 2 (non-exact data): FP64 minimum, then smallest id at it,
// among nodes inside the FP32 error bound of the pass-0 minimum.
__global__ void k_cb_scan(const float *__restrict__ D, int64_t n, int d, int metric,
                          const int *reached, const int32_t *deg, int R, const int *free_list,
                          ConnState *st, ErrModel em, int pass, int rch) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    unsigned long long *sbest = reinterpret_cast<unsigned long long *>(cb_smem);
    float *rv = reinterpret_cast<float *>(sbest + CB_B);
    __shared__ int s_need[CB_B];
    __shared__ int s_nneed;
    if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < st->b && c < st->ns_cap; ++i)
            if (st->flag[i]) s_need[c++] = i;
        s_nneed = c;
        if (blockIdx.x == 0) {
            for (int j = 0; j < c; ++j) st->need[j] = s_need[j];
            st->nneed = c;
        }
    }
    __syncthreads();
    const int nneed = s_nneed, nfree = st->nfree;
    if (nneed == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, team = tid >> 3, li = lane & 7;
    const int nteam = blockDim.x / 8, nch = d / 4;
    for (int c0 = 0; c0 < nneed; c0 += rch) {
        const int cn = min(rch, nneed - c0);
        for (int t = tid; t < cn * nch; t += blockDim.x) {
            int j = t / nch, c = t % nch;
            int r = st->r[s_need[c0 + j]];
            reinterpret_cast<float4 *>(rv)[j * nch + c] =
                reinterpret_cast<const float4 *>(D + (int64_t)r * d)[c];
        }
        for (int j = tid; j < cn; j += blockDim.x) sbest[j] = ~0ull;
        __syncthreads();
        for (int base = blockIdx.x * nteam; base < nfree; base += gridDim.x * nteam) {
            const int t = base + team;
            const int x = t < nfree ? free_list[t] : -1;
            const bool ok = x >= 0 && reached[x] && deg[x] < R;
            const float4 *xr = reinterpret_cast<const float4 *>(D + (int64_t)(ok ? x : 0) * d);
            for (int j = 0; j < cn; ++j) {
                float s = team8_dist(reinterpret_cast<const float4 *>(rv + (size_t)j * d), xr, nch, li,
                                     metric);
                if (!ok || li != 0) continue;
                const int i = s_need[c0 + j];
                if (pass > 0 && st->best[i] == ~0ull) continue;
                if (pass == 0) {
                    atomicMin(&sbest[j], pack_sid(s, x));
                    continue;
                }
                float bmin = __uint_as_float((unsigned)(st->best[i] >> 32));
                if (s - 2.f * em.err(s) > bmin + 2.f * em.err(bmin)) continue;
                double s64 = dist64_rows(rv + (size_t)j * d, D + (int64_t)x * d, d, metric);
                unsigned long long b64 = (unsigned long long)__double_as_longlong(s64);
                if (pass == 1) atomicMin(&st->best64[i], b64);
                else if (b64 == st->best64[i]) atomicMin(&st->best_id[i], x);
            }
        }
        __syncthreads();
        if (pass == 0)
            for (int j = tid; j < cn; j += blockDim.x)
                if (sbest[j] != ~0ull) atomicMin(&st->best[s_need[c0 + j]], sbest[j]);
        __syncthreads();
    }
}

// commit the batch's rounds in id order (one CTA).  For each round the
// argmin over r's kNN list restricted to the nodes reached and free *now*
// is recomputed: when it exists it is the global argmin (ball argument),
// whatever was reached earlier in the batch.  Otherwise the scan result of
// the batch start competes with the free nodes reached earlier in the batch
// (measured by teams of eight threads); a round without a scan result whose
// list qualifier filled up ends the batch.
constexpr int CTC = 256;  // threads of the commit CTA

__device__ void list_argmin(const float *__restrict__ D, int64_t n, int d, int metric,
                            const int *reached, const int32_t *deg, int R,
                            const int32_t *__restrict__ knn, int K, int r, const float *rq,
                            ErrModel em, int exact, unsigned long long *s_b,
                            unsigned long long *s_b64, int *s_bid, float *s_cs, int *s_ci) {
    const int tid = threadIdx.x, lane = tid & 31, team = tid >> 3, li = lane & 7;
    const int nteam = blockDim.x / 8, nch = d / 4;
    if (tid == 0) {
        *s_b = ~0ull;
        *s_b64 = ~0ull;
        *s_bid = INT_MAX;
    }
    __syncthreads();
    for (int base = 0; base < K; base += nteam) {
        const int j = base + team;
        int x = j < K ? knn[(int64_t)r * K + j] : -1;
        bool ok = x >= 0 && x < n && reached[x] && deg[x] < R;
        if (!__any_sync(0xffffffffu, ok)) {
            if (li == 0 && j < K) s_ci[j] = -1;
            continue;
        }
        float s = team8_dist(reinterpret_cast<const float4 *>(rq),
                             reinterpret_cast<const float4 *>(D + (int64_t)(ok ? x : r) * d), nch,
                             li, metric);
        if (li == 0 && j < K) {
            s_cs[j] = ok ? s : INFINITY;
            s_ci[j] = ok ? x : -1;
            if (ok) atomicMin(s_b, pack_sid(s, x));
        }
    }
    __syncthreads();
    if (exact || *s_b == ~0ull) {
        if (tid == 0 && *s_b != ~0ull) *s_bid = (int)(*s_b & 0xffffffffu);
        __syncthreads();
        return;
    }
    const float bmin = __uint_as_float((unsigned)(*s_b >> 32));
    for (int j = tid; j < K; j += blockDim.x) {
        if (s_ci[j] < 0) continue;
        float s = s_cs[j];
        if (s - 2.f * em.err(s) > bmin + 2.f * em.err(bmin)) continue;
        double s64 = dist64_rows(rq, D + (int64_t)s_ci[j] * d, d, metric);
        atomicMin(s_b64, (unsigned long long)__double_as_longlong(s64));
    }
    __syncthreads();
    for (int j = tid; j < K; j += blockDim.x) {
        if (s_ci[j] < 0) continue;
        float s = s_cs[j];
        if (s - 2.f * em.err(s) > bmin + 2.f * em.err(bmin)) continue;
        double s64 = dist64_rows(rq, D + (int64_t)s_ci[j] * d, d, metric);
        if ((unsigned long long)__double_as_longlong(s64) == *s_b64) atomicMin(s_bid, s_ci[j]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CTC)
k_cb_commit(const float *__restrict__ D, int64_t n, int d, int metric, int32_t *nbr, int32_t *deg,
            int R, int *reached, int *queue, ConnState *st, const int32_t *__restrict__ knn,
            int K, ErrModel em, int exact, int *err) {
    extern __shared__ __align__(16) float cm_rq[];  // r's vector [d]
    __shared__ int s_tail, s_stop, s_nb_id, s_lid, s_nfree;
    __shared__ unsigned long long s_nb, s_nb64, s_lb, s_lb64;
    __shared__ int s_r[CB_B], s_scan[CB_B], s_bid[CB_B];
    __shared__ unsigned long long s_best64[CB_B], s_best[CB_B];
    __shared__ float s_cs[256];
    __shared__ int s_ci[256];
    __shared__ int s_added, s_full, s_fast;
    const int b = st->b;
    if (b == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, team = tid >> 3, li = lane & 7;
    const int nteam = CTC / 8, nch = d / 4;
    for (int i = tid; i < b; i += CTC) {
        s_r[i] = st->r[i];
        s_best[i] = st->best[i];
        s_best64[i] = st->best64[i];
        s_bid[i] = st->best_id[i];
        s_scan[i] = 0;
    }
    if (tid == 0) {
        s_tail = 0;
        s_stop = 0;
        s_added = 0;
        s_full = 0;
        s_fast = 0;
    }
    __syncthreads();
    for (int j = tid; j < st->nneed; j += CTC) s_scan[st->need[j]] = 1;
    __syncthreads();
    for (int i = 0; i < b; ++i) {
        const int r = s_r[i];
        if (reached[r]) continue;
        for (int c = tid; c < nch; c += CTC)
            reinterpret_cast<float4 *>(cm_rq)[c] = reinterpret_cast<const float4 *>(D + (int64_t)r * d)[c];
        __syncthreads();
        int q = -1;
        // a scanned round had no list qualifier at the batch start: members
        // that qualify now were reached in this batch and are among the
        // nodes checked below, so its list need not be measured again
        if (!s_scan[i]) {
            list_argmin(D, n, d, metric, reached, deg, R, knn, knn ? K : 0, r, cm_rq, em, exact,
                        &s_lb, &s_lb64, &s_lid, s_cs, s_ci);
        } else if (tid == 0) {
            s_lid = INT_MAX;
        }
        __syncthreads();
        if (s_lid != INT_MAX) {
            q = s_lid;
            if (tid == 0) s_fast += 1;
        } else if (!s_scan[i]) {  // its list qualifier filled up: redo in the next batch
            if (tid == 0) {
                st->cursor = r;
                st->conflicts += 1;
                s_stop = 1;
            }
            __syncthreads();
            break;
        } else {
            int p;
            float ps = INFINITY;
            double ps64 = INFINITY;
            if (exact) {
                unsigned long long pk = s_best[i];
                p = pk == ~0ull ? -1 : (int)(pk & 0xffffffffu);
                if (p >= 0) ps = __uint_as_float((unsigned)(pk >> 32));
            } else {
                p = s_bid[i] == INT_MAX ? -1 : s_bid[i];
                if (p >= 0) ps64 = __longlong_as_double((long long)s_best64[i]);
            }
            if (p >= 0 && deg[p] >= R) {  // filled by an earlier commit
                if (tid == 0) {
                    st->cursor = r;
                    st->conflicts += 1;
                    s_stop = 1;
                }
                __syncthreads();
                break;
            }
            // free nodes reached earlier in this batch compete with p
            const int nr = s_tail;
            if (tid == 0) {
                s_nb = ~0ull;
                s_nb64 = ~0ull;
                s_nb_id = INT_MAX;
            }
            __syncthreads();
            for (int base = 0; base < nr; base += nteam) {
                const int t = base + team;
                const int x = t < nr ? queue[t] : -1;
                const bool ok = x >= 0 && deg[x] < R;
                if (!__any_sync(0xffffffffu, ok)) continue;
                float s = team8_dist(reinterpret_cast<const float4 *>(cm_rq),
                                     reinterpret_cast<const float4 *>(D + (int64_t)(ok ? x : r) * d),
                                     nch, li, metric);
                if (!ok || li != 0) continue;
                if (exact) {
                    atomicMin(&s_nb, pack_sid(s, x));
                } else {
                    double s64 = dist64_rows(D + (int64_t)x * d, cm_rq, d, metric);
                    atomicMin(&s_nb64, (unsigned long long)__double_as_longlong(s64));
                }
            }
            __syncthreads();
            if (!exact && s_nb64 != ~0ull) {
                for (int t = tid; t < nr; t += CTC) {
                    int x = queue[t];
                    if (deg[x] >= R) continue;
                    double s64 = dist64_rows(D + (int64_t)x * d, cm_rq, d, metric);
                    if ((unsigned long long)__double_as_longlong(s64) == s_nb64)
                        atomicMin(&s_nb_id, x);
                }
                __syncthreads();
            }
            q = p;
            if (exact) {
                if (s_nb != ~0ull && (p < 0 || s_nb < pack_sid(ps, p))) q = (int)(s_nb & 0xffffffffu);
            } else if (s_nb_id != INT_MAX) {
                double qs = __longlong_as_double((long long)s_nb64);
                if (p < 0 || qs < ps64 || (qs == ps64 && s_nb_id < p)) q = s_nb_id;
            }
            if (tid == 0 && q >= 0) s_full += 1;
        }
        if (tid == 0) {
            if (q < 0) {
                record_error(err, DERR_NO_SLOT, r);
                st->cursor = (int)n;
                s_stop = 2;
            } else {
                int dq = deg[q];
                nbr[(int64_t)q * R + dq] = r;
                deg[q] = dq + 1;
                s_added += 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        const int before = s_tail;
        block_bfs_append(nbr, deg, R, n, reached, queue, r, &s_tail);
        // a large reached set would make every later round of the batch
        // measure against it: restart from a fresh batch instead
        if (s_tail - before > 256 && i + 1 < b) {
            if (tid == 0) {
                st->cursor = s_r[i + 1];
                st->cut = 1;
                s_stop = 3;
            }
            __syncthreads();
            break;
        }
    }
    if (tid == 0) {
        st->added += s_added;
        st->full_rounds += s_full;
        st->fast_rounds += s_fast;
        if (!s_stop) st->cursor = s_r[b - 1] + 1 < n ? s_r[b - 1] + 1 : (int)n;
    }
    (void)s_nfree;
}



// ------------------------------------------------- connect, exact data
// For exact data the rounds of a batch are decided from work done for all
// of them at once, again reproducing the one-round-at-a-time result:
//  * the argmin over the nodes reached and free at the batch start, for
//    every round, by one tensor-core pass over all points (pg_tc_argmin);
//  * the closure of every round: the nodes BFS from r_i reaches through
//    nodes unreached at the batch start.  Edges added during the batch start
//    at reached nodes, so round i's BFS reaches exactly its closure minus
//    what earlier rounds reached, and the nodes reached before round i are
//    the batch-start set plus the closures of the committed rounds j < i.
//    A round j < i that was skipped had r_j inside an earlier committed
//    closure, which then contains all of closure j; so "committed j < i"
//    may be read as "every j < i" in both uses below;
//  * for every round, the argmin over the closures of all earlier rounds
//    (free at the batch start) and whether r_i lies in one of them.
// A single thread then walks the rounds in order: a round whose r lies in
// an earlier closure is skipped; otherwise its node is the smaller of the
// two argmins.  Only the chosen node's free slot needs checking (both
// sources cover a superset of the nodes free now); when it filled up during
// the batch, the batch ends there.  A closure longer than CX_C nodes ends
// the batch after its round, which is then reached by a full BFS.
constexpr int CX_C = 2048;       // closure capacity per round
constexpr int CX_H = 4096;       // hash slots of one closure BFS (> CX_C + threads)
constexpr int CX_PAIRS = 32768;  // closure nodes one round compares against

struct ConnX {
    int cursor, added, full_rounds, fast_rounds, conflicts, b, big_rounds, nfree;
    int r[CB_B];
    int comp_n[CB_B];  // closure sizes; CX_C + 1: overflowed
    int ready[CB_B];   // the closure pass covered this round
    int skip[CB_B];    // r_i lies in an earlier round's closure
    unsigned long long best[CB_B];  // argmin over the batch-start reached free nodes
    unsigned long long cmin[CB_B];  // argmin over the earlier closures' free nodes
};

__global__ void __launch_bounds__(CT) k_cx_select(const int *reached, int64_t n, ConnX *st) {
    __shared__ int s_wcnt[CT / 32];
    __shared__ int s_b;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int from = st->cursor;
    if (tid == 0) s_b = 0;
    for (int i = tid; i < CB_B; i += CT) {
        st->best[i] = ~0ull;
        st->cmin[i] = ~0ull;
        st->ready[i] = 0;
        st->skip[i] = 0;
        st->comp_n[i] = 0;
    }
    __syncthreads();
    for (int64_t base = from; base < n; base += CT) {
        if (s_b >= CB_B) break;
        const int64_t x = base + tid;
        const bool un = x < n && !reached[x];
        const unsigned bal = __ballot_sync(0xffffffffu, un);
        if (lane == 0) s_wcnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < CT / 32; ++w) {
            const int c = s_wcnt[w];
            if (w < wid) before += c;
            total += c;
        }
        const int pos = s_b + before + __popc(bal & ((1u << lane) - 1));
        if (un && pos < CB_B) st->r[pos] = (int)x;
        __syncthreads();
        if (tid == 0) s_b = min(CB_B, s_b + total);
        __syncthreads();
    }
    if (tid == 0) {
        st->b = s_b;
        if (s_b == 0) st->cursor = (int)n;
    }
}

// closure of round blockIdx.x: BFS from r over nodes unreached at the batch
// start, with an exact hash set in shared memory
__global__ void __launch_bounds__(256) k_cx_comp(const int32_t *nbr, const int32_t *deg, int R,
                                                 int64_t n, const int *reached, ConnX *st,
                                                 int *comp) {
    __shared__ int set[CX_H];
    __shared__ int s_tail, s_big;
    const int i = blockIdx.x, tid = threadIdx.x;
    if (i >= st->b) return;
    int *q = comp + (size_t)i * CX_C;
    volatile int *big = &s_big;
    for (int h = tid; h < CX_H; h += blockDim.x) set[h] = -1;
    __syncthreads();
    const int r = st->r[i];
    if (tid == 0) {
        set[((unsigned)r * 2654435761u) >> 20] = r;
        q[0] = r;
        s_tail = 1;
        s_big = 0;
    }
    __syncthreads();
    int head = 0, tail = 1;
    while (head < tail) {
        const int pairs = (tail - head) * R;
        for (int t = tid; t < pairs && !*big; t += blockDim.x) {
            const int x = q[head + t / R];
            const int j = t % R;
            if (j >= min(deg[x], R)) continue;
            const int y = nbr[(int64_t)x * R + j];
            if (y < 0 || y >= n || reached[y]) continue;
            unsigned h = ((unsigned)y * 2654435761u) >> 20;
            int probe = 0;
            for (; probe < CX_H; ++probe) {
                const int old = atomicCAS(&set[h], -1, y);
                if (old == -1) {
                    const int pos = atomicAdd(&s_tail, 1);
                    if (pos < CX_C) q[pos] = y;
                    else *big = 1;
                    break;
                }
                if (old == y) break;
                h = (h + 1) & (CX_H - 1);
            }
            if (probe == CX_H) *big = 1;
        }
        __syncthreads();
        if (*big) break;
        head = tail;
        tail = s_tail;
        __syncthreads();
    }
    if (tid == 0) st->comp_n[i] = (s_big || s_tail > CX_C) ? CX_C + 1 : s_tail;
}

// Every (round i, node x of an earlier round's closure) pair, spread over
// the grid: r_i in a closure marks i skipped; a free x competes for cmin[i].
// Rounds behind an overflowed closure or past CX_PAIRS nodes are left out
// (the walk stops before them).
__global__ void __launch_bounds__(256) k_cx_pair(const float *__restrict__ D, int d, int metric,
                                                 const int32_t *deg, int R, ConnX *st,
                                                 const int *comp) {
    __shared__ int s_pre[CB_B + 1];        // closure nodes of rounds < i
    __shared__ long long s_acc[CB_B + 1];  // pairs of rounds < i
    __shared__ int s_last;                 // rounds [0, s_last) take part
    const int tid = threadIdx.x, lane = tid & 31, li = lane & 7;
    const int b = st->b;
    if (tid == 0) {
        int pre = 0, last = b;
        long long acc = 0;
        for (int i = 0; i < b; ++i) {
            s_pre[i] = pre;
            s_acc[i] = acc;
            if (pre > CX_PAIRS) {
                last = i;
                break;
            }
            acc += pre;
            const int c = st->comp_n[i];
            if (c > CX_C) {  // the walk ends at round i
                last = i + 1;
                s_pre[i + 1] = pre;
                s_acc[i + 1] = acc;
                break;
            }
            pre += c;
        }
        if (last == b) {
            s_pre[b] = pre;
            s_acc[b] = acc;
        }
        s_last = last;
    }
    __syncthreads();
    const int last = s_last;
    const long long total = s_acc[last];
    if (blockIdx.x == 0)
        for (int i = tid; i < b; i += blockDim.x) st->ready[i] = i < last;
    const int nch = d / 4;
    const long long nteam = (long long)gridDim.x * (blockDim.x / 8);
    for (long long f0 = (long long)blockIdx.x * (blockDim.x / 8); f0 < total; f0 += nteam) {
        const long long f = f0 + (tid >> 3);
        int i = 0, x = -1, r = 0;
        if (f < total) {
            int lo = 0, hi = last - 1;  // last i with s_acc[i] <= f
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_acc[mid] <= f) lo = mid;
                else hi = mid - 1;
            }
            i = lo;
            const int t = (int)(f - s_acc[i]);  // < s_pre[i]
            int jl = 0, jh = i - 1;             // last j with s_pre[j] <= t
            while (jl < jh) {
                const int mid = (jl + jh + 1) >> 1;
                if (s_pre[mid] <= t) jl = mid;
                else jh = mid - 1;
            }
            x = comp[(size_t)jl * CX_C + (t - s_pre[jl])];
            r = st->r[i];
        }
        const bool cand = x >= 0 && x != r && deg[x] < R;
        if (li == 0 && x >= 0 && x == r) st->skip[i] = 1;
        if (!__any_sync(0xffffffffu, cand)) continue;
        const float s = team8_dist(reinterpret_cast<const float4 *>(D + (int64_t)r * d),
                                   reinterpret_cast<const float4 *>(D + (int64_t)(cand ? x : r) * d),
                                   nch, li, metric);
        if (li == 0 && cand) atomicMin(&st->cmin[i], pack_sid(s, x));
    }
}

// the rounds of the batch in order (one thread), then the edges, the
// reached marks and, after an overflowed closure, the BFS from its round
constexpr int CXD = 256;  // threads of the decide CTA

__global__ void __launch_bounds__(CXD)
k_cx_decide(int32_t *nbr, int32_t *deg, int R, int64_t n, int *reached, int *queue, ConnX *st,
            const int *comp, int *err) {
    __shared__ unsigned long long s_c[CB_B];
    __shared__ int s_r[CB_B], s_cn[CB_B], s_ready[CB_B], s_skip[CB_B], s_scan[CB_B];
    __shared__ int s_prev[CB_B], s_done[CB_B], s_rank[CB_B], s_d0[CB_B];
    __shared__ int s_stop, s_stop_i, s_tail;
    const int b = st->b;
    if (b == 0) return;
    const int tid = threadIdx.x;
    for (int i = tid; i < b; i += CXD) {
        const unsigned long long bs = st->best[i], cm = st->cmin[i];
        s_c[i] = bs <= cm ? bs : cm;
        s_scan[i] = bs <= cm;
        s_r[i] = st->r[i];
        s_cn[i] = st->comp_n[i];
        s_ready[i] = st->ready[i];
        s_skip[i] = st->skip[i];
        s_done[i] = 0;
        s_rank[i] = 0;
    }
    __syncthreads();
    // the previous round with the same candidate node, and that node's degree
    for (int i = tid; i < b; i += CXD) {
        int prev = -1;
        if (s_c[i] != ~0ull)
            for (int j = i - 1; j >= 0; --j)
                if (s_c[j] == ~0ull ? false : (unsigned)s_c[j] == (unsigned)s_c[i]) {
                    prev = j;
                    break;
                }
        s_prev[i] = prev;
        s_d0[i] = s_c[i] != ~0ull ? deg[(int)(s_c[i] & 0xffffffffu)] : 0;
    }
    __syncthreads();
    if (tid == 0) {
        int stop = 0, stop_i = b;
        for (int i = 0; i < b; ++i) {
            if (!s_ready[i]) {
                stop = 4;
                stop_i = i;
                break;
            }
            if (s_skip[i]) continue;  // r_i was reached by an earlier round
            if (s_c[i] == ~0ull) {
                stop = 2;
                stop_i = i;
                break;
            }
            int cnt = 0;  // edges its node took earlier in this batch
            for (int j = s_prev[i]; j >= 0; j = s_prev[j]) cnt += s_done[j];
            if (s_d0[i] + cnt >= R) {
                stop = 1;
                stop_i = i;
                break;
            }
            s_done[i] = 1;
            s_rank[i] = cnt;
            if (s_cn[i] > CX_C) {  // committed; its closure overflowed
                stop = 3;
                stop_i = i;
                break;
            }
        }
        s_stop = stop;
        s_stop_i = stop_i;
        s_tail = 0;
    }
    __syncthreads();
    const int stop = s_stop, stop_i = s_stop_i;
    // edges: the k-th edge of a node goes to slot deg0 + k
    int added = 0, scanned = 0;
    for (int i = tid; i < b; i += CXD) {
        if (!s_done[i]) continue;
        const int p = (int)(s_c[i] & 0xffffffffu);
        nbr[(int64_t)p * R + s_d0[i] + s_rank[i]] = s_r[i];
        bool last = true;
        for (int j = i + 1; j < b; ++j) last = last && !(s_done[j] && (unsigned)s_c[j] == (unsigned)p);
        if (last) deg[p] = s_d0[i] + s_rank[i] + 1;
        ++added;
        scanned += s_scan[i];
    }
    // reached marks of the committed closures (an overflowed one is left to the BFS)
    for (int i = 0; i < b; ++i) {
        if (!s_done[i] || s_cn[i] > CX_C) continue;
        for (int t = tid; t < s_cn[i]; t += CXD) reached[comp[(size_t)i * CX_C + t]] = 1;
    }
    if (added) {
        atomicAdd(&st->added, added);
        atomicAdd(&st->full_rounds, scanned);
        atomicAdd(&st->fast_rounds, added - scanned);
    }
    __syncthreads();
    if (stop == 3) block_bfs_append(nbr, deg, R, n, reached, queue, s_r[stop_i], &s_tail);
    if (tid == 0) {
        if (stop == 1) st->conflicts += 1;
        if (stop == 3) st->big_rounds += 1;
        if (stop == 2) {
            record_error(err, DERR_NO_SLOT, s_r[stop_i]);
            st->cursor = (int)n;
        } else if (stop == 1 || stop == 4) {
            st->cursor = s_r[stop_i];
        } else if (stop == 3 && stop_i + 1 < b) {
            st->cursor = s_r[stop_i + 1];
        } else {
            st->cursor = s_r[b - 1] + 1 < n ? s_r[b - 1] + 1 : (int)n;
        }
    }
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

// Batches of the exact-data connect (see ConnX); the state starts from the
// reached set and cursor of `init`.
static pg_status connect_exact(pg_ctx *ctx, const float *D, int64_t n, int32_t d, int32_t *nbr,
                               int32_t *deg, int32_t R, int *reached, int *queue,
                               const ConnState *init, int64_t *host_added) {
    TcArgmin tc;
    PG_TRY(pg_tc_argmin_init(ctx, D, n, d, deg, R, tc));
    Scratch<ConnX> st;
    Scratch<int> comp;
    PG_TRY(st.alloc(ctx, 1));
    PG_TRY(comp.alloc(ctx, (size_t)CB_B * CX_C));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(st.p, 0, sizeof(ConnX), ctx->stream));
    // cursor and free-list length from the common set-up
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(&st.p->cursor, &init->cursor, sizeof(int),
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(&st.p->nfree, &init->nfree, sizeof(int),
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    // One group = 8 batches of 6 launches each, the same launches every time
    // (all state lives in ConnX): the loop is launch-bound, so the group is
    // captured once as a CUDA graph and replayed (direct launches if the
    // capture is refused).  Per-kernel timers only on the direct path.
    auto issue_group = [&](bool timed) -> pg_status {
        for (int g = 0; g < 8; ++g) {
            if (timed) pg_timer_begin(ctx, TM_CSELECT);
            k_cx_select<<<1, CT, 0, ctx->stream>>>(reached, n, st.p);
            PG_LAUNCHED(ctx);
            if (timed) pg_timer_end(ctx, TM_CSELECT);
            if (timed) pg_timer_begin(ctx, TM_CSCAN);
            PG_TRY(pg_tc_argmin(ctx, tc, D, st.p->r, &st.p->b, reached, deg, R, st.p->best));
            if (timed) pg_timer_end(ctx, TM_CSCAN);
            if (timed) pg_timer_begin(ctx, TM_CFAST);
            k_cx_comp<<<CB_B, 256, 0, ctx->stream>>>(nbr, deg, R, n, reached, st.p, comp.p);
            PG_LAUNCHED(ctx);
            k_cx_pair<<<ctx->num_sms * 2, 256, 0, ctx->stream>>>(D, d, 0, deg, R, st.p, comp.p);
            PG_LAUNCHED(ctx);
            if (timed) pg_timer_end(ctx, TM_CFAST);
            if (timed) pg_timer_begin(ctx, TM_CCOMMIT);
            k_cx_decide<<<1, CXD, 0, ctx->stream>>>(nbr, deg, R, n, reached, queue, st.p, comp.p,
                                                   ctx->d_err);
            PG_LAUNCHED(ctx);
            if (timed) pg_timer_end(ctx, TM_CCOMMIT);
        }
        return PG_OK;
    };
    struct GraphExec {
        cudaGraphExec_t e = nullptr;
        ~GraphExec() {
            if (e) cudaGraphExecDestroy(e);
        }
    } exec;
    int64_t per_group = 0;
    {
        // captured on a private stream (the context's stream may be the legacy
        // default stream, which cannot capture); replayed on the context's
        const int64_t l0 = ctx->launches;
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess) {
            cudaStream_t saved = ctx->stream;
            ctx->stream = cap;
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const pg_status cs = issue_group(false);
                const cudaError_t e = cudaStreamEndCapture(cap, &graph);
                if (cs == PG_OK && e == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec.e, graph, 0) != cudaSuccess)
                    exec.e = nullptr;
                if (graph) cudaGraphDestroy(graph);
            }
            ctx->stream = saved;
            cudaStreamDestroy(cap);
        }
        cudaGetLastError();  // a refused capture leaves no sticky error
        per_group = ctx->launches - l0;
        ctx->launches = l0;
    }
    const int64_t max_groups = n / 8 + 2;
    for (int64_t group = 0;; ++group) {
        if (group > max_groups)
            return pg_fail(ctx, PG_ERR_INTERNAL, "connect: no progress after %lld batches",
                           (long long)(group * 8));
        if (exec.e) {
            PG_TRY_CUDA(ctx, cudaGraphLaunch(exec.e, ctx->stream));
            ctx->launches += per_group;
        } else {
            PG_TRY(issue_group(true));
        }
        int h[8];
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, st.p, sizeof h, cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PG_TRY(pg_sync_check(ctx, "connect"));
        memcpy(h, ctx->h_pinned, sizeof h);
        if (h[0] >= n) {
            if (host_added) *host_added = h[1];
            ctx->connect_edges += h[1];
            ctx->connect_full_rounds += h[2];
            ctx->connect_why_full += h[4];
            ctx->connect_free += h[7];
            return PG_OK;
        }
    }
}

pg_status pg_connect_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              int32_t *nbr, int32_t *deg, int32_t R, int64_t ep,
                              const DataFacts &facts, const int32_t *knn, int32_t K,
                              int64_t *host_added) {
    Scratch<int> reached, queue, fcnt, freel;
    Scratch<ConnState> st;
    PG_TRY(reached.alloc(ctx, (size_t)n));
    PG_TRY(queue.alloc(ctx, (size_t)n * 2));
    PG_TRY(fcnt.alloc(ctx, 2));
    PG_TRY(freel.alloc(ctx, (size_t)n));
    PG_TRY(st.alloc(ctx, 1));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(reached.p, 0, (size_t)n * 4, ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(st.p, 0, sizeof(ConnState), ctx->stream));
    pg_timer_begin(ctx, TM_CONNECT);
    k_free_list<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(deg, n, R, freel.p, st.p);
    PG_LAUNCHED(ctx);
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
    if (metric == PG_METRIC_L2SQ && facts.exact && facts.bf16_exact && pg_tc_argmin_supported(d)) {
        PG_TRY(connect_exact(ctx, D, n, d, nbr, deg, R, reached.p, queue.p, st.p, host_added));
        pg_timer_end(ctx, TM_CONNECT);
        return PG_OK;
    }
    const ErrModel em = pg_err_model(metric, d, facts, false);
    const int m = metric == PG_METRIC_L2SQ ? 0 : 1;
    const bool exact = facts.exact != 0;
    const size_t smem_r = (size_t)d * 4;
    int rch = (int)std::min<size_t>(CB_B, (size_t)(96 * 1024 - CB_B * 8) / ((size_t)d * 4));
    if (rch < 1) rch = 1;
    const size_t smem_scan = CB_B * 8 + (size_t)rch * d * 4;
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(k_cb_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_scan));
    const int grid = ctx->num_sms * 4;
    // every batch commits at least its first round
    const int64_t max_groups = n / 8 + 2;
    for (int64_t group = 0;; ++group) {
        if (group > max_groups)
            return pg_fail(ctx, PG_ERR_INTERNAL, "connect: no progress after %lld batches",
                           (long long)(group * 8));
        for (int g = 0; g < 8; ++g) {
            pg_timer_begin(ctx, TM_CSELECT);
            k_cb_select<<<1, CT, 0, ctx->stream>>>(reached.p, n, st.p);
            PG_LAUNCHED(ctx);
            pg_timer_end(ctx, TM_CSELECT);
            pg_timer_begin(ctx, TM_CFAST);
            k_cb_fast<<<CB_B / 8, 256, 0, ctx->stream>>>(n, reached.p, deg, R, knn, knn ? K : 0,
                                                          st.p);
            PG_LAUNCHED(ctx);
            pg_timer_end(ctx, TM_CFAST);
            for (int pass = 0; pass < (exact ? 1 : 3); ++pass) {
                pg_timer_begin(ctx, TM_CSCAN);
                k_cb_scan<<<grid, 256, smem_scan, ctx->stream>>>(D, n, d, m, reached.p, deg, R,
                                                                 freel.p, st.p, em, pass, rch);
                PG_LAUNCHED(ctx);
                pg_timer_end(ctx, TM_CSCAN);
            }
            pg_timer_begin(ctx, TM_CCOMMIT);
            k_cb_commit<<<1, CTC, smem_r, ctx->stream>>>(D, n, d, m, nbr, deg, R, reached.p,
                                                         queue.p, st.p, knn, knn ? K : 0, em,
                                                         exact ? 1 : 0, ctx->d_err);
            PG_LAUNCHED(ctx);
            pg_timer_end(ctx, TM_CCOMMIT);
        }
        int h[8];
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, st.p, sizeof h, cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PG_TRY(pg_sync_check(ctx, "connect"));
        memcpy(h, ctx->h_pinned, sizeof h);
        if (h[0] >= n) {
            if (host_added) *host_added = h[1];
            ctx->connect_edges += h[1];
            ctx->connect_full_rounds += h[2];
            ctx->connect_why_full += h[4];
            ctx->connect_free += h[7];
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

// ---------------------------------------- connectivity with edge replacement
// A reading for graphs whose reached nodes are all full (the paper's
// connectivity step only says that extra edges link the components): when
// no reached node has a free slot for the smallest unreached id r, the
// reached node p nearest to r that still holds an edge not added by this
// step gives up the last such edge in its list (its farthest original
// neighbour) for r, and the reached set is recomputed from ep.  Until the
// first such round the step equals the plain one, which therefore runs
// batched as above; each refusal is followed by one replacement and a new
// plain pass from the changed graph.  Every replacement removes an original
// edge and every plain link grows the reached set, so the loop ends.
namespace {

struct RepState {
    unsigned long long key32;  // exact data: FP32 bits << 32 | id; else min FP32 bits
    unsigned long long key64;  // min FP64 bits among the candidates inside the bound
    int id64;                  // smallest id at that FP64 minimum
};

// Argmin over reached nodes x with orig[x] > 0 (an original edge left) of
// (s(x, r), x); one warp per node.  Exact data: one pass on packed keys.
// Otherwise pass 0 takes the FP32 minimum, pass 1 the FP64 minimum among
// nodes whose FP32 distance lies within the error bounds of it, pass 2 the
// smallest id at that FP64 value.
__global__ void k_rep_scan(const float *__restrict__ D, int64_t n, int d, int metric, int64_t r,
                           const int *__restrict__ reached, const int32_t *__restrict__ orig,
                           ErrModel em, int exact, int pass, RepState *st) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float *xr = D + r * d;
    const float smin = __uint_as_float((unsigned)(exact ? 0u : st->key32));
    for (int64_t x = w0; x < n; x += nw) {
        if (!reached[x] || orig[x] <= 0) continue;
        const float *xx = D + x * d;
        float acc = 0.f;
        if (metric == 0) {
            for (int c = lane; c < d; c += 32) {
                const float t = xx[c] - xr[c];
                acc = fmaf(t, t, acc);
            }
        } else {
            for (int c = lane; c < d; c += 32) acc = fmaf(xx[c], xr[c], acc);
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const float s = metric == 0 ? acc : fmaxf(2.f - 2.f * acc, 0.f);
        if (lane != 0) continue;
        if (exact) {
            atomicMin(&st->key32, ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)x);
        } else if (pass == 0) {
            atomicMin(&st->key32, (unsigned long long)__float_as_uint(s));
        } else if (s - em.err(s) <= smin + em.err(smin)) {
            const double s64 = dist64_rows(xx, xr, d, metric);
            const unsigned long long b = (unsigned long long)__double_as_longlong(s64);
            if (pass == 1) atomicMin(&st->key64, b);
            else if (b == st->key64) atomicMin(&st->id64, (int)x);
        }
    }
}

// node p gives up its last original edge for r
__global__ void k_rep_replace(int32_t *nbr, int R, int32_t *orig, int p, int r) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int slot = orig[p] - 1;
        nbr[(int64_t)p * R + slot] = r;
        orig[p] = slot;
    }
}

__global__ void k_rep_mark(int *reached, int64_t ep, int *queue) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        reached[ep] = 1;
        queue[0] = (int)ep;
    }
}

__global__ void k_deg_sum(const int32_t *deg, const int32_t *deg0, int64_t n,
                          unsigned long long *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long v = i < n ? (long long)deg[i] - (long long)deg0[i] : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

}  // namespace

// The connectivity step with edge replacement (see above).  *host_added
// (may be NULL) = edges added, replacements included; *host_replaced (may be
// NULL) = replacements.  PG_ERR_CAPACITY when a refused round finds no
// reached node with an original edge either.
pg_status pg_connect_replace_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                      pg_metric metric, int32_t *nbr, int32_t *deg, int32_t R,
                                      int64_t ep, const DataFacts &facts, const int32_t *knn,
                                      int32_t K, int64_t *host_added, int64_t *host_replaced) {
    Scratch<int32_t> deg0, orig;
    Scratch<int> reached, queue, fcnt;
    Scratch<RepState> st;
    Scratch<unsigned long long> sum;
    PG_TRY(deg0.alloc(ctx, (size_t)n));
    PG_TRY(orig.alloc(ctx, (size_t)n));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(deg0.p, deg, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(orig.p, deg, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    const ErrModel em = pg_err_model(metric, d, facts, false);
    const int m = metric == PG_METRIC_L2SQ ? 0 : 1;
    const int exact = facts.exact ? 1 : 0;
    int64_t replaced = 0;
    for (int64_t round = 0;; ++round) {
        if (round > n + 1)
            return pg_fail(ctx, PG_ERR_INTERNAL, "connect: no progress after %lld replacements",
                           (long long)round);
        pg_status s = pg_connect_internal(ctx, D, n, d, metric, nbr, deg, R, ep, facts, knn, K,
                                          nullptr);
        if (s == PG_OK) break;
        if (ctx->last_derr != DERR_NO_SLOT) return s;
        const int64_t r = ctx->last_err_info;
        if (r < 0 || r >= n) return pg_fail(ctx, PG_ERR_INTERNAL, "connect: refused node %lld",
                                            (long long)r);
        // the reached set from ep on the graph as the plain pass left it
        if (!reached.p) {
            PG_TRY(reached.alloc(ctx, (size_t)n));
            PG_TRY(queue.alloc(ctx, (size_t)n * 2));
            PG_TRY(fcnt.alloc(ctx, 1));
            PG_TRY(st.alloc(ctx, 1));
        }
        PG_TRY_CUDA(ctx, cudaMemsetAsync(reached.p, 0, (size_t)n * 4, ctx->stream));
        k_rep_mark<<<1, 32, 0, ctx->stream>>>(reached.p, ep, queue.p);
        PG_LAUNCHED(ctx);
        int *fa = queue.p, *fb = queue.p + n;
        int fcount = 1;
        while (fcount > 0) {
            PG_TRY_CUDA(ctx, cudaMemsetAsync(fcnt.p, 0, sizeof(int), ctx->stream));
            k_bfs_level<<<(fcount + 255) / 256, 256, 0, ctx->stream>>>(nbr, deg, R, n, reached.p,
                                                                       fa, fcount, fb, fcnt.p);
            PG_LAUNCHED(ctx);
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, fcnt.p, sizeof(int),
                                             cudaMemcpyDeviceToHost, ctx->stream));
            PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            memcpy(&fcount, ctx->h_pinned, sizeof(int));
            std::swap(fa, fb);
        }
        // the reached node nearest to r that still holds an original edge
        RepState init{~0ull, ~0ull, INT_MAX};
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(st.p, &init, sizeof init, cudaMemcpyHostToDevice,
                                         ctx->stream));
        const unsigned grid = (unsigned)ctx->num_sms * 8;
        for (int pass = 0; pass < (exact ? 1 : 3); ++pass) {
            k_rep_scan<<<grid, 256, 0, ctx->stream>>>(D, n, d, m, r, reached.p, orig.p, em, exact,
                                                      pass, st.p);
            PG_LAUNCHED(ctx);
        }
        RepState h;
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(&h, st.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY(pg_sync_check(ctx, "connect replacement"));
        const int p = exact ? (h.key32 == ~0ull ? -1 : (int)(h.key32 & 0xffffffffu))
                            : (h.id64 == INT_MAX ? -1 : h.id64);
        if (p < 0)
            return pg_fail(ctx, PG_ERR_CAPACITY,
                           "connect: no reached node has a free slot or an original edge "
                           "(unreached node %lld)", (long long)r);
        k_rep_replace<<<1, 32, 0, ctx->stream>>>(nbr, R, orig.p, p, (int)r);
        PG_LAUNCHED(ctx);
        ++replaced;
    }
    if (host_added) {
        PG_TRY(sum.alloc(ctx, 1));
        PG_TRY_CUDA(ctx, cudaMemsetAsync(sum.p, 0, 8, ctx->stream));
        k_deg_sum<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(deg, deg0.p, n, sum.p);
        PG_LAUNCHED(ctx);
        unsigned long long v = 0;
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, sum.p, 8, cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PG_TRY(pg_sync_check(ctx, "connect"));
        memcpy(&v, ctx->h_pinned, 8);
        *host_added = (int64_t)v + replaced;
    }
    if (host_replaced) *host_replaced = replaced;
    return PG_OK;
}

extern "C" pg_status pg_connect_replace(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                        pg_metric metric, int32_t *nbr, int32_t *deg, int32_t R,
                                        int64_t ep, int64_t *host_added,
                                        int64_t *host_replaced) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !nbr || !deg) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n >= INT_MAX || d < 4 || d % 4 || d > 8192 || R < 1 || R > 64)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "bad n / d / R");
    if (ep < 0 || ep >= n) return pg_fail(ctx, PG_ERR_INVALID_ARG, "ep out of range");
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, D, n, d, metric, &facts));
    return pg_connect_replace_internal(ctx, D, n, d, metric, nbr, deg, R, ep, facts, nullptr, 0,
                                       host_added, host_replaced);
}
