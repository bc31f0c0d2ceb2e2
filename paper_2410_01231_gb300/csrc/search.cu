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
//
// Exactness.  On integer rows whose partial sums stay below 2^24 (and
// queries inside the rows' value range) every FP32 distance is exact.  On
// other rows the pool order is decided by an exact comparator: two FP32
// distances further apart than their rigorous rounding bounds are ordered
// by FP32; nearer ones by their FP64 distances with the CPU reference's
// sequential order, computed on first need and kept beside the pool entry.
// The pool, its truncation at L, the expansion order and the output are
// therefore those of Algorithm 1 on FP64 distances.
//
// FP8-screened queries rank the expansion candidates by distances from the
// index's FP8 E4M3 rows (decoded row scale * e against the FP32 query: the
// squared L2 distance, or the chord from the dot product); at the end the
// whole pool is re-measured in FP32 and the k best by (s, id) are returned.
#include <cuda_fp8.h>

#include <algorithm>
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
    const uint8_t *F8;  // FP8 E4M3 rows of D (screened queries) or nullptr
    const float *f8scale;
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
    int cert;   // near ties decided in FP64 (else every FP32 distance is exact)
    float rel;  // L2: |s32 - s64| <= rel * s32
    float nm;   // largest squared row norm of D (chord bound)
};

// the pool arrays hold an even number of slots, so that the query row that
// follows the table and the staging area starts on a 16-byte boundary
__host__ __device__ inline int pool_slots(int L) { return (L + 1) & ~1; }

// certified mode adds the FP64 distance of every pool entry and of the 32
// staged candidates (NaN until computed) in front of the rest
__host__ __device__ inline size_t search_warp_smem(int L, int hbits, int d, bool cert) {
    size_t b = (size_t)pool_slots(L) * 8 + ((size_t)4 << hbits) + 32 * 8 + (size_t)d * 4;
    if (cert) b += (size_t)pool_slots(L) * 8 + 32 * 8;
    return (b + 15) & ~(size_t)15;
}

// Exact comparator of the certified mode: distances further apart than the
// sum of their bounds are ordered by FP32, others by (FP64, id).
struct ExactCmp {
    int metric;
    float rel;   // L2 bound relative to the FP32 value
    float abs2;  // chord: twice the absolute bound
    const float *q;
    const float *D;
    int d;
    __device__ __forceinline__ bool near(float a, float b) const {
        const float diff = fabsf(a - b);
        return metric == 0 ? diff <= 2.02f * rel * fmaxf(a, b) : diff <= abs2;
    }
    __device__ __forceinline__ double s64(int id) const {
        return dist64_rows(q, D + (int64_t)id * d, d, metric);
    }
    // FP64 distance of a pool or staging slot, computed on first need
    __device__ __forceinline__ double cached(double *slot, int id) const {
        double v = *slot;
        if (v != v) {
            v = s64(id);
            *slot = v;
        }
        return v;
    }
};

// (s, id) order of a candidate (s, *a64, aid) against slot (t, *b64, bid)
__device__ __forceinline__ bool xless(const ExactCmp &X, float a, double *a64, int aid, float b,
                                      double *b64, int bid) {
    if (!X.near(a, b)) return a < b;
    const double x = X.cached(a64, aid), y = X.cached(b64, bid);
    return x < y || (x == y && aid < bid);
}

// Exact lower bound of (s, id) in the pool [0, size) (sorted in exact order):
// a bracket on the FP32 keys widened by twice the bound (keys may be out of
// FP32 order only inside a near-tie run), then exact comparisons inside.
// *dup = the id is present.
__device__ __forceinline__ int pool_lower_bound_exact(const ExactCmp &X, const float *pd,
                                                      const int *pi, double *pd64, int size,
                                                      float s, double *s64, int id, bool *dup) {
    const float w = X.metric == 0 ? 4.2f * X.rel * s : 2.1f * X.abs2;
    const float lo_key = s - w, hi_key = s + w;
    int a = 0, hi = size;
    while (a < hi) {
        const int mid = (a + hi) >> 1;
        if (pd[mid] < lo_key) a = mid + 1;
        else hi = mid;
    }
    int b = a;
    hi = size;
    while (b < hi) {
        const int mid = (b + hi) >> 1;
        if (pd[mid] <= hi_key) b = mid + 1;
        else hi = mid;
    }
    int pos = a;
    *dup = false;
    for (int i = a; i < b; ++i) {
        const int eid = pi[i] & ID_MASK;
        if (eid == id) {
            *dup = true;
            return i;
        }
        if (xless(X, pd[i], pd64 + i, eid, s, s64, id)) pos = i + 1;
    }
    return pos;
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

// Two E4M3 codes (the low and high byte of a 16-bit word) as floats.
__device__ __forceinline__ float2 f8x2_to_float2(unsigned w16) {
    const __half2 h(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)w16, __NV_E4M3));
    return __half22float2(h);
}

// One FP8 row against the query, by a team of eight lanes: kL2 sums
// (sc e_i - q_i)^2 -- the squared distance to the decoded row, whose error
// grows with |x - q| and not with |x| --, otherwise sums e_i q_i.  Rows whose
// width is a multiple of 16 are read 16 codes a load, others 4 codes a load.
template <bool kL2>
__device__ __forceinline__ float team8_f8(const float4 *__restrict__ q,
                                          const uint8_t *__restrict__ row, int d, int li,
                                          float sc) {
    float acc = 0.f;
    auto four = [&](unsigned w, const float4 qa) {
        const float2 a = f8x2_to_float2(w & 0xffffu), b = f8x2_to_float2(w >> 16);
        if (kL2) {
            const float t0 = fmaf(a.x, sc, -qa.x), t1 = fmaf(a.y, sc, -qa.y);
            const float t2 = fmaf(b.x, sc, -qa.z), t3 = fmaf(b.y, sc, -qa.w);
            acc = fmaf(t0, t0, acc);
            acc = fmaf(t1, t1, acc);
            acc = fmaf(t2, t2, acc);
            acc = fmaf(t3, t3, acc);
        } else {
            acc = fmaf(a.x, qa.x, acc);
            acc = fmaf(a.y, qa.y, acc);
            acc = fmaf(b.x, qa.z, acc);
            acc = fmaf(b.y, qa.w, acc);
        }
    };
    if ((d & 15) == 0) {
        const uint4 *x = reinterpret_cast<const uint4 *>(row);
        for (int c = li; c < (d >> 4); c += 8) {
            const uint4 w = __ldg(x + c);
            four(w.x, q[c * 4 + 0]);
            four(w.y, q[c * 4 + 1]);
            four(w.z, q[c * 4 + 2]);
            four(w.w, q[c * 4 + 3]);
        }
    } else {
        const unsigned *x = reinterpret_cast<const unsigned *>(row);
        for (int c = li; c < (d >> 2); c += 8) four(__ldg(x + c), q[c]);
    }
    return warp_sum8(acc);
}

// screened distance of FP8 row v to the query: squared L2 to the decoded
// row, or the chord 2 - 2 sc <e, q> of unit rows
__device__ __forceinline__ float team8_dist_f8(const SearchParams &P, const float4 *q, int v,
                                               int li) {
    const uint8_t *row = P.F8 + (int64_t)v * P.d;
    const float sc = __ldg(P.f8scale + v);
    if (P.metric == 0) return team8_f8<true>(q, row, P.d, li, sc);
    return fmaxf(2.f - 2.f * sc * team8_f8<false>(q, row, P.d, li, sc), 0.f);
}

// Register bitonic sort of one (s, s64, id, pos) per lane across the warp
// by the exact comparator; a lane that needs the partner's FP64 distance
// computes it from the partner's id (the same value the partner computes).
__device__ __forceinline__ void warp_sort32_exact(const ExactCmp &X, float &key, double &k64,
                                                  int &id, int &pos) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= 32; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            float ok = __shfl_xor_sync(0xffffffffu, key, j);
            double o64 = __shfl_xor_sync(0xffffffffu, k64, j);
            int oi = __shfl_xor_sync(0xffffffffu, id, j);
            int op = __shfl_xor_sync(0xffffffffu, pos, j);
            const bool lower = (lane & j) == 0;
            const bool up = (lane & k) == 0;
            bool other_less, mine_less;
            if (id == INT_MAX || oi == INT_MAX) {  // empty slots sort last
                other_less = pair_less(ok, oi, key, id);
                mine_less = pair_less(key, id, ok, oi);
            } else {
                other_less = xless(X, ok, &o64, oi, key, &k64, id);
                mine_less = xless(X, key, &k64, id, ok, &o64, oi);
            }
            const bool take_other = (lower == up) ? other_less : mine_less;
            if (take_other) {
                key = ok;
                k64 = o64;
                id = oi;
                pos = op;
            }
        }
    }
}

template <bool kF8, bool kCert>
__device__ void search_one(const SearchParams &P, int64_t qi, unsigned char *ws,
                           unsigned long long &n_exp, unsigned long long &n_eval,
                           unsigned long long &n_rerank) {
    const int lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int L = P.L, d = P.d, nch = d / 4;
    const int Lp = pool_slots(L);
    constexpr bool cert = kCert;
    double *pd64 = reinterpret_cast<double *>(ws);  // certified mode only
    double *nd64 = pd64 + Lp;
    float *pdA = reinterpret_cast<float *>(cert ? reinterpret_cast<unsigned char *>(nd64 + 32) : ws);
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
    constexpr bool f8 = kF8;  // FP8 rows (P.F8) in use
    ExactCmp X{P.metric, P.rel, 0.f, q, P.D, d};
    if (cert && P.metric != 0) {
        // chord bound with the larger of the rows' and the query's norms
        __syncwarp();
        float qq = 0.f;
        for (int c = lane; c < d; c += 32) qq = fmaf(q[c], q[c], qq);
        for (int o = 16; o; o >>= 1) qq += __shfl_xor_sync(0xffffffffu, qq, o);
        const double u = 5.9604644775390625e-08, nm = fmax((double)P.nm, (double)qq * 1.001);
        X.abs2 = (float)(2.0 * ((2.0 * ((d + 7) / 8 + 8) * u * nm + u * (2.0 + 2.0 * nm)) * 1.01 +
                                1e-12));
    }
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
    } else if (f8) {
        s0 = team8_dist_f8(P, q4, start, li);
    } else {
        s0 = team8_dist(q4, reinterpret_cast<const float4 *>(P.D + (int64_t)start * d), nch, li,
                        P.metric);
    }
    int size = 1, cursor = 0;
    const double nan64 = __longlong_as_double(0x7ff8000000000000ll);
    if (lane == 0) {
        pdA[0] = s0;
        piA[0] = start;
        if (cert) pd64[0] = nan64;
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
            } else if (f8) {
                for (int b0 = 0; b0 < cnt; b0 += 4) {
                    int i = b0 + team;
                    float s = team8_dist_f8(P, q4, ni[i < cnt ? i : 0], li);
                    if (li == 0 && i < cnt) nd[i] = s;
                }
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
            double s64 = nan64;  // certified mode: FP64 distance once computed
            int cpos = L;        // certified mode: exact slot against the pool
            if (lane < cnt) {
                s = nd[lane];
                id = ni[lane];
                if (cert) {
                    bool dup = false;
                    cpos = pool_lower_bound_exact(X, pdA, piA, pd64, size, s, &s64, id, &dup);
                    if (dup || cpos >= L) id = INT_MAX;
                } else if (size == L && !pair_less(s, id, pdA[L - 1], piA[L - 1] & ID_MASK)) {
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
            if (m2 > 1 && !cert && m2 <= 8) {
                // few survivors: each takes its rank among them (ids are
                // distinct, so (s, id) orders them strictly) and lane r then
                // reads the survivor of rank r back from the staging area
                int rank = 0;
                for (unsigned bits = live; bits; bits &= bits - 1) {
                    const int b = __ffs(bits) - 1;
                    const float os = __shfl_sync(0xffffffffu, s, b);
                    const int oi = __shfl_sync(0xffffffffu, id, b);
                    rank += pair_less(os, oi, s, id) ? 1 : 0;
                }
                __syncwarp();
                if (id != INT_MAX) {
                    nd[rank] = s;
                    ni[rank] = id;
                }
                __syncwarp();
                s = lane < m2 ? nd[lane] : INFINITY;
                id = lane < m2 ? ni[lane] : INT_MAX;
            } else if (m2 > 1) {
                if (cert) warp_sort32_exact(X, s, s64, id, cpos);
                else warp_sort32(s, id);  // survivors first, ascending
            } else {
                const int src = __ffs(live) - 1;
                s = __shfl_sync(0xffffffffu, s, src);
                id = __shfl_sync(0xffffffffu, id, src);
                s64 = __shfl_sync(0xffffffffu, s64, src);
                cpos = __shfl_sync(0xffffffffu, cpos, src);
                if (lane != 0) {
                    s = INFINITY;
                    id = INT_MAX;
                }
            }
            __syncwarp();
            if (lane < m2) {
                nd[lane] = s;
                ni[lane] = id;
                if (cert) nd64[lane] = s64;
            }
            // final slots of the new entries, against the pool before the merge
            int mydst = L;
            if (lane < m2)
                mydst = lane + (cert ? cpos : pool_lower_bound(pdA, piA, size, s, id));
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
                double e64 = nan64;
                if (i < size) {
                    es = pdA[i];
                    eid = piA[i];
                    const int key = eid & ID_MASK;
                    if (cert) e64 = pd64[i];
                    int lo = 0, hi = m2;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        const bool less = cert ? xless(X, nd[mid], nd64 + mid, ni[mid], es, &e64, key)
                                               : pair_less(nd[mid], ni[mid], es, key);
                        if (less) lo = mid + 1;
                        else hi = mid;
                    }
                    dst = i + lo;
                }
                __syncwarp();
                if (dst < L) {
                    pdA[dst] = es;
                    piA[dst] = eid;
                    if (cert) pd64[dst] = e64;
                }
                __syncwarp();
            }
            if (mydst < L) {
                pdA[mydst] = s;
                piA[mydst] = id;
                if (cert) pd64[mydst] = s64;
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
    } else if (f8 && !bad) {
        // re-measure the pool in FP32 (bit 31 now marks "returned")
        for (int b0 = 0; b0 < size; b0 += 4) {
            const int i = b0 + team;
            const int id = piA[i < size ? i : 0] & ID_MASK;
            const float s = team8_dist(q4, reinterpret_cast<const float4 *>(P.D + (int64_t)id * d),
                                       nch, li, P.metric);
            __syncwarp();
            if (li == 0 && i < size) {
                pdA[i] = s;
                piA[i] = id;
            }
        }
        n_rerank += (unsigned long long)size;
        __syncwarp();
        // the k best by (s, id): one warp-wide minimum per output slot
        for (int t = 0; t < P.k; ++t) {
            float bs = INFINITY;
            int bid = INT_MAX, bpos = -1;
            for (int i = lane; i < size; i += 32) {
                const int e = piA[i];
                if (!(e & EXP_BIT) && pair_less(pdA[i], e, bs, bid)) {
                    bs = pdA[i];
                    bid = e;
                    bpos = i;
                }
            }
            for (int o = 16; o; o >>= 1) {
                const float os = __shfl_xor_sync(0xffffffffu, bs, o);
                const int oid = __shfl_xor_sync(0xffffffffu, bid, o);
                const int opos = __shfl_xor_sync(0xffffffffu, bpos, o);
                if (pair_less(os, oid, bs, bid)) {
                    bs = os;
                    bid = oid;
                    bpos = opos;
                }
            }
            if (lane == 0) {
                P.out_i[qi * P.k + t] = bpos >= 0 ? bid : -1;
                P.out_s[qi * P.k + t] = bpos >= 0 ? bs : INFINITY;
                if (bpos >= 0) piA[bpos] |= EXP_BIT;
            }
            __syncwarp();
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

template <bool kF8, bool kCert>
__global__ void __launch_bounds__(SW * 32, 8) k_search(SearchParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *ws = smem + (size_t)wid * search_warp_smem(P.L, P.hbits, P.d, P.cert);
    unsigned long long n_exp = 0, n_eval = 0, n_rerank = 0;
    for (;;) {
        int64_t qi = 0;
        if (lane == 0) qi = atomicAdd(P.qcounter, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= P.nq) break;
        search_one<kF8, kCert>(P, qi, ws, n_exp, n_eval, n_rerank);
    }
    if (lane == 0) {
        // algorithmic bytes: one row per evaluation (FP8 rows also their
        // scale), one adjacency row per expansion, one FP32 row per re-measure
        const unsigned long long row =
            P.D8 ? (unsigned long long)P.d : P.F8 ? (unsigned long long)P.d + 4ull : 4ull * P.d;
        atomicAdd(P.counters + CNT_SEARCH_EXP, n_exp);
        atomicAdd(P.counters + CNT_SEARCH_EVAL, n_eval);
        atomicAdd(P.counters + CNT_SEARCH_BYTES,
                  n_eval * row + n_exp * 4ull * P.R + n_rerank * 4ull * P.d);
    }
}

std::mutex search_launch_mu;

}  // namespace

pg_status pg_search_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             const int32_t *nbr, const int32_t *deg, int32_t R,
                             const int32_t *rows, const float *Q, int64_t nq,
                             const int32_t *starts, int32_t k, int32_t L, int self,
                             int32_t *out_i, float *out_s, const uint8_t *D8, const F8Rows *f8,
                             const DataFacts *facts) {
    if (nq == 0) return PG_OK;
    SearchParams P;
    // exactness: rows (and query rows) whose FP32 distances are exact need
    // no FP64 decisions; facts given by the caller cover the queries too
    DataFacts fd;
    if (facts) {
        fd = *facts;
    } else {
        PG_TRY(pg_data_facts(ctx, D, n, d, metric, &fd));
        if (!self) PG_TRY(pg_query_facts(ctx, Q, nq, d, metric, &fd));
    }
    const bool exact = fd.exact != 0;
    const ErrModel em = pg_err_model(metric, d, fd, false);
    P.cert = !exact && !(self && D8) && !(!self && f8 && f8->q8);
    P.rel = em.rel;
    P.nm = fd.max_norm2;
    P.D = D;
    P.D8 = self ? D8 : nullptr;
    P.F8 = !self && f8 ? f8->q8 : nullptr;
    P.f8scale = P.F8 ? f8->scale : nullptr;
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
    if (search_warp_smem(L, hb, d, P.cert) * SW > 227 * 1024)
        return pg_fail(ctx, PG_ERR_CAPACITY, "search: pool/table do not fit shared memory");
    // the shared-memory attribute is per kernel, not per launch: searches
    // of other contexts on other threads (the serving workers) may set a
    // different size, so setting it and launching are one critical section
    std::lock_guard<std::mutex> lk(search_launch_mu);
    void (*kern)(SearchParams) =
        P.F8 ? k_search<true, false> : (P.cert ? k_search<false, true> : k_search<false, false>);
    // a configuration: visited-table bits * 16 + CTAs per SM (0: the
    // occupancy limit)
    auto launch = [&](int cfg, const SearchParams &Q, bool timed) -> pg_status {
        const int hbits = cfg >> 4;
        SearchParams R2 = Q;
        R2.hbits = hbits;
        const size_t smem = search_warp_smem(L, hbits, d, R2.cert) * SW;
        PG_TRY_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        int bps = 0;
        PG_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, SW * 32, smem));
        if (bps < 1) bps = 1;
        if ((cfg & 15) > 0) bps = std::min(bps, cfg & 15);
        const int64_t want = (nq + SW - 1) / SW;
        const int64_t grid = std::min<int64_t>((int64_t)ctx->num_sms * bps, want);
        PG_TRY_CUDA(ctx, cudaMemsetAsync(qc.p, 0, sizeof(int), ctx->stream));
        if (timed) pg_timer_begin(ctx, TM_SEARCH);
        kern<<<(unsigned)grid, SW * 32, smem, ctx->stream>>>(R2);
        PG_LAUNCHED(ctx);
        if (timed) pg_timer_end(ctx, TM_SEARCH);
        return PG_OK;
    };
    int cfg = hb << 4;
    if (ctx->autotune && nq >= 4096) {
        const TuneKey key{ctx->device, TUNE_SEARCH, d, L * 256 + R,
                          (P.D8 ? 1 : 0) | (P.F8 ? 2 : 0) | (P.cert ? 4 : 0) | (self ? 8 : 0) |
                              P.metric * 16};
        if (!pg_tune_lookup(key, &cfg)) {
            Scratch<unsigned long long> junk;
            PG_TRY(junk.alloc(ctx, PG_CNT_SLOTS));
            SearchParams Q = P;
            Q.counters = junk.p;
            std::vector<int> cands;
            for (int hbits = std::max(9, hb - 1); hbits <= std::min(13, hb + 1); ++hbits) {
                if (search_warp_smem(L, hbits, d, P.cert) * SW > 227 * 1024) continue;
                cands.push_back(hbits << 4);
                cands.push_back((hbits << 4) | 4);
            }
            std::vector<std::pair<int, float>> tried;
            PG_TRY(pg_tune_time(ctx, cands, [&](int c) { return launch(c, Q, false); }, &cfg,
                                &tried));
            char label[160];
            snprintf(label, sizeof label,
                     "k_search d=%d L=%d R=%d rows=%s%s%s (table bits*16 + CTAs/SM cap)", d, L, R,
                     P.D8 ? "bytes" : (P.F8 ? "fp8" : "fp32"), P.cert ? " certified" : "",
                     self ? " self" : "");
            pg_tune_store(key, cfg, tried, label);
        }
    }
    return launch(cfg, P, true);
}

// One warp per row: scale = max|x| / 448 (1 for a zero row), codes of
// x * (1 / scale) rounded to nearest E4M3 (saturating).
__global__ void k_make_f8(const float *D, int64_t r0, int64_t r1, int d, uint8_t *q8,
                          float *scale) {
    const int lane = threadIdx.x & 31;
    const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (r >= r1) return;
    const float *x = D + r * d;
    float mx = 0.f;
    for (int c = lane; c < d; c += 32) mx = fmaxf(mx, fabsf(x[c]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float sc = mx > 0.f ? mx / 448.f : 1.f;
    const float inv = 1.f / sc;
    for (int c = lane; c < d; c += 32)
        q8[r * d + c] = (uint8_t)__nv_cvt_float_to_fp8(x[c] * inv, __NV_SATFINITE, __NV_E4M3);
    if (lane == 0) scale[r] = sc;
}

pg_status pg_make_f8(pg_ctx *ctx, const float *D, int64_t r0, int64_t r1, int32_t d, uint8_t *q8,
                     float *scale) {
    if (r1 <= r0) return PG_OK;
    const int64_t warps = r1 - r0;
    k_make_f8<<<(unsigned)((warps + 7) / 8), 256, 0, ctx->stream>>>(D, r0, r1, d, q8, scale);
    PG_LAUNCHED(ctx);
    return PG_OK;
}

extern "C" pg_status pg_encode_fp8(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                   uint8_t *codes, float *scale) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D || !codes || !scale) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 0 || n >= INT_MAX) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 0 <= n < 2^31");
    if (d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need d % 4 == 0 and 4 <= d <= 8192");
    PG_TRY(pg_make_f8(ctx, D, 0, n, d, codes, scale));
    return pg_sync_check(ctx, "pg_encode_fp8");
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
    if (!pg_build_precision(precision))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "acquisition takes FP32 or BF16 screening");
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
    if (!pg_build_precision(precision))
        return pg_fail(ctx, PG_ERR_INVALID_ARG,
                       "pg_search_graph takes FP32 (FP8 screening needs an index)");
    if (!Q || !starts || !out_ids || !out_dist)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (nq < 0 || k < 1 || k > L) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= k <= L");
    PG_TRY(pg_search_internal(ctx, D, n, d, metric, nbr, deg, R, rows, Q, nq, starts, k, L, 0,
                              out_ids, out_dist, nullptr));
    return pg_sync_check(ctx, "pg_search_graph");
}
