// prune.cu -- alpha-pruning (Section 4.1 rule in the scan of Prune,
// Algorithm 3) and the reverse-edge union (Algorithm 2,
// Algorithm 5).
//
// One warp prunes one point u.  Candidate distances s(u,v) are computed by
// four teams of eight lanes (128-bit loads), the row is sorted by (s, id)
// in shared memory, repeated ids are dropped, and near-tie runs are
// re-ordered by their FP64 distance.  The scan then tests each candidate v
// against the kept set four kept points at a time (one per team), stopping
// at the first occluder; every comparison inside its FP32 error bound is
// re-decided in FP64 with the CPU reference's summation order.
// Rows longer than the shared-memory capacity of the warp kernel go to a
// one-warp-per-CTA kernel with a large dynamic buffer.
#include <climits>
#include <cmath>

#include "pg_internal.cuh"

namespace {

constexpr int PW = 8;            // warps per CTA (fast kernel)
constexpr int CMAX = 256;        // candidates per row, fast kernel
constexpr int CMAX_LONG = 8192;  // candidates per row, long-row kernel
constexpr int RMAX = 64;

struct PruneParams {
    const float *D;
    const uint8_t *D8;  // byte shadow of D (exact byte data) or nullptr
    int64_t n;          // points (ids must lie below n)
    int64_t rows;       // candidate rows (== n unless self_ids is given)
    const int32_t *self_ids;  // point id of each row, or nullptr (row = point)
    int d;
    int metric;
    const int64_t *off;
    const int32_t *cand;
    int R;
    double cos_a;
    float cos_af;
    int alpha60;
    int exact;
    int count_ties;      // count decisions with relative margin below 1e-5
    ErrModel em;
    int32_t *nbr;
    int32_t *deg;
    int *err;
    unsigned long long *counters;
    int *long_list;      // rows deferred to the long-row kernel
    int *long_count;
    int *row_counter;    // dynamic row fetch
    int cap;             // capacity of this kernel
    // K2P reuse (Section 5.4): the previous pruning of the same points with
    // an angle <= this one, N_prev [rows][prev_R] / deg, or nullptr
    const int32_t *prev_nbr;
    const int32_t *prev_deg;
    int prev_R;
};

// shared layout of one warp: c64[cap], cs[cap], ci[cap], runid[cap],
// kid[RMAX], ks[RMAX], kpos[RMAX], kchk[RMAX], uq[d] (FP32 row, or the byte
// row and the scanned candidate's byte row), cold[cap]
__host__ __device__ inline size_t warp_smem_bytes(int cap, int d) {
    return (size_t)cap * (4 + 4 + 4 + 8 + 1) + RMAX * (4 + 4 + 4 + 4) + (size_t)d * 4 + 64;
}

// s(v, w) of two byte rows (lane li's chunk of v already in vreg when
// d <= 128); the kept rows are re-read through L1
__device__ __forceinline__ float kept_dist_u8(const uint8_t *__restrict__ xv8, uint4 vreg,
                                              const uint8_t *__restrict__ xw8, int d, int li) {
    const int nch16 = d >> 4;
    const uint4 *w16 = reinterpret_cast<const uint4 *>(xw8);
    if (nch16 <= 8) {
        const uint4 w = li < nch16 ? __ldg(w16 + li) : make_uint4(0u, 0u, 0u, 0u);
        return (float)team8_sum_u(sq_diff_u8(vreg, w, 0u));
    }
    unsigned acc = 0;
    for (int c = li; c < nch16; c += 8)
        acc = sq_diff_u8(__ldg(reinterpret_cast<const uint4 *>(xv8) + c), __ldg(w16 + c), acc);
    return (float)team8_sum_u(acc);
}

struct RowStats {
    unsigned long long cands = 0, scanned = 0, tests = 0, rechecks = 0, flips = 0, edges = 0;
    unsigned long long ties = 0;  // decisions with relative margin below 1e-5
};

// Relative margin of a distance comparison a < b below 1e-5 (the tie
// budget's definition: |a - b| / max(a, b)).
__device__ __forceinline__ bool near_tie(float a, float b) {
    return fabsf(a - b) < 1e-5f * fmaxf(a, b);
}

// Relative margin of the angle clause below 1e-5:
// |(s_uw + s_vw - s_uv) - 2 cos(alpha) sqrt(s_uw s_vw)| / (s_uw + s_vw + s_uv).
__device__ __forceinline__ bool near_tie_angle(float suw, float svw, float suv, float ca) {
    const float lhs = (suw + svw) - suv, rhs = 2.f * ca * sqrtf(suw * svw);
    return fabsf(lhs - rhs) < 1e-5f * (suw + svw + suv);
}

// REG: byte rows of at most 128 bytes and R <= 32; lane l keeps the row of
// the l-th kept point in registers, so a candidate is tested against every
// kept point at once.
template <bool REG>
__device__ void prune_row(const PruneParams &P, int64_t row, const int32_t *cand, int64_t cnt,
                          unsigned char *wsmem, RowStats &st) {
    const int64_t u = P.self_ids ? (int64_t)P.self_ids[row] : row;  // the point being pruned
    const int lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int cap = P.cap;
    double *c64 = reinterpret_cast<double *>(wsmem);
    float *cs = reinterpret_cast<float *>(c64 + cap);
    int *ci = reinterpret_cast<int *>(cs + cap);
    int *runid = ci + cap;
    int *kid = runid + cap;
    float *ks = reinterpret_cast<float *>(kid + RMAX);
    int *kpos = reinterpret_cast<int *>(ks + RMAX);
    int *kchk = kpos + RMAX;
    float *uq = reinterpret_cast<float *>(kchk + RMAX);
    const int d = P.d, nch = d / 4;
    unsigned char *cold = reinterpret_cast<unsigned char *>(uq + d);
    const float *D = P.D;
    const uint8_t *D8 = P.D8;

    if (D8) {
        for (int c = lane; c < (d >> 4); c += 32)
            reinterpret_cast<uint4 *>(uq)[c] = __ldg(reinterpret_cast<const uint4 *>(D8 + u * d) + c);
    } else {
        for (int c = lane; c < nch; c += 32)
            reinterpret_cast<float4 *>(uq)[c] = __ldg(reinterpret_cast<const float4 *>(D + u * d) + c);
    }
    __syncwarp();

    // 1. s(u, v) for every candidate; invalid entries sort last
    if (D8) {
        for (int64_t base = 0; base < cnt; base += 32) {
            const int64_t j = base + lane;
            int v = j < cnt ? cand[j] : -1;
            if (j < cnt && (v >= P.n || v < -1)) record_error(P.err, DERR_BAD_ID, u);
            const bool ok = v >= 0 && v != u && v < P.n;
            if (j < cnt) ci[j] = ok ? v : -1;
            __syncwarp();
            batch_dist_u8(D8, d, reinterpret_cast<const uint4 *>(uq), ci + base,
                          (int)(cnt - base < 32 ? cnt - base : 32), cs + base);
            __syncwarp();
            if (j < cnt && ci[j] < 0) ci[j] = INT_MAX;
        }
    } else {
        for (int64_t base = 0; base < cnt; base += 4) {
            int64_t j = base + team;
            int v = j < cnt ? cand[j] : -1;
            bool ok = v >= 0 && v != u && v < P.n;
            if (j < cnt && (v >= P.n || v < -1)) record_error(P.err, DERR_BAD_ID, u);
            int row = ok ? v : (int)u;
            float s = team8_dist(reinterpret_cast<const float4 *>(uq),
                                 reinterpret_cast<const float4 *>(D + (int64_t)row * d), nch, li,
                                 P.metric);
            if (li == 0 && j < cnt) {
                cs[j] = ok ? s : INFINITY;
                ci[j] = ok ? v : INT_MAX;
            }
        }
    }
    int P2 = 32;
    while (P2 < cnt) P2 <<= 1;
    for (int j = (int)cnt + lane; j < P2; j += 32) {
        cs[j] = INFINITY;
        ci[j] = INT_MAX;
    }
    __syncwarp();
    warp_bitonic_sort(cs, ci, P2);

    // 2. drop repeated ids (adjacent after the sort) and invalid entries
    int m = 0;
    for (int base = 0; base < P2; base += 32) {
        int j = base + lane;
        float s = cs[j];
        int id = ci[j];
        bool keep = id != INT_MAX && (j == 0 || ci[j - 1] != id);
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {
            int dst = m + __popc(bal & ((1u << lane) - 1));
            cs[dst] = s;
            ci[dst] = id;
        }
        m += __popc(bal);
        __syncwarp();
    }
    st.cands += m;

    // 3. near-tie runs: FP64 distances and re-order within each run
    for (int j = lane; j < m; j += 32) {
        runid[j] = j;
        c64[j] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: not computed
    }
    __syncwarp();
    if (!P.exact) {
        bool any = false;
        for (int j = 1 + lane; j < m; j += 32) {
            float a = cs[j - 1], b = cs[j];
            int c = less_certain(a, P.em.err(a), b, P.em.err(b));
            if (c != 1) any = true;
        }
        if (__any_sync(0xffffffffu, any)) {
            if (lane == 0) {
                for (int j = 1; j < m; ++j) {
                    float a = cs[j - 1], b = cs[j];
                    if (less_certain(a, P.em.err(a), b, P.em.err(b)) != 1) runid[j] = runid[j - 1];
                }
            }
            __syncwarp();
            for (int j = lane; j < m; j += 32) {
                bool inrun = (j > 0 && runid[j] == runid[j - 1]) || (j + 1 < m && runid[j + 1] == j);
                if (inrun) c64[j] = dist64_rows(uq, D + (int64_t)ci[j] * d, d, P.metric);
            }
            __syncwarp();
            if (lane == 0) {
                int j = 0;
                while (j < m) {
                    int e = j;
                    while (e + 1 < m && runid[e + 1] == runid[j]) ++e;
                    for (int a = j + 1; a <= e; ++a) {  // insertion sort by (c64, id)
                        double kd = c64[a];
                        int kidv = ci[a];
                        float kf = cs[a];
                        int b = a - 1;
                        while (b >= j && (c64[b] > kd || (c64[b] == kd && ci[b] > kidv))) {
                            c64[b + 1] = c64[b];
                            ci[b + 1] = ci[b];
                            cs[b + 1] = cs[b];
                            --b;
                        }
                        c64[b + 1] = kd;
                        ci[b + 1] = kidv;
                        cs[b + 1] = kf;
                    }
                    st.rechecks += (e > j) ? (unsigned long long)(e - j + 1) : 0ull;
                    j = e + 1;
                }
            }
            __syncwarp();
        }
    }

    // 3b. K2P (Section 5.4): cold[j] marks a candidate that the previous
    // pruning of u kept.  It was then tested against every member of
    // N_prev(u) that precedes it and none occluded it; the test of a pair
    // depends only on u, v and w (and a larger angle occludes less), and the
    // scan order only on s(u, .), so such a candidate is tested only against
    // kept members that are not in N_prev(u).
    const bool reuse = P.prev_nbr != nullptr;
    if (reuse) {
        int pd = P.prev_deg[row];
        pd = pd < 0 ? 0 : (pd > P.prev_R ? P.prev_R : pd);
        const int32_t *pr = P.prev_nbr + row * P.prev_R;
        const int p0 = lane < pd ? pr[lane] : -2;
        const int p1 = lane + 32 < pd ? pr[lane + 32] : -2;
        for (int base = 0; base < m; base += 32) {
            const int jj = base + lane;
            const int v = jj < m ? ci[jj] : -3;
            bool hit = false;
            for (int t = 0; t < pd; ++t) {
                const int pv = __shfl_sync(0xffffffffu, t < 32 ? p0 : p1, t & 31);
                hit |= pv == v;
            }
            if (jj < m) cold[jj] = hit ? 1 : 0;
        }
        __syncwarp();
    }

    // 4. the scan
    int kept = 0;
    int j = 0;
    if constexpr (REG) {
        const int nch16 = d >> 4;  // <= 8
        uint4 *vrow = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(uq) + d);
        uint4 kr[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) kr[c] = make_uint4(0u, 0u, 0u, 0u);
        float ksl = 0.f;  // s(u, w) of this lane's kept point
        bool kold = false;  // this lane's kept point is in N_prev(u) (K2P)
        for (; j < m && kept < P.R; ++j) {
            const int v = ci[j];
            const float suv = cs[j];
            const bool vold = reuse && cold[j];
            const bool mine = lane < kept && !(vold && kold);
            if (P.count_ties && mine && near_tie(ksl, suv)) st.ties++;
            const bool work = mine && ksl < suv;
            bool occ = false;
            const bool loaded = __any_sync(0xffffffffu, work);
            if (loaded) {
                if (lane < nch16)
                    vrow[lane] = __ldg(reinterpret_cast<const uint4 *>(D8 + (int64_t)v * d) + lane);
                __syncwarp();
            }
            if (work) {  // exact data: the comparisons are exact
                unsigned acc = 0;
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < nch16) acc = sq_diff_u8(vrow[c], kr[c], acc);
                const float svw = (float)acc;
                st.tests++;
                if (P.count_ties && near_tie(svw, suv)) st.ties++;
                if (svw < suv) {
                    int c3 = 1;
                    if (!P.alpha60) {
                        if (P.count_ties && near_tie_angle(ksl, svw, suv, P.cos_af)) st.ties++;
                        c3 = angle_certain(ksl, P.em.err(ksl), svw, P.em.err(svw), suv,
                                           P.em.err(suv), P.cos_af);
                        if (c3 < 0) {
                            c3 = angle_exceeds64((double)ksl, (double)svw, (double)suv, P.cos_a);
                            st.rechecks++;
                            const bool naive =
                                ((ksl + svw) - suv) < 2.f * P.cos_af * sqrtf(ksl * svw);
                            if ((c3 != 0) != naive) st.flips++;
                        }
                    }
                    occ = c3 != 0;
                }
            }
            if (!__any_sync(0xffffffffu, occ)) {
                if (lane == kept) {
                    if (loaded) {
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (c < nch16) kr[c] = vrow[c];
                    } else {
                        const uint4 *xv = reinterpret_cast<const uint4 *>(D8 + (int64_t)v * d);
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (c < nch16) kr[c] = __ldg(xv + c);
                    }
                    ksl = suv;
                    kold = vold;
                }
                if (lane == 0) {
                    kid[kept] = v;
                    ks[kept] = suv;
                    kpos[kept] = j;
                }
                ++kept;
            }
            __syncwarp();
        }
    } else {
    for (; j < m && kept < P.R; ++j) {
        const int v = ci[j];
        const float suv = cs[j];
        const float euv = P.em.err(suv);
        const float *xv = D + (int64_t)v * d;
        const uint8_t *xv8 = D8 ? D8 + (int64_t)v * d : nullptr;
        // K2P: a candidate kept last time is tested only against new members
        const bool vold = reuse && cold[j];
        int nchk = kept;
        if (vold) {
            nchk = 0;
            for (int base = 0; base < kept; base += 32) {
                const int t = base + lane;
                const bool need = t < kept && !cold[kpos[t]];
                const unsigned bal = __ballot_sync(0xffffffffu, need);
                if (need) kchk[nchk + __popc(bal & ((1u << lane) - 1))] = t;
                nchk += __popc(bal);
            }
            __syncwarp();
        }
        uint4 vreg = make_uint4(0u, 0u, 0u, 0u);
        if (D8 && li < (d >> 4) && (d >> 4) <= 8 && nchk > 0)
            vreg = __ldg(reinterpret_cast<const uint4 *>(xv8) + li);
        bool occluded = false;
        for (int kb = 0; kb < nchk && !occluded; kb += 4) {
            const int ti = kb + team;
            const bool active = ti < nchk;
            const int t = active ? (vold ? kchk[ti] : ti) : 0;
            const int w = active ? kid[t] : v;
            const float svw =
                D8 ? kept_dist_u8(xv8, vreg, D8 + (int64_t)w * d, d, li)
                   : team8_dist(reinterpret_cast<const float4 *>(xv),
                                reinterpret_cast<const float4 *>(D + (int64_t)w * d), nch, li,
                                P.metric);
            bool occ = false;
            if (active && li == 0) {
                const int wpos = kpos[t];
                const float suw = ks[t];
                if (P.count_ties && near_tie(suw, suv)) st.ties++;
                bool c1;
                if (P.exact) c1 = suw < suv;
                else if (runid[wpos] != runid[j]) c1 = true;  // separated by a certain gap
                else c1 = c64[wpos] < c64[j];
                if (c1) {
                    st.tests++;
                    if (P.count_ties && near_tie(svw, suv)) st.ties++;
                    const float evw = P.em.err(svw);
                    int c2 = P.exact ? (svw < suv) : less_certain(svw, evw, suv, euv);
                    double s64vw = -1.0, s64uv = c64[j], s64uw = c64[wpos];
                    if (c2 < 0) {
                        s64vw = dist64_rows(xv, D + (int64_t)w * d, d, P.metric);
                        if (!(s64uv == s64uv)) s64uv = dist64_rows(uq, xv, d, P.metric);
                        c2 = s64vw < s64uv;
                        st.rechecks++;
                        if ((c2 != 0) != (svw < suv)) st.flips++;
                    }
                    if (c2) {
                        int c3 = 1;
                        if (!P.alpha60) {
                            if (P.count_ties && near_tie_angle(suw, svw, suv, P.cos_af)) st.ties++;
                            c3 = angle_certain(suw, P.em.err(suw), svw, evw, suv, euv, P.cos_af);
                            if (c3 < 0) {
                                if (P.exact) {  // the FP32 distances are the exact values
                                    s64vw = (double)svw;
                                    s64uv = (double)suv;
                                    s64uw = (double)suw;
                                }
                                if (s64vw < 0.0) s64vw = dist64_rows(xv, D + (int64_t)w * d, d, P.metric);
                                if (!(s64uv == s64uv)) s64uv = dist64_rows(uq, xv, d, P.metric);
                                if (!(s64uw == s64uw))
                                    s64uw = dist64_rows(uq, D + (int64_t)w * d, d, P.metric);
                                c3 = angle_exceeds64(s64uw, s64vw, s64uv, P.cos_a);
                                st.rechecks++;
                                bool naive = ((suw + svw) - suv) < 2.f * P.cos_af * sqrtf(suw * svw);
                                if ((c3 != 0) != naive) st.flips++;
                            }
                        }
                        occ = c3 != 0;
                    }
                }
            }
            occluded = __any_sync(0xffffffffu, occ);
        }
        if (!occluded) {
            if (lane == 0) {
                kid[kept] = v;
                ks[kept] = suv;
                kpos[kept] = j;
            }
            ++kept;
            __syncwarp();
        }
    }
    }
    st.scanned += j;
    st.edges += kept;
    for (int t = lane; t < P.R; t += 32) P.nbr[row * P.R + t] = t < kept ? kid[t] : -1;
    if (lane == 0) P.deg[row] = kept;
    __syncwarp();
}

__device__ void flush_stats(const PruneParams &P, RowStats &st, unsigned long long rows, bool lng) {
    const int lane = threadIdx.x & 31;
    // per-lane counters (tests/rechecks/flips live on team leaders)
    unsigned long long v[5] = {st.tests, st.rechecks, st.flips, st.ties, 0};
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) {
        atomicAdd(P.counters + CNT_ROWS, rows);
        atomicAdd(P.counters + CNT_CANDS, st.cands);
        atomicAdd(P.counters + CNT_SCANNED, st.scanned);
        atomicAdd(P.counters + CNT_OCCL, v[0]);
        atomicAdd(P.counters + CNT_RECHECK, v[1]);
        atomicAdd(P.counters + CNT_FLIP, v[2]);
        atomicAdd(P.counters + CNT_EDGES, st.edges);
        if (v[3]) atomicAdd(P.counters + CNT_NEAR_TIE, v[3]);
        if (lng) atomicAdd(P.counters + CNT_LONG, rows);
        // algorithmic bytes: each examined candidate's row plus (id, distance),
        // and the point's own row
        const unsigned long long row = P.D8 ? (unsigned long long)P.d : 4ull * P.d;
        atomicAdd(P.counters + CNT_PRUNE_BYTES, st.cands * (row + 8) + rows * row);
    }
}

template <bool REG>
__global__ void __launch_bounds__(PW * 32, REG ? 3 : 2) k_prune(PruneParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *ws = smem + (size_t)wid * warp_smem_bytes(CMAX, P.d);
    RowStats st;
    unsigned long long rows = 0;
    for (;;) {
        int64_t u = 0;
        if (lane == 0) u = atomicAdd(P.row_counter, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= P.rows) break;
        int64_t a = P.off[u], b = P.off[u + 1];
        if (b < a) {
            if (lane == 0) {
                record_error(P.err, DERR_BAD_ID, u);
                P.deg[u] = 0;
            }
            for (int t = lane; t < P.R; t += 32) P.nbr[u * P.R + t] = -1;
            continue;
        }
        if (b - a > CMAX) {
            if (lane == 0) {
                int slot = atomicAdd(P.long_count, 1);
                P.long_list[slot] = (int)u;
            }
            continue;
        }
        prune_row<REG>(P, u, P.cand + a, b - a, ws, st);
        ++rows;
    }
    flush_stats(P, st, rows, false);
}

__global__ void __launch_bounds__(32) k_prune_long(PruneParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    RowStats st;
    unsigned long long rows = 0;
    const int total = *P.long_count;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        int64_t u = P.long_list[i];
        int64_t a = P.off[u], b = P.off[u + 1];
        if (b - a > CMAX_LONG) {
            if (lane == 0) {
                record_error(P.err, DERR_CAPACITY, u);
                P.deg[u] = 0;
            }
            for (int t = lane; t < P.R; t += 32) P.nbr[u * P.R + t] = -1;
            continue;
        }
        prune_row<false>(P, u, P.cand + a, b - a, smem, st);
        ++rows;
    }
    flush_stats(P, st, rows, true);
}

// ---------------------------------------------------------- prefix scan
__global__ void k_scan_blocks(const int32_t *in, int64_t n, int64_t *out, int64_t *blk_sum) {
    __shared__ int64_t s[1024];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive within block
    if (threadIdx.x == 1023) blk_sum[blockIdx.x] = s[1023];
}

__global__ void k_scan_sums(int64_t *blk_sum, int64_t nb) {
    // single thread: block counts are small (n / 1024)
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t run = 0;
        for (int64_t b = 0; b < nb; ++b) {
            int64_t t = blk_sum[b];
            blk_sum[b] = run;
            run += t;
        }
        blk_sum[nb] = run;
    }
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *blk_sum, int64_t nb) {
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += blk_sum[i / 1024];
    if (i == 0) out[n] = blk_sum[nb];
}

// ------------------------------------------------------- reverse union
__global__ void k_union_count(const int32_t *nbr, const int32_t *deg, int64_t n, int R, int32_t *cnt,
                              int *err) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int dv = deg[v];
    if (dv < 0 || dv > R) {
        record_error(err, DERR_BAD_ID, v);
        return;
    }
    atomicAdd(&cnt[v], dv);
    for (int j = 0; j < dv; ++j) {
        int w = nbr[v * R + j];
        if (w < 0 || w >= n) {
            record_error(err, DERR_BAD_ID, v);
            continue;
        }
        atomicAdd(&cnt[w], 1);
    }
}

__global__ void k_union_own(const int32_t *nbr, const int32_t *deg, int64_t n, int R,
                            const int64_t *off, int32_t *ids, int64_t *cursor) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int du = deg[u];
    if (du < 0 || du > R) du = 0;
    int64_t o = off[u];
    for (int j = 0; j < du; ++j) ids[o + j] = nbr[u * R + j];
    cursor[u] = o + du;
}

__global__ void k_union_scatter(const int32_t *nbr, const int32_t *deg, int64_t n, int R,
                                int32_t *ids, unsigned long long *cursor) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int dv = deg[v];
    if (dv < 0 || dv > R) return;
    for (int j = 0; j < dv; ++j) {
        int w = nbr[v * R + j];
        if (w < 0 || w >= n) continue;
        unsigned long long pos = atomicAdd(&cursor[w], 1ull);
        ids[pos] = (int32_t)v;
    }
}

}  // namespace

pg_status pg_scan_counts(pg_ctx *ctx, const int32_t *cnt, int64_t n, int64_t *off) {
    int64_t nb = (n + 1023) / 1024;
    Scratch<int64_t> bs;
    PG_TRY(bs.alloc(ctx, (size_t)nb + 1));
    if (nb > 0) {
        k_scan_blocks<<<(unsigned)nb, 1024, 0, ctx->stream>>>(cnt, n, off, bs.p);
        PG_LAUNCHED(ctx);
    }
    k_scan_sums<<<1, 32, 0, ctx->stream>>>(bs.p, nb);
    PG_LAUNCHED(ctx);
    k_scan_add<<<(unsigned)(nb > 0 ? nb : 1), 1024, 0, ctx->stream>>>(off, n, bs.p, nb);
    PG_LAUNCHED(ctx);
    return PG_OK;
}

pg_status pg_reverse_union_internal(pg_ctx *ctx, const int32_t *nbr, const int32_t *deg, int64_t n,
                                    int32_t R, int64_t *off, int32_t *ids) {
    Scratch<int32_t> cnt;
    PG_TRY(cnt.alloc(ctx, (size_t)n));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(cnt.p, 0, (size_t)n * 4, ctx->stream));
    unsigned g = (unsigned)((n + 255) / 256);
    k_union_count<<<g, 256, 0, ctx->stream>>>(nbr, deg, n, R, cnt.p, ctx->d_err);
    PG_LAUNCHED(ctx);
    PG_TRY(pg_scan_counts(ctx, cnt.p, n, off));
    Scratch<int64_t> cursor;
    PG_TRY(cursor.alloc(ctx, (size_t)n));
    k_union_own<<<g, 256, 0, ctx->stream>>>(nbr, deg, n, R, off, ids, cursor.p);
    PG_LAUNCHED(ctx);
    pg_timer_begin(ctx, TM_UNION);
    k_union_scatter<<<g, 256, 0, ctx->stream>>>(nbr, deg, n, R, ids,
                                                reinterpret_cast<unsigned long long *>(cursor.p));
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_UNION);
    return PG_OK;
}

pg_status pg_prune_internal(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                            const int64_t *off, const int32_t *cand, int32_t R, double alpha_deg,
                            const DataFacts &facts, int32_t *nbr, int32_t *deg,
                            const uint8_t *D8, int64_t rows, const int32_t *self_ids,
                            const int32_t *prev_nbr, const int32_t *prev_deg, int32_t prev_R) {
    PruneParams P;
    P.prev_nbr = prev_nbr;
    P.prev_deg = prev_deg;
    P.prev_R = prev_R;
    P.D = D;
    P.D8 = D8;
    P.n = n;
    P.rows = rows > 0 ? rows : n;
    P.self_ids = self_ids;
    P.d = d;
    P.metric = metric == PG_METRIC_L2SQ ? 0 : 1;
    P.off = off;
    P.cand = cand;
    P.R = R;
    P.cos_a = std::cos(alpha_deg * M_PI / 180.0);
    P.cos_af = (float)P.cos_a;
    P.alpha60 = alpha_deg == 60.0;
    P.exact = facts.exact;
    P.count_ties = ctx->count_ties;
    P.em = pg_err_model(metric, d, facts, false);
    P.nbr = nbr;
    P.deg = deg;
    P.err = ctx->d_err;
    P.counters = ctx->d_counters;
    Scratch<int> ints;
    PG_TRY(ints.alloc(ctx, (size_t)P.rows + 4));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(ints.p, 0, 4 * sizeof(int), ctx->stream));
    P.row_counter = ints.p;
    P.long_count = ints.p + 1;
    P.long_list = ints.p + 4;
    P.cap = CMAX;
    size_t smem = warp_smem_bytes(CMAX, d) * PW;
    // byte rows of <= 128 bytes and R <= 32: kept rows held in registers
    const bool reg = D8 && R <= 32 && d <= 128;
    auto kern = reg ? k_prune<true> : k_prune<false>;
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    int blocks_per_sm = 0;
    PG_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, PW * 32,
                                                                   smem));
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    // CTAs per SM: the occupancy limit, or the autotuner's choice
    int bps = blocks_per_sm;
    if (ctx->autotune && blocks_per_sm > 1) {
        const TuneKey key{ctx->device, TUNE_PRUNE, d, R,
                          (reg ? 2 : (D8 ? 1 : 0)) + 4 * (prev_nbr != nullptr) + 8 * P.metric};
        int cfg = 0;
        if (pg_tune_lookup(key, &cfg)) {
            bps = cfg;
        } else {
            Scratch<unsigned long long> junk;
            PG_TRY(junk.alloc(ctx, PG_CNT_SLOTS));
            std::vector<int> cands;
            for (int c = 1; c <= blocks_per_sm; ++c) cands.push_back(c);
            auto run = [&](int c) -> pg_status {
                PruneParams Q = P;
                Q.counters = junk.p;
                PG_TRY_CUDA(ctx, cudaMemsetAsync(ints.p, 0, 4 * sizeof(int), ctx->stream));
                kern<<<ctx->num_sms * c, PW * 32, smem, ctx->stream>>>(Q);
                PG_LAUNCHED(ctx);
                return PG_OK;
            };
            std::vector<std::pair<int, float>> tried;
            PG_TRY(pg_tune_time(ctx, cands, run, &bps, &tried));
            char label[128];
            snprintf(label, sizeof label, "k_prune d=%d R=%d rows=%s%s CTAs/SM", d, R,
                     reg ? "bytes-in-registers" : (D8 ? "bytes" : "fp32"),
                     prev_nbr ? " k2p" : "");
            pg_tune_store(key, bps, tried, label);
            PG_TRY_CUDA(ctx, cudaMemsetAsync(ints.p, 0, 4 * sizeof(int), ctx->stream));
        }
    }
    pg_timer_begin(ctx, TM_PRUNE);
    kern<<<ctx->num_sms * bps, PW * 32, smem, ctx->stream>>>(P);
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_PRUNE);
    P.cap = CMAX_LONG;
    size_t smem_long = warp_smem_bytes(CMAX_LONG, d);
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(k_prune_long,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_long));
    pg_timer_begin(ctx, TM_PRUNE);
    k_prune_long<<<ctx->num_sms, 32, smem_long, ctx->stream>>>(P);
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_PRUNE);
    return PG_OK;
}

// Launch of the pruning kernels on scratch the caller provides (no
// allocation, no context): ints holds >= n + 4 ints, err 4 ints, counters
// PG_CNT_SLOTS values.  Used by the allocation-free entry point only.
cudaError_t pg_prune_launch_on(cudaStream_t stream, int num_sms, const float *D, int64_t n,
                               int32_t d, pg_metric metric, const int64_t *off,
                               const int32_t *cand, int32_t R, double alpha_deg,
                               const DataFacts &facts, int32_t *nbr, int32_t *deg, int *ints,
                               int *err, unsigned long long *counters) {
    PruneParams P;
    P.prev_nbr = nullptr;
    P.prev_deg = nullptr;
    P.prev_R = 0;
    P.D = D;
    P.D8 = nullptr;
    P.n = n;
    P.rows = n;
    P.self_ids = nullptr;
    P.d = d;
    P.metric = metric == PG_METRIC_L2SQ ? 0 : 1;
    P.off = off;
    P.cand = cand;
    P.R = R;
    P.cos_a = std::cos(alpha_deg * M_PI / 180.0);
    P.cos_af = (float)P.cos_a;
    P.alpha60 = alpha_deg == 60.0;
    P.exact = facts.exact;
    P.count_ties = 0;
    P.em = pg_err_model(metric, d, facts, false);
    P.nbr = nbr;
    P.deg = deg;
    P.err = err;
    P.counters = counters;
    P.row_counter = ints;
    P.long_count = ints + 1;
    P.long_list = ints + 4;
    P.cap = CMAX;
    cudaError_t e = cudaMemsetAsync(ints, 0, 4 * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const size_t smem = warp_smem_bytes(CMAX, d) * PW;
    e = cudaFuncSetAttribute(k_prune<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_prune<false>, PW * 32, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    k_prune<false><<<num_sms * bps, PW * 32, smem, stream>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    P.cap = CMAX_LONG;
    const size_t smem_long = warp_smem_bytes(CMAX_LONG, d);
    e = cudaFuncSetAttribute(k_prune_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_long);
    if (e != cudaSuccess) return e;
    k_prune_long<<<num_sms, 32, smem_long, stream>>>(P);
    return cudaGetLastError();
}

static pg_status check_common(pg_ctx *ctx, const float *D, int64_t n, int32_t d) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!D) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null D");
    if (n < 1 || n >= INT_MAX) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= n < 2^31");
    if (d < 4 || d % 4 || d > 8192)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need d % 4 == 0 and 4 <= d <= 8192");
    return PG_OK;
}

static pg_status prune_entry(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             const int64_t *cand_off, const int32_t *cand_ids,
                             const int32_t *prev_nbr, const int32_t *prev_deg, int32_t prev_R,
                             int32_t R, double alpha_deg, pg_precision precision, int32_t *nbr,
                             int32_t *deg, pg_prune_stats *host_stats, const char *what) {
    PG_TRY(check_common(ctx, D, n, d));
    if (!cand_off || !cand_ids || !nbr || !deg)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (R < 1 || R > RMAX) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= R <= %d", RMAX);
    if (!(alpha_deg >= 0.0 && alpha_deg <= 180.0))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 0 <= alpha <= 180");
    if (!pg_build_precision(precision))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "pruning takes FP32 or BF16 screening");
    DataFacts facts;
    PG_TRY(pg_data_facts(ctx, D, n, d, metric, &facts));
    Scratch<uint8_t> d8;
    if (pg_u8_usable(facts, metric, d, precision)) PG_TRY(pg_make_u8(ctx, D, n, d, d8));
    if (host_stats) PG_TRY(pg_reset_counters(ctx));
    PG_TRY(pg_prune_internal(ctx, D, n, d, metric, cand_off, cand_ids, R, alpha_deg, facts, nbr,
                             deg, d8.p, 0, nullptr, prev_nbr, prev_deg, prev_R));
    if (host_stats) {
        unsigned long long c[PG_CNT_SLOTS];
        PG_TRY(pg_read_counters(ctx, c));
        host_stats->rows = (int64_t)c[CNT_ROWS];
        host_stats->candidates = (int64_t)c[CNT_CANDS];
        host_stats->scanned = (int64_t)c[CNT_SCANNED];
        host_stats->occlusion_tests = (int64_t)c[CNT_OCCL];
        host_stats->fp64_rechecks = (int64_t)c[CNT_RECHECK];
        host_stats->fp64_flips = (int64_t)c[CNT_FLIP];
        host_stats->edges = (int64_t)c[CNT_EDGES];
        host_stats->long_rows = (int64_t)c[CNT_LONG];
        host_stats->near_ties = (int64_t)c[CNT_NEAR_TIE];
        return PG_OK;
    }
    return pg_sync_check(ctx, what);
}

extern "C" pg_status pg_prune(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                              const int64_t *cand_off, const int32_t *cand_ids, int32_t R,
                              double alpha_deg, pg_precision precision, int32_t *nbr,
                              int32_t *deg, pg_prune_stats *host_stats) {
    return prune_entry(ctx, D, n, d, metric, cand_off, cand_ids, nullptr, nullptr, 0, R,
                       alpha_deg, precision, nbr, deg, host_stats, "pg_prune");
}

extern "C" pg_status pg_prune_k2p(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                  pg_metric metric, const int64_t *cand_off,
                                  const int32_t *cand_ids, const int32_t *prev_nbr,
                                  const int32_t *prev_deg, int32_t prev_R, int32_t R,
                                  double alpha_deg, pg_precision precision, int32_t *nbr,
                                  int32_t *deg, pg_prune_stats *host_stats) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!prev_nbr || !prev_deg) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null previous lists");
    if (prev_R < 1 || prev_R > RMAX)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= prev_R <= %d", RMAX);
    return prune_entry(ctx, D, n, d, metric, cand_off, cand_ids, prev_nbr, prev_deg, prev_R, R,
                       alpha_deg, precision, nbr, deg, host_stats, "pg_prune_k2p");
}

extern "C" pg_status pg_reverse_union(pg_ctx *ctx, const int32_t *nbr, const int32_t *deg,
                                      int64_t n, int32_t R, int64_t *off, int32_t *ids,
                                      int64_t ids_capacity, int64_t *host_total) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!nbr || !deg || !off || !ids) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n >= INT_MAX || R < 1 || R > RMAX)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= n < 2^31 and 1 <= R <= %d", RMAX);
    if (ids_capacity < 2 * n * (int64_t)R)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "ids capacity must be >= 2*n*R");
    PG_TRY(pg_reverse_union_internal(ctx, nbr, deg, n, R, off, ids));
    if (host_total) {
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, off + n, sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY(pg_sync_check(ctx, "pg_reverse_union"));
        memcpy(host_total, ctx->h_pinned, sizeof(int64_t));
        return PG_OK;
    }
    return pg_sync_check(ctx, "pg_reverse_union");
}
