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
static_assert(BM == 8 * (NT / 32) && BN == 128, "warp w owns rows 8w .. 8w + 7 over all columns");
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
    // The next k-block of A and B is read into registers while the current
    // one is multiplied from shared memory (the last block of a column tile
    // prefetches the first block of the next tile); the per-accumulator
    // summation order is unchanged.
    float4 ra[2], rb[2][2];
    auto load_tiles = [&](int64_t c0, int kb) {
        const int k0 = kb * BK;
        {
            const int r = tid >> 2, kq = tid & 3;
            const int64_t g = row0 + r;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kk = kq * 4 + h * 16;
                ra[h] = (g < nq && k0 + kk < d)
                            ? *reinterpret_cast<const float4 *>(Q + g * d + k0 + kk)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = (tid >> 2) + h * 64, kq = tid & 3;
            const int64_t g = c0 + r;
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int kk = kq * 4 + h2 * 16;
                rb[h][h2] = (g < n && k0 + kk < d)
                                ? __ldg(reinterpret_cast<const float4 *>(X + g * d + k0 + kk))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    auto store_tiles = [&]() {
        {
            const int r = tid >> 2, kq = tid & 3;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kk = kq * 4 + h * 16;
                sm.As[kk + 0][r] = ra[h].x;
                sm.As[kk + 1][r] = ra[h].y;
                sm.As[kk + 2][r] = ra[h].z;
                sm.As[kk + 3][r] = ra[h].w;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = (tid >> 2) + h * 64, kq = tid & 3;
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int kk = kq * 4 + h2 * 16;
                sm.Bs[kk + 0][r] = rb[h][h2].x;
                sm.Bs[kk + 1][r] = rb[h][h2].y;
                sm.Bs[kk + 2][r] = rb[h][h2].z;
                sm.Bs[kk + 3][r] = rb[h][h2].w;
            }
        }
    };
    load_tiles(0, 0);
    for (int64_t col0 = 0; col0 < n; col0 += BN) {
        // column norms of this thread's eight columns, read before the tile
        float xnv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cl = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
            const int64_t gc = col0 + cl;
            xnv[j] = metric == 0 ? xnorm[gc < n ? gc : 0] : 0.f;
        }
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        for (int kb = 0; kb < nkb; ++kb) {
            store_tiles();
            __syncthreads();
            if (kb + 1 < nkb) load_tiles(col0, kb + 1);
            else if (col0 + BN < n) load_tiles(col0 + BN, 0);
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
                if (metric == 0) s = fmaxf(sm.qn[r] + xnv[j] - 2.f * acc[i][j], 0.f);
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
        // warp wid holds every column of rows 8 wid .. 8 wid + 7 (its two ty
        // values), so their buffers, counts and thresholds are its own: the
        // filter, the merges and the appends synchronise the warp only
        __syncwarp();
        // merge rows that could overflow
        for (int r = 8 * wid; r < 8 * wid + 8; ++r) {
            if (sm.cnt[r] + sm.pend[r] > BUF) {
                int64_t g = row0 + r;
                merge_row(sm, r, wid, K, out_s + g * K, out_i + g * K);
            }
        }
        __syncwarp();
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
        __syncwarp();
        if (lane < 8) sm.pend[8 * wid + lane] = 0;
        __syncwarp();
    }
    __syncthreads();
    for (int r = wid; r < BM; r += NT / 32) {
        int64_t g = row0 + r;
        if (g < nq) merge_row(sm, r, wid, K, out_s + g * K, out_i + g * K);
    }
}

// Re-order near-tie runs of each sorted row by FP64 distance (one warp per
// row).  Rows hold Kx entries; ties are judged with the per-pair error
// bound of the norm form.  Lane 0 finds the runs that reach the first K
// entries, every lane computes FP64 distances of their members, lane 0
// re-orders them.  A run that reaches the last stored entry cannot be
// closed inside the row: the row goes to fail[] (recomputed with more
// entries) unless fail is null (then it is only counted).  The first K
// entries are written to the output.
__global__ void __launch_bounds__(256) k_knn_fix(
    const float *__restrict__ Q, const float *__restrict__ X, int64_t nq, int d, int metric,
    const float *__restrict__ qnorm, const float *__restrict__ xnorm, float rel, float abs_err,
    int Kx, int K, int32_t *__restrict__ ids, float *__restrict__ ds, int32_t *__restrict__ out_i,
    float *__restrict__ out_s, unsigned long long *counters, int *fail, int *nfail) {
    __shared__ double c64[8][256];
    __shared__ int cut[8];
    const int w = threadIdx.x >> 5;
    int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + w;
    int lane = threadIdx.x & 31;
    if (q >= nq) return;
    int32_t *ri = ids + q * Kx;
    float *rs = ds + q * Kx;
    const float *qrow = Q + q * d;
    const double nan64 = __longlong_as_double(0x7ff8000000000000ll);
    auto err = [&](int j) -> float {
        int id = ri[j];
        if (id < 0) return 0.f;
        if (metric == 0) return rel * (qnorm[q] + xnorm[id] + fabsf(qnorm[q] + xnorm[id] - rs[j]));
        return abs_err;
    };
    for (int j = lane; j < Kx; j += 32) c64[w][j] = nan64;
    __syncwarp();
    // lane 0 marks the members of runs that start before K (end: cut)
    if (lane == 0) {
        int j = 0, end = 0;
        while (j < Kx && ri[j] >= 0 && j < K) {
            int e = j;
            while (e + 1 < Kx && ri[e + 1] >= 0 && rs[e + 1] - rs[e] <= err(e) + err(e + 1)) ++e;
            if (e > j)
                for (int t = j; t <= e; ++t) c64[w][t] = 0.0;  // to compute
            end = e + 1;
            j = e + 1;
        }
        cut[w] = end;
    }
    __syncwarp();
    for (int j = lane; j < cut[w]; j += 32)
        if (c64[w][j] == 0.0) c64[w][j] = dist64_rows(qrow, X + (int64_t)ri[j] * d, d, metric);
    __syncwarp();
    if (lane == 0) {
        unsigned long long rechecked = 0, unresolved = 0;
        int j = 0;
        while (j < cut[w]) {
            if (c64[w][j] != c64[w][j]) {
                ++j;
                continue;
            }
            int e = j;
            while (e + 1 < cut[w] && c64[w][e + 1] == c64[w][e + 1]) ++e;
            for (int a = j + 1; a <= e; ++a) {  // insertion sort by (FP64, id)
                const double kd = c64[w][a];
                const int ki = ri[a];
                int b = a - 1;
                while (b >= j && (c64[w][b] > kd || (c64[w][b] == kd && ri[b] > ki))) {
                    c64[w][b + 1] = c64[w][b];
                    ri[b + 1] = ri[b];
                    --b;
                }
                c64[w][b + 1] = kd;
                ri[b + 1] = ki;
            }
            rechecked += (unsigned long long)(e - j + 1);
            if (e == Kx - 1 && K < Kx) ++unresolved;
            j = e + 1;
        }
        if (rechecked) atomicAdd(counters + CNT_KNN_RECHECK, rechecked);
        if (unresolved) {
            if (fail) fail[atomicAdd(nfail, 1)] = (int)q;
            else atomicAdd(counters + CNT_KNN_UNRESOLVED, unresolved);
        }
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

// ------------------------------------------------------ certified screen
// The screened form on rows that are not BF16-exact.  Rows are centred on
// the column means (L2 only: distances do not change) and split into BF16
// hi + lo parts; the tile kernel contracts [hi | hi | lo] with [hi | lo | hi]
// (hi.hi + hi.lo + lo.hi) and keeps each row's Ks nearest by that screened
// distance.  k_knn_certify re-measures those Ks in FP32, re-orders near-tie
// runs by FP64 distance, and accepts the row only if a rigorous bound shows
// that no point outside the shortlist can come nearer than the K-th; other
// rows take the FP32 tiles.  The result equals the FP32 form's.

// Column sums of X (FP32 atomics; the mean only has to be some vector
// close to the centre: any shift leaves the distances unchanged).
__global__ void k_col_sums(const float *__restrict__ X, int64_t n, int d, int64_t rows_per_block,
                           float *sums) {
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= d) return;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(n, r0 + rows_per_block);
    float acc = 0.f;
    for (int64_t r = r0; r < r1; ++r) acc += X[r * d + c];
    atomicAdd(sums + c, acc);
}

// One warp per row: xh = x - mean (L2) or x (chord); hi = bf16(xh),
// lo = bf16(xh - hi) (xh - hi is exact in FP32); xq row [hi | hi | lo],
// xc row [hi | lo | hi], zero columns up to dp3; norms[r] = |xh|^2 in FP32
// (L2) or 1 (chord: the tiles then give 2 - 2<x, y>); *maxn = the largest
// |xh|^2 (float bits, non-negative, so integer order).
__global__ void k_split_rows(const float *__restrict__ X, int64_t n, int d, int dp3,
                             const float *__restrict__ colsum, float inv_n, int center,
                             __nv_bfloat16 *__restrict__ xq, __nv_bfloat16 *__restrict__ xc,
                             float *__restrict__ norms, unsigned *maxn) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *x = X + r * d;
    __nv_bfloat16 *q = xq + r * dp3, *c = xc + r * dp3;
    float acc = 0.f;
    for (int i = lane; i < d; i += 32) {
        const float v = center ? x[i] - colsum[i] * inv_n : x[i];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        q[i] = hi;
        q[d + i] = hi;
        q[2 * d + i] = lo;
        c[i] = hi;
        c[d + i] = lo;
        c[2 * d + i] = hi;
        acc = fmaf(v, v, acc);
    }
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    for (int i = 3 * d + lane; i < dp3; i += 32) {
        q[i] = z;
        c[i] = z;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        norms[r] = center ? acc : 1.f;
        atomicMax(maxn, __float_as_uint(acc));
    }
}

// Rigorous bound on |s_screen - s| for a row of squared norm na against any
// point of squared norm <= nb (norms of the centred rows for L2, of the rows
// for the chord); d the width, dp3 the contraction length.  Terms: the
// dropped lo.lo and the hi/lo residuals (3 2^-16 |x||y|, twice for -2<x,y>),
// the FP32 accumulation of dp3 exact products (dp3 2^-23 / (1 - dp3 2^-23)
// of their magnitudes, allowing truncating adders), the FP32 row norms
// (d 2^-23 relative), the final additions (2^-22 relative), and for L2 the
// rounding of the centring (2^-24 |xh| per row moves sqrt(s) by at most
// delta = 2^-24 (|x| + |y|)).
__device__ __forceinline__ float screen_bound(float na, float nb, int d, int dp3, int center) {
    const double a = sqrt((double)na) * 1.0001, b = sqrt((double)nb) * 1.0001;
    const double u16 = 1.52587890625e-05, u23 = 1.1920928955078125e-07;
    const double g = dp3 * u23 / (1.0 - dp3 * u23);
    double e = 2.0 * (3.001 * u16 + 1.02 * g) * a * b;
    if (center) {
        const double dl = 5.9604644775390625e-08 * 1.001 * (a + b);
        e += d * u23 * (a * a + b * b) + 2.3841857910156250e-07 * 1.01 * (a + b) * (a + b) +
             2.0 * (a + b) * dl + dl * dl;
    } else {
        e += 2.3841857910156250e-07 * 1.01 * (2.0 + 2.0 * a * b);
    }
    return (float)(e * 1.01 + 1e-12);
}

// One warp per row r: the Ks screened candidates (sid / ssc [n][Ks], sorted
// by screened distance) re-measured in FP32 (difference form / chord, the
// arithmetic of the FP32 gathers, error rel * s or abs_err), sorted by
// (s, id), near-tie runs that reach the first K re-ordered by FP64
// distance.  The row is certified when the exact K-th distance (FP64 if
// resolved, else FP32 plus its bound) is below the last screened distance
// minus screen_bound: every point outside the shortlist is then strictly
// farther.  Certified rows are written (FP64 distances rounded to FP32, as
// the FP32 form writes them); others go to fail[] for the FP32 tiles.
__global__ void __launch_bounds__(256) k_knn_certify(
    const float *__restrict__ X, int64_t n, int d, int metric, const int32_t *__restrict__ sid,
    const float *__restrict__ ssc, int Ks, int K, float rel, float abs_err,
    const float *__restrict__ norms, const unsigned *__restrict__ maxn, int dp3, int center,
    int32_t *__restrict__ out_i, float *__restrict__ out_s, int *fail, int *nfail,
    unsigned long long *counters) {
    __shared__ float ks[8][128];
    __shared__ int kid[8][128];
    __shared__ double c64[8][128];
    __shared__ double k64[8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, team = lane >> 3, li = lane & 7;
    const int64_t r = (int64_t)blockIdx.x * 8 + w;
    if (r >= n) return;
    const float *xr = X + r * d;
    const float4 *q4 = reinterpret_cast<const float4 *>(xr);
    for (int j = lane; j < 128; j += 32) {
        ks[w][j] = INFINITY;
        kid[w][j] = INT_MAX;
    }
    __syncwarp();
    int m = 0;
    for (int b0 = 0; b0 < Ks; b0 += 32) {
        const int j = b0 + lane;
        m += __popc(__ballot_sync(0xffffffffu, j < Ks && sid[r * Ks + j] >= 0));
    }
    for (int b0 = 0; b0 < Ks; b0 += 4) {
        const int j = b0 + team;
        const int id = j < Ks ? sid[r * Ks + j] : -1;
        const float sv = team8_dist(q4, reinterpret_cast<const float4 *>(X + (int64_t)(id >= 0 ? id : 0) * d),
                                    d / 4, li, metric);
        if (li == 0 && id >= 0) {
            ks[w][j] = sv;
            kid[w][j] = id;
        }
    }
    __syncwarp();
    warp_bitonic_sort(ks[w], kid[w], 128);
    float na = center ? norms[r] : 0.f;
    if (!center) {
        for (int c = lane; c < d; c += 32) na = fmaf(xr[c], xr[c], na);
        for (int o = 16; o; o >>= 1) na += __shfl_xor_sync(0xffffffffu, na, o);
    }
    auto err = [&](int j) -> float { return metric == 0 ? rel * ks[w][j] : abs_err; };
    const double nan64 = __longlong_as_double(0x7ff8000000000000ll);
    for (int j = lane; j < 128; j += 32) c64[w][j] = nan64;
    __syncwarp();
    // lane 0 marks the members of the near-tie runs that reach the first K
    if (lane == 0) {
        int j = 0, ok = 1, end = 0;
        while (ok && j < m && j < K) {
            int e = j;
            while (e + 1 < m && ks[w][e + 1] - ks[w][e] <= err(e) + err(e + 1)) ++e;
            if (e > j) {
                if (e == m - 1 && m == Ks) ok = 0;  // the run may continue outside the shortlist
                for (int t = j; t <= e; ++t) c64[w][t] = 0.0;  // to compute
            }
            end = e + 1;
            j = e + 1;
        }
        k64[w] = ok ? (double)end : -1.0;
    }
    __syncwarp();
    const int cut = k64[w] < 0.0 ? 0 : (int)k64[w];
    for (int j = lane; j < cut; j += 32)
        if (c64[w][j] == 0.0) c64[w][j] = dist64_rows(xr, X + (int64_t)kid[w][j] * d, d, metric);
    __syncwarp();
    if (lane == 0) {
        int ok = k64[w] >= 0.0;
        unsigned long long rechecked = 0;
        double kth = -1.0;  // exact K-th distance when resolved in FP64
        int j = 0;
        while (ok && j < cut) {
            if (c64[w][j] != c64[w][j]) {
                ++j;
                continue;
            }
            int e = j;
            while (e + 1 < cut && c64[w][e + 1] == c64[w][e + 1]) ++e;
            for (int a = j + 1; a <= e; ++a) {  // insertion sort by (FP64, id)
                const double kd = c64[w][a];
                const int ki = kid[w][a];
                int b = a - 1;
                while (b >= j && (c64[w][b] > kd || (c64[w][b] == kd && kid[w][b] > ki))) {
                    c64[w][b + 1] = c64[w][b];
                    kid[w][b + 1] = kid[w][b];
                    --b;
                }
                c64[w][b + 1] = kd;
                kid[w][b + 1] = ki;
            }
            if (j <= K - 1 && e >= K - 1) kth = c64[w][K - 1];
            rechecked += (unsigned long long)(e - j + 1);
            j = e + 1;
        }
        if (ok) {
            if (m < Ks) {
                ok = m == n - 1;  // the shortlist holds every other point
            } else {
                const double up = kth >= 0.0 ? kth : (double)ks[w][K - 1] + (double)err(K - 1);
                const float nb = __uint_as_float(*maxn);
                const double lower =
                    (double)ssc[r * Ks + Ks - 1] - (double)screen_bound(na, nb, d, dp3, center);
                ok = up < lower;
            }
        }
        if (rechecked) atomicAdd(counters + CNT_KNN_RECHECK, rechecked);
        if (!ok) {
            fail[atomicAdd(nfail, 1)] = (int)r;
            atomicAdd(counters + CNT_KNN_FALLBACK, 1ull);
        }
        k64[w] = ok ? 1.0 : 0.0;
    }
    __syncwarp();
    if (k64[w] == 0.0) return;
    for (int t = lane; t < K; t += 32) {
        const int id = t < m ? kid[w][t] : -1;
        out_i[r * K + t] = id;
        out_s[r * K + t] = id >= 0 ? (float)dist64_rows(xr, X + (int64_t)id * d, d, metric) : INFINITY;
    }
}

// Rows the screen could not certify: their K + 1 nearest by the FP32 tiles
// (the row itself among them unless K + 1 duplicates of it come first),
// written without the row itself.
__global__ void k_knn_fallback_scatter(const int *__restrict__ fail, int nf,
                                       const int32_t *__restrict__ gi, const float *__restrict__ gs,
                                       int K, int32_t *__restrict__ out_i, float *__restrict__ out_s,
                                       int drop_self = 1) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    const int64_t u = fail[t];
    const int kin = K + drop_self;  // entries of an input row
    int w = 0;
    for (int j = 0; j < kin && w < K; ++j) {
        const int id = gi[(int64_t)t * kin + j];
        if (drop_self && id == (int)u) continue;
        out_i[u * K + w] = id;
        out_s[u * K + w] = gs[(int64_t)t * kin + j];
        ++w;
    }
    for (; w < K; ++w) {
        out_i[u * K + w] = -1;
        out_s[u * K + w] = INFINITY;
    }
}

__global__ void k_gather_fail_rows(const float *__restrict__ X, int d, const int *__restrict__ fail,
                                   int nf, float *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nch = d / 4;
    if (t >= (int64_t)nf * nch) return;
    const int64_t r = t / nch, c = t % nch;
    reinterpret_cast<float4 *>(out)[r * nch + c] =
        reinterpret_cast<const float4 *>(X + (int64_t)fail[r] * d)[c];
}

}  // namespace

bool pg_knn_tc_supported(int d, int K);
int pg_knn_tc_max_k();
pg_status pg_knn_tc_split(pg_ctx *ctx, Scratch<__nv_bfloat16> &xc, Scratch<__nv_bfloat16> &xq,
                          int64_t n, int dp3, const float *norms, int32_t K, int32_t *ids,
                          float *dist, double work);
pg_status pg_knn_tc(pg_ctx *ctx, const float *D, int64_t n, int32_t d, const float *Q, int64_t nq,
                    int self, int32_t K, const float *xnorm, const float *qnorm, int32_t *ids,
                    float *dist);

namespace {

pg_status knn_core(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                   const float *Q, int64_t nq, int self, int32_t K, pg_precision precision,
                   int32_t *ids, float *dist, int kx_extra = 8);

pg_status knn_screened(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                       int32_t K, int Ks, int dp3, const DataFacts &facts, int32_t *ids,
                       float *dist) {
    const int center = metric == PG_METRIC_L2SQ;
    Scratch<float> csum, nrm, ss;
    Scratch<unsigned> mx;
    Scratch<__nv_bfloat16> xq, xc;
    Scratch<int32_t> si;
    Scratch<int> fail;
    PG_TRY(csum.alloc(ctx, (size_t)d));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(csum.p, 0, (size_t)d * 4, ctx->stream));
    if (center) {
        const int64_t rpb = std::max<int64_t>(64, (n + ctx->num_sms * 4 - 1) / (ctx->num_sms * 4));
        const dim3 g((unsigned)((n + rpb - 1) / rpb), (unsigned)((d + 255) / 256));
        k_col_sums<<<g, 256, 0, ctx->stream>>>(D, n, d, rpb, csum.p);
        PG_LAUNCHED(ctx);
    }
    PG_TRY(xq.alloc(ctx, (size_t)(n * dp3)));
    PG_TRY(xc.alloc(ctx, (size_t)(n * dp3)));
    PG_TRY(nrm.alloc(ctx, (size_t)n));
    PG_TRY(mx.alloc(ctx, 1));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(mx.p, 0, sizeof(unsigned), ctx->stream));
    k_split_rows<<<(unsigned)((n * 32 + 255) / 256), 256, 0, ctx->stream>>>(
        D, n, d, dp3, csum.p, (float)(1.0 / (double)n), center, xq.p, xc.p, nrm.p, mx.p);
    PG_LAUNCHED(ctx);
    PG_TRY(si.alloc(ctx, (size_t)(n * Ks)));
    PG_TRY(ss.alloc(ctx, (size_t)(n * Ks)));
    // the contraction the tensor cores run: 3d (padded) columns per pair
    PG_TRY(pg_knn_tc_split(ctx, xc, xq, n, dp3, nrm.p, Ks, si.p, ss.p,
                           2.0 * (double)n * (double)n * (double)dp3));
    PG_TRY(fail.alloc(ctx, (size_t)n + 1));
    PG_TRY_CUDA(ctx, cudaMemsetAsync(fail.p + n, 0, sizeof(int), ctx->stream));
    const ErrModel em = pg_err_model(metric, d, facts, false);
    k_knn_certify<<<(unsigned)((n + 7) / 8), 256, 0, ctx->stream>>>(
        D, n, d, metric == PG_METRIC_L2SQ ? 0 : 1, si.p, ss.p, Ks, K, em.rel, em.abs_, nrm.p,
        mx.p, dp3, center, ids, dist, fail.p, fail.p + n, ctx->d_counters);
    PG_LAUNCHED(ctx);
    int nf = 0;
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, fail.p + n, sizeof(int),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PG_TRY(pg_sync_check(ctx, "screened knn"));
    memcpy(&nf, ctx->h_pinned, sizeof(int));
    if (nf > 0) {
        Scratch<float> Qf, gs;
        Scratch<int32_t> gi;
        PG_TRY(Qf.alloc(ctx, (size_t)nf * d));
        PG_TRY(gi.alloc(ctx, (size_t)nf * (K + 1)));
        PG_TRY(gs.alloc(ctx, (size_t)nf * (K + 1)));
        const int64_t tot = (int64_t)nf * (d / 4);
        k_gather_fail_rows<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(D, d, fail.p,
                                                                                 nf, Qf.p);
        PG_LAUNCHED(ctx);
        PG_TRY(knn_core(ctx, D, n, d, metric, Qf.p, nf, 0, K + 1, PG_PREC_FP32, gi.p, gs.p));
        k_knn_fallback_scatter<<<(unsigned)((nf + 255) / 256), 256, 0, ctx->stream>>>(
            fail.p, nf, gi.p, gs.p, K, ids, dist);
        PG_LAUNCHED(ctx);
    }
    return PG_OK;
}

pg_status knn_core(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                   const float *Q, int64_t nq, int self, int32_t K, pg_precision precision,
                   int32_t *ids, float *dist, int kx_extra) {
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
    // Other data in the screened form (self kNN): the certified hi/lo
    // screen for the Ks = min(120, max(2K, K + 8)) nearest, then FP32 tiles
    // for the rows it cannot certify.  The result equals the FP32 form's.
    const int Ks = std::min(pg_knn_tc_max_k(), std::max(2 * K, K + 8));
    const int dp3 = (3 * d + 63) / 64 * 64;
    if (self && precision == PG_PREC_BF16_SCREEN && !(facts.exact && facts.bf16_exact) &&
        Ks >= K + 8 && n > Ks && pg_knn_tc_supported(dp3, Ks))
        return knn_screened(ctx, D, n, d, metric, K, Ks, dp3, facts, ids, dist);
    // rows hold Kx entries when ties must be resolved in FP64 afterwards
    int Kx = facts.exact ? K : (int)std::min<int64_t>((int64_t)K + kx_extra, KMAX);
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
        // rows whose near-tie run reaches the last stored entry are redone
        // with more entries (while the tiles can hold more)
        const bool redo = Kx < KMAX && K + (self ? 1 : 0) <= KMAX;
        Scratch<int> fail;
        if (redo) {
            PG_TRY(fail.alloc(ctx, (size_t)nq + 1));
            PG_TRY_CUDA(ctx, cudaMemsetAsync(fail.p + nq, 0, sizeof(int), ctx->stream));
        }
        k_knn_fix<<<(unsigned)((nq + 7) / 8), 256, 0, ctx->stream>>>(
            Qp, D, nq, d, metric == PG_METRIC_L2SQ ? 0 : 1, qnp, xn.p, em.rel, em.abs_, Kx, K, ti,
            ts, ids, dist, ctx->d_counters, redo ? fail.p : nullptr, redo ? fail.p + nq : nullptr);
        PG_LAUNCHED(ctx);
        if (redo) {
            int nf = 0;
            PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, fail.p + nq, sizeof(int),
                                             cudaMemcpyDeviceToHost, ctx->stream));
            PG_TRY(pg_sync_check(ctx, "knn fix"));
            memcpy(&nf, ctx->h_pinned, sizeof(int));
            if (nf > 0) {
                const int Kr = K + (self ? 1 : 0);
                Scratch<float> Qf, gs;
                Scratch<int32_t> gi;
                PG_TRY(Qf.alloc(ctx, (size_t)nf * d));
                PG_TRY(gi.alloc(ctx, (size_t)nf * Kr));
                PG_TRY(gs.alloc(ctx, (size_t)nf * Kr));
                const int64_t tot = (int64_t)nf * (d / 4);
                k_gather_fail_rows<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(
                    Qp, d, fail.p, nf, Qf.p);
                PG_LAUNCHED(ctx);
                PG_TRY(knn_core(ctx, D, n, d, metric, Qf.p, nf, 0, Kr, PG_PREC_FP32, gi.p, gs.p,
                                std::min(KMAX, 8 * kx_extra)));
                k_knn_fallback_scatter<<<(unsigned)((nf + 255) / 256), 256, 0, ctx->stream>>>(
                    fail.p, nf, gi.p, gs.p, K, ids, dist, self ? 1 : 0);
                PG_LAUNCHED(ctx);
            }
        }
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
