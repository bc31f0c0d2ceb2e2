// knn_tc.cu -- exact kNN distance tiles on the 5th-generation tensor cores
// (tcgen05, sm_103a) with a fused per-row top-K.
//
// s(q, x) = |q|^2 + |x|^2 - 2<q, x>, the dot products on tcgen05.mma
// kind::f16 (BF16 inputs, FP32 accumulation in TMEM).  Used when every value
// of D is an integer of magnitude <= 256 and every partial sum stays below
// 2^24: then the BF16 copy is exact and the tensor-core sums are exact
// integers, so the result equals the FP32 and FP64 definitions bit for bit.
//
// CTA = 10 warps for rows of at most 128 dims (6 for wider rows).  The
// epilogue threads first write the CTA's two 128-row query tiles into TMEM
// (one row per lane, two BF16 per 32-bit column), so the MMAs read only
// the candidate tiles from shared memory and every candidate tile feeds
// the MMAs of both query tiles (half the candidate bytes per product of a
// one-tile CTA).  Warp 0 issues TMA loads (128B-swizzled K-major tiles) of
// 128-row candidate tiles through a 3-stage ring.  Warp 1 owns the TMEM
// allocation and issues the MMAs (M128 N128 K16 steps, A from TMEM) into
// three FP32 accumulator buffers of 128 columns, rotating over the
// (candidate tile, query tile) pairs.  Warps 2-9 are the epilogue, four per
// query tile: thread t of a group owns query row t of its tile; it reads
// its accumulator row with tcgen05.ld.32x32b.x32, screens
// 32 columns at a time by their minimum against its current K-th distance
// and keeps a private max-heap of its K best in shared memory (sorted once
// at the end).  For the graph the points are spatially ordered first, and
// each CTA scans the tiles around its own rows before the rest.  Every mbarrier
// wait is bounded by a deadline; on expiry the kernel records an error,
// drains its outstanding MMAs, frees TMEM and returns.
#include <cuda.h>

#include <climits>
#include <cstring>

#include "pg_internal.cuh"

namespace {

constexpr int TM = 128;       // query rows per CTA = TMEM lanes
constexpr int TN = 128;       // candidate columns per tile
constexpr int STAGES = 3;     // candidate-tile ring
constexpr int KTC = 64;       // largest K of the resident-query kernel
constexpr int KTCK = 120;     // largest K of the k-blocked kernel (shared-memory fit)
constexpr int NTHREADS = 192;
constexpr int ACC_COLS = 256;  // two accumulator buffers of TN columns

// Instruction descriptor of tcgen05.mma kind::f16: D = F32 (bits 4-5),
// A = B = BF16 (bits 7-9, 10-12), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete; false once the CTA aborted or
// the 2-second deadline passed (which aborts the CTA and records the error).
// `backoff` threads (the single-thread producer and MMA roles) sleep between
// polls so that they leave issue slots to the epilogue warps.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, int *err,
                          bool backoff = false) {
    const uint64_t t0 = gtimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (backoff) __nanosleep(64);
        if ((it & 63) == 63) {
            if (*abort) return false;
            if (gtimer() - t0 > 2000000000ull) {
                *abort = 1;
                record_error(err, DERR_TIMEOUT, (long long)blockIdx.x);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); start address >> 4 in bits 0-13, LBO at 16-29
// (unused for swizzled K-major), SBO at 32-45, fixed 0b001 at 46-48,
// swizzle mode 2 (128B) at 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t a) {
    uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
}

// D (TMEM) [+]= A (TMEM, lane = row, a 32-bit column = two consecutive
// BF16 of a row) x B (shared memory descriptor)
__device__ __forceinline__ void umma_bf16_ts(uint32_t dtmem, uint32_t atmem, uint64_t bd,
                                             uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(dtmem),
        "r"(atmem), "l"(bd), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 columns of the warp's TMEM lane quarter from 32 registers per thread
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
        "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
        "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void epi_barrier(int nthreads = 128) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Named barrier of the epilogue threads that also ORs a flag over them, so
// that every epilogue thread takes the same abort decision.
__device__ __forceinline__ bool epi_barrier_or(int nthreads, bool flag) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
        " bar.red.or.pred po, 1, %2, pi;\n selp.u32 %0, 1, 0, po;\n}"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(nthreads)
        : "memory");
    return r != 0;
}


// Per-row max-heap of the K best (s, id) pairs in shared memory, layout
// [pos][TM]: element pos of row r at pos * TM + r, so a thread's accesses
// always fall in its own bank.  The root is the K-th best once the heap is
// full; thr / thr_id mirror it (+inf / INT_MAX while filling).
__device__ __forceinline__ void heap_push(float *Hs, int *Hi, int row, int K, int &cnt, float s,
                                          int id, float &thr, int &thr_id) {
    int pos;
    if (cnt < K) {
        pos = cnt++;
        while (pos > 0) {
            const int par = (pos - 1) >> 1;
            const float ps = Hs[par * TM + row];
            const int pi = Hi[par * TM + row];
            if (!pair_less(ps, pi, s, id)) break;
            Hs[pos * TM + row] = ps;
            Hi[pos * TM + row] = pi;
            pos = par;
        }
    } else {
        pos = 0;
        for (;;) {
            int c = 2 * pos + 1;
            if (c >= K) break;
            float cs = Hs[c * TM + row];
            int ci = Hi[c * TM + row];
            if (c + 1 < K) {
                const float c2 = Hs[(c + 1) * TM + row];
                const int i2 = Hi[(c + 1) * TM + row];
                if (pair_less(cs, ci, c2, i2)) {
                    c = c + 1;
                    cs = c2;
                    ci = i2;
                }
            }
            if (!pair_less(s, id, cs, ci)) break;
            Hs[pos * TM + row] = cs;
            Hi[pos * TM + row] = ci;
            pos = c;
        }
    }
    Hs[pos * TM + row] = s;
    Hi[pos * TM + row] = id;
    if (cnt == K) {
        thr = Hs[row];
        thr_id = Hi[row];
    }
}

// In-place heap sort of a row's heap into ascending (s, id) order.
__device__ __forceinline__ void heap_sort(float *Hs, int *Hi, int row, int cnt) {
    for (int end = cnt - 1; end > 0; --end) {
        const float ts = Hs[end * TM + row];
        const int ti = Hi[end * TM + row];
        Hs[end * TM + row] = Hs[row];
        Hi[end * TM + row] = Hi[row];
        int pos = 0;
        for (;;) {
            int c = 2 * pos + 1;
            if (c >= end) break;
            float cs = Hs[c * TM + row];
            int ci = Hi[c * TM + row];
            if (c + 1 < end) {
                const float c2 = Hs[(c + 1) * TM + row];
                const int i2 = Hi[(c + 1) * TM + row];
                if (pair_less(cs, ci, c2, i2)) {
                    c = c + 1;
                    cs = c2;
                    ci = i2;
                }
            }
            if (!pair_less(ts, ti, cs, ci)) break;
            Hs[pos * TM + row] = cs;
            Hi[pos * TM + row] = ci;
            pos = c;
        }
        Hs[pos * TM + row] = ts;
        Hi[pos * TM + row] = ti;
    }
}

struct TcLayout {
    uint32_t a, b, ls, li, nbuf, cnt, bars, misc, total;
};

// H = 1: four epilogue warps, one per TMEM lane quarter, each thread one
// row and all 128 columns of a tile; 3 candidate stages.  H = 2: eight
// epilogue warps, two per lane quarter taking 64 columns each, so two
// threads and two heaps per row (merged at the end); 2 candidate stages.
// QT = 2 (H = 1, dp <= 128): two 128-row query tiles per CTA, both in TMEM,
// so that every candidate tile feeds twice the MMAs; eight epilogue warps,
// one group of four per query tile; three accumulator buffers rotating
// over the (candidate tile, query tile) pairs; 3 candidate stages.
// KB (k-blocked, any dp): the query tile is not resident; every stage holds
// one 64-column block of the query tile and of the candidate tile, and the
// MMAs of a tile accumulate over the blocks; H = 1, 3 stages, K <= KTCK.
__host__ __device__ constexpr int tc_threads(int H, int QT = 1) { return 64 + 128 * H * QT; }
__host__ __device__ constexpr int tc_stages(int H, bool KB = false) {
    return KB ? 3 : (H == 1 ? 3 : 2);
}
__host__ __device__ constexpr int tc_kcap(bool KB) { return KB ? KTCK : KTC; }
constexpr uint32_t KB_STAGE = (uint32_t)(TM + TN) * 64 * 2;  // bytes of one k-blocked stage

__host__ __device__ inline TcLayout tc_layout(int dp, int H, bool KB = false, int QT = 1) {
    TcLayout L;
    uint32_t o = 0;
    L.a = o;  // unused: the resident query tiles live in TMEM
    L.b = o;
    o += KB ? tc_stages(H, KB) * KB_STAGE : (uint32_t)tc_stages(H) * TN * dp * 2;
    L.ls = o;  // H x QT x [kcap][TM] per-row heaps: distances
    o += (uint32_t)(H * QT) * tc_kcap(KB) * TM * 4;
    L.li = o;  // H x QT x [kcap][TM] ids
    o += (uint32_t)(H * QT) * tc_kcap(KB) * TM * 4;
    L.nbuf = o;  // 32 column norms per epilogue warp
    o += (uint32_t)(H * QT) * TM * 4;
    L.cnt = o;  // entries of the second heap of every row (H = 2)
    o += H == 2 ? TM * 4 : 0;
    L.bars = o;
    o += 24 * 8;
    L.misc = o;
    o += 16;
    L.total = o;
    return L;
}

// perm (nullable): position -> original id of spatially ordered points (Q
// is D itself); lists hold original ids, rows are written back in original
// order.  rotate: scan the tiles around the CTA's rows first.
template <int H, bool KB, int QT>
__global__ void __launch_bounds__(tc_threads(H, QT), 1)
k_knn_tc(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapX,
         const __nv_bfloat16 *__restrict__ qrows, int64_t nq, int64_t n, int dp,
         const float *__restrict__ qnorm,
         const float *__restrict__ xnorm, const float *__restrict__ xcmin, int K,
         int self_exclude, int32_t *__restrict__ out_i,
         float *__restrict__ out_s, int *err, const int32_t *__restrict__ perm, int rotate,
         unsigned long long *progress, int resident) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    static_assert(QT == 1 || (QT == 2 && H == 1 && !KB), "two query tiles: H = 1, resident");
    constexpr int STG = tc_stages(H, KB), NEPI = 128 * H * QT, KCAP = tc_kcap(KB);
    // accumulator buffers of TN columns: two (QT = 1) or three rotating over
    // the (candidate tile, query tile) pairs (QT = 2)
    constexpr int NACC = QT == 2 ? 3 : 2;
    // resident variants: accumulators in columns [0, NACC TN), query tile qt
    // in [ABASE + qt dp / 2, ...) (two BF16 of a row per 32-bit column);
    // dp / 2 <= 64 when QT = 2
    constexpr uint32_t ABASE = (uint32_t)NACC * TN;
    constexpr uint32_t TMEM_COLS = KB ? (uint32_t)ACC_COLS : 512u;
    const TcLayout Ly = tc_layout(dp, H, KB, QT);
    uint8_t *B = sm + Ly.b;
    float *Ls0 = reinterpret_cast<float *>(sm + Ly.ls);
    int *Li0 = reinterpret_cast<int *>(sm + Ly.li);
    float *nbuf = reinterpret_cast<float *>(sm + Ly.nbuf);
    int *cntbuf = reinterpret_cast<int *>(sm + Ly.cnt);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + Ly.bars);
    // acc_full[b * QT + qt]: buffer b holds a finished tile of query tile qt
    // (one barrier per consumer group, so each group waits on every phase of
    // its own barriers in order); acc_empty[b]: the group that read buffer b
    // has released it
    uint64_t *a_full = bars, *b_full = bars + 1, *b_empty = bars + 1 + STG;
    uint64_t *acc_full = bars + 1 + 2 * STG, *acc_empty = acc_full + NACC * QT;
    uint64_t *drain = acc_empty + NACC;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + Ly.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + Ly.misc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TM * QT;
    const int nkb = dp / 64;
    const int ntiles = (int)((n + TN - 1) / TN);
    const uint32_t b_bytes = (uint32_t)TN * dp * 2;
    // With `rotate` (spatially sorted points) the scan first covers a window
    // of `pre` tiles around the CTA's own rows, where its nearest candidates
    // are, so the thresholds tighten early; then every other tile in a
    // common cyclic order.  A CTA starts that cycle where the CTAs already
    // running are: `progress` counts the tiles issued by all CTAs, so
    // progress / resident is the position every resident CTA has reached if
    // each started the same way, and concurrent CTAs read the same candidate
    // tiles at about the same time and share them in L2.  Every role walks
    // the same order (the start is read once and shared).
    const int pre = rotate ? min(16, ntiles) : 0;
    const int w0 =
        rotate ? max(0, min((int)((row0 + TM * QT / 2) / TN) - pre / 2, ntiles - pre)) : 0;
    const int nrest = max(1, ntiles - pre);
    int *start_slot = reinterpret_cast<int *>(sm + Ly.misc + 8);

    if (threadIdx.x == 0) {
        mbar_init(a_full, KB ? 1 : NEPI);  // resident: every epilogue thread stages its row
        for (int s = 0; s < STG; ++s) {
            mbar_init(b_full + s, 1);
            mbar_init(b_empty + s, 1);
        }
        for (int a = 0; a < NACC * QT; ++a) mbar_init(acc_full + a, 1);
        for (int a = 0; a < NACC; ++a) mbar_init(acc_empty + a, NEPI / QT);
        mbar_init(drain, 1);
        *abort = 0;
        *start_slot = progress ? (int)((atomicAdd(progress, 0ull) / (unsigned long long)resident) %
                                       (unsigned long long)nrest)
                               : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int start = *start_slot;
    auto tile_at = [&](int t) {
        if (t < pre) return w0 + t;
        int k = t - pre + start;
        if (k >= nrest) k -= nrest;
        return k < w0 ? k : k + pre;
    };

    if (warp == 0) {
        if (lane == 0 && KB) {  // ---------------- TMA producer, k-blocked
            int issued = 0;
            bool ok = true;
            for (int t = 0; ok && t < ntiles; ++t) {
                for (int kb = 0; kb < nkb; ++kb) {
                    const int it = t * nkb + kb, s = it % STG;
                    if (!mbar_wait(b_empty + s, ((it / STG) & 1) ^ 1, abort, err, true)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = B + (size_t)s * KB_STAGE;
                    mbar_expect_tx(b_full + s, KB_STAGE);
                    tma_load_2d(st, &mapQ, b_full + s, kb * 64, (int)row0);
                    tma_load_2d(st + TM * 128, &mapX, b_full + s, kb * 64, tile_at(t) * TN);
                    if (kb == 0 && progress) atomicAdd(progress, 1ull);
                    issued = it + 1;
                }
            }
            if (*abort) {  // let the copies already issued land before TMEM is freed
                for (int it = max(0, issued - STG); it < issued; ++it) {
                    uint64_t t0 = gtimer();
                    while (!mbar_try_wait(b_full + it % STG, (it / STG) & 1) &&
                           gtimer() - t0 < 1000000000ull) {
                    }
                }
            }
        } else if (lane == 0) {  // ---------------- TMA producer
            int issued = 0;
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % STG;
                if (!mbar_wait(b_empty + s, ((t / STG) & 1) ^ 1, abort, err, true)) break;
                mbar_expect_tx(b_full + s, b_bytes);
                for (int kb = 0; kb < nkb; ++kb)
                    tma_load_2d(B + (size_t)s * TN * dp * 2 + kb * TN * 128, &mapX, b_full + s,
                                kb * 64, tile_at(t) * TN);
                if (progress) atomicAdd(progress, 1ull);
                issued = t + 1;
            }
            if (*abort) {  // let the copies already issued land before TMEM is freed
                for (int t = max(0, issued - STG); t < issued; ++t) {
                    uint64_t t0 = gtimer();
                    while (!mbar_try_wait(b_full + t % STG, (t / STG) & 1) &&
                           gtimer() - t0 < 1000000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && KB) {  // ---------------- MMA issuer, k-blocked
            bool ok = true;
            for (int t = 0; ok && t < ntiles; ++t) {
                const int a = t & 1;
                if (!mbar_wait(acc_empty + a, ((t >> 1) & 1) ^ 1, abort, err, true)) break;
                for (int kb = 0; kb < nkb; ++kb) {
                    const int it = t * nkb + kb, s = it % STG;
                    if (!mbar_wait(b_full + s, (it / STG) & 1, abort, err, true)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = saddr(B + (size_t)s * KB_STAGE), b0 = a0 + TM * 128;
                    for (int k = 0; k < 4; ++k)
                        umma_bf16(tmem + a * TN, sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32),
                                  (kb > 0 || k > 0) ? 1u : 0u);
                    umma_commit(b_empty + s);
                }
                if (ok) umma_commit(acc_full + a);
            }
            umma_commit(drain);
            uint64_t t0 = gtimer();
            while (!mbar_try_wait(drain, 0) && gtimer() - t0 < 1000000000ull) {
            }
        } else if (lane == 0) {  // ---------------- MMA issuer
            bool ok = mbar_wait(a_full, 0, abort, err, true);
            for (int t = 0; ok && t < ntiles; ++t) {
                const int s = t % STG;
                if (!mbar_wait(b_full + s, (t / STG) & 1, abort, err, true)) break;
                const uint32_t b0 = saddr(B + (size_t)s * TN * dp * 2);
                for (int qt = 0; qt < QT; ++qt) {
                    // pair j = QT t + qt goes to buffer j % NACC, its (j / NACC)-th use
                    const int j = QT * t + qt, a = j % NACC;
                    if (!mbar_wait(acc_empty + a, ((j / NACC) & 1) ^ 1, abort, err, true)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aq = tmem + ABASE + (uint32_t)(qt * (dp / 2));
                    for (int k = 0; k < dp / 16; ++k) {
                        const int kb = k >> 2, koff = (k & 3) * 32;
                        umma_bf16_ts(tmem + a * TN, aq + 8 * k,
                                     sw128_desc(b0 + kb * TN * 128 + koff), k > 0 ? 1u : 0u);
                    }
                    umma_commit(acc_full + a * QT + qt);
                }
                if (!ok) break;
                umma_commit(b_empty + s);
            }
            // every MMA issued above has completed once `drain` flips
            umma_commit(drain);
            uint64_t t0 = gtimer();
            while (!mbar_try_wait(drain, 0) && gtimer() - t0 < 1000000000ull) {
            }
        }
    } else {  // ---------------------------------------- epilogue
        const int q = warp & 3;               // TMEM lane quarter
        const int grp = (warp - 2) >> 2;      // group of four warps
        const int half = QT == 1 ? grp : 0;   // column half (H = 2)
        const int qt = QT == 1 ? 0 : grp;     // query tile (QT = 2)
        const int c_lo = half * (4 / H);
        float *Ls = Ls0 + grp * KCAP * TM;
        int *Li = Li0 + grp * KCAP * TM;
        const int row = q * 32 + lane;
        const int64_t g = row0 + qt * TM + row;
        const bool live = g < nq;
        const float nqr = live ? qnorm[g] : 0.f;
        if (!KB) {
            // the query tile into TMEM: thread `row` writes its row (zeros
            // past nq) to columns [ABASE + qt dp / 2, ... + dp / 2) of its lane
            if (half == 0) {
                const uint4 *src = reinterpret_cast<const uint4 *>(qrows + (live ? g : 0) * dp);
                for (int b = 0; b < dp / 64; ++b) {
                    uint32_t r[32];
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4) {
                        const uint4 v = live ? __ldg(src + b * 8 + c4) : make_uint4(0u, 0u, 0u, 0u);
                        r[4 * c4 + 0] = v.x;
                        r[4 * c4 + 1] = v.y;
                        r[4 * c4 + 2] = v.z;
                        r[4 * c4 + 3] = v.w;
                    }
                    tmem_st32(tmem + ((uint32_t)(q * 32) << 16) +
                                  (ABASE + (uint32_t)(qt * (dp / 2) + 32 * b)), r);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            tc_fence_before();
            mbar_arrive(a_full);
        }
        int count = 0;
        float thr = INFINITY;  // the heap's K-th pair once full
        int thr_id = INT_MAX;
        // Column norms: lane j of a warp loads the norm of column j of each
        // 32-column chunk it processes, one tile ahead, and stages it in the
        // warp's own 32-float slot right before the chunk: no barrier across
        // warps inside the tile loop.
        constexpr int NCH = 4 / H;  // chunks of one thread per tile
        float *wn = nbuf + (warp - 2) * 32;
        auto colnorm = [&](int t, int c) -> float {
            if (t >= ntiles) return INFINITY;
            const int64_t col = (int64_t)tile_at(t) * TN + c * 32 + lane;
            return col < n ? xnorm[col] : INFINITY;
        };
        // the smallest column norm of each 32-column chunk (one value for the
        // whole warp), also one tile ahead
        auto chunkmin = [&](int t, int c) -> float {
            return t < ntiles ? xcmin[(int64_t)tile_at(t) * (TN / 32) + c] : INFINITY;
        };
        float nxt[NCH], nxm[NCH];
#pragma unroll
        for (int ci = 0; ci < NCH; ++ci) {
            nxt[ci] = colnorm(0, c_lo + ci);
            nxm[ci] = chunkmin(0, c_lo + ci);
        }
        for (int t = 0; t < ntiles; ++t) {
            // the buffer of pair QT t + qt; this group's (t / NACC)-th use of it
            const int a = (QT * t + qt) % NACC;
            const int64_t colbase = (int64_t)tile_at(t) * TN;
            float cur[NCH], cum[NCH];
#pragma unroll
            for (int ci = 0; ci < NCH; ++ci) {
                cur[ci] = nxt[ci];
                cum[ci] = nxm[ci];
                nxt[ci] = colnorm(t + 1, c_lo + ci);
                nxm[ci] = chunkmin(t + 1, c_lo + ci);
            }
            mbar_wait(acc_full + a * QT + qt, (t / NACC) & 1, abort, err);
            // a warp that sees the abort leaves; the others leave at their
            // next check (no epilogue barrier inside this loop)
            if (__any_sync(0xffffffffu, *abort != 0)) break;
            tc_fence_after();
#pragma unroll
            for (int ci = 0; ci < NCH; ++ci) {
                const int c = c_lo + ci;
                __syncwarp();  // lanes that pushed into their heaps rejoin before the load
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * TN + c * 32), v);
                // lower bound of the chunk's distances for this row: |q|^2 +
                // (smallest column norm) - 2 (largest dot product).  Every
                // operation is correctly rounded, hence monotone, so the bound
                // never exceeds a column's computed distance: a chunk whose
                // bound is above the K-th distance holds no candidate, and
                // most chunks are dismissed by it without the column norms.
                float vx[4] = {v[0], v[1], v[2], v[3]};
#pragma unroll
                for (int j = 4; j < 32; ++j) vx[j & 3] = fmaxf(vx[j & 3], v[j]);
                const float vmax = fmaxf(fmaxf(vx[0], vx[1]), fmaxf(vx[2], vx[3]));
                const bool need = live && nqr + fmaf(-2.f, vmax, cum[ci]) <= thr;
                if (!__any_sync(0xffffffffu, need)) continue;
                __syncwarp();
                wn[lane] = cur[ci];
                __syncwarp();
                if (!need) continue;
                float nbv[32];
                const float4 *nb4 = reinterpret_cast<const float4 *>(wn);
#pragma unroll
                for (int j4 = 0; j4 < 8; ++j4) {
                    const float4 t4 = nb4[j4];
                    nbv[j4 * 4 + 0] = t4.x;
                    nbv[j4 * 4 + 1] = t4.y;
                    nbv[j4 * 4 + 2] = t4.z;
                    nbv[j4 * 4 + 3] = t4.w;
                }
                float m = INFINITY;
#pragma unroll
                for (int j = 0; j < 32; ++j) m = fminf(m, fmaf(-2.f, v[j], nbv[j]));
                // rare: this row may accept a column of the chunk (ties with
                // the K-th distance are decided by id); each thread pushes
                // into its own heap, independently of the other lanes
                if (!(live && nqr + m <= thr)) continue;
                float sv[32];
                unsigned mask = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    sv[j] = fmaxf(nqr + fmaf(-2.f, v[j], nbv[j]), 0.f);
                    if (sv[j] <= thr) mask |= 1u << j;
                }
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float s = sv[j];
                    if (!(s <= thr)) continue;
                    const int64_t col = colbase + c * 32 + j;
                    if (col >= n || (self_exclude && col == g)) continue;
                    const int id = perm ? perm[col] : (int)col;
                    if (!pair_less(s, id, thr, thr_id)) continue;
                    heap_push(Ls, Li, row, K, count, s, id, thr, thr_id);
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty + a);
        }
        heap_sort(Ls, Li, row, count);
        if (H == 2) {
            // the row's two sorted lists (disjoint columns) -> its K best,
            // merged backwards into the first half's list
            if (half == 1) cntbuf[row] = count;
            epi_barrier(NEPI);
            if (half == 0) {
                const float *Bs = Ls0 + KCAP * TM;
                const int *Bi = Li0 + KCAP * TM;
                const int na0 = count, nb0 = cntbuf[row];
                const int total = min(K, na0 + nb0);
                int i = 0, j = 0;
                for (int t = 0; t < total; ++t) {
                    if (j >= nb0 || (i < na0 && pair_less(Ls[i * TM + row], Li[i * TM + row],
                                                          Bs[j * TM + row], Bi[j * TM + row])))
                        ++i;
                    else
                        ++j;
                }
                for (int p = total - 1; p >= 0; --p) {
                    const bool takeA =
                        j == 0 || (i > 0 && pair_less(Bs[(j - 1) * TM + row], Bi[(j - 1) * TM + row],
                                                      Ls[(i - 1) * TM + row], Li[(i - 1) * TM + row]));
                    if (takeA) {
                        --i;
                        Ls[p * TM + row] = Ls[i * TM + row];
                        Li[p * TM + row] = Li[i * TM + row];
                    } else {
                        --j;
                        Ls[p * TM + row] = Bs[j * TM + row];
                        Li[p * TM + row] = Bi[j * TM + row];
                    }
                }
                count = total;
            }
        }
        __syncwarp();
        // the first half's warps write their 32 rows (coalesced along each
        // row); a permuted point's row goes back to its original position
        if (half == 0) {
            for (int rr = 0; rr < 32; ++rr) {
                const int r2 = q * 32 + rr;
                const int64_t gp = row0 + qt * TM + r2;
                const int cnt2 = __shfl_sync(0xffffffffu, count, rr);
                if (gp >= nq) continue;
                const int64_t g2 = perm ? (int64_t)perm[gp] : gp;
                for (int j = lane; j < K; j += 32) {
                    out_i[g2 * K + j] = j < cnt2 ? Li[j * TM + r2] : -1;
                    out_s[g2 * K + j] = j < cnt2 ? Ls[j * TM + r2] : INFINITY;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// FP32 rows -> BF16 rows padded with zeros to dp columns

// ---------------------------------------------------------------------------
// Split-column argmin on the tensor cores (the free-node scan of the
// connectivity step).  Every CTA takes the same <= 128 query rows and a
// contiguous range of candidate tiles; a column c takes part only while
// reached[c] != 0 and deg[c] < R (a masked column's norm is staged as +inf).
// Each row's smallest (s, c) of the range goes to best[row] by atomicMin on
// the key (FP32 bits << 32 | c): s >= 0, so the key order is the (s, id)
// order.  Same roles, barriers and deadlines as k_knn_tc.
struct ArgLayout {
    uint32_t a, b, nbuf, bars, misc, total;
};

__host__ __device__ inline ArgLayout arg_layout(int dp) {
    ArgLayout L;
    uint32_t o = 0;
    L.a = o;
    o += (uint32_t)TM * dp * 2;
    L.b = o;
    o += (uint32_t)STAGES * TN * dp * 2;
    L.nbuf = o;
    o += 2 * TN * 4;
    L.bars = o;
    o += 16 * 8;
    L.misc = o;
    o += 16;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(NTHREADS, 1)
k_argmin_tc(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapX,
            const int *__restrict__ nrows_p, int64_t n, int dp, const float *__restrict__ qnorm,
            const float *__restrict__ xnorm, const int *__restrict__ cid,
            const int *__restrict__ reached,
            const int32_t *__restrict__ deg, int R, int tiles_per_cta,
            unsigned long long *__restrict__ best, int *err) {
    const int ntiles_all = (int)((n + TN - 1) / TN);
    const int t0 = blockIdx.x * tiles_per_cta;
    const int ntiles = min(ntiles_all - t0, tiles_per_cta);
    const int nrows = *nrows_p;
    if (ntiles <= 0 || nrows <= 0) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const ArgLayout Ly = arg_layout(dp);
    uint8_t *A = sm + Ly.a;
    uint8_t *B = sm + Ly.b;
    float *nbuf = reinterpret_cast<float *>(sm + Ly.nbuf);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + Ly.bars);
    uint64_t *a_full = bars, *b_full = bars + 1, *b_empty = bars + 1 + STAGES;
    uint64_t *acc_full = bars + 1 + 2 * STAGES, *acc_empty = bars + 3 + 2 * STAGES;
    uint64_t *drain = bars + 5 + 2 * STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + Ly.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + Ly.misc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = dp / 64;
    const uint32_t a_bytes = (uint32_t)TM * dp * 2, b_bytes = (uint32_t)TN * dp * 2;

    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(b_full + s, 1);
            mbar_init(b_empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(acc_full + a, 1);
            mbar_init(acc_empty + a, 128);
        }
        mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_slot)),
                     "r"(ACC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // ---------------- TMA producer
            mbar_expect_tx(a_full, a_bytes);
            for (int kb = 0; kb < nkb; ++kb) tma_load_2d(A + kb * TM * 128, &mapQ, a_full, kb * 64, 0);
            int issued = 0;
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % STAGES;
                if (!mbar_wait(b_empty + s, ((t / STAGES) & 1) ^ 1, abort, err, true)) break;
                mbar_expect_tx(b_full + s, b_bytes);
                for (int kb = 0; kb < nkb; ++kb)
                    tma_load_2d(B + (size_t)s * TN * dp * 2 + kb * TN * 128, &mapX, b_full + s,
                                kb * 64, (t0 + t) * TN);
                issued = t + 1;
            }
            if (*abort) {
                for (int t = max(0, issued - STAGES); t < issued; ++t) {
                    uint64_t w0 = gtimer();
                    while (!mbar_try_wait(b_full + t % STAGES, (t / STAGES) & 1) &&
                           gtimer() - w0 < 1000000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------- MMA issuer
            bool ok = mbar_wait(a_full, 0, abort, err, true);
            for (int t = 0; ok && t < ntiles; ++t) {
                const int s = t % STAGES, a = t & 1;
                if (!mbar_wait(b_full + s, (t / STAGES) & 1, abort, err, true)) break;
                if (!mbar_wait(acc_empty + a, ((t >> 1) & 1) ^ 1, abort, err, true)) break;
                tc_fence_after();
                const uint32_t a0 = saddr(A), b0 = saddr(B + (size_t)s * TN * dp * 2);
                for (int k = 0; k < dp / 16; ++k) {
                    const int kb = k >> 2, koff = (k & 3) * 32;
                    umma_bf16(tmem + a * TN, sw128_desc(a0 + kb * TM * 128 + koff),
                              sw128_desc(b0 + kb * TN * 128 + koff), k > 0 ? 1u : 0u);
                }
                umma_commit(b_empty + s);
                umma_commit(acc_full + a);
            }
            umma_commit(drain);
            uint64_t w0 = gtimer();
            while (!mbar_try_wait(drain, 0) && gtimer() - w0 < 1000000000ull) {
            }
        }
    } else {  // ---------------------------------------- epilogue
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const bool live = row < nrows;
        const float nqr = live ? qnorm[row] : 0.f;
        float bs = INFINITY;
        int bid = INT_MAX;
        // column value of tile t for this thread's column: the norm, or +inf
        // for a masked column; loaded one tile ahead
        auto colval = [&](int t) -> float {
            const int64_t c = (int64_t)(t0 + t) * TN + row;
            if (t >= ntiles || c >= n) return INFINITY;
            const int x = cid[c];
            const int rc = reached[x];
            const int dc = deg[x];
            const float xc = xnorm[c];
            return (rc && dc < R) ? xc : INFINITY;
        };
        float next = colval(0);
        for (int t = 0; t < ntiles; ++t) {
            const int a = t & 1;
            const int64_t colbase = (int64_t)(t0 + t) * TN;
            nbuf[a * TN + row] = next;
            next = colval(t + 1);
            mbar_wait(acc_full + a, (t >> 1) & 1, abort, err);
            if (epi_barrier_or(128, *abort != 0)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < TN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * TN + c * 32), v);
                float m = INFINITY;
#pragma unroll
                for (int j = 0; j < 32; ++j) m = fminf(m, fmaf(-2.f, v[j], nbuf[a * TN + c * 32 + j]));
                // columns rise through the range, so a strictly smaller value
                // is the only way to a new (s, id) minimum
                if (live && nqr + m < bs) {
                    int jm = 0;
#pragma unroll
                    for (int j = 31; j >= 0; --j)
                        if (fmaf(-2.f, v[j], nbuf[a * TN + c * 32 + j]) == m) jm = j;
                    bs = nqr + m;
                    bid = cid[colbase + c * 32 + jm];  // ascending ids: ties keep the smallest
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty + a);
        }
        if (live && bid != INT_MAX && !*abort)
            atomicMin(best + row, ((unsigned long long)__float_as_uint(fmaxf(bs, 0.f)) << 32) |
                                      (unsigned)bid);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ACC_COLS)
                     : "memory");
    }
}

__global__ void k_free_flags(const int32_t *deg, int64_t n, int R, int32_t *flag) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) flag[x] = deg[x] < R ? 1 : 0;
}

__global__ void k_free_scatter(const int32_t *flag, const int64_t *off, int64_t n, int *cid) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n && flag[x]) cid[off[x]] = (int)x;
}

// rows ids[0..m) of D to BF16 [m][dp] (zero padded) with their FP32
// squared norms; one warp per row
__global__ void k_gather_bf16_rows(const float *__restrict__ D, int d, int dp, const int *ids,
                                   int64_t m, __nv_bfloat16 *__restrict__ out,
                                   float *__restrict__ norms) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const float *src = D + (int64_t)ids[row] * d;
    float acc = 0.f;
    for (int c = lane; c < dp; c += 32) {
        const float x = c < d ? src[c] : 0.f;
        acc = fmaf(x, x, acc);
        out[row * dp + c] = __float2bfloat16_rn(x);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) norms[row] = acc;
}

// <= 128 rows ids[0..*count) of D to BF16 [128][dp] (zero rows past the
// count) with their FP32 squared norms; one warp per row
__global__ void k_tc_gather_rows(const float *__restrict__ D, int d, int dp, const int *ids,
                                 const int *count, __nv_bfloat16 *__restrict__ out,
                                 float *__restrict__ norms) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= TM) return;
    const bool live = row < *count;
    const float *src = live ? D + (int64_t)ids[row] * d : nullptr;
    float acc = 0.f;
    for (int c = lane; c < dp; c += 32) {
        const float x = live && c < d ? src[c] : 0.f;
        acc = fmaf(x, x, acc);
        out[(int64_t)row * dp + c] = __float2bfloat16_rn(x);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) norms[row] = acc;
}

__global__ void k_tc_norms(const float *__restrict__ D, int64_t n, int d, float *__restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    float acc = 0.f;
    for (int c = lane; c < d; c += 32) acc = fmaf(D[r * d + c], D[r * d + c], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = acc;
}

__global__ void k_to_bf16(const float *__restrict__ X, int64_t n, int d, int dp,
                          __nv_bfloat16 *__restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * dp) return;
    int64_t r = t / dp;
    int c = (int)(t % dp);
    out[t] = __float2bfloat16_rn(c < d ? X[r * d + c] : 0.f);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

pg_status make_map(pg_ctx *ctx, CUtensorMap *map, const __nv_bfloat16 *base, int64_t rows, int dp) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return pg_fail(ctx, PG_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return pg_fail(ctx, PG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PG_OK;
}

}  // namespace

// Kernel variant for dp columns and K neighbours: the resident-query kernel
// with two query tiles per CTA (both in TMEM: dp <= 128), else with one
// query tile and one heap per row, else two heaps per row, else the
// k-blocked kernel.
struct TcVariant {
    int H;
    bool KB;
    int QT;
};

static TcVariant tc_variant(int dp, int K) {
    const uint32_t cap = 227 * 1024 - 1024;
    if (K <= KTC && dp <= 128 && tc_layout(dp, 1, false, 2).total <= cap) return {1, false, 2};
    if (K <= KTC && tc_layout(dp, 1).total <= cap) return {1, false, 1};
    if (K <= KTC && tc_layout(dp, 2).total <= cap) return {2, false, 1};
    return {1, true, 1};
}

bool pg_knn_tc_supported(int d, int K) {
    const int dp = (d + 63) / 64 * 64;
    return K >= 1 && K <= KTCK && d <= 8192 && tc_layout(dp, 1, true).total + 1024 <= 227 * 1024;
}

int pg_knn_tc_max_k() { return KTCK; }


namespace {

__global__ void k_gather_bf16(const __nv_bfloat16 *__restrict__ src, const int32_t *__restrict__ idx,
                              int64_t m, int dp, __nv_bfloat16 *__restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nch = dp / 8;  // 16-byte chunks
    if (t >= m * nch) return;
    const int64_t r = t / nch, c = t % nch;
    reinterpret_cast<uint4 *>(dst)[r * nch + c] =
        reinterpret_cast<const uint4 *>(src)[(int64_t)idx[r] * nch + c];
}

__global__ void k_gather_f32(const float *__restrict__ src, const int32_t *__restrict__ idx,
                             int64_t m, float *__restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) dst[t] = src[idx[t]];
}

// smallest of each 32 consecutive column norms (+inf past n)
__global__ void k_chunk_min(const float *__restrict__ xn, int64_t n, int64_t nch, float *out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    float m = INFINITY;
    for (int64_t i = c * 32; i < min(n, c * 32 + 32); ++i) m = fminf(m, xn[i]);
    out[c] = m;
}

__global__ void k_pivot_ids(int32_t *ids, int p, int64_t n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < p) ids[t] = (int32_t)((int64_t)t * n / p);
}

__global__ void k_bucket_count(const int32_t *__restrict__ bucket, int64_t n, int32_t *cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) atomicAdd(&cnt[max(bucket[t], 0)], 1);
}

__global__ void k_bucket_scatter(const int32_t *__restrict__ bucket, int64_t n,
                                 unsigned long long *cursor, int32_t *perm) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) perm[atomicAdd(&cursor[max(bucket[t], 0)], 1ull)] = (int32_t)t;
}

}  // namespace

// The tile launch on prepared BF16 copies [rows][dp]: xc the candidate
// rows; for self mode the query rows are xc itself or, when xq_sep is
// given, the same points in another layout (the hi/lo split of the
// screened form); otherwise qext holds nq external query rows.  The copies
// are released once the spatially ordered ones are made.
static pg_status tc_knn_run(pg_ctx *ctx, Scratch<__nv_bfloat16> &xc,
                            Scratch<__nv_bfloat16> *xq_sep, const __nv_bfloat16 *qext, int64_t n,
                            int64_t nq, int dp, int self, int32_t K, const float *xnorm,
                            const float *qnorm, int32_t *ids, float *dist, double work) {
    Scratch<__nv_bfloat16> pb, xs, xqs;
    Scratch<int32_t> pid, asg, perm, cnt;
    Scratch<float> adist, pn, xsn;
    Scratch<int64_t> boff;
    const __nv_bfloat16 *qp = self ? (xq_sep ? xq_sep->p : xc.p) : qext;
    const TcVariant V = tc_variant(dp, K);
    const size_t smem = tc_layout(dp, V.H, V.KB, V.QT).total + 1024;
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(
                         V.KB ? k_knn_tc<1, true, 1>
                              : (V.QT == 2 ? k_knn_tc<1, false, 2>
                                           : (V.H == 2 ? k_knn_tc<2, false, 1> : k_knn_tc<1, false, 1>)),
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int rows_per_cta = TM * V.QT;
    // one launch of the chosen variant
    // tiles issued by all CTAs of a launch (the common start of each cycle)
    Scratch<unsigned long long> prog;
    PG_TRY(prog.alloc(ctx, 2));
    auto launch = [&](unsigned grid, const CUtensorMap &mq_, const CUtensorMap &mx_,
                      const __nv_bfloat16 *qrows_, int64_t nq_, int64_t n_, const float *qn_,
                      const float *xn_, int K_, int self_, int32_t *oi, float *os,
                      const int32_t *perm_, int rot) -> pg_status {
        PG_TRY_CUDA(ctx, cudaMemsetAsync(prog.p, 0, 8, ctx->stream));
        // chunk minima of the candidates' norms, padded to whole tiles
        const int64_t nch = (n_ + TN - 1) / TN * (TN / 32);
        Scratch<float> cmin;
        PG_TRY(cmin.alloc(ctx, (size_t)nch));
        k_chunk_min<<<(unsigned)((nch + 255) / 256), 256, 0, ctx->stream>>>(xn_, n_, nch, cmin.p);
        PG_LAUNCHED(ctx);
        const int res = ctx->num_sms;  // one CTA per SM (shared memory)
        if (V.KB)
            k_knn_tc<1, true, 1><<<grid, tc_threads(1), smem, ctx->stream>>>(
                mq_, mx_, qrows_, nq_, n_, dp, qn_, xn_, cmin.p, K_, self_, oi, os, ctx->d_err, perm_, rot,
                prog.p, res);
        else if (V.QT == 2)
            k_knn_tc<1, false, 2><<<grid, tc_threads(1, 2), smem, ctx->stream>>>(
                mq_, mx_, qrows_, nq_, n_, dp, qn_, xn_, cmin.p, K_, self_, oi, os, ctx->d_err, perm_, rot,
                prog.p, res);
        else if (V.H == 2)
            k_knn_tc<2, false, 1><<<grid, tc_threads(2), smem, ctx->stream>>>(
                mq_, mx_, qrows_, nq_, n_, dp, qn_, xn_, cmin.p, K_, self_, oi, os, ctx->d_err, perm_, rot,
                prog.p, res);
        else
            k_knn_tc<1, false, 1><<<grid, tc_threads(1), smem, ctx->stream>>>(
                mq_, mx_, qrows_, nq_, n_, dp, qn_, xn_, cmin.p, K_, self_, oi, os, ctx->d_err, perm_, rot,
                prog.p, res);
        return PG_OK;
    };
    const int32_t *permp = nullptr;
    const __nv_bfloat16 *xp = xc.p;
    const float *xnp = xnorm, *qnp = qnorm;
    if (self && n >= 16384) {
        // ---- spatial order: nearest pivot, then a counting sort by pivot
        const int P = (int)std::min<int64_t>(4096, std::max<int64_t>(64, n / 1024));
        PG_TRY(pid.alloc(ctx, (size_t)P));
        PG_TRY(pb.alloc(ctx, (size_t)P * dp));
        PG_TRY(pn.alloc(ctx, (size_t)P));
        PG_TRY(asg.alloc(ctx, (size_t)n));
        PG_TRY(adist.alloc(ctx, (size_t)n));
        k_pivot_ids<<<(P + 255) / 256, 256, 0, ctx->stream>>>(pid.p, P, n);
        PG_LAUNCHED(ctx);
        k_gather_bf16<<<(unsigned)(((int64_t)P * dp / 8 + 255) / 256), 256, 0, ctx->stream>>>(
            xc.p, pid.p, P, dp, pb.p);
        PG_LAUNCHED(ctx);
        k_gather_f32<<<(P + 255) / 256, 256, 0, ctx->stream>>>(xnorm, pid.p, P, pn.p);
        PG_LAUNCHED(ctx);
        CUtensorMap mqa, mpa;
        PG_TRY(make_map(ctx, &mqa, qp, n, dp));
        PG_TRY(make_map(ctx, &mpa, pb.p, P, dp));
        PG_TRY(launch((unsigned)((n + rows_per_cta - 1) / rows_per_cta), mqa, mpa, qp, n, P, xnorm,
                      pn.p, 1, 0, asg.p, adist.p, nullptr, 0));
        PG_LAUNCHED(ctx);
        PG_TRY(cnt.alloc(ctx, (size_t)P));
        PG_TRY(boff.alloc(ctx, (size_t)P + 1));
        PG_TRY(perm.alloc(ctx, (size_t)n));
        PG_TRY_CUDA(ctx, cudaMemsetAsync(cnt.p, 0, (size_t)P * 4, ctx->stream));
        const unsigned gn = (unsigned)((n + 255) / 256);
        k_bucket_count<<<gn, 256, 0, ctx->stream>>>(asg.p, n, cnt.p);
        PG_LAUNCHED(ctx);
        PG_TRY(pg_scan_counts(ctx, cnt.p, P, boff.p));
        k_bucket_scatter<<<gn, 256, 0, ctx->stream>>>(
            asg.p, n, reinterpret_cast<unsigned long long *>(boff.p), perm.p);
        PG_LAUNCHED(ctx);
        PG_TRY(xs.alloc(ctx, (size_t)(n * dp)));
        PG_TRY(xsn.alloc(ctx, (size_t)n));
        k_gather_bf16<<<(unsigned)((n * dp / 8 + 255) / 256), 256, 0, ctx->stream>>>(
            xc.p, perm.p, n, dp, xs.p);
        PG_LAUNCHED(ctx);
        k_gather_f32<<<gn, 256, 0, ctx->stream>>>(xnorm, perm.p, n, xsn.p);
        PG_LAUNCHED(ctx);
        xc.release();
        permp = perm.p;
        xp = xs.p;
        qp = xs.p;
        if (xq_sep) {
            PG_TRY(xqs.alloc(ctx, (size_t)(n * dp)));
            k_gather_bf16<<<(unsigned)((n * dp / 8 + 255) / 256), 256, 0, ctx->stream>>>(
                xq_sep->p, perm.p, n, dp, xqs.p);
            PG_LAUNCHED(ctx);
            xq_sep->release();
            qp = xqs.p;
        }
        xnp = xsn.p;
        qnp = xsn.p;
    }
    CUtensorMap mq, mx;
    PG_TRY(make_map(ctx, &mx, xp, n, dp));
    PG_TRY(make_map(ctx, &mq, qp, self ? n : nq, dp));
    const unsigned grid = (unsigned)((nq + rows_per_cta - 1) / rows_per_cta);
    pg_timer_begin(ctx, TM_KNN);
    PG_TRY(launch(grid, mq, mx, qp, nq, n, qnp, xnp, K, self, ids, dist, permp, permp ? 1 : 0));
    PG_LAUNCHED(ctx);
    pg_timer_end(ctx, TM_KNN, work);
    return PG_OK;
}

// Exact kNN of Q (or of D itself when self) on the tensor cores; the caller
// guarantees BF16-exact integer data.  xnorm/qnorm are FP32 squared norms.
// For the graph (self) the points are first ordered by their nearest of
// ~n/1024 pivots (a kNN with K = 1 on the same kernel), so that every CTA
// meets its rows' neighbours in its first tiles; lists hold original ids and
// rows are written back in original order, so the result does not depend
// on the order.
pg_status pg_knn_tc(pg_ctx *ctx, const float *D, int64_t n, int32_t d, const float *Q, int64_t nq,
                    int self, int32_t K, const float *xnorm, const float *qnorm, int32_t *ids,
                    float *dist) {
    const int dp = (d + 63) / 64 * 64;
    Scratch<__nv_bfloat16> xb, qb;
    PG_TRY(xb.alloc(ctx, (size_t)(n * dp)));
    k_to_bf16<<<(unsigned)((n * dp + 255) / 256), 256, 0, ctx->stream>>>(D, n, d, dp, xb.p);
    PG_LAUNCHED(ctx);
    if (!self) {
        PG_TRY(qb.alloc(ctx, (size_t)(nq * dp)));
        k_to_bf16<<<(unsigned)((nq * dp + 255) / 256), 256, 0, ctx->stream>>>(Q, nq, d, dp, qb.p);
        PG_LAUNCHED(ctx);
    }
    return tc_knn_run(ctx, xb, nullptr, qb.p, n, nq, dp, self, K, xnorm, qnorm, ids, dist,
                      2.0 * (double)nq * (double)n * (double)d);
}

// Self kNN on the hi/lo split copies of the screened form: xq rows
// [hi | hi | lo] and xc rows [hi | lo | hi] (dp3 columns), so that one
// contraction gives hi.hi + hi.lo + lo.hi; norms are the rows' FP32 squared
// norms (1 for the chord).  work: the algorithmic flops to report.
pg_status pg_knn_tc_split(pg_ctx *ctx, Scratch<__nv_bfloat16> &xc, Scratch<__nv_bfloat16> &xq,
                          int64_t n, int dp3, const float *norms, int32_t K, int32_t *ids,
                          float *dist, double work) {
    return tc_knn_run(ctx, xc, &xq, nullptr, n, n, dp3, 1, K, norms, norms, ids, dist, work);
}

// ------------------------------------------------ split-column argmin (host)
bool pg_tc_argmin_supported(int d) {
    const int dp = (d + 63) / 64 * 64;
    return dp <= 256 && arg_layout(dp).total + 1024 <= 227 * 1024;
}

pg_status pg_tc_argmin_init(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                            const int32_t *deg, int R, TcArgmin &t) {
    t.d = d;
    t.dp = (d + 63) / 64 * 64;
    // the points with a free slot, in ascending id order (flags, scan, scatter)
    Scratch<int32_t> flag;
    Scratch<int64_t> off;
    PG_TRY(flag.alloc(ctx, (size_t)n));
    PG_TRY(off.alloc(ctx, (size_t)n + 1));
    k_free_flags<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(deg, n, R, flag.p);
    PG_LAUNCHED(ctx);
    PG_TRY(pg_scan_counts(ctx, flag.p, n, off.p));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, off.p + n, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PG_TRY(pg_sync_check(ctx, "argmin candidates"));
    int64_t m = 0;
    memcpy(&m, ctx->h_pinned, sizeof m);
    t.n = m;
    const int64_t ma = std::max<int64_t>(m, 1);  // a tensor map needs a row
    PG_TRY(t.cid.alloc(ctx, (size_t)ma));
    PG_TRY(t.xb.alloc(ctx, (size_t)(ma * t.dp)));
    PG_TRY(t.xn.alloc(ctx, (size_t)ma));
    PG_TRY(t.qb.alloc(ctx, (size_t)TM * t.dp));
    PG_TRY(t.qn.alloc(ctx, (size_t)TM));
    if (m == 0) PG_TRY_CUDA(ctx, cudaMemsetAsync(t.xb.p, 0, (size_t)t.dp * 2, ctx->stream));
    k_free_scatter<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(flag.p, off.p, n, t.cid.p);
    PG_LAUNCHED(ctx);
    if (m > 0) {
        k_gather_bf16_rows<<<(unsigned)((m + 7) / 8), 256, 0, ctx->stream>>>(D, d, t.dp, t.cid.p, m,
                                                                             t.xb.p, t.xn.p);
        PG_LAUNCHED(ctx);
    }
    static_assert(sizeof(t.mapx) >= sizeof(CUtensorMap), "tensor map storage");
    PG_TRY(make_map(ctx, reinterpret_cast<CUtensorMap *>(t.mapx), t.xb.p, ma, t.dp));
    PG_TRY(make_map(ctx, reinterpret_cast<CUtensorMap *>(t.mapq), t.qb.p, TM, t.dp));
    const size_t smem = arg_layout(t.dp).total + 1024;
    PG_TRY_CUDA(ctx, cudaFuncSetAttribute(k_argmin_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    return PG_OK;
}

pg_status pg_tc_argmin(pg_ctx *ctx, TcArgmin &t, const float *D, const int *ids, const int *count,
                       const int *reached, const int32_t *deg, int R, unsigned long long *best) {
    k_tc_gather_rows<<<TM / 8, 256, 0, ctx->stream>>>(D, t.d, t.dp, ids, count, t.qb.p, t.qn.p);
    PG_LAUNCHED(ctx);
    const int ntiles = (int)((t.n + TN - 1) / TN);
    const int grid = std::max(1, std::min(ctx->num_sms, ntiles));
    const int per = (ntiles + grid - 1) / grid;
    const size_t smem = arg_layout(t.dp).total + 1024;
    k_argmin_tc<<<(unsigned)grid, NTHREADS, smem, ctx->stream>>>(
        *reinterpret_cast<const CUtensorMap *>(t.mapq), *reinterpret_cast<const CUtensorMap *>(t.mapx),
        count, t.n, t.dp, t.qn.p, t.xn.p, t.cid.p, reached, deg, R, per, best, ctx->d_err);
    PG_LAUNCHED(ctx);
    return PG_OK;
}
