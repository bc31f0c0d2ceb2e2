// noalloc.cu -- alpha-pruning for callers that cannot allocate device
// memory.
//
// Some callers may not call cudaMalloc (or anything that allocates) at the
// point where they prune: allocators and runtimes that own every device
// allocation themselves, or processes that must keep their footprint fixed
// after start-up.  pg_prune_noalloc does the same work as pg_prune but takes
// all of its scratch from one file-scope device array of fixed size, so it
// allocates nothing at all: no device memory, no host heap, no library
// context.  The call is synchronous: it waits on the caller's stream twice
// (for the data facts and for the device error word) and copies both to
// host stack buffers, so it may not be made on a stream that is being
// captured into a CUDA graph.
#include <climits>
#include <cstring>
#include <mutex>

#include "pg_internal.cuh"

__global__ void k_data_facts(const float *__restrict__ D, int64_t n, int d, float *blk_out);
cudaError_t pg_prune_launch_on(cudaStream_t stream, int num_sms, const float *D, int64_t n,
                               int32_t d, pg_metric metric, const int64_t *off,
                               const int32_t *cand, int32_t R, double alpha_deg,
                               const DataFacts &facts, int32_t *nbr, int32_t *deg, int *ints,
                               int *err, unsigned long long *counters);

namespace {

constexpr int64_t MAX_N = PG_PRUNE_NOALLOC_MAX_N;
constexpr int FACT_BLOCKS = 2048;  // >= 4 blocks per SM on any current GPU
constexpr size_t OFF_INTS = 0;
constexpr size_t OFF_FACTS = OFF_INTS + (size_t)(MAX_N + 4) * 4;
constexpr size_t OFF_ERR = OFF_FACTS + (size_t)FACT_BLOCKS * 4 * 4;
constexpr size_t OFF_CNT = OFF_ERR + 64;
constexpr size_t SCRATCH_BYTES = OFF_CNT + PG_CNT_SLOTS * 8;

// The one scratch area of this entry point; every GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_prune_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
unsigned char *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  Host code
// cannot use the array's name as a device address; the address is looked
// up once per device, with that device current.
cudaError_t scratch_for(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_prune_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

pg_status from_cuda(cudaError_t e) {
    return e == cudaSuccess ? PG_OK : (e == cudaErrorMemoryAllocation ? PG_ERR_OOM : PG_ERR_CUDA);
}

}  // namespace

extern "C" pg_status pg_prune_noalloc(void *cuda_stream, const float *D, int64_t n, int32_t d,
                                      pg_metric metric, const int64_t *cand_off,
                                      const int32_t *cand_ids, int32_t R, double alpha_deg,
                                      int32_t *nbr, int32_t *deg) {
    if (!D || !cand_off || !cand_ids || !nbr || !deg) return PG_ERR_INVALID_ARG;
    if (n < 1 || d < 4 || d % 4 || d > 8192 || R < 1 || R > 64) return PG_ERR_INVALID_ARG;
    if (!(alpha_deg >= 0.0 && alpha_deg <= 180.0)) return PG_ERR_INVALID_ARG;
    if (metric < PG_METRIC_L2SQ || metric > PG_METRIC_IP) return PG_ERR_INVALID_ARG;
    if (n > MAX_N) return PG_ERR_CAPACITY;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= MAX_DEVICES)) return PG_ERR_CAPACITY;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned char *base = nullptr;
    if (e == cudaSuccess) e = scratch_for(dev, &base);
    if (e != cudaSuccess) return from_cuda(e);
    int *ints = reinterpret_cast<int *>(base + OFF_INTS);
    float *facts_blk = reinterpret_cast<float *>(base + OFF_FACTS);
    int *err = reinterpret_cast<int *>(base + OFF_ERR);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(base + OFF_CNT);
    // the area keeps the previous call's contents: clear what must start at 0
    e = cudaMemsetAsync(err, 0, 4 * sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, PG_CNT_SLOTS * 8, stream);
    if (e != cudaSuccess) return from_cuda(e);

    // arithmetic facts of D (same rules as every other entry point)
    const int blocks = sms * 4 < FACT_BLOCKS ? sms * 4 : FACT_BLOCKS;
    k_data_facts<<<blocks, 256, 0, stream>>>(D, n, d, facts_blk);
    e = cudaGetLastError();
    float h[FACT_BLOCKS * 4];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, facts_blk, (size_t)blocks * 4 * sizeof(float),
                            cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return from_cuda(e);
    const DataFacts f = pg_reduce_facts(h, blocks, n, d, metric);

    e = pg_prune_launch_on(stream, sms, D, n, d, metric, cand_off, cand_ids, R, alpha_deg, f, nbr,
                           deg, ints, err, cnt);
    int herr[4] = {0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return from_cuda(e);
    switch (herr[0]) {
    case DERR_NONE: return PG_OK;
    case DERR_BAD_ID: return PG_ERR_DEVICE_CHECK;
    case DERR_CAPACITY: return PG_ERR_CAPACITY;
    case DERR_TIMEOUT: return PG_ERR_TIMEOUT;
    default: return PG_ERR_INTERNAL;
    }
}
