// tune.cu -- the launch-configuration autotuner of the persistent kernels.
//
// The pruning and beam-search kernels fetch rows / queries from an atomic
// counter, so any grid gives the same result; what changes with the
// configuration is the speed: CTAs per SM (occupancy) for both, and the
// size of the search's visited table (shared memory per warp against
// re-evaluations of forgotten nodes).  With tuning on (pg_ctx_set_autotune),
// the first call for a key (kernel, width, degree or pool, row form) on a
// device times every candidate on that call's own input with CUDA events
// and keeps the fastest; later calls with the key take it from this
// process-wide table.  pg_autotune_report lists the table.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "pg_internal.cuh"

namespace {

struct Entry {
    int config = -1;
    std::vector<std::pair<int, float>> tried;  // (config, ms)
    std::string label;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int, int, int>, Entry> g_table;

}  // namespace

bool pg_tune_lookup(const TuneKey &k, int *config) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(std::make_tuple(k.device, k.kernel, k.d, k.p, k.form));
    if (it == g_table.end() || it->second.config < 0) return false;
    *config = it->second.config;
    return true;
}

void pg_tune_store(const TuneKey &k, int config, const std::vector<std::pair<int, float>> &tried,
                   const char *label) {
    std::lock_guard<std::mutex> lk(g_mu);
    Entry &e = g_table[std::make_tuple(k.device, k.kernel, k.d, k.p, k.form)];
    e.config = config;
    e.tried = tried;
    e.label = label;
}

pg_status pg_tune_time(pg_ctx *ctx, const std::vector<int> &configs,
                       const std::function<pg_status(int)> &run, int *best,
                       std::vector<std::pair<int, float>> *tried) {
    cudaEvent_t a, b;
    PG_TRY_CUDA(ctx, cudaEventCreate(&a));
    PG_TRY_CUDA(ctx, cudaEventCreate(&b));
    float best_ms = 0.f;
    *best = configs.front();
    pg_status st = PG_OK;
    for (int c : configs) {
        cudaEventRecord(a, ctx->stream);
        st = run(c);
        if (st != PG_OK) break;
        cudaEventRecord(b, ctx->stream);
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) {
            st = pg_cuda_fail(ctx, e, "autotune timing");
            break;
        }
        tried->push_back({c, ms});
        if (tried->size() == 1 || ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

extern "C" pg_status pg_ctx_set_autotune(pg_ctx *ctx, int enable) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    ctx->autotune = enable ? 1 : 0;
    return PG_OK;
}

extern "C" int64_t pg_autotune_report(char *buf, int64_t cap) {
    std::string out;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const auto &kv : g_table) {
            const Entry &e = kv.second;
            char line[256];
            snprintf(line, sizeof line, "%s -> %d (", e.label.c_str(), e.config);
            out += line;
            for (size_t i = 0; i < e.tried.size(); ++i) {
                snprintf(line, sizeof line, "%s%d:%.3f", i ? " " : "", e.tried[i].first,
                         e.tried[i].second);
                out += line;
            }
            out += " ms)\n";
        }
    }
    if (buf && cap > 0) {
        const size_t m = std::min<size_t>(out.size(), (size_t)cap - 1);
        memcpy(buf, out.data(), m);
        buf[m] = 0;
    }
    return (int64_t)out.size() + 1;
}
