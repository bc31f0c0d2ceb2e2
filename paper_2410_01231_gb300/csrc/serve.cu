// serve.cu -- serving loop over a growable index: a request queue of query
// batches and insertion batches drained by one host worker thread that owns
// the context and the index while the server runs.
//
// Requests run in submission order, so completion is monotone: ticket t is
// done once the worker has finished every request up to t.  Consecutive
// query requests with the same (k, beam, upper_beam) are merged into one
// search launch of up to max_batch queries (continuous batching); an
// insertion batch (Algorithm 4 on a snapshot, pg_index_insert) runs alone,
// after every earlier query and before every later one, so a query always
// sees exactly the points inserted before it was submitted.
//
// While the server runs, the context belongs to the worker thread: the
// submit functions, called from other threads, only validate and enqueue;
// a refused submission returns its status without touching the context's
// error message (which the worker may be writing).
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "pg_internal.cuh"

namespace {

struct Req {
    int64_t ticket = 0;
    int kind = 0;  // 0 query, 1 insert
    const float *host = nullptr;
    int64_t rows = 0;
    int k = 0, beam = 0, upper_beam = 1, ef = 0;
    int32_t *out_ids = nullptr;
    float *out_dist = nullptr;
};

}  // namespace

struct pg_server {
    pg_ctx *ctx = nullptr;
    pg_index *index = nullptr;
    int device = 0;
    int d = 0;
    int max_batch = 1024;
    int64_t queue_limit = 0;  // pending requests admitted at most (0: no limit)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> queue;
    bool stopping = false;
    int64_t next_ticket = 1;
    int64_t last_done = 0;
    std::unordered_map<int64_t, int> failed;  // ticket -> status
    int64_t n_batches = 0, n_requests = 0, n_queries = 0, n_inserted = 0;
    std::thread worker;
};

namespace {

pg_status run_queries(pg_server *s, const std::vector<Req> &batch) {
    pg_ctx *ctx = s->ctx;
    int64_t total = 0;
    for (const Req &r : batch) total += r.rows;
    const int k = batch[0].k, d = s->d;
    Scratch<float> Q, dist;
    Scratch<int32_t> ids;
    PG_TRY(Q.alloc(ctx, (size_t)(total * d)));
    PG_TRY(ids.alloc(ctx, (size_t)(total * k)));
    PG_TRY(dist.alloc(ctx, (size_t)(total * k)));
    int64_t at = 0;
    for (const Req &r : batch) {
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(Q.p + at * d, r.host, (size_t)(r.rows * d) * 4,
                                         cudaMemcpyHostToDevice, ctx->stream));
        at += r.rows;
    }
    PG_TRY(pg_search(ctx, s->index, Q.p, total, k, batch[0].beam, batch[0].upper_beam, 0,
                     PG_PREC_FP32, ids.p, dist.p));
    at = 0;
    for (const Req &r : batch) {
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(r.out_ids, ids.p + at * k, (size_t)(r.rows * k) * 4,
                                         cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(r.out_dist, dist.p + at * k, (size_t)(r.rows * k) * 4,
                                         cudaMemcpyDeviceToHost, ctx->stream));
        at += r.rows;
    }
    return pg_sync_check(ctx, "serve query");
}

pg_status run_insert(pg_server *s, const Req &r) {
    pg_ctx *ctx = s->ctx;
    Scratch<float> X;
    PG_TRY(X.alloc(ctx, (size_t)(r.rows * s->d)));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(X.p, r.host, (size_t)(r.rows * s->d) * 4,
                                     cudaMemcpyHostToDevice, ctx->stream));
    return pg_index_insert(ctx, s->index, X.p, r.rows, r.ef, r.upper_beam);
}

bool same_query_shape(const Req &a, const Req &b) {
    return a.kind == 0 && b.kind == 0 && a.k == b.k && a.beam == b.beam &&
           a.upper_beam == b.upper_beam;
}

void worker_main(pg_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Req> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [s] { return s->stopping || !s->queue.empty(); });
            if (s->queue.empty()) break;  // stopping and drained
            batch.push_back(s->queue.front());
            s->queue.pop_front();
            if (batch[0].kind == 0) {
                int64_t total = batch[0].rows;
                while (!s->queue.empty() && same_query_shape(batch[0], s->queue.front()) &&
                       total + s->queue.front().rows <= s->max_batch) {
                    total += s->queue.front().rows;
                    batch.push_back(s->queue.front());
                    s->queue.pop_front();
                }
            }
        }
        const pg_status st = batch[0].kind == 0 ? run_queries(s, batch) : run_insert(s, batch[0]);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->last_done = batch.back().ticket;
            if (st != PG_OK)
                for (const Req &r : batch) s->failed[r.ticket] = (int)st;
            s->n_batches += 1;
            s->n_requests += (int64_t)batch.size();
            for (const Req &r : batch) (r.kind == 0 ? s->n_queries : s->n_inserted) += r.rows;
        }
        s->cv_done.notify_all();
    }
}

pg_status submit(pg_server *s, Req r, int64_t *ticket) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return PG_ERR_INVALID_ARG;  // the server is stopping
        if (s->queue_limit > 0 && s->next_ticket - 1 - s->last_done >= s->queue_limit)
            return PG_ERR_CAPACITY;  // admission refused: the queue is full
        r.ticket = s->next_ticket++;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r.ticket;
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_serve_start(pg_ctx *ctx, pg_index *index, int32_t max_batch,
                                    pg_server **out) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!index || !out) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (max_batch < 1 || max_batch > 65536)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= max_batch <= 65536");
    pg_server *s = new (std::nothrow) pg_server();
    if (!s) return pg_fail(ctx, PG_ERR_OOM, "host allocation");
    s->ctx = ctx;
    s->index = index;
    s->device = ctx->device;
    s->d = pg_index_dim(index);
    s->max_batch = max_batch;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PG_OK;
}

extern "C" pg_status pg_serve_submit_query(pg_server *s, const float *Q, int64_t nq, int32_t k,
                                           int32_t beam, int32_t upper_beam, int32_t *out_ids,
                                           float *out_dist, int64_t *ticket) {
    if (!s) return PG_ERR_INVALID_ARG;
    if (!Q || !out_ids || !out_dist || !ticket) return PG_ERR_INVALID_ARG;
    if (nq < 1 || k < 1 || beam < k || beam > 256 || upper_beam < 1 || upper_beam > 256)
        return PG_ERR_INVALID_ARG;
    Req r;
    r.kind = 0;
    r.host = Q;
    r.rows = nq;
    r.k = k;
    r.beam = beam;
    r.upper_beam = upper_beam;
    r.out_ids = out_ids;
    r.out_dist = out_dist;
    return submit(s, r, ticket);
}

extern "C" pg_status pg_serve_submit_insert(pg_server *s, const float *X, int64_t m, int32_t ef,
                                            int32_t upper_beam, int64_t *ticket) {
    if (!s) return PG_ERR_INVALID_ARG;
    if (!X || !ticket) return PG_ERR_INVALID_ARG;
    if (m < 1 || ef < 1 || ef > 256 || upper_beam < 1 || upper_beam > 256)
        return PG_ERR_INVALID_ARG;
    Req r;
    r.kind = 1;
    r.host = X;
    r.rows = m;
    r.ef = ef;
    r.upper_beam = upper_beam;
    return submit(s, r, ticket);
}

extern "C" pg_status pg_serve_wait(pg_server *s, int64_t ticket, double timeout_s,
                                   int32_t *done) {
    if (!s || !done) return PG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [s, ticket] { return s->last_done >= ticket; };
    if (timeout_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    *done = ready() ? 1 : 0;
    if (!*done) return PG_OK;
    auto it = s->failed.find(ticket);
    return it == s->failed.end() ? PG_OK : (pg_status)it->second;
}

extern "C" pg_status pg_serve_set_queue_limit(pg_server *s, int64_t limit) {
    if (!s || limit < 0) return PG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->queue_limit = limit;
    return PG_OK;
}

extern "C" pg_status pg_serve_stats(pg_server *s, int64_t *host_stats4) {
    if (!s || !host_stats4) return PG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    host_stats4[0] = s->n_batches;
    host_stats4[1] = s->n_requests;
    host_stats4[2] = s->n_queries;
    host_stats4[3] = s->n_inserted;
    return PG_OK;
}

extern "C" pg_status pg_serve_stop(pg_server *s) {
    if (!s) return PG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return PG_OK;
}
