// serve.cu -- serving loop over a growable index: a request queue of query
// batches and insertion batches, a dispatcher thread and `slots` worker
// threads, each worker with its own context (own CUDA stream, scratch and
// error word), so that query launches of different requests overlap on the
// device.
//
// Dispatch is in submission order.  Consecutive query requests with the
// same (k, beam, upper_beam, precision) are merged into one group of at most max_batch
// queries (continuous batching); a group is admitted to a worker once a
// worker is free and the device scratch of the groups in flight plus its
// own fits the HBM budget of the server's context (a group that could never
// fit fails with PG_ERR_BUDGET).  An insertion batch (Algorithm 4 on a
// snapshot, pg_index_insert) takes a free worker beside the query groups in
// flight: it builds the next version of the index in copies of the layer
// arrays while those groups keep searching the version they started on
// (epoch snapshots), publishes it when it ends, and nothing submitted after
// it is dispatched before then: a query sees exactly the points inserted
// before it was submitted, however the work overlaps.  Tickets complete out
// of order; pg_serve_wait waits for one ticket.
//
// The scheduler below is host-only and takes its work as callbacks, so the
// same code runs with simulated work on a machine without a GPU
// (pg_serve_simulate).  While the server runs, the context and the index
// belong to it: the submit functions, called from other threads, only
// validate and enqueue; a refused submission returns its status without
// touching the context's error message (which the dispatcher may be
// writing).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <set>
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
    pg_precision precision = PG_PREC_FP32;  // queries: distance form of the search
    int32_t *out_ids = nullptr;
    float *out_dist = nullptr;
    int64_t shape = 0;  // simulated requests: merge key
    std::chrono::steady_clock::time_point submitted;
};

struct Group {
    std::vector<Req> reqs;
    int64_t rows = 0;
    size_t bytes = 0;
    bool insert = false;
    std::shared_ptr<void> pinned;  // the index version a query group searches
};

enum { SLOT_IDLE = 0, SLOT_ASSIGNED, SLOT_RUNNING };

struct Sched {
    // configuration and work
    int nslots = 1;
    int64_t max_batch = 1024;
    size_t budget = 0;  // bytes of device scratch in flight at most (0: no limit)
    std::function<bool(const Req &, const Req &)> mergeable;
    std::function<size_t(const Group &)> group_bytes;
    std::function<pg_status(int, const Group &)> run_group;
    std::function<pg_status(int, const Req &)> run_insert;
    // pins the current version of the index for a query group being
    // dispatched (with mu held): the group searches it wherever its worker
    // starts, so it sees exactly the insertions submitted before it
    std::function<std::shared_ptr<void>()> pin;

    // state, under mu
    std::mutex mu;
    std::condition_variable cv_work, cv_free, cv_slot, cv_done;
    std::deque<Req> queue;
    bool stopping = false, slots_exit = false;
    int64_t next_ticket = 1, completed = 0, queue_limit = 0;
    pg_precision precision = PG_PREC_FP32;  // taken by query requests when submitted
    int64_t done_below = 1;          // every ticket below it is done
    std::set<int64_t> done_above;    // done tickets at or above done_below
    std::unordered_map<int64_t, int> failed;  // ticket -> status
    std::vector<int> slot_state;
    std::vector<Group> slot_job;
    int busy = 0;
    bool insert_running = false;  // an insertion is on a worker: nothing after it starts
    size_t bytes_in_flight = 0;
    int64_t n_groups = 0, n_requests = 0, n_queries = 0, n_inserted = 0, max_in_flight = 0,
            admission_waits = 0;
    // seconds from submission to completion of the last kLatRing tickets
    static constexpr int64_t kLatRing = int64_t(1) << 16;
    std::vector<double> latency = std::vector<double>((size_t)kLatRing, 0.0);
    std::thread dispatcher;
    std::vector<std::thread> workers;
    std::function<void()> thread_init;  // run first on every thread (device binding)

    bool is_done(int64_t t) const { return t < done_below || done_above.count(t) != 0; }

    // with mu held
    void complete(const std::vector<Req> &reqs, pg_status st) {
        const auto now = std::chrono::steady_clock::now();
        for (const Req &r : reqs) {
            latency[(size_t)(r.ticket % kLatRing)] =
                std::chrono::duration<double>(now - r.submitted).count();
            if (st != PG_OK) failed[r.ticket] = (int)st;
            done_above.insert(r.ticket);
            ++completed;
            ++n_requests;
            (r.kind == 0 ? n_queries : n_inserted) += r.rows;
        }
        ++n_groups;
        while (!done_above.empty() && *done_above.begin() == done_below) {
            done_above.erase(done_above.begin());
            ++done_below;
        }
        cv_done.notify_all();
    }

    void worker_main(int s) {
        if (thread_init) thread_init();
        for (;;) {
            Group g;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_slot.wait(lk, [&] {
                    return slots_exit || slot_state[(size_t)s] == SLOT_ASSIGNED;
                });
                if (slot_state[(size_t)s] != SLOT_ASSIGNED) return;  // exit with nothing assigned
                slot_state[(size_t)s] = SLOT_RUNNING;
                g = std::move(slot_job[(size_t)s]);
            }
            const pg_status st = g.insert ? run_insert(s, g.reqs[0]) : run_group(s, g);
            g.pinned.reset();
            {
                std::lock_guard<std::mutex> lk(mu);
                complete(g.reqs, st);
                slot_state[(size_t)s] = SLOT_IDLE;
                --busy;
                bytes_in_flight -= g.bytes;
                if (g.insert) insert_running = false;
            }
            cv_free.notify_all();
        }
    }

    void dispatcher_main() {
        if (thread_init) thread_init();
        for (;;) {
            Group g;
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
            if (queue.empty()) break;  // stopping and drained
            // A group is formed only once it can start (a free worker), so
            // requests that arrive while the workers are busy join it:
            // batching follows the load.
            const bool insertion = queue.front().kind == 1;
            auto can_start = [&] { return busy < nslots; };
            if (!can_start()) {
                ++admission_waits;
                cv_free.wait(lk, can_start);
            }
            g.reqs.push_back(queue.front());
            g.rows = queue.front().rows;
            queue.pop_front();
            if (insertion) {
                // The insertion runs on a worker beside the query groups in
                // flight, which search the version of the index they started
                // on; it publishes the next version when it ends, and
                // nothing submitted after it is dispatched before then.
                g.insert = true;
                int s = 0;
                while (slot_state[(size_t)s] != SLOT_IDLE) ++s;
                slot_state[(size_t)s] = SLOT_ASSIGNED;
                slot_job[(size_t)s] = std::move(g);
                ++busy;
                max_in_flight = std::max<int64_t>(max_in_flight, busy);
                insert_running = true;
                cv_slot.notify_all();
                cv_free.wait(lk, [&] { return !insert_running; });
                continue;
            }
            while (!queue.empty() && mergeable(g.reqs[0], queue.front()) &&
                   g.rows + queue.front().rows <= max_batch) {
                g.rows += queue.front().rows;
                g.reqs.push_back(queue.front());
                queue.pop_front();
            }
            g.bytes = group_bytes(g);
            if (budget && g.bytes > budget) {
                complete(g.reqs, PG_ERR_BUDGET);
                continue;
            }
            auto fits = [&] { return !budget || bytes_in_flight + g.bytes <= budget; };
            if (!fits()) {
                ++admission_waits;
                cv_free.wait(lk, fits);
            }
            if (pin) g.pinned = pin();
            int s = 0;
            while (slot_state[(size_t)s] != SLOT_IDLE) ++s;
            slot_state[(size_t)s] = SLOT_ASSIGNED;
            bytes_in_flight += g.bytes;
            slot_job[(size_t)s] = std::move(g);
            ++busy;
            max_in_flight = std::max<int64_t>(max_in_flight, busy);
            cv_slot.notify_all();
        }
        std::unique_lock<std::mutex> lk(mu);
        cv_free.wait(lk, [&] { return busy == 0; });
        slots_exit = true;
        cv_slot.notify_all();
    }

    // false if a thread could not be started (the others are joined again)
    bool start() {
        slot_state.assign((size_t)nslots, SLOT_IDLE);
        slot_job.resize((size_t)nslots);
        try {
            for (int s = 0; s < nslots; ++s) workers.emplace_back(&Sched::worker_main, this, s);
            dispatcher = std::thread(&Sched::dispatcher_main, this);
        } catch (const std::exception &) {
            {
                std::lock_guard<std::mutex> lk(mu);
                stopping = slots_exit = true;
            }
            cv_slot.notify_all();
            cv_work.notify_all();
            for (auto &t : workers)
                if (t.joinable()) t.join();
            if (dispatcher.joinable()) dispatcher.join();
            return false;
        }
        return true;
    }

    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stopping = true;
        }
        cv_work.notify_all();
        if (dispatcher.joinable()) dispatcher.join();
        for (auto &t : workers)
            if (t.joinable()) t.join();
    }

    pg_status submit(Req r, int64_t *ticket) {
        {
            std::lock_guard<std::mutex> lk(mu);
            if (stopping) return PG_ERR_INVALID_ARG;  // the server is stopping
            if (queue_limit > 0 && next_ticket - 1 - completed >= queue_limit)
                return PG_ERR_CAPACITY;  // admission refused: the queue is full
            r.ticket = next_ticket++;
            r.submitted = std::chrono::steady_clock::now();
            if (r.kind == 0) r.precision = precision;
            queue.push_back(r);
        }
        cv_work.notify_one();
        *ticket = r.ticket;
        return PG_OK;
    }

    // enqueue several requests at once (the dispatcher sees all of them)
    pg_status submit_all(std::vector<Req> &rs) {
        {
            std::lock_guard<std::mutex> lk(mu);
            if (stopping) return PG_ERR_INVALID_ARG;
            for (Req &r : rs) {
                r.ticket = next_ticket++;
                r.submitted = std::chrono::steady_clock::now();
                queue.push_back(r);
            }
        }
        cv_work.notify_one();
        return PG_OK;
    }

    pg_status wait(int64_t ticket, double timeout_s, int32_t *done) {
        std::unique_lock<std::mutex> lk(mu);
        if (ticket < 1 || ticket >= next_ticket) return PG_ERR_INVALID_ARG;
        auto ready = [&] { return is_done(ticket); };
        // at most a day per call: longer durations would overflow the clock
        if (timeout_s > 0)
            cv_done.wait_for(lk, std::chrono::duration<double>(std::min(timeout_s, 86400.0)),
                             ready);
        *done = ready() ? 1 : 0;
        if (!*done) return PG_OK;
        auto it = failed.find(ticket);
        return it == failed.end() ? PG_OK : (pg_status)it->second;
    }

    pg_status latency_of(int64_t ticket, double *seconds) {
        std::lock_guard<std::mutex> lk(mu);
        if (ticket < 1 || ticket >= next_ticket || ticket <= next_ticket - 1 - kLatRing ||
            !is_done(ticket))
            return PG_ERR_INVALID_ARG;
        *seconds = latency[(size_t)(ticket % kLatRing)];
        return PG_OK;
    }

    void stats(int64_t *out, int count) {
        std::lock_guard<std::mutex> lk(mu);
        const int64_t v[6] = {n_groups, n_requests, n_queries, n_inserted, max_in_flight,
                              admission_waits};
        for (int i = 0; i < count && i < 6; ++i) out[i] = v[i];
    }
};

}  // namespace

struct pg_server {
    pg_ctx *ctx = nullptr;
    pg_index *index = nullptr;
    int device = 0;
    int d = 0;
    std::vector<cudaStream_t> streams;
    std::vector<pg_ctx *> slot_ctx;
    Sched sched;
};

namespace {

size_t query_group_bytes(int d, const Group &g) {
    // queries, results and the search's own scratch (entry, next entry and
    // its distance per query)
    const int64_t k = g.reqs[0].k;
    return (size_t)g.rows * ((size_t)d * 4 + (size_t)k * 8 + 12);
}

pg_status run_queries(pg_ctx *ctx, int d, const Group &g) {
    const IndexSnap &sn = *static_cast<const IndexSnap *>(g.pinned.get());
    const int64_t total = g.rows;
    const int k = g.reqs[0].k;
    Scratch<float> Q, dist;
    Scratch<int32_t> ids;
    PG_TRY(Q.alloc(ctx, (size_t)(total * d)));
    PG_TRY(ids.alloc(ctx, (size_t)(total * k)));
    PG_TRY(dist.alloc(ctx, (size_t)(total * k)));
    int64_t at = 0;
    for (const Req &r : g.reqs) {
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(Q.p + at * d, r.host, (size_t)(r.rows * d) * 4,
                                         cudaMemcpyHostToDevice, ctx->stream));
        at += r.rows;
    }
    PG_TRY(pg_search_pinned(ctx, sn, Q.p, total, k, g.reqs[0].beam, g.reqs[0].upper_beam, 0,
                            g.reqs[0].precision, ids.p, dist.p));
    at = 0;
    for (const Req &r : g.reqs) {
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(r.out_ids, ids.p + at * k, (size_t)(r.rows * k) * 4,
                                         cudaMemcpyDeviceToHost, ctx->stream));
        PG_TRY_CUDA(ctx, cudaMemcpyAsync(r.out_dist, dist.p + at * k, (size_t)(r.rows * k) * 4,
                                         cudaMemcpyDeviceToHost, ctx->stream));
        at += r.rows;
    }
    return pg_sync_check(ctx, "serve query");
}

pg_status run_insert(pg_server *s, int slot, const Req &r) {
    pg_ctx *ctx = s->slot_ctx[(size_t)slot];
    Scratch<float> X;
    PG_TRY(X.alloc(ctx, (size_t)(r.rows * s->d)));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(X.p, r.host, (size_t)(r.rows * s->d) * 4,
                                     cudaMemcpyHostToDevice, ctx->stream));
    return pg_index_insert(ctx, s->index, X.p, r.rows, r.ef, r.upper_beam);
}

bool same_query_shape(const Req &a, const Req &b) {
    return a.kind == 0 && b.kind == 0 && a.k == b.k && a.beam == b.beam &&
           a.upper_beam == b.upper_beam && a.precision == b.precision;
}

void release_slots(pg_server *s) {
    for (pg_ctx *c : s->slot_ctx) pg_ctx_destroy(c);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    s->slot_ctx.clear();
    s->streams.clear();
}

}  // namespace

extern "C" pg_status pg_serve_start(pg_ctx *ctx, pg_index *index, int32_t max_batch,
                                    int32_t slots, pg_server **out) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!index || !out) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if (max_batch < 1 || max_batch > 65536)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= max_batch <= 65536");
    if (slots < 1 || slots > 16) return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 1 <= slots <= 16");
    pg_server *s = new (std::nothrow) pg_server();
    if (!s) return pg_fail(ctx, PG_ERR_OOM, "host allocation");
    s->ctx = ctx;
    s->index = index;
    s->device = ctx->device;
    s->d = pg_index_dim(index);
    // one context per worker, each on its own non-blocking stream, created
    // on the server's device (the caller's current device is restored)
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    pg_status st = PG_OK;
    for (int i = 0; i < slots && st == PG_OK; ++i) {
        cudaStream_t stream = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            st = pg_cuda_fail(ctx, e, "pg_serve_start stream");
            break;
        }
        s->streams.push_back(stream);
        pg_ctx *c = nullptr;
        st = pg_ctx_create(stream, 0, &c);
        if (st != PG_OK) {
            pg_fail(ctx, st, "pg_serve_start: worker context");
            break;
        }
        s->slot_ctx.push_back(c);
    }
    cudaSetDevice(prev);
    if (st != PG_OK) {
        release_slots(s);
        delete s;
        return st;
    }
    Sched &q = s->sched;
    q.nslots = slots;
    q.max_batch = max_batch;
    q.budget = ctx->budget;
    q.mergeable = same_query_shape;
    const int d = s->d;
    q.group_bytes = [d](const Group &g) { return query_group_bytes(d, g); };
    q.run_group = [s](int slot, const Group &g) {
        return run_queries(s->slot_ctx[(size_t)slot], s->d, g);
    };
    q.pin = [s]() -> std::shared_ptr<void> { return std::make_shared<IndexSnap>(s->index); };
    q.run_insert = [s](int slot, const Req &r) { return run_insert(s, slot, r); };
    const int dev = s->device;
    q.thread_init = [dev] { cudaSetDevice(dev); };
    if (!q.start()) {
        release_slots(s);
        delete s;
        return pg_fail(ctx, PG_ERR_INTERNAL, "pg_serve_start: cannot start the worker threads");
    }
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
    return s->sched.submit(r, ticket);
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
    return s->sched.submit(r, ticket);
}

extern "C" pg_status pg_serve_wait(pg_server *s, int64_t ticket, double timeout_s,
                                   int32_t *done) {
    if (!s || !done) return PG_ERR_INVALID_ARG;
    return s->sched.wait(ticket, timeout_s, done);
}

extern "C" pg_status pg_serve_latency(pg_server *s, int64_t ticket, double *seconds) {
    if (!s || !seconds) return PG_ERR_INVALID_ARG;
    return s->sched.latency_of(ticket, seconds);
}

extern "C" pg_status pg_serve_set_queue_limit(pg_server *s, int64_t limit) {
    if (!s || limit < 0) return PG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->sched.mu);
    s->sched.queue_limit = limit;
    return PG_OK;
}

extern "C" pg_status pg_serve_set_precision(pg_server *s, pg_precision precision) {
    if (!s) return PG_ERR_INVALID_ARG;
    if (precision != PG_PREC_FP32 && precision != PG_PREC_BF16_SCREEN &&
        precision != PG_PREC_FP8_SCREEN)
        return PG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->sched.mu);
    s->sched.precision = precision;
    return PG_OK;
}

extern "C" pg_status pg_serve_set_budget(pg_server *s, int64_t bytes) {
    if (!s || bytes < 0) return PG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->sched.mu);
        s->sched.budget = (size_t)bytes;
    }
    s->sched.cv_free.notify_all();
    return PG_OK;
}

extern "C" pg_status pg_serve_stats(pg_server *s, int64_t *host_stats, int32_t count) {
    if (!s || !host_stats || count < 0) return PG_ERR_INVALID_ARG;
    s->sched.stats(host_stats, count);
    return PG_OK;
}

extern "C" pg_status pg_serve_stop(pg_server *s) {
    if (!s) return PG_ERR_INVALID_ARG;
    s->sched.stop();
    release_slots(s);
    delete s;
    return PG_OK;
}

// ------------------------------------------------------------- simulation

extern "C" pg_status pg_serve_simulate(int32_t slots, int32_t max_batch, int64_t budget_bytes,
                                       int32_t count, const int32_t *kind, const int32_t *rows,
                                       const int32_t *shape, int32_t work_us,
                                       int64_t bytes_per_row, int64_t *start_seq,
                                       int64_t *end_seq, int32_t *slot_of, int64_t *group_of,
                                       int64_t *version_of, int64_t *host_stats6) {
    if (slots < 1 || slots > 16 || max_batch < 1 || budget_bytes < 0 || count < 0 ||
        work_us < 0 || work_us > 100000 || bytes_per_row < 0)
        return PG_ERR_INVALID_ARG;
    if (count && (!kind || !rows || !shape || !start_seq || !end_seq || !slot_of || !group_of))
        return PG_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i)
        if ((kind[i] != 0 && kind[i] != 1) || rows[i] < 1) return PG_ERR_INVALID_ARG;
    std::atomic<int64_t> seq{0}, group_id{0}, version{0};
    Sched q;
    q.nslots = slots;
    q.max_batch = max_batch;
    q.budget = (size_t)budget_bytes;
    q.mergeable = [](const Req &a, const Req &b) {
        return a.kind == 0 && b.kind == 0 && a.shape == b.shape;
    };
    q.group_bytes = [bytes_per_row](const Group &g) { return (size_t)(g.rows * bytes_per_row); };
    // an insertion publishes version + 1 when it ends; a query group
    // records the version pinned when it was dispatched
    auto simulate = [&](int s, const std::vector<Req> &reqs, int64_t units, int64_t ver) {
        const int64_t g = group_id++;
        const int64_t t0 = seq++;
        std::this_thread::sleep_for(std::chrono::microseconds((int64_t)work_us * (1 + units / 64)));
        if (ver < 0) ver = ++version;
        const int64_t t1 = seq++;
        for (const Req &r : reqs) {
            const size_t i = (size_t)(r.ticket - 1);
            start_seq[i] = t0;
            end_seq[i] = t1;
            slot_of[i] = s;
            group_of[i] = g;
            if (version_of) version_of[i] = ver;
        }
        return PG_OK;
    };
    q.run_group = [&](int s, const Group &g) {
        return simulate(s, g.reqs, g.rows, *static_cast<const int64_t *>(g.pinned.get()));
    };
    q.run_insert = [&](int slot, const Req &r) {
        return simulate(slot, std::vector<Req>{r}, r.rows, -1);
    };
    q.pin = [&]() -> std::shared_ptr<void> { return std::make_shared<int64_t>(version.load()); };
    if (!q.start()) return PG_ERR_INTERNAL;
    std::vector<Req> reqs((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        reqs[(size_t)i].kind = kind[i];
        reqs[(size_t)i].rows = rows[i];
        reqs[(size_t)i].shape = shape[i];
    }
    pg_status st = q.submit_all(reqs);
    for (int64_t t = 1; t <= count && st == PG_OK; ++t) {
        int32_t done = 0;
        const pg_status w = q.wait(t, 60.0, &done);
        if (!done) st = PG_ERR_TIMEOUT;
        else if (w != PG_OK && w != PG_ERR_BUDGET) st = w;
    }
    q.stop();
    if (host_stats6) q.stats(host_stats6, 6);
    return st;
}
