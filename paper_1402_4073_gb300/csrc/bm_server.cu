// Serving loop: continuous batching of arriving queries over a resident
// pool, admission by device memory, overlapping batches on several streams.
//
// A request holds a copy of its query.  It waits in a FIFO until the
// scheduler thread can give it an output slot from the server's device
// arena (admission by memory: a slot is one output bitmap plus alignment)
// and a batch position.  Whenever a stream is free the scheduler launches
// every admitted waiting request (up to max_batch) as one bm_threshold_batch
// on that stream, so requests that arrive while other batches run join the
// next batch and their work overlaps on the GPU.  A host callback after each
// batch stamps its completion time and wakes waiters.  A request's slot is
// returned when the caller collects or releases the result.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "bm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double us_since(Clock::time_point t0, Clock::time_point t1) {
    return std::chrono::duration<double, std::micro>(t1 - t0).count();
}

struct Request {
    uint64_t ticket = 0;
    std::vector<uint32_t> ids;
    std::vector<uint64_t> table;
    bm_query q{};
    int32_t slot = -1;
    int32_t path = 0;
    uint64_t card = 0;
    Clock::time_point t_submit, t_launch, t_done;
    Clock::time_point deadline = Clock::time_point::max();  // drop if still waiting after this
    bool done = false;
};

struct Batch {
    Clock::time_point t_launch;
    uint64_t inputs = 0;  // ids of the batch's requests, repeats counted
    cudaStream_t stream = nullptr;
    uint64_t* d_cards = nullptr;
    uint64_t* h_cards = nullptr;  // pinned
    std::vector<Request*> reqs;
    std::vector<int32_t> paths;  // path each request ran on, filled before the callback
    bool busy = false;
    struct bm_server* srv = nullptr;
};

}  // namespace

struct bm_server {
    bm_pool* pool = nullptr;
    bm_server_config cfg{};
    uint64_t slot_bytes = 0;
    uint32_t n_slots = 0;
    uint8_t* d_arena = nullptr;
    std::vector<int32_t> free_slots;
    std::vector<Batch> batches;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request*> waiting;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;

    // running estimates of a batch's time, microseconds: a fixed part (from
    // batches of few inputs) and a time per input id (from large ones); a
    // request's work grows with its number of inputs
    double est_fixed_us = 100.0, est_us_per_input = 0.1;
    uint64_t waiting_inputs = 0;  // ids of the requests waiting for admission

    // statistics
    uint64_t submitted = 0, completed = 0, refused = 0, batches_run = 0, batched_queries = 0;
    uint64_t cancelled = 0, expired = 0;
    uint32_t max_batch_seen = 0;
    int last_error = BM_OK;
};

namespace {

void CUDART_CB on_batch_done(void* arg) {
    Batch* b = static_cast<Batch*>(arg);
    bm_server* s = b->srv;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = 0; i < b->reqs.size(); ++i) {
            Request* r = b->reqs[i];
            r->card = b->h_cards[i];
            r->path = b->paths[i];
            r->t_done = now;
            r->done = true;
        }
        s->completed += b->reqs.size();
        // the batch's time updates the estimates the latency objective uses
        const double exec = us_since(b->t_launch, now);
        const double ni = (double)b->inputs;
        if (ni <= 2048) {
            const double fixed = std::max(5.0, exec - s->est_us_per_input * ni);
            s->est_fixed_us = 0.9 * s->est_fixed_us + 0.1 * fixed;
        } else {
            const double per = std::max(1e-3, (exec - s->est_fixed_us) / ni);
            s->est_us_per_input = 0.8 * s->est_us_per_input + 0.2 * per;
        }
        b->inputs = 0;
        b->reqs.clear();
        b->busy = false;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
}

// Launch one batch of admitted requests on stream b.stream.  Called without
// the server lock: CUDA calls inside (allocation, frees) may wait for the
// device, and the device may be waiting for a host callback that needs the
// lock.
int launch_batch(bm_server* s, Batch& b, const std::vector<bm_query>& qs) {
    b.paths.assign(qs.size(), 0);
    int rc = bm_threshold_batch(s->pool, qs.data(), (uint32_t)qs.size(), b.d_cards, b.paths.data(),
                                b.stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(b.h_cards, b.d_cards, 8 * qs.size(), cudaMemcpyDeviceToHost, b.stream) !=
        cudaSuccess)
        return BM_ECUDA;
    if (cudaLaunchHostFunc(b.stream, on_batch_done, &b) != cudaSuccess) return BM_ECUDA;
    return BM_OK;
}

void scheduler(bm_server* s) {
    cudaSetDevice(s->pool->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // wakes on submissions, completions and releases; at least every
        // millisecond while requests wait, to expire their deadlines
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(1), [&] {
            if (s->stop) return true;
            if (s->waiting.empty() || s->free_slots.empty()) return false;
            for (auto& b : s->batches)
                if (!b.busy) return true;
            return false;
        });
        if (s->stop) break;
        if (s->cfg.batch_window_us) {
            // let a batch grow for a short window when the GPU has room
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(s->cfg.batch_window_us));
            lk.lock();
            if (s->stop) break;
        }
        {
            // requests whose deadline passed while they waited complete as
            // expired; with a latency objective, so do those that could not
            // finish within it even in a batch of their own
            const auto now = Clock::now();
            const auto slo = std::chrono::microseconds(s->cfg.slo_us);
            bool expired = false;
            for (auto it = s->waiting.begin(); it != s->waiting.end();) {
                const auto alone = std::chrono::microseconds(
                    (int64_t)(s->est_fixed_us + s->est_us_per_input * (double)(*it)->q.n));
                if ((*it)->deadline <= now ||
                    (s->cfg.slo_us && (*it)->t_submit + slo <= now + alone)) {
                    Request* r = *it;
                    s->waiting_inputs -= r->q.n;
                    r->done = true;
                    r->t_launch = r->t_done = now;
                    r->path = BM_ETIMEOUT;
                    s->expired += 1;
                    it = s->waiting.erase(it);
                    expired = true;
                } else {
                    ++it;
                }
            }
            if (expired) s->cv_done.notify_all();
        }
        for (auto& b : s->batches) {
            if (b.busy || s->waiting.empty() || s->free_slots.empty()) continue;
            // with a latency objective, the batch is sized so that its oldest
            // request (the front) can still complete within it: its inputs'
            // estimated time fits the front's remaining budget
            double budget_inputs = 1e300;
            if (s->cfg.slo_us) {
                const double age = us_since(s->waiting.front()->t_submit, Clock::now());
                const double budget = (double)s->cfg.slo_us - age - s->est_fixed_us;
                budget_inputs = budget / s->est_us_per_input;
            }
            std::vector<Request*> take;
            double inputs = 0.0;
            while (!s->waiting.empty() && !s->free_slots.empty() &&
                   take.size() < s->cfg.max_batch) {
                Request* r = s->waiting.front();
                if (!take.empty() && inputs + (double)r->q.n > budget_inputs) break;
                inputs += (double)r->q.n;
                s->waiting_inputs -= r->q.n;
                s->waiting.pop_front();
                r->slot = s->free_slots.back();
                s->free_slots.pop_back();
                r->q.out_words =
                    reinterpret_cast<uint64_t*>(s->d_arena + (uint64_t)r->slot * s->slot_bytes);
                take.push_back(r);
            }
            b.reqs = take;
            b.inputs = (uint64_t)inputs;
            b.busy = true;
            const auto now = Clock::now();
            b.t_launch = now;
            std::vector<bm_query> qs(take.size());
            for (size_t i = 0; i < take.size(); ++i) {
                take[i]->t_launch = now;
                qs[i] = take[i]->q;
            }
            // Once the lock is dropped the batch may complete and its requests be
            // collected and freed, so they are not touched again on success.
            const size_t nb = take.size();
            lk.unlock();
            int rc = launch_batch(s, b, qs);
            lk.lock();
            if (rc) {
                // the batch could not run: its requests complete with the error
                s->last_error = rc;
                const auto t = Clock::now();
                for (Request* r : take) {
                    r->done = true;
                    r->t_done = t;
                    r->path = rc;
                }
                b.reqs.clear();
                b.inputs = 0;
                b.busy = false;
                s->cv_done.notify_all();
            } else {
                s->batches_run += 1;
                s->batched_queries += nb;
                s->max_batch_seen = std::max<uint32_t>(s->max_batch_seen, (uint32_t)nb);
            }
            if (s->stop) break;
        }
    }
}

}  // namespace

extern "C" {

int bm_server_create(bm_pool* pool, const bm_server_config* cfg, bm_server** out) {
    if (!pool || !cfg || !out) return BM_EINVAL;
    if (cfg->max_batch == 0 || cfg->max_inflight == 0 || cfg->max_inflight > 4 ||
        cfg->max_queue == 0 || cfg->reserved)
        return BM_EINVAL;
    *out = nullptr;
    bm_pool_info_t info;
    bm_pool_info(pool, &info);
    bm_server* s = new bm_server();
    s->pool = pool;
    s->cfg = *cfg;
    s->slot_bytes = (info.words * 8 + 255) & ~(uint64_t)255;
    const uint64_t n = cfg->mem_budget / s->slot_bytes;
    if (n == 0) {
        delete s;
        return BM_ENOMEM;
    }
    s->n_slots = (uint32_t)std::min<uint64_t>(n, 1u << 30);
    if (cudaSetDevice(pool->device) != cudaSuccess ||
        cudaMalloc(&s->d_arena, (size_t)s->n_slots * s->slot_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return BM_ENOMEM;
    }
    s->free_slots.reserve(s->n_slots);
    for (int32_t i = (int32_t)s->n_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->batches.resize(cfg->max_inflight);
    for (auto& b : s->batches) {
        b.srv = s;
        if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&b.d_cards, 8ull * cfg->max_batch) != cudaSuccess ||
            cudaHostAlloc(&b.h_cards, 8ull * cfg->max_batch, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            bm_server_destroy(s);
            return BM_ENOMEM;
        }
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return BM_OK;
}

int bm_server_destroy(bm_server* s) {
    if (!s) return BM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto& b : s->batches) {
        if (b.stream) cudaStreamSynchronize(b.stream);
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.d_cards) cudaFree(b.d_cards);
        if (b.h_cards) cudaFreeHost(b.h_cards);
    }
    if (s->d_arena) cudaFree(s->d_arena);
    for (auto& kv : s->reqs) delete kv.second;  // every submitted request, waiting or not
    delete s;
    return BM_OK;
}

int bm_server_submit(bm_server* s, const bm_query* q, uint64_t* ticket) {
    return bm_server_submit_deadline(s, q, 0, ticket);
}

int bm_server_submit_deadline(bm_server* s, const bm_query* q, uint64_t deadline_us,
                              uint64_t* ticket) {
    if (!s || !q || !ticket || !q->ids || q->n == 0 || q->n > BM_N_MAX || q->reserved)
        return BM_EINVAL;
    if (q->kind > BM_KIND_TABLE || q->path < BM_PATH_AUTO || q->path > BM_PATH_RLE)
        return BM_EINVAL;
    if (q->kind == BM_KIND_TABLE && !q->table) return BM_EINVAL;
    {
        // ids are checked here so that a bad request never joins a batch
        std::lock_guard<std::mutex> plk(s->pool->mu);
        int rc = bm::validate_ids(s->pool, q->ids, q->n, q->path);
        if (rc) return rc;
    }
    Request* r = new Request();
    r->ids.assign(q->ids, q->ids + q->n);
    if (q->kind == BM_KIND_TABLE) r->table.assign(q->table, q->table + (q->n + 1 + 63) / 64);
    r->q = *q;
    r->q.ids = r->ids.data();
    r->q.table = r->table.empty() ? nullptr : r->table.data();
    r->t_submit = Clock::now();
    if (deadline_us) r->deadline = r->t_submit + std::chrono::microseconds(deadline_us);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        bool refuse = s->waiting.size() >= s->cfg.max_queue;
        if (s->cfg.slo_us && !refuse) {
            // admission by the latency objective: the work ahead of this request
            // (waiting and in flight) must drain within it
            uint64_t ahead = s->waiting_inputs + q->n;
            for (const auto& b : s->batches) ahead += b.inputs;
            refuse = s->est_fixed_us + s->est_us_per_input * (double)ahead > s->cfg.slo_us;
        }
        if (refuse) {
            s->refused += 1;
            delete r;
            return BM_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->waiting.push_back(r);
        s->waiting_inputs += r->q.n;
        s->submitted += 1;
        *ticket = r->ticket;
    }
    s->cv_sched.notify_one();
    return BM_OK;
}

int bm_server_wait(bm_server* s, uint64_t ticket, uint32_t timeout_ms) {
    if (!s) return BM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return BM_ERANGE;
    Request* r = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
        return BM_ETIMEOUT;
    return r->path < 0 ? r->path : BM_OK;
}

int bm_server_result(bm_server* s, uint64_t ticket, uint64_t* host_words, uint64_t* card,
                     double* latency_us, double* queue_us, int32_t* path) {
    if (!s) return BM_EINVAL;
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return BM_ERANGE;
        r = it->second;
        if (!r->done) return BM_ENOTREADY;
    }
    int rc = r->path < 0 ? r->path : BM_OK;
    if (!rc && host_words) {
        // the request's batch has completed (its host callback ran), so the slot holds the result
        if (cudaMemcpy(host_words, r->q.out_words, s->pool->words * 8, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            rc = BM_ECUDA;
    }
    if (card) *card = r->card;
    if (latency_us) *latency_us = us_since(r->t_submit, r->t_done);
    if (queue_us) *queue_us = us_since(r->t_submit, r->t_launch);
    if (path) *path = r->path;
    return rc;
}

int bm_server_cancel(bm_server* s, uint64_t ticket) {
    if (!s) return BM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return BM_ERANGE;
        Request* r = it->second;
        auto w = std::find(s->waiting.begin(), s->waiting.end(), r);
        if (w == s->waiting.end()) return BM_EBUSY;  // admitted: it runs to completion
        s->waiting.erase(w);
        s->waiting_inputs -= r->q.n;
        s->reqs.erase(it);
        s->cancelled += 1;
        delete r;
    }
    s->cv_sched.notify_one();
    return BM_OK;
}

int bm_server_release(bm_server* s, uint64_t ticket) {
    if (!s) return BM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return BM_ERANGE;
        Request* r = it->second;
        if (!r->done) return BM_ENOTREADY;
        if (r->slot >= 0) s->free_slots.push_back(r->slot);
        s->reqs.erase(it);
        delete r;
    }
    s->cv_sched.notify_one();
    return BM_OK;
}

int bm_server_replay(bm_server* s, const bm_query* qs, uint32_t n, const double* arrival_s,
                     double* latency_us, double* queue_us, uint64_t* cards, int32_t* status,
                     double* wall_s) {
    if (!s || !qs || !arrival_s || n == 0) return BM_EINVAL;
    std::vector<uint64_t> tickets(n, 0);
    std::vector<int32_t> st(n, BM_OK);
    std::atomic<uint32_t> submitted{0};
    std::atomic<bool> submit_done{false};
    // collector: results in submission order, each slot released at once
    std::thread collector([&] {
        bool stalled = false;
        for (uint32_t i = 0; i < n; ++i) {
            while (submitted.load() <= i && !submit_done.load())
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            if (i >= submitted.load()) break;
            if (st[i] != BM_OK) continue;
            // a request gets at most 10 s; after one never completes the rest get 100 ms each
            int rc = bm_server_wait(s, tickets[i], stalled ? 100 : 10000);
            if (rc != BM_OK) {
                double lat = 0, qu = 0;
                st[i] = rc;
                if (bm_server_result(s, tickets[i], nullptr, nullptr, &lat, &qu, nullptr) ==
                    BM_ENOTREADY) {
                    stalled = true;  // the wait itself ran out
                    continue;
                }
                // completed without a result: dropped (deadline, objective) or failed
                if (latency_us) latency_us[i] = lat;
                if (queue_us) queue_us[i] = qu;
                bm_server_release(s, tickets[i]);
                continue;
            }
            double lat = 0, qu = 0;
            uint64_t c = 0;
            st[i] = bm_server_result(s, tickets[i], nullptr, &c, &lat, &qu, nullptr);
            if (latency_us) latency_us[i] = lat;
            if (queue_us) queue_us[i] = qu;
            if (cards) cards[i] = c;
            bm_server_release(s, tickets[i]);
        }
    });
    const auto t0 = Clock::now();
    for (uint32_t i = 0; i < n; ++i) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                                  std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
            const auto left = due - Clock::now();
            if (left > std::chrono::microseconds(200))
                std::this_thread::sleep_for(left - std::chrono::microseconds(100));
        }
        st[i] = bm_server_submit(s, &qs[i], &tickets[i]);
        submitted.store(i + 1);
    }
    submit_done.store(true);
    collector.join();
    if (wall_s) *wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    if (status) memcpy(status, st.data(), 4ull * n);
    return BM_OK;
}

int bm_server_stats(bm_server* s, bm_server_stats_t* out) {
    if (!s || !out) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->refused = s->refused;
    out->batches = s->batches_run;
    out->batched_queries = s->batched_queries;
    out->waiting = (uint32_t)s->waiting.size();
    out->free_slots = (uint32_t)s->free_slots.size();
    out->total_slots = s->n_slots;
    out->max_batch_seen = s->max_batch_seen;
    out->cancelled = s->cancelled;
    out->expired = s->expired;
    out->last_error = s->last_error;
    return BM_OK;
}

}  // extern "C"
