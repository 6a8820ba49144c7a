// cr_serve.cu -- serving runtime: a request queue in front of one batch (cr_batch.cu).
//
// Callers submit solve requests from any thread; one server thread owns the batch and the
// GPU work.  Its loop: admit queued requests in arrival order while their multipliers fit
// under the memory cap (cr_batch_instance_bytes) and the active-slot limit allows; run
// check_every iterations of every active instance (one graph block); retire the instances
// that converged or reached their iteration cap -- copy (y, xi) to the request, free the
// instance's device memory, record its latency -- and loop.  Requests that arrive while
// others are running join at the next block boundary, so their work shares the same
// launches (continuous batching).  The server thread waits on a condition variable when
// there is nothing to run; every wait is bounded.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cr_host.h"

using namespace crh;

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    int N = 0, n = 0;
    double tol = 0.0;
    long long max_iter = 0;
    std::vector<double> X, ybar;     // host copies of the inputs (released at admission)
    std::vector<double> y, xi;       // result
    int state = 0;                   // 0 queued, 1 running, 2 done
    int status = CR_OK;
    cr_gap_info info{};
    int batch_id = -1;
    long long bytes = 0;
    clk::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct cr_server {
    cr_options opt{};
    long long mem_cap = 0, mem_used = 0;
    int max_active = 0;
    int device = 0;
    void *stream = nullptr;
    cr_batch *batch = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<long long> queue;
    std::unordered_map<long long, Request *> reqs;
    std::unordered_map<int, long long> by_batch;
    long long next_id = 0;
    bool stop = false;
    int fatal = CR_OK;
    char fatal_msg[256] = "";
    std::thread th;
    // statistics
    long long completed = 0, converged = 0, admitted = 0;
    double busy_s = 0.0;
    std::vector<double> latencies;
    clk::time_point t_start;
};

namespace {

void server_loop(cr_server *s) {
    cudaSetDevice(s->device);
    std::vector<long long> running;
    for (;;) {
        // ---- admission (arrival order, memory cap, slot limit)
        std::vector<Request *> to_add;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (running.empty() && s->queue.empty() && !s->stop)
                s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            if (s->stop) break;
            while (!s->queue.empty() && (int)(running.size() + to_add.size()) < s->max_active) {
                Request *r = s->reqs[s->queue.front()];
                if (s->mem_used + r->bytes > s->mem_cap && !(running.empty() && to_add.empty())) break;
                s->queue.pop_front();
                s->mem_used += r->bytes;
                to_add.push_back(r);
            }
        }
        for (Request *r : to_add) {
            int bid = -1;
            cr_status st = cr_batch_add(s->batch, r->X.data(), r->ybar.data(), r->N, r->n, r->tol, r->max_iter, &bid);
            std::lock_guard<std::mutex> lk(s->mu);
            r->t_admit = clk::now();
            r->X.clear();
            r->X.shrink_to_fit();
            r->ybar.clear();
            r->ybar.shrink_to_fit();
            if (st != CR_OK) {
                r->state = 2;
                r->status = st;
                r->t_done = r->t_admit;
                s->mem_used -= r->bytes;
                ++s->completed;
                s->cv_done.notify_all();
                continue;
            }
            r->state = 1;
            r->batch_id = bid;
            s->by_batch[bid] = r->id;
            running.push_back(r->id);
            ++s->admitted;
        }
        if (running.empty()) continue;
        // ---- one block of iterations for everything on the GPU
        const auto t0 = clk::now();
        int active = 0;
        cr_status st = cr_batch_step(s->batch, s->opt.check_every, &active);
        const double dt = std::chrono::duration<double>(clk::now() - t0).count();
        if (st != CR_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->fatal = st;
            snprintf(s->fatal_msg, sizeof(s->fatal_msg), "%s", cr_last_error());
            for (long long id : running) {
                Request *r = s->reqs[id];
                r->state = 2;
                r->status = st;
                r->t_done = clk::now();
            }
            s->cv_done.notify_all();
            break;
        }
        // ---- retirement
        std::vector<long long> still;
        for (long long id : running) {
            Request *r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = s->reqs[id];
            }
            int done = 0, status = CR_OK;
            cr_gap_info info{};
            cr_batch_poll(s->batch, r->batch_id, &done, &status, &info);
            if (!done) {
                still.push_back(id);
                continue;
            }
            std::vector<double> y((size_t)r->N), xi((size_t)r->N * r->n);
            cr_status pst = cr_batch_primal(s->batch, r->batch_id, y.data(), xi.data());
            cr_batch_remove(s->batch, r->batch_id);
            std::lock_guard<std::mutex> lk(s->mu);
            r->y.swap(y);
            r->xi.swap(xi);
            r->info = info;
            r->status = pst != CR_OK ? pst : status;
            r->state = 2;
            r->t_done = clk::now();
            s->mem_used -= r->bytes;
            s->by_batch.erase(r->batch_id);
            ++s->completed;
            if (r->status == CR_OK) ++s->converged;
            s->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
            s->cv_done.notify_all();
        }
        running.swap(still);
        std::lock_guard<std::mutex> lk(s->mu);
        s->busy_s += dt;
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t i = std::min(v.size() - 1, (size_t)floor(q * (double)(v.size() - 1) + 0.5));
    return v[i];
}

}  // namespace

extern "C" {

CR_API cr_status cr_server_create(const cr_options *opt, long long mem_cap_bytes, int max_active, void *stream,
                                  cr_server **out) {
    if (!out || mem_cap_bytes <= 0 || max_active < 1) {
        set_err("bad argument to cr_server_create");
        return CR_EINVAL;
    }
    *out = nullptr;
    cr_server *s = new (std::nothrow) cr_server();
    if (!s) {
        set_err("host allocation failed");
        return CR_ENOMEM;
    }
    if (opt)
        s->opt = *opt;
    else
        cr_default_options(&s->opt);
    if (s->opt.check_every < 1) s->opt.check_every = 1;
    s->mem_cap = mem_cap_bytes;
    s->max_active = max_active;
    s->stream = stream;
    cudaGetDevice(&s->device);
    cr_status st = cr_batch_create(&s->opt, stream, &s->batch);
    if (st != CR_OK) {
        delete s;
        return st;
    }
    s->t_start = clk::now();
    try {
        s->th = std::thread(server_loop, s);
    } catch (...) {
        cr_batch_destroy(s->batch);
        delete s;
        set_err("could not start the server thread");
        return CR_ENOMEM;
    }
    *out = s;
    return CR_OK;
}

CR_API cr_status cr_server_submit(cr_server *s, const double *X, const double *ybar, long long N, int n,
                                  double rel_gap_tol, long long max_iter, long long *req_id) {
    if (!s || !X || !ybar || !req_id || N < 2 || N > (1LL << 30) || n < 1 || n > CR_MAX_N_BATCH ||
        !(rel_gap_tol >= 0.0) || max_iter < 0) {
        set_err("bad argument to cr_server_submit");
        return CR_EINVAL;
    }
    long long bytes = cr_batch_instance_bytes(N, n);
    if (s->opt.step_rule == CR_STEP_ADAPTIVE)  // third multiplier buffer, candidate C^T and row sums
        bytes += N * ((N + 31) / 32 * 32) * 4 + 8 * N * (n + 1) + 4 * N * ((N + 511) / 512 + 1);
    if (bytes > s->mem_cap) {
        set_err("request needs %lld bytes, above the server's cap of %lld", bytes, s->mem_cap);
        return CR_ENOMEM;
    }
    Request *r = new (std::nothrow) Request();
    if (!r) {
        set_err("host allocation failed");
        return CR_ENOMEM;
    }
    r->N = (int)N;
    r->n = n;
    r->tol = rel_gap_tol;
    r->max_iter = max_iter;
    r->bytes = bytes;
    try {
        r->X.resize((size_t)N * n);
        r->ybar.resize((size_t)N);
    } catch (...) {
        delete r;
        set_err("host allocation failed");
        return CR_ENOMEM;
    }
    // inputs may be host or device memory: copy with unified addressing
    cudaError_t e = cudaMemcpy(r->X.data(), X, sizeof(double) * N * n, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(r->ybar.data(), ybar, sizeof(double) * N, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        delete r;
        set_err("input copy failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != CR_OK) {
            delete r;
            set_err("server stopped: %s", s->fatal_msg);
            return (cr_status)s->fatal;
        }
        r->id = s->next_id++;
        r->t_submit = clk::now();
        s->reqs[r->id] = r;
        s->queue.push_back(r->id);
        *req_id = r->id;
    }
    s->cv_work.notify_one();
    return CR_OK;
}

CR_API cr_status cr_server_poll(cr_server *s, long long req_id, int *state, int *status, cr_gap_info *info,
                                double *latency_s) {
    if (!s) {
        set_err("server is NULL");
        return CR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) {
        set_err("unknown request %lld", req_id);
        return CR_EINVAL;
    }
    const Request *r = it->second;
    if (state) *state = r->state;
    if (status) *status = r->status;
    if (info) *info = r->info;
    if (latency_s)
        *latency_s = r->state == 2 ? std::chrono::duration<double>(r->t_done - r->t_submit).count() : -1.0;
    return CR_OK;
}

CR_API cr_status cr_server_wait(cr_server *s, long long req_id, double timeout_s) {
    if (!s || !(timeout_s >= 0.0)) {
        set_err("bad argument to cr_server_wait");
        return CR_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) {
        set_err("unknown request %lld", req_id);
        return CR_EINVAL;
    }
    Request *r = it->second;
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
    while (r->state != 2) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2) {
            set_err("request %lld not finished within %.3f s", req_id, timeout_s);
            return CR_ETIMEOUT;
        }
    }
    return CR_OK;
}

CR_API cr_status cr_server_result(cr_server *s, long long req_id, double *y, double *xi) {
    if (!s) {
        set_err("server is NULL");
        return CR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) {
        set_err("unknown request %lld", req_id);
        return CR_EINVAL;
    }
    Request *r = it->second;
    if (r->state != 2) {
        set_err("request %lld is not finished", req_id);
        return CR_EINVAL;
    }
    if (r->y.empty()) {
        set_err("request %lld has no result (status %d)", req_id, r->status);
        return (cr_status)(r->status != CR_OK ? r->status : CR_EINVAL);
    }
    cudaError_t e = cudaSuccess;
    if (y) e = cudaMemcpy(y, r->y.data(), sizeof(double) * r->y.size(), cudaMemcpyDefault);
    if (xi && e == cudaSuccess) e = cudaMemcpy(xi, r->xi.data(), sizeof(double) * r->xi.size(), cudaMemcpyDefault);
    if (e != cudaSuccess) {
        set_err("result copy failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    return CR_OK;
}

CR_API cr_status cr_server_release(cr_server *s, long long req_id) {
    if (!s) {
        set_err("server is NULL");
        return CR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end() || it->second->state != 2) {
        set_err("request %lld is unknown or not finished", req_id);
        return CR_EINVAL;
    }
    delete it->second;
    s->reqs.erase(it);
    return CR_OK;
}

CR_API cr_status cr_server_stats(cr_server *s, cr_serve_stats *out) {
    if (!s || !out) {
        set_err("bad argument to cr_server_stats");
        return CR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->converged = s->converged;
    out->queued = (long long)s->queue.size();
    out->running = (long long)s->by_batch.size();
    out->mem_used = s->mem_used;
    out->mem_cap = s->mem_cap;
    out->p50_s = percentile(s->latencies, 0.50);
    out->p99_s = percentile(s->latencies, 0.99);
    out->elapsed_s = std::chrono::duration<double>(clk::now() - s->t_start).count();
    out->busy_s = s->busy_s;
    return CR_OK;
}

CR_API void cr_server_destroy(cr_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    cr_batch_destroy(s->batch);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
