// Serving: continuous batching of minimisation requests on one GPU.
//
// Fused mode: the running requests whose children go through the term-table
// FP32-then-FP64 kernel are advanced in steps: every such request whose
// previous generation has finished joins the next step, which enqueues a
// generation of each of them with a single fused child-evaluation launch
// over all their children (batch_generation); the other requests advance as
// below.
//
// gb_submit copies a request (objective, bounds, options) and returns at once.
// A worker thread admits queued requests in arrival order while the device
// memory they need fits the server's budget and a slot is free, runs every
// admitted request's generations on that request's own stream -- advancing
// whichever request's previous generation has finished, so the requests'
// kernels overlap on the device -- and retires finished requests, which frees
// their memory and slots for the next ones.  Each request's search depends
// only on its own state, so its result is the same alone and in a mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gb_launch.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    // copy of the submitted problem
    std::vector<gb_node> nodes;
    int32_t root = 0, n = 0;
    std::vector<std::vector<double>> tables;
    std::vector<double> l, u;
    double tol = 0.0;
    gb_options opt{};
    // state
    enum { QUEUED, RUNNING, DONE } phase = QUEUED;
    gb_problem* prob = nullptr;
    size_t reserved = 0;
    gb_status status = GB_OK;
    std::string error;
    gb_result result{};
    Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct gb_server {
    size_t budget = 0, in_use = 0;
    int device = 0, max_active = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> running;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_id = 1;
    bool stop = false;
    int fused = 0;
    GbBatchCtx* batch = nullptr;   // worker thread only
    bool batch_failed = false;     // could not set up the fused step: requests advance on their own
    std::thread worker;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

void finish_request(gb_server* S, const std::shared_ptr<Request>& r, gb_status st) {
    r->t_done = Clock::now();
    r->status = st;
    r->result.status = st;
    r->result.queue_ms = ms_between(r->t_submit, r->t_start);
    r->result.latency_ms = ms_between(r->t_submit, r->t_done);
    std::lock_guard<std::mutex> lk(S->mu);
    r->phase = Request::DONE;
    S->in_use -= r->reserved;
    r->reserved = 0;
}

void worker_loop(gb_server* S) {
    for (;;) {
        // ---- admission -------------------------------------------------------
        std::vector<std::shared_ptr<Request>> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->running.empty() && S->queue.empty())
                S->cv.wait(lk, [S] { return S->stop || !S->queue.empty(); });
            if (S->stop) return;
            while (!S->queue.empty() && (int)(S->running.size() + admit.size()) < S->max_active) {
                auto& r = S->queue.front();
                size_t need = r->opt.pool_bytes;
                bool alone = S->running.empty() && admit.empty();
                if (S->in_use + need > S->budget && !alone) break;   // wait for memory to free up
                r->reserved = need;
                S->in_use += need;
                admit.push_back(r);
                S->queue.pop_front();
            }
        }
        for (auto& r : admit) {
            r->t_start = Clock::now();
            std::vector<const double*> tp(r->tables.size());
            std::vector<int64_t> tl(r->tables.size());
            for (size_t t = 0; t < r->tables.size(); t++) tp[t] = r->tables[t].data(), tl[t] = (int64_t)r->tables[t].size();
            gb_status st = gb_create_problem(r->nodes.data(), (int32_t)r->nodes.size(), r->root,
                                             tp.empty() ? nullptr : tp.data(), tl.empty() ? nullptr : tl.data(),
                                             (int32_t)r->tables.size(), r->n, r->l.data(), r->u.data(), r->tol,
                                             &r->opt, &r->prob);
            if (st == GB_OK) st = solve_begin(r->prob);
            if (st != GB_OK) {
                r->error = gb_last_error();
                if (r->prob) gb_destroy_problem(r->prob);
                r->prob = nullptr;
                finish_request(S, r, st);
                continue;
            }
            S->running.push_back(r);
        }
        // ---- advance every request whose previous generation has finished ----
        bool progressed = false;
        int fused;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            fused = S->fused;
        }
        if (fused && !S->batch && !S->batch_failed) {
            S->batch = batch_create(S->device);
            S->batch_failed = S->batch == nullptr;
        }
        std::vector<gb_problem*> step;   // fusable requests ready for their next generation
        for (size_t k = 0; k < S->running.size();) {
            auto r = S->running[k];
            int done;
            if (fused && S->batch && solve_fusable(r->prob)) {
                const int c = solve_check(r->prob, false);   // launched by the fused step below
                if (c == 0) step.push_back(r->prob);
                done = c > 0;
            } else {
                done = solve_advance(r->prob, false);
            }
            if (!done) {
                k++;
                continue;
            }
            progressed = true;
            gb_status st = solve_finish(r->prob, &r->result, true);
            if (st != GB_OK) r->error = gb_last_error();
            gb_destroy_problem(r->prob);
            r->prob = nullptr;
            S->running.erase(S->running.begin() + k);
            finish_request(S, r, st);
        }
        if (!step.empty()) {   // every ready request joins this step; the others are still running theirs
            for (size_t b = 0; b < step.size(); b += GB_BATCH_MAX) {
                const int k = (int)std::min<size_t>(GB_BATCH_MAX, step.size() - b);
                if (batch_generation(step.data() + b, k, S->batch, 4) != GB_OK) {
                    // a failed enqueue ends those requests with the error
                    for (int i = 0; i < k; i++) solve_abort(step[b + i], GB_E_CUDA);
                }
            }
            progressed = true;
        }
        if (!progressed && !S->running.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

gb_status gb_server_create(size_t pool_budget_bytes, int32_t device, int32_t max_active, gb_server** out) {
    if (!out || pool_budget_bytes == 0 || max_active < 1) return gb_internal_fail(GB_E_INVALID, "bad server arguments");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return gb_internal_fail(GB_E_CUDA, "no CUDA device available");
    // keep freed request memory in the device's stream-ordered pool (up to the
    // budget) instead of returning it to the driver at every synchronisation
    cudaMemPool_t mp;
    if (cudaSetDevice(device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess) {
        uint64_t keep = pool_budget_bytes;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    gb_server* S = new gb_server();
    S->budget = pool_budget_bytes;
    S->device = device;
    S->max_active = max_active;
    S->worker = std::thread([S] {
        cudaSetDevice(S->device);
        gb_pdl_thread(false);   // many requests share the SMs: no early-started blocks waiting on them
        worker_loop(S);
    });
    *out = S;
    return GB_OK;
}

gb_status gb_submit(gb_server* S, const gb_node* dag, int32_t n_nodes, int32_t root, const double* const* tables,
                    const int64_t* table_lens, int32_t n_tables, int32_t n, const double* l, const double* u,
                    double tol, const gb_options* opt, uint64_t* request_id) {
    if (!S || !dag || n_nodes < 1 || n < 1 || !l || !u || !request_id || n_tables < 0 ||
        (n_tables > 0 && (!tables || !table_lens)))
        return gb_internal_fail(GB_E_INVALID, "bad gb_submit arguments");
    auto r = std::make_shared<Request>();
    r->nodes.assign(dag, dag + n_nodes);
    r->root = root;
    r->n = n;
    for (int t = 0; t < n_tables; t++) {
        if (table_lens[t] < 0) return gb_internal_fail(GB_E_INVALID, "negative table length");
        r->tables.emplace_back(tables[t], tables[t] + table_lens[t]);
    }
    r->l.assign(l, l + n);
    r->u.assign(u, u + n);
    r->tol = tol;
    gb_default_options(&r->opt);
    if (opt) r->opt = *opt;
    r->opt.device = S->device;
    if (opt == nullptr || opt->pool_bytes == 0) r->opt.pool_bytes = S->budget / (size_t)S->max_active;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return gb_internal_fail(GB_E_BUSY, "server is shutting down");
        r->id = S->next_id++;
        S->all[r->id] = r;
        S->queue.push_back(r);
    }
    S->cv.notify_one();
    *request_id = r->id;
    return GB_OK;
}

gb_status gb_server_set_fused(gb_server* S, int32_t fused) {
    if (!S) return gb_internal_fail(GB_E_INVALID, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    S->fused = fused ? 1 : 0;
    return GB_OK;
}

gb_status gb_poll(gb_server* S, uint64_t id, gb_result* out) {
    if (!S || !out) return gb_internal_fail(GB_E_INVALID, "bad gb_poll arguments");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(id);
        if (it == S->all.end()) return gb_internal_fail(GB_E_INVALID, "unknown request id");
        if (it->second->phase != Request::DONE) return GB_E_BUSY;
        r = it->second;
        S->all.erase(it);
    }
    *out = r->result;                       // ownership of the host arrays passes to the caller
    std::memset(&r->result, 0, sizeof(r->result));
    if (r->status != GB_OK && !r->error.empty()) gb_internal_fail(r->status, r->error.c_str());
    return r->status;
}

gb_status gb_server_destroy(gb_server* S) {
    if (!S) return GB_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    batch_destroy(S->batch);
    for (auto& r : S->running)
        if (r->prob) gb_destroy_problem(r->prob);
    for (auto& kv : S->all) gb_free_result(&kv.second->result);
    delete S;
    return GB_OK;
}

}  // extern "C"
