// Serving: continuous batching of step requests over resident scenes (see
// include/ipc.h). Worker threads, one per slot, each own a CUDA stream;
// admission and results live under one mutex.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ipc.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    unsigned long long ticket;
    ipc_scene* scene;
    int n_steps;
    Clock::time_point submitted;
};

struct Result {
    bool done = false;
    int code = IPC_OK;
    ipc_step_stats stats{};
    double latency_ms = 0.0;
};

}  // namespace

struct ipc_server {
    ipc_server_cfg cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::deque<Request> queue;
    std::unordered_map<unsigned long long, Result> results;
    std::unordered_set<ipc_scene*> running;
    unsigned long long next_ticket = 1;
    int n_running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    // index of the first admissible queued request, or -1 (mu held)
    int admissible() {
        for (size_t i = 0; i < queue.size(); ++i) {
            if (running.count(queue[i].scene)) continue;
            if (n_running > 0 && cfg.min_free_bytes > 0) {
                size_t fr = 0, tot = 0;
                if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr < cfg.min_free_bytes) return -1;
            }
            return (int)i;
        }
        return -1;
    }

    void work(int slot) {
        cudaSetDevice(device);
        cudaStream_t st = streams[slot];
        for (;;) {
            Request rq;
            {
                std::unique_lock<std::mutex> lk(mu);
                int idx = -1;
                work_cv.wait(lk, [&] {
                    idx = admissible();
                    return idx >= 0 || (stop && queue.empty());
                });
                if (idx < 0) return;  // stopping with nothing left
                rq = queue[idx];
                queue.erase(queue.begin() + idx);
                running.insert(rq.scene);
                ++n_running;
            }
            ipc_step_stats stats{};
            int code = ipc_step(rq.scene, rq.n_steps, st, &stats);
            cudaStreamSynchronize(st);
            const double ms = std::chrono::duration<double, std::milli>(Clock::now() - rq.submitted).count();
            {
                std::lock_guard<std::mutex> lk(mu);
                Result& r = results[rq.ticket];
                r.done = true;
                r.code = code;
                r.stats = stats;
                r.latency_ms = ms;
                running.erase(rq.scene);
                --n_running;
            }
            work_cv.notify_all();
            done_cv.notify_all();
        }
    }
};

extern "C" {

int ipc_server_create(const ipc_server_cfg* cfg, const ipc_alloc_fns* alloc, ipc_server** out) {
    (void)alloc;
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 256) return IPC_ERR_INVALID;
    ipc_server* s = new ipc_server;
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return IPC_ERR_CUDA;
    }
    for (int i = 0; i < cfg->slots; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
            delete s;
            return IPC_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    for (int i = 0; i < cfg->slots; ++i) s->workers.emplace_back([s, i] { s->work(i); });
    *out = s;
    return IPC_OK;
}

int ipc_server_submit(ipc_server* s, ipc_scene* scene, int n_steps, unsigned long long* ticket) {
    if (!s || !scene || n_steps < 0) return IPC_ERR_INVALID;
    unsigned long long t;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return IPC_ERR_INVALID;
        t = s->next_ticket++;
        s->results[t] = Result{};
        s->queue.push_back(Request{t, scene, n_steps, Clock::now()});
    }
    s->work_cv.notify_all();
    if (ticket) *ticket = t;
    return IPC_OK;
}

static int take_result(ipc_server* s, unsigned long long ticket, ipc_step_stats* stats, double* latency_ms) {
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return IPC_ERR_INVALID;
    if (!it->second.done) return IPC_PENDING;
    const Result r = it->second;
    s->results.erase(it);
    if (stats) *stats = r.stats;
    if (latency_ms) *latency_ms = r.latency_ms;
    return r.code;
}

int ipc_server_poll(ipc_server* s, unsigned long long ticket, ipc_step_stats* stats, double* latency_ms) {
    if (!s) return IPC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    return take_result(s, ticket, stats, latency_ms);
}

int ipc_server_wait(ipc_server* s, unsigned long long ticket, double timeout_ms, ipc_step_stats* stats,
                    double* latency_ms) {
    if (!s) return IPC_ERR_INVALID;
    // NaN or <= 0: no wait; the cap keeps the conversion to microseconds
    // defined (1e12 ms is about 30 years)
    const double ms = timeout_ms > 0.0 ? (timeout_ms < 1e12 ? timeout_ms : 1e12) : 0.0;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::microseconds((long long)(ms * 1e3));
    s->done_cv.wait_until(lk, until, [&] {
        auto it = s->results.find(ticket);
        return it == s->results.end() || it->second.done;
    });
    return take_result(s, ticket, stats, latency_ms);
}

void ipc_server_destroy(ipc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->work_cv.notify_all();
    for (std::thread& t : s->workers) t.join();
    for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
    delete s;
}

}  // extern "C"
