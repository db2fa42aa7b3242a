// Serving loop with continuous batching: jobs are admitted while their
// device footprint fits the HBM budget and a stream slot is free; admitted
// jobs run concurrently on their own streams and keep their state resident
// until they finish; finished jobs free their slot and memory for the next.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "internal.h"

namespace tusq {
size_t exec_footprint(const tusq_plan_t *p, const tusq_run_opts *o);
int exec_create(const tusq_plan_t *p, const tusq_run_opts *o, cudaStream_t st, tusq_exec **out);
int exec_launch(tusq_exec *e, double *probs, cudaStream_t st);
int exec_finish(tusq_exec *e, tusq_run_info_t *info);
void exec_free(tusq_exec *e);
}  // namespace tusq

using namespace tusq;

namespace {
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t id = 0;
    const tusq_plan_t *plan = nullptr;
    tusq_run_opts opts{};
    double *probs = nullptr;
    size_t footprint = 0;
    double t_submit = 0, t_done = 0;
    int status = TUSQ_OK;
    bool done = false;
    int slot = -1;
    tusq_exec *exec = nullptr;
    cudaEvent_t ev = nullptr;
};
}  // namespace

struct tusq_server {
    size_t budget = 0, in_use = 0;
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Job> jobs;
    uint64_t next_id = 1;
    size_t outstanding = 0;
    std::atomic<bool> stop{false};
    std::thread worker;

    void loop() {
        cudaSetDevice(device);
        while (!stop.load()) {
            bool did = false;
            // 1. retire finished jobs
            std::vector<uint64_t> running;
            {
                std::lock_guard<std::mutex> g(mu);
                for (auto &kv : jobs)
                    if (kv.second.exec && !kv.second.done) running.push_back(kv.first);
            }
            for (uint64_t id : running) {
                Job *j;
                {
                    std::lock_guard<std::mutex> g(mu);
                    j = &jobs[id];
                }
                cudaError_t q = cudaEventQuery(j->ev);
                if (q == cudaErrorNotReady) continue;
                int rc = exec_finish(j->exec, nullptr);
                exec_free(j->exec);
                cudaEventDestroy(j->ev);
                std::lock_guard<std::mutex> g(mu);
                j->exec = nullptr;
                j->status = (q == cudaSuccess) ? rc : TUSQ_ECUDA;
                j->t_done = now_s();
                j->done = true;
                in_use -= j->footprint;
                slot_busy[j->slot] = false;
                outstanding--;
                did = true;
                cv.notify_all();
            }
            // 2. admit queued jobs (FIFO) while memory and a slot are free
            while (true) {
                uint64_t id;
                int slot = -1;
                Job *j;
                {
                    std::lock_guard<std::mutex> g(mu);
                    if (queue.empty()) break;
                    id = queue.front();
                    j = &jobs[id];
                    if (in_use + j->footprint > budget) break;
                    for (size_t s = 0; s < slot_busy.size(); ++s)
                        if (!slot_busy[s]) { slot = (int)s; break; }
                    if (slot < 0) break;
                    queue.pop_front();
                    slot_busy[slot] = true;
                    in_use += j->footprint;
                    j->slot = slot;
                }
                cudaStream_t st = streams[slot];
                tusq_exec *e = nullptr;
                int rc = exec_create(j->plan, &j->opts, st, &e);
                if (rc == TUSQ_OK) rc = exec_launch(e, j->probs, st);
                cudaEvent_t ev = nullptr;
                if (rc == TUSQ_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                    rc = TUSQ_ECUDA;
                if (rc == TUSQ_OK && cudaEventRecord(ev, st) != cudaSuccess) rc = TUSQ_ECUDA;
                std::lock_guard<std::mutex> g(mu);
                if (rc != TUSQ_OK) {
                    if (e) exec_free(e);
                    if (ev) cudaEventDestroy(ev);
                    j->status = rc;
                    j->done = true;
                    j->t_done = now_s();
                    in_use -= j->footprint;
                    slot_busy[slot] = false;
                    outstanding--;
                    cv.notify_all();
                } else {
                    j->exec = e;
                    j->ev = ev;
                }
                did = true;
            }
            if (!did) {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait_for(lk, std::chrono::microseconds(50));
            }
        }
    }
};

extern "C" {

int tusq_server_create(size_t hbm_budget_bytes, int n_streams, tusq_server **out) {
    if (!out || hbm_budget_bytes == 0 || n_streams < 1 || n_streams > 64) {
        set_error("tusq_server_create: bad argument");
        return TUSQ_EINVAL;
    }
    tusq_server *s = new (std::nothrow) tusq_server;
    if (!s) { set_error("tusq_server_create: out of host memory"); return TUSQ_ENOMEM; }
    s->budget = hbm_budget_bytes;
    cudaGetDevice(&s->device);
    s->streams.resize(n_streams);
    s->slot_busy.assign(n_streams, false);
    for (auto &st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("tusq_server_create: cudaStreamCreate failed");
            for (auto &x : s->streams) if (x) cudaStreamDestroy(x);
            delete s;
            return TUSQ_ECUDA;
        }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return TUSQ_OK;
}

int tusq_submit(tusq_server *s, const tusq_plan_t *p, const tusq_run_opts *opts, double *probs_dev,
                uint64_t *job_id) {
    if (!s || !p || !probs_dev || !job_id) { set_error("tusq_submit: NULL argument"); return TUSQ_EINVAL; }
    tusq_run_opts o;
    tusq_run_opts_default(&o);
    if (opts) o = *opts;
    if (o.snapshot_bytes == 0) o.snapshot_bytes = (uint64_t)8 * ((uint64_t)(o.precision == TUSQ_C128 ? 16 : 8) << p->n);
    Job j;
    j.plan = p;
    j.opts = o;
    j.probs = probs_dev;
    j.footprint = exec_footprint(p, &o);
    if (j.footprint > s->budget) {
        set_error("tusq_submit: job footprint exceeds the server's HBM budget");
        return TUSQ_ENOMEM_ADMIT;
    }
    j.t_submit = now_s();
    std::lock_guard<std::mutex> g(s->mu);
    j.id = s->next_id++;
    s->jobs[j.id] = j;
    s->queue.push_back(j.id);
    s->outstanding++;
    *job_id = j.id;
    s->cv.notify_all();
    return TUSQ_OK;
}

int tusq_poll(tusq_server *s, uint64_t job_id, int *done, double *latency_s) {
    if (!s || !done) { set_error("tusq_poll: NULL argument"); return TUSQ_EINVAL; }
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) { set_error("tusq_poll: unknown job id"); return TUSQ_ENOTFOUND; }
    *done = it->second.done ? 1 : 0;
    if (it->second.done) {
        if (latency_s) *latency_s = it->second.t_done - it->second.t_submit;
        if (it->second.status != TUSQ_OK) {
            set_error("tusq_poll: job failed");
            return it->second.status;
        }
    }
    return TUSQ_OK;
}

int tusq_server_drain(tusq_server *s) {
    if (!s) { set_error("tusq_server_drain: NULL server"); return TUSQ_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [s] { return s->outstanding == 0; });
    for (auto &kv : s->jobs)
        if (kv.second.status != TUSQ_OK) {
            set_error("tusq_server_drain: a job failed");
            return kv.second.status;
        }
    return TUSQ_OK;
}

void tusq_server_free(tusq_server *s) {
    if (!s) return;
    tusq_server_drain(s);
    s->stop = true;
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
