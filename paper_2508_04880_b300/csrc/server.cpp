// Serving loop with continuous batching: jobs are admitted while their
// device footprint fits the HBM budget and a stream slot is free; admitted
// jobs run concurrently on their own streams and keep their state resident
// until they finish; finished jobs free their slot and memory for the next.
//
// Host work is split so that the admission thread never compiles: a pool of
// compile threads turns each submitted job's plan into its device program
// (the schedule compile, seconds for large trees) as soon as it is
// submitted; the admission thread only retires finished jobs, and admits
// compiled ones in submission order -- allocating their buffers, uploading
// the program and launching the traversal on the job's stream.
#include <cuda_runtime.h>

#include <algorithm>
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
int exec_prepare(const tusq_plan_t *p, const tusq_run_opts *o, tusq_exec **out);
int exec_materialize(tusq_exec *e, cudaStream_t st);
int exec_launch(tusq_exec *e, double *probs, cudaStream_t st);
int exec_finish(tusq_exec *e, tusq_run_info_t *info);
void exec_free(tusq_exec *e);
}  // namespace tusq

using namespace tusq;

namespace {
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum JobState { J_COMPILING = 0, J_READY = 1, J_RUNNING = 2, J_DONE = 3 };

struct Job {
    uint64_t id = 0;
    const tusq_plan_t *plan = nullptr;
    tusq_run_opts opts{};
    double *probs = nullptr;
    size_t footprint = 0;
    double t_submit = 0, t_done = 0;
    int status = TUSQ_OK;
    int state = J_COMPILING;
    bool done = false;
    int slot = -1;
    tusq_exec *exec = nullptr;        // prepared on a compile thread, materialised at admission
    cudaEvent_t ev_start = nullptr;   // on the job's stream, around its traversal
    cudaEvent_t ev_end = nullptr;
    float dev_start_ms = -1.f, dev_end_ms = -1.f;   // since the server's reference event
};
}  // namespace

struct tusq_server {
    size_t budget = 0, in_use = 0;
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    cudaEvent_t ref = nullptr;          // device-time origin of the job intervals
    std::mutex mu;
    std::condition_variable cv;         // admission thread and drain
    std::condition_variable cv_compile; // compile threads
    std::deque<uint64_t> compile_q;     // submitted, not yet compiled
    std::deque<uint64_t> admit_q;       // submitted, not yet admitted (submission order)
    std::map<uint64_t, Job> jobs;
    uint64_t next_id = 1;
    size_t outstanding = 0;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::vector<std::thread> compilers;

    // Compile thread: prepare each submitted job's device program.
    void compile_loop() {
        cudaSetDevice(device);
        for (;;) {
            uint64_t id;
            const tusq_plan_t *plan;
            tusq_run_opts opts;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_compile.wait(lk, [this] { return stop.load() || !compile_q.empty(); });
                if (compile_q.empty()) return;      // stopping
                id = compile_q.front();
                compile_q.pop_front();
                plan = jobs[id].plan;
                opts = jobs[id].opts;
            }
            tusq_exec *e = nullptr;
            const int rc = exec_prepare(plan, &opts, &e);
            std::lock_guard<std::mutex> g(mu);
            Job &j = jobs[id];
            if (rc != TUSQ_OK) {
                j.status = rc;
                j.state = J_DONE;
                j.done = true;
                j.t_done = now_s();
                admit_q.erase(std::find(admit_q.begin(), admit_q.end(), id));
                outstanding--;
            } else {
                j.exec = e;
                j.state = J_READY;
            }
            cv.notify_all();
        }
    }

    // Retire the running jobs whose traversal has finished.
    bool retire() {
        bool did = false;
        std::vector<uint64_t> running;
        {
            std::lock_guard<std::mutex> g(mu);
            for (auto &kv : jobs)
                if (kv.second.state == J_RUNNING) running.push_back(kv.first);
        }
        for (uint64_t id : running) {
            Job *j;
            {
                std::lock_guard<std::mutex> g(mu);
                j = &jobs[id];
            }
            const cudaError_t q = cudaEventQuery(j->ev_end);
            if (q == cudaErrorNotReady) continue;
            const int rc = exec_finish(j->exec, nullptr);
            float t0 = -1.f, t1 = -1.f;
            if (q == cudaSuccess) {
                cudaEventElapsedTime(&t0, ref, j->ev_start);
                cudaEventElapsedTime(&t1, ref, j->ev_end);
            }
            exec_free(j->exec);
            cudaEventDestroy(j->ev_start);
            cudaEventDestroy(j->ev_end);
            std::lock_guard<std::mutex> g(mu);
            j->exec = nullptr;
            j->status = (q == cudaSuccess) ? rc : TUSQ_ECUDA;
            j->dev_start_ms = t0;
            j->dev_end_ms = t1;
            j->t_done = now_s();
            j->state = J_DONE;
            j->done = true;
            in_use -= j->footprint;
            slot_busy[j->slot] = false;
            outstanding--;
            did = true;
            cv.notify_all();
        }
        return did;
    }

    // Admit compiled jobs in submission order while memory and a slot are
    // free; a compiled job that does not fit blocks the ones behind it (no
    // overtaking by smaller jobs), a job still compiling does not.
    bool admit() {
        bool did = false;
        for (;;) {
            uint64_t id = 0;
            int slot = -1;
            Job *j = nullptr;
            {
                std::lock_guard<std::mutex> g(mu);
                for (uint64_t cand : admit_q) {
                    Job &c = jobs[cand];
                    if (c.state != J_READY) continue;
                    if (in_use + c.footprint > budget) break;
                    for (size_t s = 0; s < slot_busy.size(); ++s)
                        if (!slot_busy[s]) { slot = (int)s; break; }
                    if (slot < 0) break;
                    id = cand;
                    j = &c;
                    break;
                }
                if (!j) return did;
                admit_q.erase(std::find(admit_q.begin(), admit_q.end(), id));
                slot_busy[slot] = true;
                in_use += j->footprint;
                j->slot = slot;
                j->state = J_RUNNING;
            }
            cudaStream_t st = streams[slot];
            tusq_exec *e = j->exec;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            int rc = exec_materialize(e, st);    // frees e on failure
            if (rc != TUSQ_OK) e = nullptr;
            if (rc == TUSQ_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
                rc = TUSQ_ECUDA;
            if (rc == TUSQ_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = TUSQ_ECUDA;
            if (rc == TUSQ_OK) rc = exec_launch(e, j->probs, st);
            if (rc == TUSQ_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = TUSQ_ECUDA;
            std::lock_guard<std::mutex> g(mu);
            if (rc != TUSQ_OK) {
                if (e) exec_free(e);
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
                j->exec = nullptr;
                j->status = rc;
                j->state = J_DONE;
                j->done = true;
                j->t_done = now_s();
                in_use -= j->footprint;
                slot_busy[slot] = false;
                outstanding--;
                cv.notify_all();
            } else {
                j->ev_start = e0;
                j->ev_end = e1;
            }
            did = true;
        }
    }

    // Admission thread: retirement, admission and launches only.
    void loop() {
        cudaSetDevice(device);
        while (!stop.load()) {
            bool did = retire();
            did = admit() || did;
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
    if (cudaEventCreate(&s->ref) != cudaSuccess || cudaEventRecord(s->ref, s->streams[0]) != cudaSuccess) {
        set_error("tusq_server_create: cudaEventCreate failed");
        for (auto &x : s->streams) cudaStreamDestroy(x);
        if (s->ref) cudaEventDestroy(s->ref);
        delete s;
        return TUSQ_ECUDA;
    }
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nc = (int)std::min(4u, std::max(1u, hw / 2));
    for (int k = 0; k < nc; ++k) s->compilers.emplace_back([s] { s->compile_loop(); });
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
    s->compile_q.push_back(j.id);
    s->admit_q.push_back(j.id);
    s->outstanding++;
    *job_id = j.id;
    s->cv_compile.notify_one();
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

int tusq_job_state(tusq_server *s, uint64_t job_id, int *state) {
    if (!s || !state) { set_error("tusq_job_state: NULL argument"); return TUSQ_EINVAL; }
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) { set_error("tusq_job_state: unknown job id"); return TUSQ_ENOTFOUND; }
    static_assert(J_COMPILING == TUSQ_JOB_COMPILING && J_READY == TUSQ_JOB_READY &&
                  J_RUNNING == TUSQ_JOB_RUNNING && J_DONE == TUSQ_JOB_DONE, "job states");
    *state = it->second.state;
    return TUSQ_OK;
}

int tusq_poll_device_interval(tusq_server *s, uint64_t job_id, double *start_ms, double *end_ms) {
    if (!s || !start_ms || !end_ms) { set_error("tusq_poll_device_interval: NULL argument"); return TUSQ_EINVAL; }
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) { set_error("tusq_poll_device_interval: unknown job id"); return TUSQ_ENOTFOUND; }
    if (!it->second.done) { set_error("tusq_poll_device_interval: job not finished"); return TUSQ_EBUSY; }
    *start_ms = it->second.dev_start_ms;
    *end_ms = it->second.dev_end_ms;
    return it->second.status;
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
    s->cv_compile.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &t : s->compilers)
        if (t.joinable()) t.join();
    for (auto &st : s->streams) cudaStreamDestroy(st);
    if (s->ref) cudaEventDestroy(s->ref);
    delete s;
}

}  // extern "C"
