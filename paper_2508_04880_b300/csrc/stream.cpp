// Streamed traversal of a wide instance tree (tusq_run_streamed): the DFS
// order is cut into chunks of about `chunk_leaves` leaves (the subtree cut
// of tusq_plan_shard, Sec. III-B), each chunk's device program is compiled
// on host threads ahead of the GPU, and the chunks traverse one after the
// other on one stream, each from its own root state, all adding into the
// caller's output.  Only the programs of the chunks in flight exist at any
// time, so the host and device memory of the program stays bounded however
// many leaves the tree has.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <future>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace tusq {
int resolve_run_opts(const tusq_plan_t *p, const tusq_run_opts *opts, tusq_run_opts &o, const char *who);
int exec_prepare(const tusq_plan_t *p, const tusq_run_opts *o, tusq_exec **out);
int exec_materialize(tusq_exec *e, cudaStream_t st);
int exec_launch(tusq_exec *e, double *probs, cudaStream_t st);
int exec_finish(tusq_exec *e, tusq_run_info_t *info);
void exec_set_accumulate(tusq_exec *e, bool on);
void exec_free(tusq_exec *e);
}  // namespace tusq

using namespace tusq;

namespace {

struct Prepared {
    tusq_plan_t *plan = nullptr;   // the chunk's own plan (owned)
    tusq_exec *exec = nullptr;     // compiled, not yet on the device
    int rc = TUSQ_OK;
    std::string err;
};

void add_info(tusq_run_info_t &sum, const tusq_run_info_t &one) {
    sum.passes += one.passes;
    sum.gate_apps += one.gate_apps;
    sum.pauli_apps += one.pauli_apps;
    sum.leaf_passes += one.leaf_passes;
    sum.checks += one.checks;
    sum.restores += one.restores;
    sum.unrecovered += one.unrecovered;
    sum.resets += one.resets;
    sum.kernel_launches += one.kernel_launches;
    sum.max_drift = std::max(sum.max_drift, one.max_drift);
    sum.state_bytes = one.state_bytes;
    sum.algorithmic_bytes += one.algorithmic_bytes;
    sum.program_bytes = std::max(sum.program_bytes, one.program_bytes);
    sum.stages += one.stages;
    sum.matrix_ops += one.matrix_ops;
    sum.diag_ops += one.diag_ops;
    sum.diag_terms += one.diag_terms;
    sum.cache_restores += one.cache_restores;
    sum.rederives += one.rederives;
    sum.dense_ops += one.dense_ops;
}

}  // namespace

extern "C" int tusq_run_streamed(const tusq_plan_t *p, const tusq_run_opts *opts, uint64_t chunk_leaves,
                                 int compile_threads, double *probs_dev, void *cuda_stream,
                                 tusq_run_info_t *info) {
    if (!p || !probs_dev || chunk_leaves == 0 || compile_threads < 0) {
        set_error("tusq_run_streamed: NULL argument, chunk_leaves == 0 or compile_threads < 0");
        return TUSQ_EINVAL;
    }
    tusq_run_opts o;
    int rc = resolve_run_opts(p, opts, o, "tusq_run_streamed");
    if (rc) return rc;
    o.subtrees = 1;       // chunks run one after the other on the caller's stream
    o.use_graph = 0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint64_t n = p->n_inst();
    const int k = (int)std::max<uint64_t>(1, (n + chunk_leaves - 1) / chunk_leaves);
    int threads = compile_threads;
    if (threads == 0) threads = (int)std::max(1u, std::thread::hardware_concurrency() / 2);
    threads = std::max(1, std::min(threads, k));
    int dev = 0;
    cudaGetDevice(&dev);

    if (cudaMemsetAsync(probs_dev, 0, sizeof(double) << p->n, st) != cudaSuccess) {
        set_error("tusq_run_streamed: cudaMemsetAsync failed");
        return TUSQ_ECUDA;
    }
    // chunk r: cut, compile (host threads, up to `threads` chunks ahead)
    auto prepare = [p, k, dev, &o](int r) {
        Prepared pr;
        cudaSetDevice(dev);
        if (k == 1) {
            pr.rc = exec_prepare(p, &o, &pr.exec);
        } else {
            pr.rc = tusq_plan_shard(p, r, k, &pr.plan);
            if (pr.rc == TUSQ_OK) pr.rc = exec_prepare(pr.plan, &o, &pr.exec);
        }
        if (pr.rc != TUSQ_OK) pr.err = tusq_last_error();
        return pr;
    };
    std::deque<std::future<Prepared>> ahead;
    int next = 0;
    int first_err = TUSQ_OK;
    auto refill = [&]() {
        while (first_err == TUSQ_OK && (int)ahead.size() < threads && next < k)
            ahead.push_back(std::async(std::launch::async, prepare, next++));
    };
    refill();
    tusq_run_info_t sum{};
    for (int r = 0; r < k && !ahead.empty(); ++r) {
        Prepared pr = ahead.front().get();
        ahead.pop_front();
        refill();
        if (pr.rc == TUSQ_OK && first_err == TUSQ_OK) {
            tusq_exec *e = pr.exec;
            pr.exec = nullptr;
            exec_set_accumulate(e, true);
            int c = exec_materialize(e, st);     // frees e on failure
            if (c == TUSQ_OK) {
                c = exec_launch(e, probs_dev, st);
                tusq_run_info_t one{};
                const int f = exec_finish(e, &one);
                if (c == TUSQ_OK) c = f;
                add_info(sum, one);
                exec_free(e);
            }
            if (c != TUSQ_OK) first_err = c;
        } else if (pr.rc != TUSQ_OK && first_err == TUSQ_OK) {
            first_err = pr.rc;
            set_error(pr.err);
        }
        if (pr.exec) exec_free(pr.exec);
        if (pr.plan) tusq_plan_free(pr.plan);
    }
    if (info) *info = sum;
    return first_err;
}
