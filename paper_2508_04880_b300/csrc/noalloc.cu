// tusq_run_noalloc: one DFTT traversal that allocates no device memory.
//
// Some callers cannot call cudaMalloc -- for example an application whose
// device memory is owned entirely by its own pool allocator and that forbids
// allocations outside it, or a plugin host that only lends out buffers it
// allocated itself.  For them this entry point keeps every scratch buffer the
// traversal needs (the state, the device program, the drift-check records,
// the reduction partials and as many branch snapshots as fit) in one
// file-scope __device__ array of fixed size, and copies the program into it.
// The caller passes only the plan and the output buffer.
//
// In host code the array's name is a host-side stand-in, not a device
// address; the device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"
#include "program.h"

namespace tusq {
void compile_program(const tusq_plan_t &P, const CompileOpts &co, Program &prog);
cudaError_t launch_pass(const PassArgs &a, int precision, int V, int grid, cudaStream_t st);
int pass_occupancy(int precision, int V, int L, int tc);
cudaError_t launch_init(void *state, int precision, uint64_t dim, int nsm, cudaStream_t st);
cudaError_t launch_finalize(const double *partials, int nparts, double *records, int depth,
                            int is_check, double *drift_log, int check, int *restore_flag,
                            int has_snapshot, double tol, unsigned long long *counters,
                            double record_bias, cudaStream_t st);
cudaError_t launch_restore(void *state, const void *snap, int precision, uint64_t dim,
                           const int *restore_flag, int check, int nsm, cudaStream_t st);
}  // namespace tusq

using namespace tusq;

// The whole scratch of tusq_run_noalloc.  Every GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TUSQ_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("tusq_run_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return TUSQ_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("tusq_run_noalloc: device ordinal out of range");
        return TUSQ_EINVAL;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("tusq_run_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return TUSQ_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return TUSQ_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of every buffer inside the scratch array.
struct Layout {
    size_t state, snaps, records, partials, drift_log, restore_flag, counters, ops, mats, matsf, tmask,
        tphi, total;
};

Layout layout_of(const Program &pg, size_t state_bytes, int n_snaps, int max_grid) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(std::max<size_t>(bytes, 16));
        return at;
    };
    L.state = take(state_bytes);
    L.records = take(sizeof(double) * 4 * std::max(pg.max_depth, 1));
    L.partials = take(sizeof(double) * 3 * max_grid);
    L.drift_log = take(sizeof(double) * std::max(pg.n_checks, 1));
    L.restore_flag = take(sizeof(int) * std::max(pg.n_checks, 1));
    L.counters = take(sizeof(unsigned long long) * 4);
    L.ops = take(sizeof(DevOp) * pg.ops.size());
    L.mats = take(sizeof(double) * pg.mats.size());
    L.matsf = take(sizeof(float) * pg.matsf.size());
    L.tmask = take(sizeof(uint64_t) * pg.term_mask.size());
    L.tphi = take(sizeof(uint64_t) * pg.term_phi.size());
    L.snaps = take(state_bytes * (size_t)n_snaps);
    L.total = o;
    return L;
}

#define NA_TRY(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_error(std::string("tusq_run_noalloc: ") + #call + ": " + cudaGetErrorString(e_)); \
            return TUSQ_ECUDA;                                                         \
        }                                                                              \
    } while (0)

}  // namespace

extern "C" int tusq_run_noalloc(const tusq_plan_t *p, const tusq_run_opts *opts, double *probs_dev,
                                void *cuda_stream, tusq_run_info_t *info) {
    if (!p || !probs_dev) {
        set_error("tusq_run_noalloc: NULL argument");
        return TUSQ_EINVAL;
    }
    tusq_run_opts o;
    tusq_run_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != TUSQ_C64 && o.precision != TUSQ_C128) {
        set_error("tusq_run_noalloc: bad precision");
        return TUSQ_EINVAL;
    }
    if (o.traversal < TUSQ_DFTT || o.traversal > TUSQ_DFTT_SNAPSHOT) {
        set_error("tusq_run_noalloc: bad traversal");
        return TUSQ_EINVAL;
    }
    if (o.max_window != 0 && (o.max_window < 4 || o.max_window > kMaxTileBits)) {
        set_error("tusq_run_noalloc: max_window must be 0 (default) or in [4, 14]");
        return TUSQ_EINVAL;
    }
    // the same range checks as tusq_run for the options this entry ignores:
    // subtrees (one traversal), use_graph (direct launches), cache_states
    // (no DFTT+Caching cache) and tc_mode (SIMT stages only)
    if (o.subtrees < -1 || o.subtrees > 16) {
        set_error("tusq_run_noalloc: subtrees must be in [-1, 16]");
        return TUSQ_EINVAL;
    }
    if (o.cache_states < -1 || o.cache_states > 64) {
        set_error("tusq_run_noalloc: cache_states must be in [-1, 64]");
        return TUSQ_EINVAL;
    }
    if (o.tc_mode < TUSQ_TC_NONE || o.tc_mode > TUSQ_TC_TF32) {
        set_error("tusq_run_noalloc: bad tc_mode");
        return TUSQ_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t amp = o.precision == TUSQ_C128 ? 16 : 8;
    const uint64_t dim = 1ULL << p->n;
    const size_t state_bytes = amp * dim;
    if (state_bytes > TUSQ_NOALLOC_SCRATCH_BYTES / 2) {
        set_error("tusq_run_noalloc: the state (" + std::to_string(state_bytes) +
                  " bytes) does not fit the " + std::to_string((size_t)TUSQ_NOALLOC_SCRATCH_BYTES) +
                  "-byte static scratch; use tusq_run");
        return TUSQ_EINVAL;
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    int nsm = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);

    // compile with as many snapshots as the scratch can hold (at most the
    // budget in the options, at most 64)
    CompileOpts co;
    co.precision = o.precision;
    co.max_window = o.max_window;
    co.traversal = o.traversal;
    co.leaf_peek = o.leaf_peek;
    co.root_reset = o.root_reset;
    co.schedule = o.schedule;
    co.checks = o.drift_tol >= 0 && o.traversal != TUSQ_FROM_SCRATCH;
    const bool want_snaps = co.checks || o.traversal == TUSQ_DFTT_SNAPSHOT;
    uint64_t budget = o.snapshot_bytes ? o.snapshot_bytes : 8 * state_bytes;
    int k = want_snaps ? (int)std::min<uint64_t>(budget / state_bytes, 64) : 0;
    k = std::min<int>(k, (int)((TUSQ_NOALLOC_SCRATCH_BYTES - state_bytes) / state_bytes));
    Program pg;
    Layout lay;
    std::vector<int> grid;
    int max_grid = 1;
    bool sized = false;   // the snapshot count has been fitted to one compile's program size
    for (;;) {
        co.snapshots = k;
        try {
            compile_program(*p, co, pg);
        } catch (const std::exception &ex) {
            set_error(std::string("tusq_run_noalloc: schedule compilation failed: ") + ex.what());
            return TUSQ_EINVAL;
        }
        grid.assign(pg.passes.size(), 1);
        max_grid = 1;
        int occ[16] = {0};
        for (size_t i = 0; i < pg.passes.size(); ++i) {
            const PassDesc &d = pg.passes[i];
            int V = std::min(pg.reg_bits, d.L);
            if (!occ[d.L]) occ[d.L] = pass_occupancy(o.precision, V, d.L, 0);
            uint64_t g = std::min<uint64_t>(d.ntiles, (uint64_t)nsm * occ[d.L]);
            grid[i] = (int)std::max<uint64_t>(g, 1);
            max_grid = std::max(max_grid, grid[i]);
        }
        lay = layout_of(pg, state_bytes, pg.n_snap_slots, max_grid);
        if (lay.total <= TUSQ_NOALLOC_SCRATCH_BYTES) break;
        if (k == 0) {
            set_error("tusq_run_noalloc: state + device program (" + std::to_string(lay.total) +
                      " bytes) exceed the " + std::to_string((size_t)TUSQ_NOALLOC_SCRATCH_BYTES) +
                      "-byte static scratch; use tusq_run");
            return TUSQ_EINVAL;
        }
        if (!sized) {
            // the snapshots the scratch leaves room for beside this program
            // (the program barely changes with the snapshot count), then at
            // most a few more compiles stepping down
            const size_t fixed = lay.total - state_bytes * (size_t)pg.n_snap_slots;
            const size_t room = fixed < TUSQ_NOALLOC_SCRATCH_BYTES ? TUSQ_NOALLOC_SCRATCH_BYTES - fixed : 0;
            k = std::min<int>(k - 1, (int)(room / state_bytes));
            sized = true;
        } else {
            --k;
        }
        if (k < 0) k = 0;
    }
    auto at = [&](size_t off) { return (void *)(base + off); };
    double *records = (double *)at(lay.records), *partials = (double *)at(lay.partials);
    double *drift_log = (double *)at(lay.drift_log);
    int *restore_flag = (int *)at(lay.restore_flag);
    unsigned long long *counters = (unsigned long long *)at(lay.counters);
    void *state = at(lay.state), *snaps = at(lay.snaps);
    // the program: the copies read pageable host memory, which may be
    // reused once cudaMemcpyAsync returns; the device writes are ordered on
    // the stream, which is synchronised before this call returns (pg lives
    // until then)
    if (!pg.ops.empty()) NA_TRY(cudaMemcpyAsync(at(lay.ops), pg.ops.data(), sizeof(DevOp) * pg.ops.size(), cudaMemcpyHostToDevice, st));
    if (!pg.mats.empty()) NA_TRY(cudaMemcpyAsync(at(lay.mats), pg.mats.data(), sizeof(double) * pg.mats.size(), cudaMemcpyHostToDevice, st));
    if (!pg.matsf.empty()) NA_TRY(cudaMemcpyAsync(at(lay.matsf), pg.matsf.data(), sizeof(float) * pg.matsf.size(), cudaMemcpyHostToDevice, st));
    if (!pg.term_mask.empty()) NA_TRY(cudaMemcpyAsync(at(lay.tmask), pg.term_mask.data(), sizeof(uint64_t) * pg.term_mask.size(), cudaMemcpyHostToDevice, st));
    if (!pg.term_phi.empty()) NA_TRY(cudaMemcpyAsync(at(lay.tphi), pg.term_phi.data(), sizeof(uint64_t) * pg.term_phi.size(), cudaMemcpyHostToDevice, st));
    // the scratch keeps the previous call's contents: clear what must start at zero
    NA_TRY(cudaMemsetAsync(probs_dev, 0, sizeof(double) * dim, st));
    NA_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * 4, st));
    NA_TRY(cudaMemsetAsync(drift_log, 0, sizeof(double) * std::max(pg.n_checks, 1), st));
    NA_TRY(cudaMemsetAsync(restore_flag, 0, sizeof(int) * std::max(pg.n_checks, 1), st));
    NA_TRY(cudaMemsetAsync(records, 0, sizeof(double) * 4 * std::max(pg.max_depth, 1), st));
    int last_grid = 1;
    uint64_t launches = 0;
    for (const Step &s : pg.steps) {
        switch (s.type) {
        case ST_INIT:
            NA_TRY(launch_init(state, o.precision, dim, nsm, st));
            break;
        case ST_PASS: {
            PassArgs a;
            a.d = pg.passes[s.pass];
            a.src = state;
            a.state = state;
            a.snap = (a.d.flags & PF_SNAPSHOT) ? (unsigned char *)snaps + state_bytes * a.d.snap : nullptr;
            a.acc = probs_dev;
            a.partials = partials;
            a.ops = (const DevOp *)at(lay.ops);
            a.mats = (const double *)at(lay.mats);
            a.matsf = (const float *)at(lay.matsf);
            a.tmask = (const uint64_t *)at(lay.tmask);
            a.tphi = (const uint64_t *)at(lay.tphi);
            a.err = nullptr;          // no dense ops here (tc_mode is not used), so nothing waits
            a.dense_skip = 0;
            a.dpool = nullptr;
            last_grid = grid[s.pass];
            NA_TRY(launch_pass(a, o.precision, std::min(pg.reg_bits, a.d.L), last_grid, st));
            break;
        }
        case ST_RECORD:
            NA_TRY(launch_finalize(partials, last_grid, records, s.depth, 0, drift_log, 0, restore_flag, 0,
                                   o.drift_tol, counters, 0.0, st));
            break;
        case ST_CHECK:
            NA_TRY(launch_finalize(partials, last_grid, records, s.depth, 1, drift_log, s.check, restore_flag,
                                   s.snap >= 0 ? 1 : 0, o.drift_tol, counters, 0.0, st));
            break;
        case ST_RESTORE:
            NA_TRY(launch_restore(state, (unsigned char *)snaps + state_bytes * s.snap, o.precision, dim,
                                  restore_flag, s.check, nsm, st));
            break;
        default:
            set_error("tusq_run_noalloc: bad step");
            return TUSQ_EINVAL;
        }
        ++launches;
    }
    unsigned long long cnt[4] = {0, 0, 0, 0};
    NA_TRY(cudaMemcpyAsync(cnt, counters, sizeof cnt, cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->passes = pg.passes_count;
        info->gate_apps = pg.gate_apps;
        info->pauli_apps = pg.pauli_apps;
        info->leaf_passes = pg.leaf_passes;
        info->checks = pg.n_checks;
        info->restores = pg.restores + cnt[0];
        info->unrecovered = cnt[1];
        info->resets = pg.resets;
        info->kernel_launches = launches;
        info->state_bytes = (double)state_bytes;
    }
    if (cnt[1]) {
        set_error("tusq_run_noalloc: drift above tolerance at a branch node without a snapshot");
        return TUSQ_EDRIFT;
    }
    return TUSQ_OK;
}
