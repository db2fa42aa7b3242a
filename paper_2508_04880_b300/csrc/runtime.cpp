// Host runtime of the DFTT engine: compiles a plan into a device program,
// owns the device buffers (state, LIFO snapshot pool, check records) and
// enqueues the traversal on a CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
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
cudaError_t launch_sum_parts(double *out, const double *const *parts, int k, uint64_t dim, int nsm,
                             cudaStream_t st);

}  // namespace tusq

using namespace tusq;

struct tusq_exec {
    Program prog;
    tusq_run_opts opts{};
    int n = 0;
    uint64_t dim = 0;
    size_t amp_bytes = 8;
    int nsm = 148;
    int V = 5;
    cudaStream_t stream = nullptr;
    // device buffers
    void *state = nullptr;
    void *snaps = nullptr;
    int n_snaps = 0;
    double *records = nullptr;
    double *partials = nullptr;
    double *drift_log = nullptr;
    int *restore_flag = nullptr;
    unsigned long long *counters = nullptr;
    DevOp *ops = nullptr;
    double *mats = nullptr;
    float *matsf = nullptr;
    uint64_t *tmask = nullptr, *tphi = nullptr;
    float *dpool = nullptr;          // B operand parts of the dense ops
    std::vector<int> grid_of_pass;
    int max_grid = 1;
    double record_bias = 0.0;
    int dense_skip = 0;             // test hook: dense ops do not issue (their waits run out)
    // prepared on the host, not yet materialised on the device: parallel
    // subtrees still to cut from `plan` (0: none)
    int pending_parts = 0;
    const tusq_plan_t *plan = nullptr;
    bool accumulate = false;        // add into the output instead of overwriting it (streamed chunks)
    uint64_t launches = 0;
    size_t footprint = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<float> prof_ms;
    std::vector<double> prof_bytes;
    std::vector<int32_t> structure;   // 8 fields per pass in launch order
    // CUDA-graph replay of the whole traversal (use_graph)
    cudaGraphExec_t gexec = nullptr;
    double *g_probs = nullptr;
    uint64_t g_launches = 0;
    // parallel subtrees (opts.subtrees > 1): one exec per chunk of the DFS
    // order on its own stream; part 0 writes the caller's buffer, the others
    // their own, summed into it after the join
    std::vector<tusq_exec *> parts;
    std::vector<tusq_plan_t *> part_plans;
    std::vector<cudaStream_t> part_st;
    std::vector<double *> part_out;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
};

namespace {

#define CUDA_TRY(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return TUSQ_ECUDA;                                                      \
        }                                                                           \
    } while (0)

template <class T>
int dmalloc(T **p, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync((void **)p, bytes, st);
    if (e != cudaSuccess) {
        set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                  cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TUSQ_ENOMEM : TUSQ_ECUDA;
    }
    return TUSQ_OK;
}

void release(tusq_exec *e) {
    void *bufs[] = {e->state, e->snaps, e->records, e->partials, e->drift_log, e->restore_flag,
                    e->counters, e->ops, e->mats, e->matsf, e->tmask, e->tphi, e->dpool};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, e->stream);
    e->state = e->snaps = nullptr;
    e->records = e->partials = e->drift_log = nullptr;
    e->restore_flag = nullptr;
    e->counters = nullptr;
    e->ops = nullptr;
    e->mats = nullptr;
    e->matsf = nullptr;
    e->tmask = e->tphi = nullptr;
    e->dpool = nullptr;
}

}  // namespace

namespace tusq {

static CompileOpts compile_opts_of(const tusq_run_opts *o, size_t state_bytes) {
    CompileOpts co;
    co.precision = o->precision;
    co.max_window = o->max_window;
    co.traversal = o->traversal;
    co.leaf_peek = o->leaf_peek;
    co.root_reset = o->root_reset;
    co.schedule = o->schedule;
    co.checks = o->drift_tol >= 0 && o->traversal != TUSQ_FROM_SCRATCH;
    bool snaps = co.checks || o->traversal == TUSQ_DFTT_SNAPSHOT;
    co.snapshots = snaps ? (int)std::min<uint64_t>(o->snapshot_bytes / state_bytes, 64) : 0;
    co.cache_states = o->cache_states;
    co.tc_mode = o->tc_mode;
    return co;
}

// Algorithmic HBM bytes of one pass: the state read, its write (and the
// snapshot write) when asked, and the FP64 accumulator read + write of a
// leaf pass.
static double pass_bytes(const PassDesc &d, double state_bytes, uint64_t dim) {
    double b = state_bytes;
    if (d.flags & PF_WRITE) b += state_bytes;
    if (d.flags & PF_SNAPSHOT) b += state_bytes;
    if (d.flags & PF_LEAF) b += 16.0 * dim;
    return b;
}

// What a launch of the program executes, known on the host.
static void static_info(const Program &pg, size_t amp_bytes, uint64_t dim, tusq_run_info_t *info) {
    std::memset(info, 0, sizeof *info);
    info->passes = pg.passes_count;
    info->gate_apps = pg.gate_apps;
    info->pauli_apps = pg.pauli_apps;
    info->leaf_passes = pg.leaf_passes;
    info->checks = pg.n_checks;
    info->resets = pg.resets;
    info->restores = pg.restores;
    info->cache_restores = pg.cache_restores;
    info->rederives = pg.rederives;
    info->state_bytes = (double)(amp_bytes * dim);
    // every pass reads the state and writes it (and a snapshot) when asked;
    // a leaf pass also reads and writes the FP64 accumulator; a reset
    // writes the state; an unconditional restore copies a snapshot
    const double sb = info->state_bytes;
    double bytes = 0;
    uint64_t launches = 0;
    for (const Step &s : pg.steps) {
        ++launches;
        if (s.type == ST_PASS) {
            const PassDesc &d = pg.passes[s.pass];
            bytes += pass_bytes(d, sb, dim);
            info->stages += d.n_stages;
            info->diag_terms += d.nterm;
            for (uint32_t k = 0; k < d.nops; ++k) {
                const int t = pg.ops[d.op0 + k].type;
                if (t == OP_DIAG) info->diag_ops++;
                else if (t == OP_DENSE) info->dense_ops++;
                else info->matrix_ops++;
            }
        } else if (s.type == ST_INIT) {
            bytes += sb;
        } else if (s.type == ST_RESTORE && s.check < 0) {
            bytes += 2 * sb;
        }
    }
    info->kernel_launches = launches;
    info->algorithmic_bytes = bytes;
    info->program_bytes = (double)(sizeof(DevOp) * pg.ops.size() + sizeof(double) * pg.mats.size() +
                                   sizeof(float) * (pg.matsf.size() + pg.dense_pool.size()) +
                                   sizeof(uint64_t) * (pg.term_mask.size() + pg.term_phi.size()));
}

// Qubits of a full pass window (the tile of one CTA).
static int tile_bits(int n, const tusq_run_opts *o) {
    int L = o->precision == TUSQ_C128 ? 12 : 13;
    if (o->max_window > 0) L = std::min(L, o->max_window);
    return std::min(L, n);
}

// subtrees = -1: enough chunks that the passes in flight offer about twice
// the CTA slots of the GPU (slots = SMs x CTAs per SM), at most 16; one
// chunk when a single pass already has that many tiles.
static int auto_subtrees(int n, const tusq_run_opts *o, uint64_t slots) {
    const uint64_t tiles = 1ull << (n - tile_bits(n, o));
    const uint64_t k = (2 * slots + tiles - 1) / tiles;
    return (int)std::min<uint64_t>(std::max<uint64_t>(k, 1), 16);
}

// Chunks a traversal is cut into: o->subtrees, or for -1 the automatic rule
// with the current device's SM count and the pass kernel's CTAs per SM.
// exec_footprint and exec_prepare both use it, so that a job admitted by its
// footprint creates no more chunks than it paid for.
static int chunk_count(const tusq_plan_t *p, const tusq_run_opts *o) {
    if (o->subtrees >= 0) return o->subtrees;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
    const int L = tile_bits(p->n, o);
    const int V = std::min(o->precision == TUSQ_C128 ? kRegBitsC128 : kRegBitsC64, L);
    return auto_subtrees(p->n, o, (uint64_t)nsm * pass_occupancy(o->precision, V, L, 0));
}

// Device bytes an exec of this plan needs (state + snapshots + program).
size_t exec_footprint(const tusq_plan_t *p, const tusq_run_opts *o) {
    size_t amp = o->precision == TUSQ_C128 ? 16 : 8;
    size_t state = amp << p->n;
    CompileOpts co = compile_opts_of(o, state);
    int K = 0;
    if (o->traversal != TUSQ_FROM_SCRATCH && p->stats.n_noninv_layers > 0)
        K = co.cache_states < 0 ? (int)std::min<uint64_t>(p->stats.n_noninv_layers, kDefaultCacheStates)
                                : co.cache_states;
    const size_t one = state * (1 + co.snapshots + K) + (1u << 20);
    const int k = chunk_count(p, o);
    const uint64_t parts = k > 1 ? std::min<uint64_t>((uint64_t)k, std::max<uint64_t>(p->n_inst(), 1)) : 1;
    return one * parts + (parts - 1) * sizeof(double) * ((size_t)1 << p->n);
}

int compile_stats(const tusq_plan_t *p, const tusq_run_opts *o, tusq_run_info_t *info) {
    size_t amp = o->precision == TUSQ_C128 ? 16 : 8;
    Program pg;
    try {
        compile_program(*p, compile_opts_of(o, amp << p->n), pg);
        fuse_restores(pg);
    } catch (const std::exception &ex) {
        set_error(std::string("tusq_compile_stats: schedule compilation failed: ") + ex.what());
        return TUSQ_EINVAL;
    }
    static_info(pg, amp, 1ULL << p->n, info);
    return TUSQ_OK;
}

int exec_create(const tusq_plan_t *p, const tusq_run_opts *o, cudaStream_t st, tusq_exec **out);
void exec_free(tusq_exec *e);

// Parallel subtrees: the plan's DFS order cut into k chunks (tusq_plan_shard),
// one exec per chunk on its own non-blocking stream, an FP64 output per
// chunk after the first.
static int create_parts(tusq_exec *e, const tusq_plan_t *p, const tusq_run_opts *o, int k_req) {
    const int k = (int)std::min<uint64_t>((uint64_t)k_req, p->n_inst());
    tusq_run_opts so = *o;
    so.subtrees = 1;
    so.use_graph = 0;
    CUDA_TRY(cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming));
    for (int r = 0; r < k; ++r) {
        tusq_plan_t *q = nullptr;
        int rc = tusq_plan_shard(p, r, k, &q);
        if (rc != TUSQ_OK) return rc;
        e->part_plans.push_back(q);
        cudaStream_t s = nullptr;
        CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        e->part_st.push_back(s);
        cudaEvent_t ev = nullptr;
        CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        e->join_ev.push_back(ev);
        tusq_exec *x = nullptr;
        rc = exec_create(q, &so, s, &x);
        if (rc != TUSQ_OK) return rc;
        e->parts.push_back(x);
        double *buf = nullptr;
        if (r > 0 && (rc = dmalloc(&buf, sizeof(double) * e->dim, s)) != TUSQ_OK) return rc;
        e->part_out.push_back(buf);
        e->footprint += x->footprint + (r ? sizeof(double) * e->dim : 0);
    }
    for (cudaStream_t s : e->part_st) CUDA_TRY(cudaStreamSynchronize(s));
    return TUSQ_OK;
}

// Host half of creating an exec: the schedule compile and the grid of every
// pass.  No device memory is touched (only device attributes are read), so
// it can run on any host thread ahead of admission.
int exec_prepare(const tusq_plan_t *p, const tusq_run_opts *o, tusq_exec **out) {
    tusq_exec *e = new (std::nothrow) tusq_exec;
    if (!e) { set_error("tusq_exec_create: out of host memory"); return TUSQ_ENOMEM; }
    e->opts = *o;
    e->n = p->n;
    e->dim = 1ULL << p->n;
    e->amp_bytes = o->precision == TUSQ_C128 ? 16 : 8;
    e->plan = p;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e->nsm <= 0) e->nsm = 148;
    const int k_parts = chunk_count(p, o);
    if (k_parts > 1 && p->n_inst() >= 2) {
        // the chunks are cut and compiled when the exec is materialised
        e->pending_parts = k_parts;
        *out = e;
        return TUSQ_OK;
    }
    const size_t state_bytes = e->amp_bytes * e->dim;
    CompileOpts co = compile_opts_of(o, state_bytes);
    try {
        compile_program(*p, co, e->prog);
        fuse_restores(e->prog);
    } catch (const std::exception &ex) {
        delete e;
        set_error(std::string("tusq_exec_create: schedule compilation failed: ") + ex.what());
        return TUSQ_EINVAL;
    }
    Program &pg = e->prog;
    e->V = pg.reg_bits;
    e->n_snaps = pg.n_snap_slots;
    // grid of every pass
    e->grid_of_pass.resize(pg.passes.size());
    int occ_cache[4][16] = {{0}};
    for (size_t i = 0; i < pg.passes.size(); ++i) {
        const PassDesc &d = pg.passes[i];
        int V = std::min(e->V, d.L);
        const int tc = pass_dense_mode(d.flags);
        int &occ = occ_cache[tc][d.L];
        if (!occ) occ = pass_occupancy(o->precision, V, d.L, tc);
        uint64_t g = std::min<uint64_t>(d.ntiles, (uint64_t)e->nsm * occ);
        e->grid_of_pass[i] = (int)std::max<uint64_t>(g, 1);
        e->max_grid = std::max(e->max_grid, e->grid_of_pass[i]);
    }
    e->footprint = state_bytes * (1 + e->n_snaps);
    *out = e;
    return TUSQ_OK;
}

// Device half: allocate the state, snapshots, records and program buffers on
// stream st and upload the program.  On failure the exec is freed.
int exec_materialize(tusq_exec *e, cudaStream_t st) {
    e->stream = st;
    if (e->pending_parts) {
        const int rc = create_parts(e, e->plan, &e->opts, e->pending_parts);
        e->pending_parts = 0;
        if (rc != TUSQ_OK) exec_free(e);
        return rc;
    }
    Program &pg = e->prog;
    const size_t state_bytes = e->amp_bytes * e->dim;
    int rc;
#define ALLOC(ptr, bytes) \
    if ((rc = dmalloc(&(ptr), (bytes), st)) != TUSQ_OK) { release(e); delete e; return rc; }
    ALLOC(e->state, state_bytes);
    if (e->n_snaps > 0) ALLOC(e->snaps, state_bytes * e->n_snaps);
    ALLOC(e->records, sizeof(double) * 4 * std::max(pg.max_depth, 1));
    ALLOC(e->partials, sizeof(double) * 3 * e->max_grid);
    ALLOC(e->drift_log, sizeof(double) * std::max(pg.n_checks, 1));
    ALLOC(e->restore_flag, sizeof(int) * std::max(pg.n_checks, 1));
    ALLOC(e->counters, sizeof(unsigned long long) * 4);
    ALLOC(e->ops, sizeof(DevOp) * std::max<size_t>(pg.ops.size(), 1));
    ALLOC(e->mats, sizeof(double) * std::max<size_t>(pg.mats.size(), 1));
    ALLOC(e->matsf, sizeof(float) * std::max<size_t>(pg.matsf.size(), 1));
    ALLOC(e->tmask, sizeof(uint64_t) * std::max<size_t>(pg.term_mask.size(), 1));
    ALLOC(e->tphi, sizeof(uint64_t) * std::max<size_t>(pg.term_phi.size(), 1));
    if (!pg.dense_pool.empty()) ALLOC(e->dpool, sizeof(float) * pg.dense_pool.size());
#undef ALLOC
    auto up = [&](void *dst, const void *src, size_t bytes) -> int {
        if (!bytes) return TUSQ_OK;
        cudaError_t ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return TUSQ_ECUDA; }
        return TUSQ_OK;
    };
    if ((rc = up(e->ops, pg.ops.data(), sizeof(DevOp) * pg.ops.size())) ||
        (rc = up(e->mats, pg.mats.data(), sizeof(double) * pg.mats.size())) ||
        (rc = up(e->matsf, pg.matsf.data(), sizeof(float) * pg.matsf.size())) ||
        (rc = up(e->tmask, pg.term_mask.data(), sizeof(uint64_t) * pg.term_mask.size())) ||
        (rc = up(e->tphi, pg.term_phi.data(), sizeof(uint64_t) * pg.term_phi.size())) ||
        (rc = up(e->dpool, pg.dense_pool.data(), sizeof(float) * pg.dense_pool.size()))) {
        release(e);
        delete e;
        return rc;
    }
    // the program's host arrays live as long as the exec, so the copies need
    // no wait here; errors of the queued work surface at the next
    // synchronisation (tusq_exec_finish)
    return TUSQ_OK;
}

int exec_create(const tusq_plan_t *p, const tusq_run_opts *o, cudaStream_t st, tusq_exec **out) {
    tusq_exec *e = nullptr;
    int rc = exec_prepare(p, o, &e);
    if (rc != TUSQ_OK) return rc;
    rc = exec_materialize(e, st);
    if (rc != TUSQ_OK) return rc;
    *out = e;
    return TUSQ_OK;
}

static int exec_launch_direct(tusq_exec *e, double *probs, cudaStream_t st) {
    Program &pg = e->prog;
    e->stream = st;
    e->launches = 0;
    if (!e->parts.empty()) {
        // fork: every part waits for the work queued before it on st; join:
        // st waits for every part, then sums the parts' outputs (fixed order)
        CUDA_TRY(cudaEventRecord(e->fork_ev, st));
        std::vector<const double *> outs;
        for (size_t r = 0; r < e->parts.size(); ++r) {
            CUDA_TRY(cudaStreamWaitEvent(e->part_st[r], e->fork_ev, 0));
            e->parts[r]->profiling = e->profiling;
            double *o = r == 0 ? probs : e->part_out[r];
            const int rc = exec_launch_direct(e->parts[r], o, e->part_st[r]);
            if (rc != TUSQ_OK) return rc;
            e->launches += e->parts[r]->launches;
            if (r) outs.push_back(o);
            CUDA_TRY(cudaEventRecord(e->join_ev[r], e->part_st[r]));
            CUDA_TRY(cudaStreamWaitEvent(st, e->join_ev[r], 0));
        }
        CUDA_TRY(launch_sum_parts(probs, outs.data(), (int)outs.size(), e->dim, e->nsm, st));
        e->launches++;
        return TUSQ_OK;
    }
    if (!e->accumulate) CUDA_TRY(cudaMemsetAsync(probs, 0, sizeof(double) * e->dim, st));
    CUDA_TRY(cudaMemsetAsync(e->counters, 0, sizeof(unsigned long long) * 4, st));
    if (pg.n_checks) {
        CUDA_TRY(cudaMemsetAsync(e->drift_log, 0, sizeof(double) * pg.n_checks, st));
        CUDA_TRY(cudaMemsetAsync(e->restore_flag, 0, sizeof(int) * pg.n_checks, st));
    }
    const size_t state_bytes = e->amp_bytes * e->dim;
    int last_grid = 1;
    size_t npass = 0;
    if (e->profiling) {
        size_t np = 0;
        for (const Step &s : pg.steps) np += (s.type == ST_PASS);
        while (e->prof_ev.size() < 2 * np) {
            cudaEvent_t ev;
            CUDA_TRY(cudaEventCreate(&ev));
            e->prof_ev.push_back(ev);
        }
        e->prof_bytes.assign(np, 0.0);
        e->prof_ms.assign(np, 0.f);
    }
    for (const Step &s : pg.steps) {
        switch (s.type) {
        case ST_INIT:
            CUDA_TRY(launch_init(e->state, e->opts.precision, e->dim, e->nsm, st));
            e->launches++;
            break;
        case ST_PASS: {
            PassArgs a;
            a.d = pg.passes[s.pass];
            a.src = a.d.src_snap >= 0 ? (const char *)e->snaps + state_bytes * a.d.src_snap : e->state;
            a.state = e->state;
            a.snap = (a.d.flags & PF_SNAPSHOT) ? (char *)e->snaps + state_bytes * a.d.snap : nullptr;
            a.acc = probs;
            a.partials = e->partials;
            a.ops = e->ops;
            a.mats = e->mats;
            a.matsf = e->matsf;
            a.tmask = e->tmask;
            a.tphi = e->tphi;
            a.err = reinterpret_cast<unsigned int *>(e->counters + 3);
            a.dense_skip = e->dense_skip;
            a.dpool = e->dpool;
            last_grid = e->grid_of_pass[s.pass];
            if (e->profiling) CUDA_TRY(cudaEventRecord(e->prof_ev[2 * npass], st));
            CUDA_TRY(launch_pass(a, e->opts.precision, std::min(e->V, a.d.L), last_grid, st));
            if (e->profiling) {
                CUDA_TRY(cudaEventRecord(e->prof_ev[2 * npass + 1], st));
                e->prof_bytes[npass] = pass_bytes(a.d, e->amp_bytes * e->dim, e->dim);
            }
            ++npass;
            e->launches++;
            break;
        }
        case ST_RECORD:
            CUDA_TRY(launch_finalize(e->partials, last_grid, e->records, s.depth, 0, e->drift_log, 0,
                                     e->restore_flag, 0, e->opts.drift_tol, e->counters,
                                     e->record_bias, st));
            e->launches++;
            break;
        case ST_CHECK:
            CUDA_TRY(launch_finalize(e->partials, last_grid, e->records, s.depth, 1, e->drift_log,
                                     s.check, e->restore_flag, s.snap >= 0 ? 1 : 0,
                                     e->opts.drift_tol, e->counters, 0.0, st));
            e->launches++;
            break;
        case ST_RESTORE:
            CUDA_TRY(launch_restore(e->state, (char *)e->snaps + state_bytes * s.snap,
                                    e->opts.precision, e->dim, e->restore_flag, s.check, e->nsm, st));
            e->launches++;
            break;
        default:
            set_error("exec_launch: bad step");
            return TUSQ_EINVAL;
        }
    }
    return TUSQ_OK;
}

int exec_finish(tusq_exec *e, tusq_run_info_t *info) {
    CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (!e->parts.empty()) {
        // the parts' counters, summed (max for the drift); their pass
        // profiles concatenated in part order
        int rc_all = TUSQ_OK;
        tusq_run_info_t sum{};
        e->prof_ms.clear();
        e->prof_bytes.clear();
        for (tusq_exec *q : e->parts) {
            tusq_run_info_t one{};
            const int rc = exec_finish(q, &one);
            if (rc != TUSQ_OK && rc_all == TUSQ_OK) rc_all = rc;
            sum.passes += one.passes;
            sum.gate_apps += one.gate_apps;
            sum.pauli_apps += one.pauli_apps;
            sum.leaf_passes += one.leaf_passes;
            sum.checks += one.checks;
            sum.restores += one.restores;
            sum.unrecovered += one.unrecovered;
            sum.resets += one.resets;
            sum.max_drift = std::max(sum.max_drift, one.max_drift);
            sum.state_bytes = one.state_bytes;
            sum.algorithmic_bytes += one.algorithmic_bytes;
            sum.program_bytes += one.program_bytes;
            sum.stages += one.stages;
            sum.matrix_ops += one.matrix_ops;
            sum.diag_ops += one.diag_ops;
            sum.diag_terms += one.diag_terms;
            sum.cache_restores += one.cache_restores;
            sum.rederives += one.rederives;
            e->prof_ms.insert(e->prof_ms.end(), q->prof_ms.begin(), q->prof_ms.end());
            e->prof_bytes.insert(e->prof_bytes.end(), q->prof_bytes.begin(), q->prof_bytes.end());
        }
        sum.kernel_launches = e->launches;
        sum.chunks = e->parts.size();
        if (info) *info = sum;
        return rc_all;
    }
    unsigned long long cnt[4] = {0};
    CUDA_TRY(cudaMemcpy(cnt, e->counters, sizeof cnt, cudaMemcpyDeviceToHost));
    double maxd = 0;
    if (e->prog.n_checks) {
        std::vector<double> log(e->prog.n_checks);
        CUDA_TRY(cudaMemcpy(log.data(), e->drift_log, sizeof(double) * log.size(),
                            cudaMemcpyDeviceToHost));
        for (double v : log) maxd = std::max(maxd, v);
    }
    if (e->profiling)
        for (size_t i = 0; i < e->prof_ms.size(); ++i)
            CUDA_TRY(cudaEventElapsedTime(&e->prof_ms[i], e->prof_ev[2 * i], e->prof_ev[2 * i + 1]));
    if (info) {
        static_info(e->prog, e->amp_bytes, e->dim, info);
        info->restores += cnt[0];
        info->unrecovered = cnt[1];
        info->kernel_launches = e->launches;
        info->max_drift = maxd;
        info->chunks = 1;
    }
    if (cnt[3]) {
        set_error("a bounded device wait for the tensor cores ran out; the traversal stopped early");
        return TUSQ_ETIMEOUT;
    }
    if (cnt[1]) {
        set_error("drift above tolerance at a branch node without a snapshot");
        return TUSQ_EDRIFT;
    }
    return TUSQ_OK;
}

// One traversal on stream st: the launch sequence directly, or (use_graph,
// non-default stream, not profiling) a CUDA graph captured from it on the
// first call and replayed while the output buffer stays the same.
int exec_launch(tusq_exec *e, double *probs, cudaStream_t st) {
    if (!e->opts.use_graph || e->profiling || st == nullptr) return exec_launch_direct(e, probs, st);
    if (!e->gexec || e->g_probs != probs) {
        if (e->gexec) {
            cudaGraphExecDestroy(e->gexec);
            e->gexec = nullptr;
        }
        CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        const int rc = exec_launch_direct(e, probs, st);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (rc != TUSQ_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) {
            set_error(std::string("tusq_exec_launch: cudaStreamEndCapture: ") + cudaGetErrorString(ce));
            return TUSQ_ECUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&e->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            e->gexec = nullptr;
            set_error(std::string("tusq_exec_launch: cudaGraphInstantiate: ") + cudaGetErrorString(ie));
            return TUSQ_ECUDA;
        }
        e->g_probs = probs;
        e->g_launches = e->launches;
    }
    e->stream = st;
    CUDA_TRY(cudaGraphLaunch(e->gexec, st));
    e->launches = e->g_launches;
    return TUSQ_OK;
}

void exec_set_accumulate(tusq_exec *e, bool on) { e->accumulate = on; }

void exec_free(tusq_exec *e) {
    if (!e) return;
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    for (size_t r = 0; r < e->parts.size(); ++r) exec_free(e->parts[r]);
    for (size_t r = 0; r < e->part_out.size(); ++r)
        if (e->part_out[r]) cudaFreeAsync(e->part_out[r], e->part_st[r]);
    for (cudaStream_t s : e->part_st) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (tusq_plan_t *q : e->part_plans) tusq_plan_free(q);
    if (e->fork_ev) cudaEventDestroy(e->fork_ev);
    for (cudaEvent_t ev : e->join_ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : e->prof_ev) cudaEventDestroy(ev);
    const bool on_device = e->state || !e->parts.empty();
    release(e);
    // a prepared exec that never reached the device has nothing queued
    if (on_device) cudaStreamSynchronize(e->stream);
    delete e;
}

}  // namespace tusq

extern "C" {

void tusq_run_opts_default(tusq_run_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = TUSQ_C64;
    o->max_window = 0;
    o->traversal = TUSQ_DFTT;
    o->leaf_peek = 1;
    o->root_reset = 1;
    o->drift_tol = 1e-6;
    o->snapshot_bytes = 0;      // 0 -> up to 64 states within 16 GiB, at least 8 (resolved at exec creation)
    o->check_every = 0;
    o->cache_states = -1;       // one per non-invertible layer, at most 8
    o->subtrees = 1;
}

// Validate and complete run options (0 snapshot bytes -> up to 64 states
// within 16 GiB, at least 8).
static int resolve_opts(const tusq_plan_t *p, const tusq_run_opts *opts, tusq_run_opts &o,
                        const char *who) {
    tusq_run_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != TUSQ_C64 && o.precision != TUSQ_C128) {
        set_error(std::string(who) + ": bad precision");
        return TUSQ_EINVAL;
    }
    if (o.subtrees < -1 || o.subtrees > 16) {
        set_error(std::string(who) + ": subtrees must be in [-1, 16]");
        return TUSQ_EINVAL;
    }
    if (o.cache_states < -1 || o.cache_states > 64) {
        set_error(std::string(who) + ": cache_states must be in [-1, 64]");
        return TUSQ_EINVAL;
    }
    if (o.traversal < TUSQ_DFTT || o.traversal > TUSQ_DFTT_SNAPSHOT) {
        set_error(std::string(who) + ": bad traversal");
        return TUSQ_EINVAL;
    }
    if (o.tc_mode < TUSQ_TC_NONE || o.tc_mode > TUSQ_TC_TF32) {
        set_error(std::string(who) + ": tc_mode must be TUSQ_TC_NONE, TUSQ_TC_TF32X3, TUSQ_TC_BF16X3 or TUSQ_TC_TF32");
        return TUSQ_EINVAL;
    }
    if (o.max_window != 0 && (o.max_window < 4 || o.max_window > kMaxTileBits)) {
        set_error(std::string(who) + ": max_window must be 0 (default) or in [4, 14]");
        return TUSQ_EINVAL;
    }
    if (o.snapshot_bytes == 0) {
        // 64 LIFO slots when they fit in 16 GiB (deep trees then rarely fall
        // back to an unchecked uncompute), never fewer than 8
        const uint64_t state = (uint64_t)(o.precision == TUSQ_C128 ? 16 : 8) << p->n;
        o.snapshot_bytes = std::max<uint64_t>(8 * state, std::min<uint64_t>(64 * state, (uint64_t)16 << 30));
    }
    return TUSQ_OK;
}

int tusq_exec_create(const tusq_plan_t *p, const tusq_run_opts *opts, void *cuda_stream,
                     tusq_exec **out) {
    if (!p || !out) { set_error("tusq_exec_create: NULL argument"); return TUSQ_EINVAL; }
    tusq_run_opts o;
    int rc = resolve_opts(p, opts, o, "tusq_exec_create");
    if (rc) return rc;
    return exec_create(p, &o, (cudaStream_t)cuda_stream, out);
}

int tusq_compile_stats(const tusq_plan_t *p, const tusq_run_opts *opts, tusq_run_info_t *out) {
    if (!p || !out) { set_error("tusq_compile_stats: NULL argument"); return TUSQ_EINVAL; }
    tusq_run_opts o;
    int rc = resolve_opts(p, opts, o, "tusq_compile_stats");
    if (rc) return rc;
    return compile_stats(p, &o, out);
}

int tusq_exec_launch(tusq_exec *e, double *probs_dev, void *cuda_stream) {
    if (!e || !probs_dev) { set_error("tusq_exec_launch: NULL argument"); return TUSQ_EINVAL; }
    return exec_launch(e, probs_dev, (cudaStream_t)cuda_stream);
}

int tusq_exec_finish(tusq_exec *e, tusq_run_info_t *info) {
    if (!e) { set_error("tusq_exec_finish: NULL exec"); return TUSQ_EINVAL; }
    return exec_finish(e, info);
}

int tusq_exec_set_dense_skip(tusq_exec *e, int on) {
    if (!e) { set_error("tusq_exec_set_dense_skip: NULL exec"); return TUSQ_EINVAL; }
    e->dense_skip = on != 0;
    for (tusq_exec *q : e->parts) q->dense_skip = on != 0;
    return TUSQ_OK;
}

int tusq_exec_set_profiling(tusq_exec *e, int on) {
    if (!e) { set_error("tusq_exec_set_profiling: NULL exec"); return TUSQ_EINVAL; }
    e->profiling = on != 0;
    return TUSQ_OK;
}

int tusq_exec_pass_structure(tusq_exec *e, uint64_t *n_passes, const int32_t **fields) {
    if (!e || !n_passes) { set_error("tusq_exec_pass_structure: NULL argument"); return TUSQ_EINVAL; }
    if (e->structure.empty()) {
        const Program &pg = e->prog;
        for (const Step &s : pg.steps) {
            if (s.type != ST_PASS) continue;
            const PassDesc &d = pg.passes[s.pass];
            int32_t f[8] = {d.n_stages, (int32_t)d.nops, 0, 0, 0, (int32_t)d.nterm, (int32_t)d.flags, d.L};
            for (uint32_t k = 0; k < d.nops; ++k) {
                int t = pg.ops[d.op0 + k].type;
                f[t == OP_MAT1 ? 2 : (t == OP_MAT2 || t == OP_DENSE) ? 3 : 4]++;
            }
            e->structure.insert(e->structure.end(), f, f + 8);
        }
    }
    *n_passes = e->structure.size() / 8;
    if (fields) *fields = e->structure.data();
    return TUSQ_OK;
}

int tusq_exec_pass_profile(tusq_exec *e, uint64_t *n_passes, const float **ms, const double **bytes) {
    if (!e || !n_passes) { set_error("tusq_exec_pass_profile: NULL argument"); return TUSQ_EINVAL; }
    *n_passes = e->prof_ms.size();
    if (ms) *ms = e->prof_ms.data();
    if (bytes) *bytes = e->prof_bytes.data();
    return TUSQ_OK;
}

int tusq_exec_set_record_bias(tusq_exec *e, double delta) {
    if (!e) { set_error("tusq_exec_set_record_bias: NULL exec"); return TUSQ_EINVAL; }
    e->record_bias = delta;
    return TUSQ_OK;
}

void tusq_exec_free(tusq_exec *e) { exec_free(e); }

int tusq_run(const tusq_plan_t *p, const tusq_run_opts *opts, double *probs_dev, void *cuda_stream) {
    tusq_exec *e = nullptr;
    int rc = tusq_exec_create(p, opts, cuda_stream, &e);
    if (rc) return rc;
    rc = tusq_exec_launch(e, probs_dev, cuda_stream);
    if (rc == TUSQ_OK) rc = tusq_exec_finish(e, nullptr);
    tusq_exec_free(e);
    return rc;
}

}  // extern "C"

namespace tusq {
// Option validation and completion as tusq_exec_create does it (for the
// other entry points built on the exec).
int resolve_run_opts(const tusq_plan_t *p, const tusq_run_opts *opts, tusq_run_opts &o, const char *who) {
    return resolve_opts(p, opts, o, who);
}
}  // namespace tusq
