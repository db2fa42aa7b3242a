// Device program of one DFTT traversal: the layout shared by the schedule
// compiler (host C++) and the CUDA kernels/runtime.
#pragma once

#include <complex>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/tusq.h"

namespace tusq {

constexpr int kMaxTileBits = 14;     // a pass tile holds at most 2^14 amplitudes
constexpr int kMaxStages = 8;        // register stages per pass
constexpr int kRegBitsC64 = 5;       // amplitudes per thread = 2^5 (complex64)
constexpr int kRegBitsC128 = 4;      // 2^4 (complex128)

enum DevOpType : int32_t { OP_MAT1 = 1, OP_MAT2 = 2, OP_DIAG = 3, OP_DENSE = 4 };

// Structure of a matrix op (DevOp::sub), chosen on the host so the kernel
// spends fewer FMAs.  MAT1: general; real entries; and the RX-type form
// [[c, -is], [-is, c]] with a scalar factored out (tangent forms, two FMAs
// per output amplitude):
//   SUB_RXT (|c| >= |s|): c [[1, -it], [-it, 1]], t = s / c in entry 0;
//   SUB_RXS (|s| >  |c|): -is [[ik, 1], [1, ik]], k = c / s in entry 0;
// the factor (c, or -is) goes into the pass's scalar (StageDesc::kre/kim).
// MAT2: general, or a swap of two basis states (CX in some basis order).
enum DevOpSub : uint32_t { SUB_GENERAL = 0, SUB_REAL = 1, SUB_RXT = 2, SUB_RXS = 3, SUB_SWAP = 4 };

#if defined(__CUDACC__)
#define TUSQ_HD __host__ __device__ __forceinline__
#else
#define TUSQ_HD inline
#endif

// Shared-memory swizzle of a tile's local index (XOR-linear bijection).
// complex64 (8-byte elements): bits 1..3 take the xor of the higher bits in
// groups of three, bit 0 stays, so a pair (2e, 2e+1) stays adjacent for
// 16-byte accesses.  complex128 (16-byte elements): bits 0..2.
TUSQ_HD uint32_t tile_swizzle(uint32_t e, bool c128) {
    if (c128) return e ^ (((e >> 3) ^ (e >> 6) ^ (e >> 9)) & 7u);
    return e ^ ((((e >> 4) ^ (e >> 7) ^ (e >> 10)) & 7u) << 1);
}

// One operation of a stage, on the register bits of that stage.
//   MAT1: 2x2 on register bit a (row-major, basis bit a).
//   MAT2: 4x4 on register bits a < b, basis index bit_a + 2*bit_b.
//   DIAG: amp(x) *= exp(2 pi i (phi0 + sum_k phi_k parity(x & mask_k))) with
//         x the global index; phases in fixed point (2^-31 turn units for
//         complex64, 2^-63 for complex128); terms sorted by their mask
//         restricted to the register bits (mu), csr[mu]..csr[mu+1];
//         mu_mask has bit mu (>= 1) set iff that group is non-empty.
struct DevOp {
    int32_t type;
    int32_t a, b;
    uint32_t mat;          // index of the 4x4 slot in the matrix pools
    uint32_t term_begin;   // DIAG: first term
    uint32_t sub;          // DevOpSub
    uint64_t phi0;         // DIAG: constant phase (fixed point)
    uint16_t csr[34];      // DIAG: term offsets per register mask mu (relative)
    int16_t sw0, sw1;      // SUB_SWAP: the two basis states exchanged (0..3)
    uint32_t mu_mask;      // DIAG: non-empty register-mask groups mu >= 1
    uint32_t code;         // the op decoded for the kernels' single dispatch (DevCode)
};
static_assert(sizeof(DevOp) % 16 == 0, "DevOp alignment");

// Kernel dispatch code of an op: MAT1 = CODE_MAT1 + 5 sub + a (sub is
// SUB_GENERAL, SUB_REAL, SUB_RXT or SUB_RXS), MAT2 = CODE_MAT2 / CODE_SWAP + the
// index of the register pair (a, b) in (0,1) (0,2) (0,3) (0,4) (1,2) (1,3)
// (1,4) (2,3) (2,4) (3,4) order, DIAG = CODE_DIAG.  A product op
// (CODE_PROD + sub) is a run of 2x2s of one form on distinct register bits:
// `a` is the mask of those bits and bit b's matrix is entries 4b..4b+3 of
// the two matrix slots starting at `mat`.
enum DevCode : uint32_t { CODE_MAT1 = 0, CODE_MAT2 = 32, CODE_SWAP = 48, CODE_DIAG = 64, CODE_PROD = 80,
                          CODE_DENSE = 96 };

// Tensor-core dense op (OP_DENSE, code CODE_DENSE, sub = the tc mode): the
// stage's 32 registers times one 32x32 complex matrix U.  `mat` is its index
// in the dense pool: Program::dense_pool holds the B operand parts of U in the
// kernels' shared-memory layout (dense_b_words(mode) words from mat *
// dense_b_words(mode)), which the kernel copies into the pass's B region (the
// last 4 dense_b_words(mode) bytes of PassDesc::prog_bytes, which count it):
// the pass's first dense op's at kernel start, every later one's as soon as
// the op before it is done, so that the copy runs behind other work.  `a` is
// the pool index of the dense op that follows in the pass, cyclically (the
// first op of the next tile after the last); a == mat: the region already
// holds it.  Program::dense_u holds U itself (row-major, 2048 doubles from
// mat * 2048) for host-side interpreters, when CompileOpts::keep_dense_u is
// set.  Dense ops with equal B parts share one pool entry.  phi0 and the
// csr[0]..csr[1] terms are diagonal terms on fixed bits only: a per-thread
// constant phase (mu_mask is 0).  b = 1 when U is unitary: each thread's
// 32-vector then keeps its norm, which the kernel restores after the
// tensor-core product.  Only 13-qubit complex64 tiles (256 threads, V = 5)
// carry dense ops.
constexpr int kDenseTileBits = 13;
constexpr double kDenseMinCost = 24.0;   // SIMT instructions per amplitude a run must cost

// FP32 words of the B operand parts of one dense op, and their encoding from
// U (row-major 32x32 complex) into the kernels' layout.
size_t dense_b_words(int mode);
void encode_dense_b(const std::complex<double> *u, int mode, float *out);

TUSQ_HD constexpr uint32_t pair_code(int lo, int hi) {
    return (uint32_t)(lo * (9 - lo) / 2 + (hi - lo - 1));
}

struct StageDesc {
    uint8_t rbits[8];      // local bit positions held in registers (ascending)
    uint8_t cpos[16];      // remaining local bit positions (ascending) -> thread bits
    uint16_t sr[32];       // swizzled shared-memory offset of register index r
    uint8_t cglob[16];     // global position of each thread bit (win[cpos[i]])
    uint64_t greg[8];      // global bit of each register bit (1 << win[rbits[i]])
    uint32_t op_begin, op_count;
    // kflag != 0: multiply every amplitude by kre + i kim when the stage
    // ends -- the product of the factors the tangent forms of the pass took
    // out (a scalar commutes with every op, so the compiler puts it on one
    // stage of the pass, preferably one that multiplies by a per-thread
    // phase anyway)
    double kre, kim;
    uint32_t kflag, kpad;
};

// Per-pass program limits: a pass's ops, matrices and diagonal terms are
// copied into shared memory next to the tile.
constexpr int kMaxStageOps = 48;
constexpr int kMaxDiagTerms = 256;
constexpr uint32_t kMaxPassProgramBytes = 40 * 1024;

enum PassFlags : uint32_t {
    PF_WRITE = 1,          // write the tile back to the state
    PF_SNAPSHOT = 2,       // also write it to the snapshot buffer
    PF_LEAF = 4,           // acc[x] += w |psi_x|^2
    PF_REDUCE = 8,         // partial sums of |psi|^2 and sum h(x) psi_x
    PF_DENSE = 16,         // has tensor-core dense ops (TMEM is allocated)
};
// A PF_DENSE pass holds its dense ops' tc mode (tusq_tc_mode) in flag bits
// 8-9: the kernels are instantiated once per mode.
constexpr int kDenseModeShift = 8;
TUSQ_HD constexpr int pass_dense_mode(uint32_t flags) {
    return (flags & PF_DENSE) ? (int)((flags >> kDenseModeShift) & 3u) : 0;
}

struct PassDesc {
    int32_t L;             // tile = 2^L amplitudes
    int32_t n_stages;
    int32_t n_cw;          // number of tile-index bits
    uint32_t flags;
    uint64_t ntiles;
    uint8_t win[16];       // local bit i <-> global bit win[i]
    uint8_t cw[40];        // global positions of the tile-index bits (ascending)
    uint64_t cwmask;       // the same positions as a mask
    uint64_t grow[32];     // global offset of load row i (local index i * T)
    uint16_t srow[32];     // swizzled shared offset of load row i
    StageDesc st[kMaxStages];
    double leaf_w;
    int32_t snap;          // snapshot slot for PF_SNAPSHOT
    int32_t src_snap;      // >= 0: load the tiles from this snapshot slot instead
                           // of the state (an unconditional restore fused into
                           // the pass that follows it); -1: from the state
    uint32_t prog_bytes;   // shared-memory bytes of the program below
    uint32_t op0, nops;    // the pass's ops: [op0, op0 + nops) of Program::ops
    uint32_t mat0, nmat;   // its matrix slots
    uint32_t term0, nterm; // its diagonal terms
};

// Host-side step of the traversal.
enum StepType : int32_t {
    ST_INIT = 1,           // state <- |0..0>
    ST_PASS = 2,           // fused pass (PassDesc index)
    ST_RECORD = 3,         // partial sums -> record[depth]
    ST_CHECK = 4,          // partial sums vs record[depth] -> drift log; flag restore
    ST_RESTORE = 5,        // if flagged: state <- snapshot[snap]
};

struct Step {
    int32_t type;
    int32_t pass;          // ST_PASS
    int32_t depth;         // ST_RECORD / ST_CHECK
    int32_t snap;          // ST_CHECK / ST_RESTORE (-1: none)
    int32_t check;         // index into the drift log
};

struct Program {
    int n = 0;
    int precision = 0;
    int reg_bits = 5;
    std::vector<Step> steps;
    std::vector<PassDesc> passes;
    std::vector<DevOp> ops;
    std::vector<double> mats;        // 32 doubles (16 complex) per matrix slot
    std::vector<float> matsf;        // the same slots in FP32 (complex64 kernels)
    // dense ops: their B operand parts (FP32 words, dense_b_words(mode) per
    // op) and their matrices U (2048 doubles per op), indexed by DevOp::mat
    std::vector<float> dense_pool;
    std::vector<double> dense_u;
    std::vector<uint64_t> term_mask;
    std::vector<uint64_t> term_phi;
    int max_depth = 0;
    int n_checks = 0;
    int n_snapshots = 0;
    // counters
    uint64_t gate_apps = 0, pauli_apps = 0, passes_count = 0, leaf_passes = 0, resets = 0;
    uint64_t restores = 0;           // unconditional snapshot restores (snapshot policy)
    uint64_t cache_restores = 0;     // returns served by a cached pre-layer state
    uint64_t rederives = 0;          // returns re-derived forward (saved state above, or |0..0>)
    int n_snap_slots = 0;            // snapshot slots the steps use (branch + cache)
};

// Arguments of one pass launch.
struct PassArgs {
    PassDesc d;
    const void *src;      // tiles are loaded from here (the state or a snapshot)
    void *state;
    void *snap;           // snapshot buffer for PF_SNAPSHOT
    double *acc;          // FP64 output for PF_LEAF
    double *partials;     // 3 doubles per CTA for PF_REDUCE
    const DevOp *ops;
    const double *mats;
    const float *matsf;
    const uint64_t *tmask;
    const uint64_t *tphi;
    unsigned int *err;    // bit 0 set when a bounded device wait ran out
    int dense_skip;       // test hook: dense ops never issue their tensor-core work
    int pad;
    const float *dpool;   // B operand parts of the dense ops (Program::dense_pool)
};

// One job of a batch launch: its steps in the batch's step array (pass,
// op, matrix and term indices already relocated into the batch arrays), its
// size and its device buffers.
struct JobDesc {
    uint32_t step0, nsteps;
    int32_t n;
    int32_t group_k;       // 0: the job runs in one CTA with its state in shared
                           // memory; k > 0: a group of k CTAs runs it with the
                           // state in global memory, meeting at a barrier after
                           // every pass
    double *acc;           // 2^n FP64 output (zeroed by the kernel)
    void *snaps;           // snapshot slots, 2^n amplitudes each
    double *records;       // 4 doubles per record depth
    void *state;           // group jobs: the state (2^n amplitudes)
    double *partials;      // group jobs: 3 doubles per group member (norm, checksum)
    unsigned int *bar;     // group jobs: barrier counter (zeroed before each launch)
};

// One entry of a CTA's group-job list: the job and the CTA's rank in its group.
struct GroupEntry {
    uint32_t job, rank;
};

// Batched jobs above one CTA's shared memory run on groups of at most
// kMaxGroupSize CTAs; the largest state a batch takes (32 MiB complex64).
constexpr int kMaxGroupSize = 16;
constexpr int kMaxGroupJobQubits = 22;

struct BatchArgs {
    const JobDesc *jobs;
    int32_t n_jobs;
    int32_t pad;
    const Step *steps;
    const PassDesc *passes;
    const DevOp *ops;
    const double *mats;
    const float *matsf;
    const uint64_t *tmask;
    const uint64_t *tphi;
    unsigned int *next_job;          // work queue head (zeroed before each launch)
    unsigned long long *counters;    // [0] restores after failed checks, [1] unrecovered drift
    double drift_tol;
    // group jobs: CTA b runs the (job, rank) entries assign[assign_off[b] ..
    // assign_off[b + 1]) in that order -- one global order of the group jobs,
    // so no two CTAs wait for each other the other way round -- then takes
    // single-CTA jobs small_ids[next_job++] until none is left
    const GroupEntry *assign;
    const uint32_t *assign_off;
    const uint32_t *small_ids;
    int32_t n_small;
    int32_t stall_test;              // test hook: group barriers wait for one member too many
    unsigned int *abort;             // set when a bounded wait ran out (group barrier or tensor cores)
    unsigned int *err;               // bit 0: a bounded wait ran out
    const float *dpool;              // B operand parts of the jobs' dense ops (relocated pool indices)
};

// Fuse every unconditional snapshot restore into the pass that follows it
// when that pass writes the state, or when the state buffer is not read
// again before the next restore or reset: the pass loads its tiles from the
// snapshot and the copy pass disappears.
void fuse_restores(Program &prog);

struct CompileOpts {
    int precision;
    int max_window;
    int traversal;
    int leaf_peek;
    int root_reset;
    bool checks;
    int snapshots;         // snapshot slots available for branch nodes
    int schedule;          // 0 lookahead window growth, 1 list order
    int cache_states = 0;  // DFTT+Caching capacity; < 0: one per layer, at most kDefaultCacheStates
    int tc_mode = TUSQ_TC_NONE;  // tensor-core dense stages (complex64 only)
    bool keep_dense_u = false;   // also store each dense op's U in Program::dense_u (host interpreters)
};

constexpr int kDefaultCacheStates = 8;

}  // namespace tusq
