/*
 * tusq.h -- C ABI of the B300 DFTT noisy-statevector engine.
 *
 * The engine implements the hot path of TUSQ (arXiv 2508.04880): the Error
 * Characterization Module (ER sampling and tallying, ER commutation,
 * pruning; Sec. III-A) on the host, and Depth-First Tree Traversal (DFTT,
 * Sec. III-B) of the resulting instance tree on one GPU, accumulating the
 * tally-weighted output distribution.
 *
 * Conventions shared with callers:
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - gate kinds: see enum tusq_gate_kind; RX/RY/RZ(t) = exp(-i t sigma/2),
 *     RZZ(t) = exp(-i t Z(x)Z/2); two-qubit gates on (q0, q1) use the local
 *     basis index 2*bit(q0) + bit(q1); CX has control q0, target q1;
 *   - Pauli codes: I=0 X=1 Y=2 Z=3; a two-qubit Pauli is 4*P(q0) + P(q1).
 *
 * Errors: every function returning int returns TUSQ_OK (0) or a negative
 * status; tusq_last_error() gives a thread-local message for the last
 * failure on the calling thread.  No function aborts the process.
 * Thread safety: distinct objects may be used from distinct threads; one
 * object must not be used concurrently.
 */
#ifndef TUSQ_ABI_H_INCLUDED
#define TUSQ_ABI_H_INCLUDED

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TUSQ_OK            0
#define TUSQ_EINVAL       -1  /* bad argument (size, index, kind, probability) */
#define TUSQ_ENOMEM       -2  /* host or device allocation failed */
#define TUSQ_ENOMEM_ADMIT -3  /* serving: job footprint exceeds the HBM budget */
#define TUSQ_ECUDA        -4  /* a CUDA runtime call failed */
#define TUSQ_EDRIFT       -5  /* drift above tolerance at a node without a snapshot */
#define TUSQ_ETIMEOUT     -6  /* a bounded device wait ran out */
#define TUSQ_EBUSY        -7  /* object in use / job not finished */
#define TUSQ_ENOTFOUND    -8  /* unknown job id */

enum tusq_gate_kind {
    TUSQ_H = 0, TUSQ_X, TUSQ_Y, TUSQ_Z, TUSQ_S, TUSQ_SDG, TUSQ_T, TUSQ_TDG,
    TUSQ_RX, TUSQ_RY, TUSQ_RZ, TUSQ_U1Q, TUSQ_CX, TUSQ_CZ, TUSQ_RZZ, TUSQ_U2Q,
    /* Non-invertible one-qubit operations (Sec. III-B2: mid-circuit
     * measurements and other channels DFTT cannot back-traverse).  Each is
     * unravelled into its two Kraus branches: the state after it is the
     * unnormalised K_m psi, m = 0, 1, and every branch is a child in the
     * instance tree, so the tally-weighted sum of |psi_leaf|^2 is the exact
     * output distribution (the branch norms carry the outcome
     * probabilities; mid-circuit records are not part of the output).
     *   RESET:   K_m = |0><m|  (measure and reset to |0>)
     *   MEASURE: K_m = |m><m|  (projective Z measurement, record discarded)
     * Paulis are not commuted across them.  Consecutive ones (no other gate
     * between) form one layer: one non-invertible edge, one cache entry. */
    TUSQ_RESET = 16, TUSQ_MEASURE = 17
};

/* Event code of a Kraus-branch choice in an instance's event list: the
 * event (j, q, TUSQ_OUTCOME1) means the non-invertible gate j on qubit q
 * takes branch m = 1; without it, m = 0.  Pauli events use codes 1..3. */
#define TUSQ_OUTCOME1 4

enum tusq_precision { TUSQ_C64 = 0, TUSQ_C128 = 1 };

/* Commutation rule sets (Sec. III-A3).  PAPER: rules 1-6 -- Pauli gates,
 * same-axis rotations RX/RY/RZ, CX.  CLIFFORD (default): additionally H, S,
 * SDG, CZ by conjugation and T, TDG, RZZ for Paulis that commute with them.
 * Every rule is exact up to a global phase, so the output is unchanged. */
enum tusq_commute_mode { TUSQ_COMMUTE_OFF = 0, TUSQ_COMMUTE_PAPER = 1, TUSQ_COMMUTE_CLIFFORD = 2 };

enum tusq_traversal {
    TUSQ_DFTT = 0,          /* uncompute back to each branch point (Sec. III-B) */
    TUSQ_FROM_SCRATCH = 1,  /* every instance from |0..0> (the plain form) */
    TUSQ_DFTT_SNAPSHOT = 2  /* DFTT that restores a branch node from its LIFO
                               snapshot when it has one (loaded by the next pass instead of
                               uncomputing), uncomputing otherwise */
};

typedef struct tusq_circuit tusq_circuit;   /* opaque, library-owned */
typedef struct tusq_plan_t tusq_plan_t;     /* opaque, immutable after tusq_plan */
typedef struct tusq_exec tusq_exec;         /* opaque device program + buffers */
typedef struct tusq_server tusq_server;     /* opaque serving loop */

/* ------------------------------------------------------------- circuits */

/* New empty circuit on n_qubits (1..34).  *out is owned by the caller and
 * released with tusq_circuit_free. */
int tusq_circuit_create(int n_qubits, tusq_circuit **out);

/* Append gate `kind` on q0 (and q1 for two-qubit kinds; pass -1 otherwise).
 * params: RX/RY/RZ/RZZ take 1 angle; U1Q takes a row-major 2x2 complex
 * matrix as 8 doubles (re, im pairs); U2Q a 4x4 one as 32 doubles; other
 * kinds take none.  The matrix of U1Q/U2Q must be unitary (checked to 1e-9).
 * Returns the gate index through the return value when >= 0. */
int tusq_circuit_add_gate(tusq_circuit *c, int kind, int q0, int q1,
                          const double *params, int n_params);

/* Attach a Pauli channel right after gate gate_index, acting on that gate's
 * qubits (Sec. II: noise as a classical mixture of Pauli circuits).
 * pauli_codes[n_terms] are the non-identity outcomes (1..3 for a one-qubit
 * gate, 1..15 for a two-qubit gate), probs[n_terms] their probabilities; the
 * identity gets 1 - sum(probs), which must be >= 0.  n_terms <= 15. */
int tusq_circuit_set_channel(tusq_circuit *c, int gate_index, int n_terms,
                             const uint8_t *pauli_codes, const double *probs);

void tusq_circuit_free(tusq_circuit *c);

/* ---------------------------------------------------------------- plans */

typedef struct {
    double alpha;       /* significance threshold, Sec. III-A4 (paper: 0.01) */
    uint32_t beta;      /* insignificant instances kept, Sec. III-A4 (paper: 100) */
    int prune;          /* 0: keep every distinct instance with weight c/S */
    int commute_mode;   /* enum tusq_commute_mode */
    int n_threads;      /* host threads for sampling/commutation; 0 = all cores */
    int device_sampling;/* 1: draw the ERs of every shot on the current CUDA device
                           (same draws, same plan); 0: on the host threads */
    int terminal_fold;  /* 1: fold the Paulis left at slot G into the readout
                           (Sec. II: the output is the computational-basis
                           distribution): Z is dropped and Y becomes X, since
                           |(Z psi)_x|^2 = |psi_x|^2 and |(Y psi)_x|^2 = |(X psi)_x|^2.
                           Lossless; instances that differ only there merge
                           before pruning.  0: keep them as slot-G events */
} tusq_plan_opts;

typedef struct {
    uint64_t shots;               /* S */
    uint64_t n_channels;          /* C */
    uint64_t n_gates;             /* G = tree height in gate slots */
    uint64_t n_raw_unique;        /* distinct ERs after tallying (Sec. III-A1) */
    uint64_t n_commuted_unique;   /* distinct instances after commutation (III-A2) */
    uint64_t n_significant;       /* |C_S| */
    uint64_t n_insignificant;     /* |C_I| */
    uint64_t n_picked;            /* min(beta, |C_I|) */
    uint64_t n_instances;         /* leaves N_l = S_final (Eq. S_final), times 2^R with R
                                     RESET / MEASURE gates (one leaf per Kraus-branch record) */
    uint64_t tree_gate_edges;     /* |E| counted in gate applications */
    uint64_t dftt_gate_apps;      /* 2|E| - G: DFTT without root resets */
    uint64_t scratch_gate_apps;   /* N_l * G: every instance from scratch */
    uint64_t dftt_pauli_apps;     /* Pauli applications of the same traversal */
    uint64_t scratch_pauli_apps;
    double seconds_sample;        /* wall time of each ECM step */
    double seconds_tally;
    double seconds_commute;
    double seconds_prune_tree;
    uint64_t n_noninvertible;     /* RESET / MEASURE gates R: each kept instance has 2^R leaves */
    uint64_t n_noninv_layers;     /* their layers (runs with no other gate between) */
    uint64_t n_ecm_instances;     /* kept instances before the Kraus-branch expansion */
} tusq_plan_stats_t;

/* Run the Error Characterization Module on the host (Sec. III-A) and build
 * the DFS-ordered instance tree (Sec. III-B):
 *   1. for shot s and channel c draw r = word (c mod 4) of Philox4x64-10 at
 *      counter (s, c/4, 0, 0), key (seed, 0); the outcome is the first k with
 *      r < T_k, T_k = floor(cdf_k * 2^64) over the cumulative probabilities
 *      (identity first, cdf_0 = 1 - sum p), the last threshold being 2^64-1;
 *   2. tally identical ERs; 3. commute each distinct ER and re-tally;
 *   4. prune (significant iff c >= alpha * c_max; min(beta, |C_I|) picks by a
 *      partial Fisher-Yates over C_I in key order with draws from key
 *      (seed, 2), j = i + r mod (|C_I| - i); weights c/S and
 *      (c/S)(C_insig / sum picked c)); 5. sort instances by their event
 *      lists, ended lists last, and record the branch slot between
 *      neighbours.
 * The result is independent of n_threads.  *out is released with
 * tusq_plan_free. */
int tusq_plan(const tusq_circuit *c, const tusq_plan_opts *opts, uint64_t shots,
              uint64_t seed, tusq_plan_t **out);

int tusq_plan_stats(const tusq_plan_t *p, tusq_plan_stats_t *out);

/* Build a plan from a caller-supplied instance list instead of running the
 * ECM: n_inst instances, instance i's events are [ev_off[i], ev_off[i+1])
 * of ev_slot / ev_qubit / ev_pauli (slot in [0, G], qubit in [0, n), Pauli
 * 1..3; at most one Pauli per (slot, qubit); TUSQ_OUTCOME1 only at slot j
 * of a RESET / MEASURE gate j on its qubit, after any Pauli there), with
 * weights[i].  No Kraus-branch expansion is done: an instance without an
 * outcome event at a non-invertible gate takes branch 0 there.  The
 * instances are sorted into DFS order and the branch slots computed as in
 * tusq_plan; counts are reported as 0.  Returns TUSQ_EINVAL on a malformed
 * list (bad slot/qubit/code, unsorted or duplicate events, two identical
 * instances). */
int tusq_plan_from_instances(const tusq_circuit *c, uint64_t n_inst, const uint64_t *ev_off,
                             const int32_t *ev_slot, const int32_t *ev_qubit,
                             const int32_t *ev_pauli, const double *weights, tusq_plan_t **out);

/* Borrowed views of the kept instances, valid until tusq_plan_free:
 * instance i's events are [ev_off[i], ev_off[i+1]) of ev_slot / ev_qubit /
 * ev_pauli (slot j = before gate j, slot G = after the last gate), sorted by
 * (slot, qubit); lcp[i] (i < n_inst - 1) is the branch slot between
 * instances i and i+1. */
int tusq_plan_export(const tusq_plan_t *p, uint64_t *n_inst, const uint64_t **ev_off,
                     const int32_t **ev_slot, const int32_t **ev_qubit,
                     const int32_t **ev_pauli, const uint64_t **counts,
                     const double **weights, const int32_t **lcp);

/* Borrowed views of an intermediate tally: stage 0 = raw ERs after
 * tallying (a = channel index, b = outcome code, c unused), stage 1 =
 * commuted event lists before pruning (a = slot, b = qubit, c = Pauli).
 * Both are sorted (ended lists last). */
int tusq_plan_export_tally(const tusq_plan_t *p, int stage, uint64_t *n, const uint64_t **off,
                           const int32_t **a, const int32_t **b, const int32_t **c,
                           const uint64_t **counts);

/* Subtree sharding for several GPUs (the parallel-subtree form of DFTT,
 * Sec. III-B): the DFS-ordered instances are cut into `world` contiguous
 * chunks of nearly equal estimated work (each chunk is a set of subtrees
 * plus the path to them); *out gets chunk `rank` as its own plan with the
 * original weights, so the sum over ranks of the ranks' output
 * distributions is the full one -- the only exchange is that FP64
 * sum-reduce, done by the caller.  An empty chunk (world > N) is a plan
 * with no instances. */
int tusq_plan_shard(const tusq_plan_t *p, int rank, int world, tusq_plan_t **out);

int tusq_plan_n_qubits(const tusq_plan_t *p);
void tusq_plan_free(tusq_plan_t *p);

/* ------------------------------------------------------------ execution */

typedef struct {
    int precision;            /* enum tusq_precision (default C64) */
    int max_window;           /* qubits per fused pass tile, 0 = default */
    int traversal;            /* enum tusq_traversal */
    int leaf_peek;            /* 1: last forward pass accumulates and skips its write */
    int root_reset;           /* 1: a branch at slot 0 resets to |0..0> instead of uncomputing */
    double drift_tol;         /* drift check threshold (1e-6); < 0 disables checks */
    uint64_t snapshot_bytes;  /* device budget for LIFO branch snapshots */
    int check_every;          /* reserved, 0 */
    int schedule;             /* fusion: 0 = grow windows by the op that admits most
                                 further ops (default), 1 = in list order */
    int use_graph;            /* 1: the first tusq_exec_launch on a non-default stream
                                 captures the whole traversal into a CUDA graph; later
                                 launches with the same output buffer replay it (one
                                 host call instead of one per pass).  Ignored on the
                                 legacy default stream and while profiling. */
    int cache_states;         /* DFTT+Caching (Sec. III-B2): capacity K of the LIFO cache of
                                 states taken just before a non-invertible layer; backtracking
                                 across such a layer restores the cached state instead of
                                 uncomputing.  When more layers are on the current path than
                                 K, the K closest to the leaf are kept and a return that finds
                                 no usable state re-derives it forward from the deepest
                                 snapshot above it, or from |0..0>.  -1 (default) = one per
                                 non-invertible layer, at most 8; 0 = no cache.  Each entry is
                                 one state of device memory on top of snapshot_bytes. */
    int subtrees;             /* parallel-subtree DFTT on one GPU (Sec. III-B, subtrees traversed
                                 in parallel when memory is free): 1 (default) = one traversal;
                                 -1 = automatic (enough chunks that the passes in flight offer
                                 about twice the GPU's CTA slots: 16 for tiny states, 1 once a
                                 single pass has that many tiles);
                                 k in 2..16 = the DFS order cut into k chunks of nearly equal work
                                 (as tusq_plan_shard), each traversed by its own exec on its own
                                 stream from its own copy of the root state, the k FP64 outputs
                                 summed in a fixed order into the caller's buffer.  Pays when one
                                 pass does not fill the GPU (small states); costs k times the
                                 state, snapshot and cache memory.  tusq_compile_stats reports
                                 the single traversal. */
    int tc_mode;              /* enum tusq_tc_mode: complex64 register stages whose ops are all
                                 independent of the thread (matrix ops on the stage's register
                                 qubits, diagonal terms within them; e.g. a layer of single-qubit
                                 gates plus the CZs among those qubits) run as one 32x32 complex
                                 matrix on the tensor cores instead of op by op (Sec. II, Eq. 1:
                                 a fused gate block applied to groups of 2^k amplitudes).
                                 TUSQ_TC_NONE (default) = never. Only 13-qubit pass tiles. */
    int group_ctas;           /* batches only: most CTAs of the group running one job above one
                                 CTA's shared memory (1..16; 0 = 16); a job never gets more CTAs
                                 than its passes have tiles */
} tusq_run_opts;

/* Tensor-core precision of the dense stages (FP32 accumulation in TMEM):
 *   TF32X3  amplitudes and matrix split into TF32 hi + lo parts, three products
 *           (hi.hi + hi.lo + lo.hi): about 1e-6 relative error per stage;
 *   BF16X3  the same split in BF16: about 1e-4 relative error per stage;
 *   TF32    one TF32 product: about 1e-3 relative error per stage.
 * Only TF32X3 is meant to meet the complex64 tolerance of the output
 * (max-abs 1e-5, total variation 1e-4) on deep circuits; the other two are
 * for error studies. */
enum tusq_tc_mode { TUSQ_TC_NONE = 0, TUSQ_TC_TF32X3 = 1, TUSQ_TC_BF16X3 = 2, TUSQ_TC_TF32 = 3 };

/* Defaults: C64, window 0, DFTT, leaf_peek 1, root_reset 1, drift_tol 1e-6,
 * snapshot_bytes 0 = 64 states when they fit in 16 GiB, else 8 states,
 * cache_states -1, subtrees 1, tc_mode TUSQ_TC_NONE. */
void tusq_run_opts_default(tusq_run_opts *o);

typedef struct {
    uint64_t passes;              /* fused full-state passes launched */
    uint64_t gate_apps;           /* gate applications executed (fwd + uncompute) */
    uint64_t pauli_apps;          /* Pauli applications executed */
    uint64_t leaf_passes;
    uint64_t checks;              /* drift checks evaluated */
    uint64_t restores;            /* snapshot restores taken (device-decided) */
    uint64_t unrecovered;         /* drift above tolerance with no snapshot */
    uint64_t resets;              /* root resets */
    uint64_t kernel_launches;
    double max_drift;             /* largest drift measure seen */
    double state_bytes;           /* bytes of one state */
    double algorithmic_bytes;     /* HBM bytes the passes must move (reads + writes) */
    double program_bytes;         /* device program copied host->device at create */
    uint64_t stages;              /* register stages over all passes */
    uint64_t matrix_ops;          /* fused 2x2 / 4x4 device ops */
    uint64_t diag_ops;            /* fused diagonal-phase device ops */
    uint64_t diag_terms;          /* their terms */
    uint64_t cache_restores;      /* DFTT+Caching: returns served by a cached pre-layer state */
    uint64_t rederives;           /* returns re-derived forward from a snapshot above or |0..0>
                                     (no usable state below a non-invertible layer) */
    uint64_t dense_ops;           /* tensor-core dense ops (tc_mode): 32x32 matrices */
    uint64_t chunks;              /* parallel-subtree chunks the traversal ran as (1: one) */
} tusq_run_info_t;

/* Compile a plan into a device program for the current device and allocate
 * the state, the snapshot pool and the check records on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  Host-side work is the
 * schedule compilation (fused passes split at branch slots); the program
 * is copied to the device once. */
int tusq_exec_create(const tusq_plan_t *p, const tusq_run_opts *opts, void *cuda_stream,
                     tusq_exec **out);

/* Enqueue one DFTT traversal on `cuda_stream`: probs_dev (caller-owned
 * device buffer of 2^n doubles) is zeroed and receives
 * sum_i w_i |psi_i(x)|^2.  Stream-ordered; returns after enqueueing.  Drift
 * checks and restores are decided on the device. */
int tusq_exec_launch(tusq_exec *e, double *probs_dev, void *cuda_stream);

/* Synchronise the stream of the last launch and fill *info; returns
 * TUSQ_EDRIFT if a check failed where no snapshot was available, or
 * TUSQ_ETIMEOUT if a bounded device wait ran out (the only waits are those of
 * the tensor-core dense stages, tc_mode != TUSQ_TC_NONE). */
int tusq_exec_finish(tusq_exec *e, tusq_run_info_t *info);

/* Host only (no GPU needed): compile the plan's device program with `opts`
 * and report what a launch would execute -- passes, gate and Pauli
 * applications, leaf passes, checks, resets, kernel launches and the
 * algorithmic HBM bytes (state reads/writes of every pass, accumulator
 * traffic of leaf passes).  Counters that only the device knows
 * (restores, drift) are zero. */
int tusq_compile_stats(const tusq_plan_t *p, const tusq_run_opts *opts, tusq_run_info_t *out);

/* Profiling: when on, the next launches record a CUDA event pair around
 * every fused pass on the launch stream.  After tusq_exec_finish,
 * tusq_exec_pass_profile returns borrowed arrays (valid until the next
 * launch or tusq_exec_free) of the last launch: per pass, its device time
 * in ms and its algorithmic HBM bytes (state read + writes, accumulator
 * traffic of leaf passes). */
int tusq_exec_set_profiling(tusq_exec *e, int on);
int tusq_exec_pass_profile(tusq_exec *e, uint64_t *n_passes, const float **ms,
                           const double **bytes);

/* Structure of every pass of the compiled program, in launch order, 8
 * integers per pass: register stages, ops, 2x2 ops, 4x4 and dense ops, diagonal ops,
 * diagonal terms, flags (1 write, 2 snapshot, 4 leaf, 8 reduce), tile
 * qubits.  Borrowed, valid until tusq_exec_free. */
int tusq_exec_pass_structure(tusq_exec *e, uint64_t *n_passes, const int32_t **fields);

/* Host hook for tests: add `delta` to the recorded norm of every record
 * taken from now on (0 = off).  Forces the drift path without touching the
 * device state. */
int tusq_exec_set_record_bias(tusq_exec *e, double delta);

/* Test hook for the bounded waits of the tensor-core dense stages: when on,
 * later launches (not already captured into a CUDA graph) skip issuing the
 * tensor-core work of every dense op, so each CTA's wait for it runs out
 * after about one second of SM clock; the kernel then records the timeout,
 * stops its CTA's work, frees its tensor memory and returns, and
 * tusq_exec_finish returns TUSQ_ETIMEOUT.  The output is then incomplete.
 * Nothing faults or hangs; the context stays usable. */
int tusq_exec_set_dense_skip(tusq_exec *e, int on);

void tusq_exec_free(tusq_exec *e);

/* tusq_exec_create + launch + finish + free. */
int tusq_run(const tusq_plan_t *p, const tusq_run_opts *opts, double *probs_dev,
             void *cuda_stream);

/* Diagnostic of the tensor-core dense stage on the current device: y_t = U x_t
 * for t = 0..255 through the same device path as a dense stage of a pass
 * (one CTA of 256 threads, each holding one vector in registers).
 *   u_host : host, row-major 32x32 complex matrix as 2048 doubles (re, im);
 *   x_dev  : device, 256 x 32 complex64 (row t = vector t), read;
 *   y_dev  : device, 256 x 32 complex64, written.
 * Synchronises the stream.  TUSQ_EINVAL for a bad mode, TUSQ_ETIMEOUT if
 * the wait for the tensor cores ran out, TUSQ_ECUDA on CUDA errors. */
int tusq_dense_check(int tc_mode, const double *u_host, const float *x_dev, float *y_dev,
                     void *cuda_stream);

/* Measured FP32 and FP64 fused multiply-add throughput of the current
 * device (TFLOP/s, 2 flops per FMA): the peaks the rooflines of the SIMT
 * pass kernels are stated against.  Own kernels (eight independent FMA
 * chains per thread, 8 CTAs of 256 threads per SM), best of three timed
 * launches after a warm-up, CUDA events on cuda_stream; takes well under a
 * second.  The SM clock during the call is the caller's to sample. */
int tusq_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops, void *cuda_stream);

/* A traversal of a wide tree with bounded program memory: the DFS order is
 * cut into ceil(N_l / chunk_leaves) chunks of nearly equal work (as
 * tusq_plan_shard, the parallel-subtree cut of Sec. III-B), and the chunks
 * traverse one after the other on cuda_stream, each from its own root state,
 * all adding into probs_dev (caller-owned device buffer of 2^n doubles, zeroed
 * first; the result is the same distribution as tusq_run's).  Each chunk's
 * device program is compiled on one of `compile_threads` host threads (0 =
 * half the cores) up to that many chunks ahead of the GPU, so compilation
 * overlaps the traversal and only the programs of the chunks in flight
 * exist.  Options as tusq_run (subtrees and use_graph are not used).
 * Synchronises the stream; fills *info (optional) with the summed counters
 * (program_bytes: the largest chunk's).  Errors as tusq_run. */
int tusq_run_streamed(const tusq_plan_t *p, const tusq_run_opts *opts, uint64_t chunk_leaves,
                      int compile_threads, double *probs_dev, void *cuda_stream, tusq_run_info_t *info);

/* ------------------------------------------------------- shot sampling */

/* Shots drawn from an output distribution on the device.  The paper samples
 * the output state vector of each kept instance s_i times (Sec. III-A1);
 * tusq_run returns the exact tally-weighted mixture, and this draws `shots`
 * outcomes from it.
 *   probs_dev  : device, 2^n_qubits doubles (e.g. tusq_run's output); need
 *                not be normalised; entries <= 0 or NaN never occur.
 *   counts_dev : device, 2^n_qubits uint64, caller-owned; overwritten with
 *                the number of shots that landed on each outcome.
 * Definition (bit-exact, independent of the device): w_x = floor(p_x 2^56),
 * C_x = w_0 + ... + w_x (exact integers), W = C_(2^n - 1); shot s takes
 * r = word 0 of Philox4x64-10 at counter (s, 0, 0, 0), key (seed, 3) and
 * lands on the first x with C_x > floor(r W / 2^64).
 * Stream-ordered on cuda_stream; scratch of 8 (2^n + 2^n / 4096 + 1) bytes is
 * allocated and freed on that stream (cudaMallocAsync); the call waits for
 * the total weight once.  Returns TUSQ_EINVAL for bad arguments or a
 * distribution without positive weight, TUSQ_ECUDA for CUDA failures. */
int tusq_sample(const double *probs_dev, int n_qubits, uint64_t shots, uint64_t seed, uint64_t *counts_dev,
                void *cuda_stream);

/* ------------------------------------------------------- batched jobs */

typedef struct tusq_batch tusq_batch;   /* opaque */

/* Many jobs in one launch (the batching of Sec. III-B's traversal across
 * independent noisy simulations), of uneven size, depth and tree shape, in
 * one persistent kernel:
 *   - a job of 5..13 qubits (complex64; 4..12 complex128) runs whole in one
 *     CTA with its state in shared memory, taken from a work queue;
 *   - a larger one, up to 22 qubits (a "group job"), runs on a group of
 *     k = min(2^(n-13), 16) CTAs (2^(n-12) for complex128) with its state in
 *     global memory: each member takes its share of every pass's tiles, and
 *     the group meets at a barrier after every step that writes the state.
 *     The host assigns group jobs to CTAs before the launch (most work first,
 *     onto the CTAs that fall free earliest, one order for all), and the
 *     launch is cooperative so that every CTA is resident; a barrier's wait
 *     is bounded (about 1 s), after which the batch stops and
 *     tusq_batch_finish returns TUSQ_ETIMEOUT.
 * A CTA first runs its group-job shares, then takes queued single-CTA jobs.
 * probs_dev[j] is job j's caller-owned device output (2^n_j doubles, zeroed
 * by the kernel).
 * use_graph != 0 records the launch into a CUDA graph on the first
 * tusq_batch_launch and replays it afterwards (needs a non-default stream).
 * Options as tusq_run (leaf peek is not used: the state never leaves the
 * CTA).  tc_mode (complex64) turns the thread-independent register-stage runs
 * of 13-qubit tiles -- 13-qubit single-CTA jobs and every group job -- into
 * tensor-core dense ops as in tusq_run; each CTA of the launch then holds 128
 * TMEM columns, and a tensor-core wait that runs out stops the batch
 * (TUSQ_ETIMEOUT).  Plans and outputs must stay alive while the batch exists. */
int tusq_batch_create(const tusq_plan_t *const *plans, uint32_t n_jobs, const tusq_run_opts *opts,
                      double *const *probs_dev, int use_graph, void *cuda_stream, tusq_batch **out);
int tusq_batch_launch(tusq_batch *b, void *cuda_stream);
/* Synchronises; *info (optional) gets the summed counters of all jobs.
 * TUSQ_ETIMEOUT if a group barrier's bounded wait ran out. */
int tusq_batch_finish(tusq_batch *b, tusq_run_info_t *info);
/* Number of group jobs (jobs above one CTA's shared memory) in the batch. */
int tusq_batch_group_jobs(const tusq_batch *b);
/* Test hook for the bounded group-barrier wait: when on, later launches make
 * every group barrier wait for one member more than the group has, a
 * dependency that never resolves; each wait runs out after about one second
 * and tusq_batch_finish returns TUSQ_ETIMEOUT.  Nothing faults or hangs; the
 * batch runs normally again once the hook is off. */
int tusq_batch_set_stall_test(tusq_batch *b, int on);
void tusq_batch_free(tusq_batch *b);

/* Autotuner: times batch launches (one warm-up, one timed) while it tunes,
 * one knob at a time from *base, the traversal policy (snapshot, uncompute,
 * from scratch), the fusion schedule (window growth by lookahead or list
 * order) and, when the batch has group jobs, the CTAs per group (16, 8, 4);
 * returns the fastest options in *best (and its time in *best_ms). */
int tusq_batch_autotune(const tusq_plan_t *const *plans, uint32_t n_jobs, const tusq_run_opts *base,
                        double *const *probs_dev, void *cuda_stream, tusq_run_opts *best,
                        double *best_ms);

/* ------------------------------------------------- allocation-free run */

/* Size of the static device scratch used by tusq_run_noalloc (32 MiB). */
#define TUSQ_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/* One traversal of `p` exactly as tusq_run computes it, but without
 * allocating any device memory: for callers that cannot call cudaMalloc --
 * e.g. an application whose device memory is owned entirely by its own pool
 * allocator, or a plugin host that only lends out buffers it allocated
 * itself.  (The paper has no counterpart; this is a deployment option.)
 *
 * All scratch -- the state, the device program, the drift-check records and
 * reduction partials, and as many branch snapshots as fit -- lives in one
 * static __device__ array of TUSQ_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until exit.  The caller passes the plan and
 * probs_dev (caller-owned device buffer of 2^n doubles, zeroed here and
 * filled with sum_i w_i |psi_i|^2) and a stream (cudaStream_t, NULL = legacy
 * default stream).  No cudaMalloc, cudaFree or allocating library routine is
 * called; host memory is used for compiling the program.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array and keeps
 * the last call's contents (what must start at zero is cleared on entry):
 * calls whose work overlaps on the GPU race with each other.  The call
 * synchronises `cuda_stream` before returning and fills *info if given.
 * Options are range-checked as by tusq_run; subtrees, use_graph, cache_states
 * and tc_mode are then ignored (one traversal, direct launches, no
 * DFTT+Caching cache, SIMT stages).
 * Errors: TUSQ_EINVAL with a message when the state (more than half the
 * scratch) or state + program do not fit -- use tusq_run then; TUSQ_ECUDA,
 * TUSQ_EDRIFT as tusq_run. */
int tusq_run_noalloc(const tusq_plan_t *p, const tusq_run_opts *opts, double *probs_dev,
                     void *cuda_stream, tusq_run_info_t *info);

/* -------------------------------------------------------------- serving */

/* A serving loop that admits jobs while their device footprint
 * (state + accumulator + snapshots) fits hbm_budget_bytes, runs admitted
 * jobs concurrently on `n_streams` CUDA streams of the current device and
 * records each job's latency (submit to completion).  A pool of host threads
 * compiles each job's device program as soon as it is submitted; one
 * admission thread retires finished jobs and admits compiled ones in
 * submission order (a compiled job that does not fit the budget is not
 * overtaken). */
int tusq_server_create(size_t hbm_budget_bytes, int n_streams, tusq_server **out);

/* Queue a job; the plan must stay alive until the job completes.  probs_dev
 * is a caller-owned device buffer of 2^n doubles.  Returns TUSQ_ENOMEM_ADMIT
 * if the job alone can never fit the budget. */
int tusq_submit(tusq_server *s, const tusq_plan_t *p, const tusq_run_opts *opts,
                double *probs_dev, uint64_t *job_id);

/* Non-blocking: *done = 1 once finished (latency_s then set). */
int tusq_poll(tusq_server *s, uint64_t job_id, int *done, double *latency_s);

/* Where a submitted job is: compiling on the server's host threads, ready
 * (compiled, waiting for memory, a stream slot or the jobs submitted before
 * it), running (admitted: its program is on the device and its traversal
 * queued on its stream) or done.  Non-blocking; TUSQ_ENOTFOUND for an
 * unknown job id. */
enum tusq_job_state { TUSQ_JOB_COMPILING = 0, TUSQ_JOB_READY = 1, TUSQ_JOB_RUNNING = 2, TUSQ_JOB_DONE = 3 };
int tusq_job_state(tusq_server *s, uint64_t job_id, int *state);

/* Device-time interval of a finished job's traversal: the CUDA events
 * recorded on its stream just before its first kernel and just after its
 * last, in ms since the server was created (comparable between jobs, e.g.
 * to see that admitted jobs ran concurrently).  TUSQ_EBUSY while the job
 * runs; the job's own status once it is done. */
int tusq_poll_device_interval(tusq_server *s, uint64_t job_id, double *start_ms, double *end_ms);

/* Block until every submitted job is done. */
int tusq_server_drain(tusq_server *s);

void tusq_server_free(tusq_server *s);

/* Thread-local message for the last non-OK status on this thread. */
const char *tusq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
