"""Thin Python binding of libtusq (the B300 DFTT noisy-statevector engine).

Argument marshalling only: every step runs in the C++ planner or in the
CUDA kernels of ``libtusq.so``.  PyTorch is used by callers for device
buffers and streams; pass ``tensor.data_ptr()`` and
``torch.cuda.current_stream().cuda_stream``.

The functions keep the C names (``tusq_plan``, ``tusq_exec_create``, ...);
``Plan`` / ``Exec`` wrap the handles so that they are freed.
The first call fails loudly (ImportError) if the shared object is missing
or does not load; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtusq.so")

TUSQ_OK, TUSQ_EINVAL, TUSQ_ENOMEM, TUSQ_ENOMEM_ADMIT, TUSQ_ECUDA, TUSQ_EDRIFT, \
    TUSQ_ETIMEOUT, TUSQ_EBUSY, TUSQ_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7, -8
C64, C128 = 0, 1
COMMUTE_OFF, COMMUTE_PAPER, COMMUTE_CLIFFORD = 0, 1, 2
DFTT, FROM_SCRATCH, DFTT_SNAPSHOT = 0, 1, 2
TC_NONE, TC_TF32X3, TC_BF16X3, TC_TF32 = 0, 1, 2, 3
JOB_COMPILING, JOB_READY, JOB_RUNNING, JOB_DONE = 0, 1, 2, 3

# Every symbol include/tusq.h declares.
EXPORTS = [
    "tusq_circuit_create", "tusq_circuit_add_gate", "tusq_circuit_set_channel", "tusq_circuit_free",
    "tusq_plan", "tusq_plan_stats", "tusq_plan_from_instances", "tusq_plan_export",
    "tusq_plan_export_tally",
    "tusq_plan_n_qubits", "tusq_plan_shard", "tusq_plan_free", "tusq_run_opts_default",
    "tusq_exec_create",
    "tusq_exec_launch", "tusq_exec_finish", "tusq_compile_stats", "tusq_exec_set_record_bias",
    "tusq_exec_set_profiling", "tusq_exec_set_dense_skip", "tusq_exec_pass_profile", "tusq_exec_pass_structure", "tusq_exec_free",
    "tusq_run", "tusq_run_noalloc", "tusq_run_streamed", "tusq_dense_check", "tusq_measure_alu_peaks", "tusq_sample", "tusq_batch_create", "tusq_batch_launch", "tusq_batch_finish",
    "tusq_batch_free", "tusq_batch_group_jobs", "tusq_batch_set_stall_test", "tusq_batch_autotune", "tusq_server_create", "tusq_submit", "tusq_poll",
    "tusq_poll_device_interval", "tusq_job_state", "tusq_server_drain",
    "tusq_server_free", "tusq_last_error",
]


class TusqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tusq error {code}: {msg}")
        self.code = code


class PlanOpts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_uint32), ("prune", ctypes.c_int),
                ("commute_mode", ctypes.c_int), ("n_threads", ctypes.c_int), ("device_sampling", ctypes.c_int),
                ("terminal_fold", ctypes.c_int)]


class PlanStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in (
        "shots", "n_channels", "n_gates", "n_raw_unique", "n_commuted_unique", "n_significant",
        "n_insignificant", "n_picked", "n_instances", "tree_gate_edges", "dftt_gate_apps",
        "scratch_gate_apps", "dftt_pauli_apps", "scratch_pauli_apps")] + \
        [(f, ctypes.c_double) for f in ("seconds_sample", "seconds_tally", "seconds_commute",
                                        "seconds_prune_tree")] + \
        [(f, ctypes.c_uint64) for f in ("n_noninvertible", "n_noninv_layers", "n_ecm_instances")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RunOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_window", ctypes.c_int), ("traversal", ctypes.c_int),
                ("leaf_peek", ctypes.c_int), ("root_reset", ctypes.c_int), ("drift_tol", ctypes.c_double),
                ("snapshot_bytes", ctypes.c_uint64), ("check_every", ctypes.c_int),
                ("schedule", ctypes.c_int), ("use_graph", ctypes.c_int), ("cache_states", ctypes.c_int),
                ("subtrees", ctypes.c_int), ("tc_mode", ctypes.c_int), ("group_ctas", ctypes.c_int)]


class RunInfo(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in (
        "passes", "gate_apps", "pauli_apps", "leaf_passes", "checks", "restores", "unrecovered",
        "resets", "kernel_launches")] + \
        [(f, ctypes.c_double) for f in ("max_drift", "state_bytes", "algorithmic_bytes",
                                        "program_bytes")] + \
        [(f, ctypes.c_uint64) for f in ("stages", "matrix_ops", "diag_ops", "diag_terms", "cache_restores",
                                        "rederives", "dense_ops", "chunks")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtusq.so is missing at {LIB_PATH}; build it with "
                          "`python -m paper_2508_04880_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i32, u64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    sig = {
        "tusq_circuit_create": (i32, [i32, P(vp)]),
        "tusq_circuit_add_gate": (i32, [vp, i32, i32, i32, P(f64), i32]),
        "tusq_circuit_set_channel": (i32, [vp, i32, i32, P(ctypes.c_uint8), P(f64)]),
        "tusq_circuit_free": (None, [vp]),
        "tusq_plan": (i32, [vp, P(PlanOpts), u64, u64, P(vp)]),
        "tusq_plan_stats": (i32, [vp, P(PlanStats)]),
        "tusq_plan_from_instances": (i32, [vp, u64, P(u64), P(ctypes.c_int32), P(ctypes.c_int32),
                                           P(ctypes.c_int32), P(f64), P(vp)]),
        "tusq_plan_export": (i32, [vp, P(u64), P(P(u64)), P(P(ctypes.c_int32)), P(P(ctypes.c_int32)),
                                   P(P(ctypes.c_int32)), P(P(u64)), P(P(f64)), P(P(ctypes.c_int32))]),
        "tusq_plan_export_tally": (i32, [vp, i32, P(u64), P(P(u64)), P(P(ctypes.c_int32)),
                                         P(P(ctypes.c_int32)), P(P(ctypes.c_int32)), P(P(u64))]),
        "tusq_plan_n_qubits": (i32, [vp]),
        "tusq_plan_shard": (i32, [vp, i32, i32, P(vp)]),
        "tusq_plan_free": (None, [vp]),
        "tusq_run_opts_default": (None, [P(RunOpts)]),
        "tusq_exec_create": (i32, [vp, P(RunOpts), vp, P(vp)]),
        "tusq_exec_launch": (i32, [vp, vp, vp]),
        "tusq_exec_finish": (i32, [vp, P(RunInfo)]),
        "tusq_exec_set_record_bias": (i32, [vp, f64]),
        "tusq_compile_stats": (i32, [vp, P(RunOpts), P(RunInfo)]),
        "tusq_exec_set_profiling": (i32, [vp, i32]),
        "tusq_exec_set_dense_skip": (i32, [vp, i32]),
        "tusq_exec_pass_profile": (i32, [vp, P(u64), P(P(ctypes.c_float)), P(P(f64))]),
        "tusq_exec_pass_structure": (i32, [vp, P(u64), P(P(ctypes.c_int32))]),
        "tusq_exec_free": (None, [vp]),
        "tusq_run": (i32, [vp, P(RunOpts), vp, vp]),
        "tusq_run_noalloc": (i32, [vp, P(RunOpts), vp, vp, P(RunInfo)]),
        "tusq_run_streamed": (i32, [vp, P(RunOpts), u64, i32, vp, vp, P(RunInfo)]),
        "tusq_dense_check": (i32, [i32, P(f64), vp, vp, vp]),
        "tusq_measure_alu_peaks": (i32, [P(f64), P(f64), vp]),
        "tusq_sample": (i32, [vp, i32, u64, u64, vp, vp]),
        "tusq_batch_create": (i32, [P(vp), ctypes.c_uint32, P(RunOpts), P(vp), i32, vp, P(vp)]),
        "tusq_batch_launch": (i32, [vp, vp]),
        "tusq_batch_finish": (i32, [vp, P(RunInfo)]),
        "tusq_batch_free": (None, [vp]),
        "tusq_batch_group_jobs": (i32, [vp]),
        "tusq_batch_set_stall_test": (i32, [vp, i32]),
        "tusq_batch_autotune": (i32, [P(vp), ctypes.c_uint32, P(RunOpts), P(vp), vp, P(RunOpts), P(f64)]),
        "tusq_server_create": (i32, [ctypes.c_size_t, i32, P(vp)]),
        "tusq_submit": (i32, [vp, vp, P(RunOpts), vp, P(u64)]),
        "tusq_poll": (i32, [vp, u64, P(i32), P(f64)]),
        "tusq_poll_device_interval": (i32, [vp, u64, P(f64), P(f64)]),
        "tusq_job_state": (i32, [vp, u64, P(i32)]),
        "tusq_server_drain": (i32, [vp]),
        "tusq_server_free": (None, [vp]),
        "tusq_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


class _LazyLib:
    """Loads libtusq.so on first use (so that the build module can be
    imported before the library exists); raises if it is missing."""
    _L = None

    def __getattr__(self, name):
        if _LazyLib._L is None:
            _LazyLib._L = _load()
        return getattr(_LazyLib._L, name)


lib = _LazyLib()


def _check(rc: int, what: str = "") -> int:
    if rc < 0:
        raise TusqError(rc, (lib.tusq_last_error() or b"").decode() or what)
    return rc


# ------------------------------------------------------------------ circuits

class Circuit:
    """Owns a tusq_circuit handle."""

    def __init__(self, n_qubits: int):
        h = ctypes.c_void_p()
        _check(lib.tusq_circuit_create(n_qubits, ctypes.byref(h)))
        self.h = h
        self.n_qubits = n_qubits

    def add_gate(self, kind: int, q0: int, q1: int = -1, params=()) -> int:
        arr = (ctypes.c_double * max(len(params), 1))(*params)
        return _check(lib.tusq_circuit_add_gate(self.h, kind, q0, q1, arr, len(params)))

    def set_channel(self, gate_index: int, codes, probs) -> None:
        c = (ctypes.c_uint8 * max(len(codes), 1))(*codes)
        p = (ctypes.c_double * max(len(probs), 1))(*probs)
        _check(lib.tusq_circuit_set_channel(self.h, gate_index, len(codes), c, p))

    def __del__(self):
        if getattr(self, "h", None):
            lib.tusq_circuit_free(self.h)
            self.h = None


def circuit_from(wc) -> Circuit:
    """Marshal a ``tusq_workloads.Circuit`` into a library circuit."""
    c = Circuit(wc.n_qubits)
    for j, (kind, q0, q1, params) in enumerate(wc.gates):
        c.add_gate(kind, q0, q1, params)
        ch = wc.channels[j]
        if ch is not None:
            c.set_channel(j, ch[0], ch[1])
    return c


# --------------------------------------------------------------------- plans

class Plan:
    """Owns a tusq_plan_t handle; exposes the stats and the exported views."""

    def __init__(self, h, n_qubits: int):
        self.h = h
        self.n_qubits = n_qubits

    def __del__(self):
        if getattr(self, "h", None):
            lib.tusq_plan_free(self.h)
            self.h = None

    def shard(self, rank: int, world: int) -> "Plan":
        """Contiguous DFS chunk `rank` of `world` (subtree sharding); the
        ranks' output distributions sum to this plan's."""
        h = ctypes.c_void_p()
        _check(lib.tusq_plan_shard(self.h, rank, world, ctypes.byref(h)))
        return Plan(h, self.n_qubits)

    def stats(self) -> dict:
        s = PlanStats()
        _check(lib.tusq_plan_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def instances(self):
        """(events per instance, counts, weights, lcp) as Python/numpy data."""
        n = ctypes.c_uint64()
        P = ctypes.POINTER
        off, sl, qb, pa = P(ctypes.c_uint64)(), P(ctypes.c_int32)(), P(ctypes.c_int32)(), P(ctypes.c_int32)()
        cnt, w, lcp = P(ctypes.c_uint64)(), P(ctypes.c_double)(), P(ctypes.c_int32)()
        _check(lib.tusq_plan_export(self.h, ctypes.byref(n), ctypes.byref(off), ctypes.byref(sl),
                                    ctypes.byref(qb), ctypes.byref(pa), ctypes.byref(cnt),
                                    ctypes.byref(w), ctypes.byref(lcp)))
        N = n.value
        offs = np.ctypeslib.as_array(off, (N + 1,)).copy()
        ne = int(offs[-1])
        s_ = np.ctypeslib.as_array(sl, (ne,)).copy() if ne else np.zeros(0, np.int32)
        q_ = np.ctypeslib.as_array(qb, (ne,)).copy() if ne else np.zeros(0, np.int32)
        p_ = np.ctypeslib.as_array(pa, (ne,)).copy() if ne else np.zeros(0, np.int32)
        inst = [tuple(zip(s_[offs[i]:offs[i + 1]].tolist(), q_[offs[i]:offs[i + 1]].tolist(),
                          p_[offs[i]:offs[i + 1]].tolist())) for i in range(N)]
        counts = np.ctypeslib.as_array(cnt, (N,)).copy() if N else np.zeros(0, np.uint64)
        weights = np.ctypeslib.as_array(w, (N,)).copy() if N else np.zeros(0)
        lcps = np.ctypeslib.as_array(lcp, (N - 1,)).copy() if N > 1 else np.zeros(0, np.int32)
        return inst, counts, weights, lcps

    def tally(self, stage: int):
        n = ctypes.c_uint64()
        P = ctypes.POINTER
        off, a, b, c, cnt = P(ctypes.c_uint64)(), P(ctypes.c_int32)(), P(ctypes.c_int32)(), \
            P(ctypes.c_int32)(), P(ctypes.c_uint64)()
        _check(lib.tusq_plan_export_tally(self.h, stage, ctypes.byref(n), ctypes.byref(off),
                                          ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(cnt)))
        N = n.value
        offs = np.ctypeslib.as_array(off, (N + 1,)).copy()
        ne = int(offs[-1])
        cols = [np.ctypeslib.as_array(x, (ne,)).copy() if ne else np.zeros(0, np.int32) for x in (a, b, c)]
        if stage == 0:
            rec = [tuple(zip(cols[0][offs[i]:offs[i + 1]].tolist(), cols[1][offs[i]:offs[i + 1]].tolist()))
                   for i in range(N)]
        else:
            rec = [tuple(zip(*(col[offs[i]:offs[i + 1]].tolist() for col in cols))) for i in range(N)]
        return rec, np.ctypeslib.as_array(cnt, (N,)).copy()


def tusq_plan(circ: Circuit, shots: int, seed: int, alpha: float = 0.01, beta: int = 100,
              prune: bool = True, commute_mode: int = COMMUTE_CLIFFORD, n_threads: int = 0,
              device_sampling: bool = False, terminal_fold: bool = False) -> Plan:
    o = PlanOpts(alpha, beta, int(bool(prune)), commute_mode, n_threads, int(bool(device_sampling)),
                 int(bool(terminal_fold)))
    h = ctypes.c_void_p()
    _check(lib.tusq_plan(circ.h, ctypes.byref(o), shots, seed, ctypes.byref(h)))
    return Plan(h, circ.n_qubits)


def tusq_plan_from_instances(circ: Circuit, instances, weights) -> Plan:
    """Plan of a caller-supplied instance list: ``instances`` is a list of
    event lists [(slot, qubit, pauli), ...] sorted by (slot, qubit)."""
    n = len(instances)
    off = np.zeros(n + 1, dtype=np.uint64)
    for i, ev in enumerate(instances):
        off[i + 1] = off[i] + len(ev)
    flat = np.array([e for ev in instances for e in ev] or [(0, 0, 0)], dtype=np.int32).reshape(-1, 3)
    s, q, p = (np.ascontiguousarray(flat[:, k]) for k in range(3))
    w = np.ascontiguousarray(weights, dtype=np.float64)
    P = ctypes.POINTER
    h = ctypes.c_void_p()
    _check(lib.tusq_plan_from_instances(circ.h, n, off.ctypes.data_as(P(ctypes.c_uint64)),
                                        s.ctypes.data_as(P(ctypes.c_int32)),
                                        q.ctypes.data_as(P(ctypes.c_int32)),
                                        p.ctypes.data_as(P(ctypes.c_int32)),
                                        w.ctypes.data_as(P(ctypes.c_double)), ctypes.byref(h)))
    return Plan(h, circ.n_qubits)


def plan(wc, shots: int, seed: int, **kw) -> Plan:
    """Convenience: marshal a workload circuit and plan it."""
    return tusq_plan(circuit_from(wc), shots, seed, **kw)


# ----------------------------------------------------------------- execution

def run_opts(**kw) -> RunOpts:
    o = RunOpts()
    lib.tusq_run_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Exec:
    """Owns a tusq_exec handle: the compiled device program and its buffers."""

    def __init__(self, plan: Plan, opts: Optional[RunOpts] = None, stream: int = 0):
        self.plan = plan
        self.opts = opts or run_opts()
        h = ctypes.c_void_p()
        _check(lib.tusq_exec_create(plan.h, ctypes.byref(self.opts), ctypes.c_void_p(stream),
                                    ctypes.byref(h)))
        self.h = h

    def launch(self, probs_ptr: int, stream: int = 0) -> None:
        _check(lib.tusq_exec_launch(self.h, ctypes.c_void_p(probs_ptr), ctypes.c_void_p(stream)))

    def finish(self) -> dict:
        info = RunInfo()
        _check(lib.tusq_exec_finish(self.h, ctypes.byref(info)))
        return info.as_dict()

    def set_record_bias(self, delta: float) -> None:
        _check(lib.tusq_exec_set_record_bias(self.h, delta))

    def set_dense_skip(self, on: bool) -> None:
        _check(lib.tusq_exec_set_dense_skip(self.h, int(bool(on))))

    def set_profiling(self, on: bool) -> None:
        _check(lib.tusq_exec_set_profiling(self.h, int(bool(on))))

    def pass_structure(self) -> np.ndarray:
        """Per pass (launch order): stages, ops, 2x2 ops, 4x4 ops, diagonal
        ops, diagonal terms, flags, tile qubits."""
        n = ctypes.c_uint64()
        f = ctypes.POINTER(ctypes.c_int32)()
        _check(lib.tusq_exec_pass_structure(self.h, ctypes.byref(n), ctypes.byref(f)))
        if n.value == 0:
            return np.zeros((0, 8), np.int32)
        return np.ctypeslib.as_array(f, (n.value * 8,)).copy().reshape(-1, 8)

    def pass_profile(self):
        """(ms per pass, algorithmic bytes per pass) of the last launch."""
        n = ctypes.c_uint64()
        ms = ctypes.POINTER(ctypes.c_float)()
        by = ctypes.POINTER(ctypes.c_double)()
        _check(lib.tusq_exec_pass_profile(self.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
        if n.value == 0:
            return np.zeros(0, np.float32), np.zeros(0)
        return (np.ctypeslib.as_array(ms, (n.value,)).copy(),
                np.ctypeslib.as_array(by, (n.value,)).copy())

    def __del__(self):
        if getattr(self, "h", None):
            lib.tusq_exec_free(self.h)
            self.h = None


def tusq_compile_stats(plan: Plan, opts: Optional[RunOpts] = None) -> dict:
    """Host-only: what a launch of this plan would execute (no GPU needed)."""
    info = RunInfo()
    _check(lib.tusq_compile_stats(plan.h, ctypes.byref(opts or run_opts()), ctypes.byref(info)))
    return info.as_dict()


def tusq_run(plan: Plan, probs_ptr: int, opts: Optional[RunOpts] = None, stream: int = 0) -> None:
    o = opts or run_opts()
    _check(lib.tusq_run(plan.h, ctypes.byref(o), ctypes.c_void_p(probs_ptr), ctypes.c_void_p(stream)))


def tusq_run_noalloc(plan: Plan, probs_ptr: int, opts: Optional[RunOpts] = None, stream: int = 0) -> dict:
    """One traversal with every scratch buffer in the library's static
    device array (no device allocation); returns the run counters."""
    o = opts or run_opts()
    info = RunInfo()
    _check(lib.tusq_run_noalloc(plan.h, ctypes.byref(o), ctypes.c_void_p(probs_ptr), ctypes.c_void_p(stream),
                                ctypes.byref(info)))
    return info.as_dict()


def tusq_run_streamed(plan: Plan, probs_ptr: int, chunk_leaves: int, opts: Optional[RunOpts] = None,
                      compile_threads: int = 0, stream: int = 0) -> dict:
    """The traversal as DFS chunks of about chunk_leaves leaves, compiled on
    host threads ahead of the GPU; returns the summed run info."""
    o = opts or run_opts()
    info = RunInfo()
    _check(lib.tusq_run_streamed(plan.h, ctypes.byref(o), chunk_leaves, compile_threads,
                                 ctypes.c_void_p(probs_ptr), ctypes.c_void_p(stream), ctypes.byref(info)),
           "tusq_run_streamed")
    return info.as_dict()


def tusq_dense_check(tc_mode: int, u, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    """y_t = U x_t (t = 0..255, vectors of 32 complex64 amplitudes) through the
    tensor-core dense-stage path; u is a 32x32 complex array."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(32, 32)).view(np.float64)
    _check(lib.tusq_dense_check(tc_mode, uu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), ctypes.c_void_p(stream)),
           "tusq_dense_check")


def tusq_measure_alu_peaks(stream: int = 0):
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.tusq_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(stream)))
    return a.value, b.value


def tusq_sample(probs_ptr: int, n_qubits: int, shots: int, seed: int, counts_ptr: int, stream: int = 0) -> None:
    """Draw `shots` outcomes from the device distribution at probs_ptr into
    the device uint64 counts at counts_ptr (both 2^n_qubits entries)."""
    _check(lib.tusq_sample(ctypes.c_void_p(probs_ptr), n_qubits, shots, seed, ctypes.c_void_p(counts_ptr),
                           ctypes.c_void_p(stream)))


def sample_torch(probs, shots: int, seed: int):
    """Shot counts (torch uint64 tensor on the probs' device) drawn from a
    torch FP64 device distribution, on torch's current stream."""
    import torch
    n = int(probs.numel()).bit_length() - 1
    if probs.dtype != torch.float64 or not probs.is_cuda or probs.numel() != 1 << n or not probs.is_contiguous():
        raise ValueError("probs must be a contiguous CUDA float64 tensor of 2^n entries")
    counts = torch.empty(1 << n, dtype=torch.uint64, device=probs.device)
    tusq_sample(probs.data_ptr(), n, shots, seed, counts.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return counts


def run_torch(plan: Plan, opts: Optional[RunOpts] = None, device: str = "cuda"):
    """Allocate a torch FP64 output on the device and run one traversal on
    torch's current stream.  Returns (probs tensor, run info)."""
    import torch
    probs = torch.empty(1 << plan.n_qubits, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream().cuda_stream
    ex = Exec(plan, opts, stream)
    ex.launch(probs.data_ptr(), stream)
    info = ex.finish()
    return probs, info


# ------------------------------------------------------------------ batching

def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(p) for p in ptrs])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


class Batch:
    """Owns a tusq_batch: many jobs (5..22 qubits complex64, 4..22 complex128)
    traversed by one persistent launch -- single-CTA jobs with the state in
    shared memory, larger ones on CTA groups -- optionally replayed from a
    captured CUDA graph."""

    def __init__(self, plans, probs_ptrs, opts: Optional[RunOpts] = None, use_graph: bool = False,
                 stream: int = 0):
        self.plans = list(plans)
        self.opts = opts or run_opts()
        pp, self._pa = _ptr_array([p.h.value for p in self.plans])
        op, self._oa = _ptr_array(list(probs_ptrs))
        h = ctypes.c_void_p()
        _check(lib.tusq_batch_create(pp, len(self.plans), ctypes.byref(self.opts), op, int(bool(use_graph)),
                                     ctypes.c_void_p(stream), ctypes.byref(h)))
        self.h = h

    def launch(self, stream: int = 0) -> None:
        _check(lib.tusq_batch_launch(self.h, ctypes.c_void_p(stream)))

    def finish(self) -> dict:
        info = RunInfo()
        _check(lib.tusq_batch_finish(self.h, ctypes.byref(info)))
        return info.as_dict()

    def group_jobs(self) -> int:
        return int(lib.tusq_batch_group_jobs(self.h))

    def set_stall_test(self, on: bool) -> None:
        _check(lib.tusq_batch_set_stall_test(self.h, int(bool(on))))

    def __del__(self):
        if getattr(self, "h", None):
            lib.tusq_batch_free(self.h)
            self.h = None


def tusq_batch_autotune(plans, probs_ptrs, base: Optional[RunOpts] = None, stream: int = 0):
    """Fastest (traversal, schedule) for this batch: returns (RunOpts, ms)."""
    pp, _pa = _ptr_array([p.h.value for p in plans])
    op, _oa = _ptr_array(list(probs_ptrs))
    best = RunOpts()
    ms = ctypes.c_double()
    _check(lib.tusq_batch_autotune(pp, len(plans), ctypes.byref(base or run_opts()), op, ctypes.c_void_p(stream),
                                   ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


# ------------------------------------------------------------------- serving

class Server:
    """Owns a tusq_server: continuous batching of jobs under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, n_streams: int = 4):
        h = ctypes.c_void_p()
        _check(lib.tusq_server_create(hbm_budget_bytes, n_streams, ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, plan: Plan, probs_ptr: int, opts: Optional[RunOpts] = None) -> int:
        o = opts or run_opts()
        jid = ctypes.c_uint64()
        _check(lib.tusq_submit(self.h, plan.h, ctypes.byref(o), ctypes.c_void_p(probs_ptr),
                               ctypes.byref(jid)))
        self._keep[jid.value] = (plan, o)
        return jid.value

    def poll(self, job_id: int):
        done = ctypes.c_int()
        lat = ctypes.c_double()
        _check(lib.tusq_poll(self.h, job_id, ctypes.byref(done), ctypes.byref(lat)))
        return bool(done.value), lat.value

    def state(self, job_id: int) -> int:
        """JOB_COMPILING, JOB_READY, JOB_RUNNING or JOB_DONE."""
        st = ctypes.c_int()
        _check(lib.tusq_job_state(self.h, job_id, ctypes.byref(st)))
        return st.value

    def device_interval(self, job_id: int):
        """(start_ms, end_ms) of a finished job's traversal on the device, in ms
        since the server was created."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib.tusq_poll_device_interval(self.h, job_id, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def drain(self) -> None:
        _check(lib.tusq_server_drain(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            lib.tusq_server_free(self.h)
            self.h = None
