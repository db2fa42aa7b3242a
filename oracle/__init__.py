"""CPU oracle for the TUSQ DFTT noisy-statevector path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``tusq_oracle.c`` (plain C,
complex128) with ctypes; it never imports the CUDA library's package, and the
library never imports it.

Functions and the paper passage each follows:

* ``philox4x64_10``          -- Philox4x64-10 (Salmon et al., SC'11) for the ER draws.
* ``gate_matrix``            -- gate conventions (Sec. II, Eq. 1 acting on 2^k amplitudes).
* ``simulate``               -- one fixed-Pauli circuit from |0..0> (Sec. II mixture).
* ``plan``                   -- ER sampling + tally (Sec. III-A1), commutation
                                (Sec. III-A2/3), pruning (Sec. III-A4, Eq. S_final),
                                DFS order and branch slots (Sec. III-B).
* ``run`` / ``run_instances``-- tally-weighted output distribution of the kept
                                instances, each simulated independently.
* ``dm_run``                 -- density-matrix simulation with Pauli channels (Sec. II).
* ``commute_one``            -- commutation of a single ER (rules 1-6, Sec. III-A3).
* ``sample``                 -- shot counts drawn from the output distribution (the
                                paper samples each leaf s_i times, Sec. III-A1).

Parity pins: tests/test_oracle_*.py.  The pruning step is a heuristic whose
accuracy against the unpruned answer is parity unpinned (only its selection
rule is pinned).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tusq_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtusq_oracle.so")
_lib = None

PSTRIDE = 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP over amplitudes)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        i32p, i64p, u64p, f64p = (P(ctypes.c_int), P(ctypes.c_int64), P(ctypes.c_uint64),
                                 P(ctypes.c_double))
        L.or_gate_matrix.argtypes = [ctypes.c_int, f64p, f64p]
        L.or_simulate.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, f64p, ctypes.c_int,
                                  i32p, i32p, i32p, ctypes.c_double, f64p, f64p]
        L.or_run_instances.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, f64p, i64p,
                                       i32p, i32p, i32p, f64p, ctypes.c_int64, ctypes.c_int64, f64p]
        L.or_dm_run.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, f64p, i32p, i32p,
                                i32p, f64p, f64p]
        L.or_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.or_plan_build.restype = ctypes.c_void_p
        L.or_plan_build.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, ctypes.c_int,
                                    i32p, i32p, i32p, f64p, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_int]
        L.or_plan_free.argtypes = [ctypes.c_void_p]
        L.or_plan_sizes.argtypes = [ctypes.c_void_p, i64p]
        L.or_plan_raw.argtypes = [ctypes.c_void_p, i64p, i32p, i32p, u64p]
        L.or_plan_keys.argtypes = [ctypes.c_void_p, i64p, i32p, i32p, i32p, u64p]
        L.or_plan_instances.argtypes = [ctypes.c_void_p, i64p, i32p, i32p, i32p, u64p, f64p, i32p]
        L.or_commute_one.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, ctypes.c_int,
                                     ctypes.c_int, i32p, i32p, i32p, i32p, i32p, ctypes.c_int]
        L.or_draw_er.restype = ctypes.c_uint64
        L.or_draw_er.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.or_draw_prune.restype = ctypes.c_uint64
        L.or_draw_prune.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_draw_sample.restype = ctypes.c_uint64
        L.or_draw_sample.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_sample.argtypes = [ctypes.c_int, f64p, ctypes.c_uint64, ctypes.c_uint64, u64p]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def philox4x64_10(ctr, key):
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_p(c, ctypes.c_uint64), _p(k, ctypes.c_uint64), _p(out, ctypes.c_uint64))
    return out


def draw_er(seed: int, shot: int, channel: int) -> int:
    return int(lib().or_draw_er(seed, shot, channel))


def draw_prune(seed: int, i: int) -> int:
    return int(lib().or_draw_prune(seed, i))


def draw_sample(seed: int, s: int) -> int:
    return int(lib().or_draw_sample(seed, s))


def sample(probs, shots: int, seed: int) -> np.ndarray:
    """Shot counts drawn from an output distribution (inverse transform on
    integer cumulative weights floor(p 2^56); see or_sample)."""
    p = np.ascontiguousarray(probs, dtype=np.float64)
    n = int(np.log2(len(p)))
    assert len(p) == 1 << n
    counts = np.zeros(len(p), dtype=np.uint64)
    rc = lib().or_sample(n, _p(p, ctypes.c_double), shots, seed, _p(counts, ctypes.c_uint64))
    if rc:
        raise ValueError(f"or_sample failed ({rc})")
    return counts


def gate_matrix(kind: int, params=()) -> np.ndarray:
    p = np.zeros(PSTRIDE, dtype=np.float64)
    p[:len(params)] = params
    out = np.zeros(32, dtype=np.float64)
    d = lib().or_gate_matrix(kind, _p(p, ctypes.c_double), _p(out, ctypes.c_double))
    if d == 0:
        raise ValueError(f"unknown gate kind {kind}")
    z = out[0:2 * d * d:2] + 1j * out[1:2 * d * d:2]
    return z.reshape(d, d)


def _circ_arrays(circ):
    kinds, q0, q1, params, ch_gate, ch_nterms, ch_codes, ch_probs = circ.flat()
    return kinds, q0, q1, params, ch_gate, ch_nterms, ch_codes, ch_probs


def simulate(circ, events=(), weight: float = 1.0, want_state: bool = False):
    """Simulate one instance.  ``events``: iterable of (slot, qubit, pauli)
    sorted by slot.  Returns (probs, state-or-None)."""
    kinds, q0, q1, params, *_ = _circ_arrays(circ)
    ev = np.array(list(events), dtype=np.int32).reshape(-1, 3)
    s, q, p = _i32(ev[:, 0]), _i32(ev[:, 1]), _i32(ev[:, 2])
    dim = 1 << circ.n_qubits
    acc = np.zeros(dim, dtype=np.float64)
    psi = np.zeros(2 * dim, dtype=np.float64) if want_state else None
    rc = lib().or_simulate(circ.n_qubits, circ.n_gates, _p(kinds, ctypes.c_int), _p(q0, ctypes.c_int),
                           _p(q1, ctypes.c_int), _p(params, ctypes.c_double), len(ev),
                           _p(s, ctypes.c_int), _p(q, ctypes.c_int), _p(p, ctypes.c_int),
                           weight, _p(acc, ctypes.c_double),
                           _p(psi, ctypes.c_double) if psi is not None else None)
    if rc:
        raise ValueError(f"or_simulate failed ({rc})")
    return acc, (psi[0::2] + 1j * psi[1::2] if psi is not None else None)


def dm_run(circ) -> np.ndarray:
    kinds, q0, q1, params, ch_gate, ch_nterms, ch_codes, ch_probs = _circ_arrays(circ)
    ch_of_gate = np.full(max(circ.n_gates, 1), -1, dtype=np.int32)
    for c, j in enumerate(ch_gate):
        ch_of_gate[j] = c
    out = np.zeros(1 << circ.n_qubits, dtype=np.float64)
    z = np.zeros(1, dtype=np.int32)
    zf = np.zeros(1, dtype=np.float64)
    rc = lib().or_dm_run(circ.n_qubits, circ.n_gates, _p(kinds, ctypes.c_int), _p(q0, ctypes.c_int),
                         _p(q1, ctypes.c_int), _p(params, ctypes.c_double),
                         _p(ch_of_gate, ctypes.c_int),
                         _p(ch_nterms if len(ch_nterms) else z, ctypes.c_int),
                         _p(ch_codes if len(ch_codes) else z, ctypes.c_int),
                         _p(ch_probs if len(ch_probs) else zf, ctypes.c_double),
                         _p(out, ctypes.c_double))
    if rc:
        raise ValueError("dm_run supports n <= 8")
    return out


@dataclasses.dataclass
class OraclePlan:
    n_qubits: int
    n_gates: int
    raw: List[tuple]            # distinct raw ERs: tuple of (channel, code), sorted
    raw_count: np.ndarray
    keys: List[tuple]           # distinct commuted keys: tuple of (slot, qubit, pauli), sorted
    key_count: np.ndarray
    inst: List[tuple]           # kept instances in DFS order
    inst_count: np.ndarray
    weights: np.ndarray
    lcp: np.ndarray
    n_sig: int
    n_insig: int
    n_pick: int
    c_max: int
    c_insig: int
    c_pick: int


def _split(off, *cols):
    return [tuple(zip(*(c[off[i]:off[i + 1]] for c in cols))) for i in range(len(off) - 1)]


def plan(circ, shots: int, seed: int, commute_mode: int = 2, prune: bool = True,
         alpha: float = 0.01, beta: int = 100, terminal_fold: bool = False) -> OraclePlan:
    kinds, q0, q1, params, ch_gate, ch_nterms, ch_codes, ch_probs = _circ_arrays(circ)
    z = np.zeros(1, dtype=np.int32)
    zf = np.zeros(1, dtype=np.float64)
    L = lib()
    h = L.or_plan_build(circ.n_qubits, circ.n_gates, _p(kinds, ctypes.c_int), _p(q0, ctypes.c_int),
                        _p(q1, ctypes.c_int), len(ch_gate),
                        _p(ch_gate if len(ch_gate) else z, ctypes.c_int),
                        _p(ch_nterms if len(ch_nterms) else z, ctypes.c_int),
                        _p(ch_codes if len(ch_codes) else z, ctypes.c_int),
                        _p(ch_probs if len(ch_probs) else zf, ctypes.c_double),
                        shots, seed, commute_mode, int(bool(prune)), alpha, beta, int(bool(terminal_fold)))
    if not h:
        raise ValueError("oracle plan: the Kraus-branch expansion exceeds 2^24 instances")
    try:
        sz = np.zeros(12, dtype=np.int64)
        L.or_plan_sizes(h, _p(sz, ctypes.c_int64))
        nr, nre, nk, nke, ni, nie = (int(v) for v in sz[:6])
        roff = np.zeros(nr + 1, np.int64); rch = np.zeros(max(nre, 1), np.int32)
        rcode = np.zeros(max(nre, 1), np.int32); rcount = np.zeros(max(nr, 1), np.uint64)
        L.or_plan_raw(h, _p(roff, ctypes.c_int64), _p(rch, ctypes.c_int), _p(rcode, ctypes.c_int),
                      _p(rcount, ctypes.c_uint64))
        koff = np.zeros(nk + 1, np.int64); ks = np.zeros(max(nke, 1), np.int32)
        kq = np.zeros(max(nke, 1), np.int32); kp = np.zeros(max(nke, 1), np.int32)
        kcount = np.zeros(max(nk, 1), np.uint64)
        L.or_plan_keys(h, _p(koff, ctypes.c_int64), _p(ks, ctypes.c_int), _p(kq, ctypes.c_int),
                       _p(kp, ctypes.c_int), _p(kcount, ctypes.c_uint64))
        ioff = np.zeros(ni + 1, np.int64); is_ = np.zeros(max(nie, 1), np.int32)
        iq = np.zeros(max(nie, 1), np.int32); ip = np.zeros(max(nie, 1), np.int32)
        icount = np.zeros(max(ni, 1), np.uint64); iw = np.zeros(max(ni, 1), np.float64)
        lcp = np.zeros(max(ni, 1), np.int32)
        L.or_plan_instances(h, _p(ioff, ctypes.c_int64), _p(is_, ctypes.c_int), _p(iq, ctypes.c_int),
                            _p(ip, ctypes.c_int), _p(icount, ctypes.c_uint64), _p(iw, ctypes.c_double),
                            _p(lcp, ctypes.c_int))
    finally:
        L.or_plan_free(h)
    return OraclePlan(circ.n_qubits, circ.n_gates,
                      _split(roff, rch, rcode), rcount[:nr], _split(koff, ks, kq, kp), kcount[:nk],
                      _split(ioff, is_, iq, ip), icount[:ni], iw[:ni], lcp[:max(ni - 1, 0)],
                      int(sz[6]), int(sz[7]), int(sz[8]), int(sz[9]), int(sz[10]), int(sz[11]))


def flatten_instances(instances):
    off = np.zeros(len(instances) + 1, dtype=np.int64)
    for i, ev in enumerate(instances):
        off[i + 1] = off[i] + len(ev)
    flat = np.array([e for ev in instances for e in ev], dtype=np.int32).reshape(-1, 3)
    return off, flat


def run_instances(circ, instances, weights, first: int = 0, count: Optional[int] = None,
                  acc: Optional[np.ndarray] = None) -> np.ndarray:
    """Sum of w_i |psi_i|^2 over instances [first, first+count), each simulated
    independently from |0..0> (no tree, no uncomputation)."""
    kinds, q0, q1, params, *_ = _circ_arrays(circ)
    count = len(instances) - first if count is None else count
    off, flat = flatten_instances(instances)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if acc is None:
        acc = np.zeros(1 << circ.n_qubits, dtype=np.float64)
    s, q, p = _i32(flat[:, 0]), _i32(flat[:, 1]), _i32(flat[:, 2])
    if len(s) == 0:
        s = q = p = np.zeros(1, np.int32)
    rc = lib().or_run_instances(circ.n_qubits, circ.n_gates, _p(kinds, ctypes.c_int),
                                _p(q0, ctypes.c_int), _p(q1, ctypes.c_int),
                                _p(params, ctypes.c_double), _p(off, ctypes.c_int64),
                                _p(s, ctypes.c_int), _p(q, ctypes.c_int), _p(p, ctypes.c_int),
                                _p(w, ctypes.c_double), first, count, _p(acc, ctypes.c_double))
    if rc:
        raise ValueError(f"or_run_instances failed ({rc})")
    return acc


def run(circ, shots: int, seed: int, commute_mode: int = 2, prune: bool = True,
        alpha: float = 0.01, beta: int = 100, terminal_fold: bool = False):
    """Full oracle: plan, then every kept instance simulated independently."""
    pl = plan(circ, shots, seed, commute_mode, prune, alpha, beta, terminal_fold)
    return run_instances(circ, pl.inst, pl.weights), pl


def commute_one(circ, er, mode: int = 2):
    """Commute one raw ER given as [(channel, code), ...] (channel = index
    among the circuit's channels in gate order)."""
    kinds, q0, q1, params, ch_gate, *_ = _circ_arrays(circ)
    er = list(er)
    chs = _i32([c for c, _ in er] or [0])
    codes = _i32([k for _, k in er] or [0])
    cap = 4 * len(er) + 8
    s = np.zeros(cap, np.int32); q = np.zeros(cap, np.int32); p = np.zeros(cap, np.int32)
    cg = ch_gate if len(ch_gate) else np.zeros(1, np.int32)
    m = lib().or_commute_one(circ.n_qubits, circ.n_gates, _p(kinds, ctypes.c_int),
                             _p(q0, ctypes.c_int), _p(q1, ctypes.c_int), _p(cg, ctypes.c_int),
                             mode, len(er), _p(chs, ctypes.c_int), _p(codes, ctypes.c_int),
                             _p(s, ctypes.c_int), _p(q, ctypes.c_int), _p(p, ctypes.c_int), cap)
    if m < 0:
        raise ValueError("commute_one overflow")
    return tuple(zip(s[:m].tolist(), q[:m].tolist(), p[:m].tolist()))
