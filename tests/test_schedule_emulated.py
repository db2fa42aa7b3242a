"""The schedule compiler's device program, interpreted on the host with the
kernels' semantics (tests/emu/program_emulator.cpp), against the oracle.
This checks the DFTT traversal (forward segments, uncompute, leaf peek,
records, checks, snapshot restores, root resets), the pass and stage
fusion, the register layouts and the diagonal-phase formula without a GPU."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_04880_b300", "csrc")
SO = os.path.join(HERE, "emu", "_build", "libprogram_emulator.so")
_emu = None


def emu():
    global _emu
    if _emu is None:
        srcs = [os.path.join(HERE, "emu", "program_emulator.cpp")] + \
            [os.path.join(CSRC, f) for f in ("compile.cpp", "plan.cpp", "capi.cpp", "dense_host.cpp")]
        deps = srcs + [os.path.join(CSRC, f) for f in ("program.h", "internal.h")]
        if not os.path.exists(SO) or any(os.path.getmtime(d) > os.path.getmtime(SO) for d in deps):
            os.makedirs(os.path.dirname(SO), exist_ok=True)
            tmp = SO + f".{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, *srcs,
                                   "-lpthread"])
            os.replace(tmp, SO)
        L = ctypes.CDLL(SO)
        L.emu_run.argtypes = [ctypes.c_void_p, ctypes.POINTER(T.RunOpts), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double)]
        _emu = L
    return _emu


def emu_run(plan, **opts):
    o = T.run_opts(**opts)
    if o.snapshot_bytes == 0:
        o.snapshot_bytes = 8 * (16 if o.precision == T.C128 else 8) << plan.n_qubits
    out = np.zeros(1 << plan.n_qubits)
    info = np.zeros(4)
    emu().emu_run(plan.h, ctypes.byref(o), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  info.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out, {"max_drift": info[0], "restores": info[1], "diag_mismatch": info[2], "passes": info[3]}


TRAV = [T.DFTT, T.FROM_SCRATCH, T.DFTT_SNAPSHOT]
# the interpreter runs in FP64; complex64 programs carry their phases in
# 2^-31-turn fixed point, which bounds their deviation
TOL = {T.C128: 1e-12, T.C64: 1e-7}


@pytest.mark.parametrize("traversal", TRAV)
@pytest.mark.parametrize("precision", [T.C128, T.C64])
@pytest.mark.parametrize("prune", [True, False])
def test_random_layers_6q(traversal, precision, prune):
    circ = W.random_layers(6, 20, 0, 1e-3, 1e-2)
    ref, _ = oracle.run(circ, 10_000, 0, prune=prune)
    got, info = emu_run(T.plan(circ, 10_000, 0, prune=prune), precision=precision, traversal=traversal)
    assert info["diag_mismatch"] < 1e-9
    assert np.abs(got - ref).max() < TOL[precision]


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (8, 4), (10, 5)])
@pytest.mark.parametrize("window", [0, 4, 6])
@pytest.mark.parametrize("precision", [T.C128, T.C64])
def test_every_gate_kind(n, seed, window, precision):
    circ = W.random_mixed(n, 40, seed, p1=3e-2, p2=6e-2)
    ref, _ = oracle.run(circ, 3000, seed, prune=False)
    pl = T.plan(circ, 3000, seed, prune=False)
    for trav in TRAV:
        for peek, reset in ((1, 1), (0, 0)):
            got, info = emu_run(pl, precision=precision, traversal=trav, max_window=window,
                                leaf_peek=peek, root_reset=reset)
            assert info["diag_mismatch"] < 1e-9
            assert np.abs(got - ref).max() < TOL[precision], (trav, peek, reset)


def test_qaoa_and_brickwork_multi_tile():
    for circ, shots in [(W.qaoa_3regular(14, 3, 4, 1e-3, 1e-2), 20_000),
                        (W.brickwork(14, 8, 2, 2e-3, 2e-2), 20_000)]:
        ref, _ = oracle.run(circ, shots, 1)
        pl = T.plan(circ, shots, 1)
        for trav in TRAV:
            got, info = emu_run(pl, precision=T.C64, traversal=trav, max_window=9)
            assert info["diag_mismatch"] < 1e-9
            assert np.abs(got - ref).max() < TOL[T.C64]


def test_forced_drift_restores():
    circ = W.brickwork(8, 8, 3, 2e-3, 2e-2)
    ref, _ = oracle.run(circ, 20_000, 5)
    got, info = emu_run(T.plan(circ, 20_000, 5), precision=T.C128, traversal=T.DFTT, drift_tol=0.0)
    assert info["restores"] > 0
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("leaf_peek", [0, 1])
@pytest.mark.parametrize("window", [0, 3])
def test_uncompute_without_drift_checks(leaf_peek, window):
    # no branch stack (drift checks off, uncompute traversal): the leaf pass
    # that skips its write must not hold ops above the node the uncompute
    # returns to, so a pass ends at every next branch node
    circ = W.random_layers(6, 20, 0, 1e-2, 3e-2)
    ref, _ = oracle.run(circ, 5000, 3)
    got, _ = emu_run(T.plan(circ, 5000, 3), precision=T.C128, traversal=T.DFTT, drift_tol=-1.0,
                     leaf_peek=leaf_peek, max_window=window)
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("tc_mode", [T.TC_TF32X3, T.TC_BF16X3])
def test_tensor_core_dense_stages(tc_mode):
    # with tc_mode, thread-independent runs of a register stage become one
    # 32x32 matrix (Sec. II, Eq. 1); the interpreter applies the FP64 matrix
    # the compiler stored, so the program's structure -- which ops were
    # absorbed, the fixed-bit phases riding along, the pass split under the
    # larger program budget -- is checked against the oracle
    for circ, shots in [(W.brickwork(14, 8, 2, 2e-3, 2e-2), 20_000),
                        (W.qaoa_3regular(14, 3, 4, 1e-3, 1e-2), 20_000)]:
        ref, _ = oracle.run(circ, shots, 1)
        pl = T.plan(circ, shots, 1)
        for trav in TRAV:
            st = T.tusq_compile_stats(pl, T.run_opts(precision=T.C64, traversal=trav, tc_mode=tc_mode))
            got, info = emu_run(pl, precision=T.C64, traversal=trav, tc_mode=tc_mode)
            assert info["diag_mismatch"] < 1e-9
            assert np.abs(got - ref).max() < TOL[T.C64], (circ.name, trav)
            if circ.name.startswith("brickwork"):
                assert st["dense_ops"] > 0
