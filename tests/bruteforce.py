"""Brute-force numpy helpers for pinning the oracle on tiny inputs.

Everything here is built from full 2^n x 2^n operators (Kronecker products
and explicit index loops), which is a different route from the oracle's
in-place amplitude-pair updates.  Only the tests use it.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg

import tusq_workloads as W

PAULI = {
    0: np.eye(2, dtype=complex),
    1: np.array([[0, 1], [1, 0]], dtype=complex),
    2: np.array([[0, -1j], [1j, 0]], dtype=complex),
    3: np.array([[1, 0], [0, -1]], dtype=complex),
}


def textbook_matrix(kind, params=()):
    """Gate matrices from their textbook definitions (expm for rotations)."""
    s2 = 1 / np.sqrt(2)
    if kind == W.H:
        return np.array([[s2, s2], [s2, -s2]], dtype=complex)
    if kind in (W.X, W.Y, W.Z):
        return PAULI[kind].copy()
    if kind == W.S:
        return np.diag([1, 1j])
    if kind == W.SDG:
        return np.diag([1, -1j])
    if kind == W.T:
        return np.diag([1, np.exp(1j * np.pi / 4)])
    if kind == W.TDG:
        return np.diag([1, np.exp(-1j * np.pi / 4)])
    if kind in (W.RX, W.RY, W.RZ):
        sig = PAULI[{W.RX: 1, W.RY: 2, W.RZ: 3}[kind]]
        return scipy.linalg.expm(-0.5j * params[0] * sig)
    if kind == W.RZZ:
        return scipy.linalg.expm(-0.5j * params[0] * np.kron(PAULI[3], PAULI[3]))
    if kind == W.CX:
        return np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    if kind == W.CZ:
        return np.diag([1, 1, 1, -1]).astype(complex)
    if kind == W.U1Q:
        p = np.asarray(params)
        return (p[0::2] + 1j * p[1::2]).reshape(2, 2)
    if kind == W.U2Q:
        p = np.asarray(params)
        return (p[0::2] + 1j * p[1::2]).reshape(4, 4)
    raise ValueError(kind)


def full_op(n, U, q0, q1=-1):
    """The 2^n x 2^n operator of a 1q gate on q0 or a 2q gate on (q0, q1)
    (local index 2*bit(q0) + bit(q1)), by an explicit index loop."""
    dim = 1 << n
    M = np.zeros((dim, dim), dtype=complex)
    if q1 < 0:
        for i in range(dim):
            for j in range(dim):
                if (i & ~(1 << q0)) != (j & ~(1 << q0)):
                    continue
                M[i, j] = U[(i >> q0) & 1, (j >> q0) & 1]
        return M
    mask = ~((1 << q0) | (1 << q1))
    for i in range(dim):
        for j in range(dim):
            if (i & mask) != (j & mask):
                continue
            li = 2 * ((i >> q0) & 1) + ((i >> q1) & 1)
            lj = 2 * ((j >> q0) & 1) + ((j >> q1) & 1)
            M[i, j] = U[li, lj]
    return M


def kraus(kind, m):
    """Kraus operator m of a reset (|0><m|) or a Z measurement (|m><m|)."""
    ket0, ketm = np.eye(2)[:, [0]], np.eye(2)[:, [m]]
    return (ket0 @ ketm.T if kind == W.RESET else ketm @ ketm.T).astype(complex)


def gate_full(circ, j):
    kind, q0, q1, params = circ.gates[j]
    U = textbook_matrix(kind, params)
    return full_op(circ.n_qubits, U, q0, q1 if kind in W.TWO_QUBIT else -1)


def pauli_full(n, q, p):
    return full_op(n, PAULI[p], q)


def state_of_instance(circ, events):
    """psi = prod over slots (gate_j . paulis_at_slot_j) |0>, full matrices."""
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    ev = sorted(events)
    for j in range(circ.n_gates + 1):
        branch = 0
        for (s, q, p) in ev:
            if s == j and p == W.OUTCOME1:
                branch = 1
            elif s == j:
                psi = pauli_full(n, q, p) @ psi
        if j < circ.n_gates and circ.gates[j][0] in W.NONINVERTIBLE:
            psi = full_op(n, kraus(circ.gates[j][0], branch), circ.gates[j][1]) @ psi
        elif j < circ.n_gates:
            psi = gate_full(circ, j) @ psi
    return psi


def channel_paulis(circ, j, code):
    """Per-qubit Paulis of a channel outcome on gate j's qubits."""
    kind, q0, q1, _ = circ.gates[j]
    if kind in W.TWO_QUBIT:
        return [(q0, code >> 2), (q1, code & 3)]
    return [(q0, code)]


def dm_bruteforce(circ):
    """rho <- U rho U^dag, then sum_k p_k P_k rho P_k after noisy gates."""
    n = circ.n_qubits
    dim = 1 << n
    rho = np.zeros((dim, dim), dtype=complex)
    rho[0, 0] = 1
    for j in range(circ.n_gates):
        kind, q0 = circ.gates[j][0], circ.gates[j][1]
        if kind in W.NONINVERTIBLE:
            # rho <- sum_m K_m rho K_m^dag
            Ks = [full_op(n, kraus(kind, m), q0) for m in (0, 1)]
            rho = sum(K @ rho @ K.conj().T for K in Ks)
        else:
            U = gate_full(circ, j)
            rho = U @ rho @ U.conj().T
        ch = circ.channels[j]
        if ch is None:
            continue
        codes, probs = ch
        new = (1 - sum(probs)) * rho
        for code, p in zip(codes, probs):
            P = np.eye(dim, dtype=complex)
            for q, pp in channel_paulis(circ, j, code):
                if pp:
                    P = pauli_full(n, q, pp) @ P
            new = new + p * (P @ rho @ P.conj().T)
        rho = new
    return np.real(np.diag(rho))


def enumerate_ers(circ):
    """Every error realization with its exact probability (product over
    channels of the chosen term's probability)."""
    chans = [(j, c) for j, c in enumerate(circ.channels) if c is not None]
    options = []
    for j, (codes, probs) in chans:
        options.append([(j, 0, 1 - sum(probs))] + [(j, c, p) for c, p in zip(codes, probs)])
    for combo in itertools.product(*options):
        prob = 1.0
        events = []
        for (j, code, p) in combo:
            prob *= p
            if code:
                for q, pp in channel_paulis(circ, j, code):
                    if pp:
                        events.append((j + 1, q, pp))
        yield prob, sorted(events)
