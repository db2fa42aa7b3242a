"""Seeded synthetic noisy circuits shaped like the paper's workloads.

This module only *generates inputs*: gate lists, gate parameters and per-gate
Pauli channels.  It holds none of the method's arithmetic (no sampling of error
realizations, no commutation, no simulation) and is the one module that both
the CUDA library's tests and the CPU oracle consume.

The paper evaluates on Supermarq circuits (Section IV-B, benchmark table:
QAOA 13-25 qubits with 130-1250 gates, adders, GHZ, QFT, ...) with
depolarizing noise p = 1e-2 or 1e-3 (Section IV-D).  Those circuits are not
available here; the generators below produce circuits with the same qubit
counts, depths, gate mixes and noise rates instead.

Interface numbering (shared with the C ABI header and the oracle, each of
which writes its own copy):

* gate kinds: H=0 X=1 Y=2 Z=3 S=4 SDG=5 T=6 TDG=7 RX=8 RY=9 RZ=10 U1Q=11
  CX=12 CZ=13 RZZ=14 U2Q=15, and the non-invertible one-qubit RESET=16
  (to |0>) and MEASURE=17 (mid-circuit Z measurement, record not output).  RX/RY/RZ(t) = exp(-i t sigma/2),
  RZZ(t) = exp(-i t Z(x)Z/2), U1Q carries a row-major 2x2 complex matrix as
  8 doubles (re, im pairs), U2Q a 4x4 one as 32 doubles.  For a two-qubit
  gate on (q0, q1) the local basis index is 2*bit(q0) + bit(q1); CX has
  control q0 and target q1.  Qubit q is bit q of the amplitude index.
* Pauli codes: I=0 X=1 Y=2 Z=3; a two-qubit Pauli is 4*P(q0) + P(q1).
* A channel is attached to a gate and acts on that gate's qubits right after
  it: a list of non-identity Pauli codes with their probabilities; the
  identity gets 1 - sum.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

H, X, Y, Z, S, SDG, T, TDG, RX, RY, RZ, U1Q, CX, CZ, RZZ, U2Q, RESET, MEASURE = range(18)
TWO_QUBIT = (CX, CZ, RZZ, U2Q)
NONINVERTIBLE = (RESET, MEASURE)     # mid-circuit reset / measurement (no parameters)
OUTCOME1 = 4                          # event code of Kraus branch 1 in an instance's event list
PARAM_STRIDE = 32          # doubles reserved per gate in flat parameter arrays
N_PARAMS = {RX: 1, RY: 1, RZ: 1, RZZ: 1, U1Q: 8, U2Q: 32}

Gate = Tuple[int, int, int, Tuple[float, ...]]          # (kind, q0, q1, params)
Channel = Tuple[Tuple[int, ...], Tuple[float, ...]]     # (codes, probs)


@dataclasses.dataclass
class Circuit:
    """A noisy circuit: gates in order, each optionally followed by a channel."""
    n_qubits: int
    gates: List[Gate] = dataclasses.field(default_factory=list)
    channels: List[Optional[Channel]] = dataclasses.field(default_factory=list)
    name: str = ""

    def add(self, kind: int, q0: int, q1: int = -1, params: Sequence[float] = (),
            channel: Optional[Channel] = None) -> None:
        self.gates.append((int(kind), int(q0), int(q1), tuple(float(p) for p in params)))
        self.channels.append(channel)

    @property
    def n_gates(self) -> int:
        return len(self.gates)

    @property
    def n_channels(self) -> int:
        return sum(1 for c in self.channels if c is not None)

    def flat(self):
        """Flat numpy arrays (kinds, q0, q1, params[G*32], ch_gate, ch_nterms,
        ch_codes[C*15], ch_probs[C*15]) used to pass the circuit over a C ABI."""
        G = self.n_gates
        kinds = np.array([g[0] for g in self.gates], dtype=np.int32)
        q0 = np.array([g[1] for g in self.gates], dtype=np.int32)
        q1 = np.array([g[2] for g in self.gates], dtype=np.int32)
        params = np.zeros(max(G, 1) * PARAM_STRIDE, dtype=np.float64)
        for j, g in enumerate(self.gates):
            params[j * PARAM_STRIDE: j * PARAM_STRIDE + len(g[3])] = g[3]
        ch_gate, ch_nterms, ch_codes, ch_probs = [], [], [], []
        for j, ch in enumerate(self.channels):
            if ch is None:
                continue
            codes, probs = ch
            ch_gate.append(j)
            ch_nterms.append(len(codes))
            ch_codes.extend(list(codes) + [0] * (15 - len(codes)))
            ch_probs.extend(list(probs) + [0.0] * (15 - len(probs)))
        return (kinds, q0, q1, params,
                np.array(ch_gate, dtype=np.int32), np.array(ch_nterms, dtype=np.int32),
                np.array(ch_codes, dtype=np.int32), np.array(ch_probs, dtype=np.float64))


# ----------------------------------------------------------------------------- channels

def depolarizing_1q(p: float) -> Channel:
    """X, Y, Z each with p/3 (Section II, the depolarizing channel)."""
    return ((1, 2, 3), (p / 3.0,) * 3)


def depolarizing_2q(p: float) -> Channel:
    """The 15 non-identity two-qubit Paulis each with p/15 (the paper does not
    define a two-qubit channel; this is the usual uniform one)."""
    return (tuple(range(1, 16)), (p / 15.0,) * 15)


def pauli_twirled_decoherence(t: float, t1: float, t2: float) -> Channel:
    """Pauli-twirled amplitude/phase damping (Section VI-A):
    pX = pY = (1 - e^{-t/T1})/4, pZ = (1 - e^{-t/T2})/2 - (1 - e^{-t/T1})/4."""
    a = (1.0 - math.exp(-t / t1)) / 4.0
    pz = (1.0 - math.exp(-t / t2)) / 2.0 - a
    return ((1, 2, 3), (a, a, pz))


def measurement_flip(p: float) -> Channel:
    """Bit flip before measurement (b = 2 children, {I, X}; Section III-B1)."""
    return ((1,), (p,))


def _noise_for(kind: int, p1: float, p2: float) -> Optional[Channel]:
    if kind in TWO_QUBIT:
        return depolarizing_2q(p2) if p2 > 0 else None
    return depolarizing_1q(p1) if p1 > 0 else None


# ----------------------------------------------------------------------------- helpers

def haar_su2(rng: np.random.Generator) -> Tuple[float, ...]:
    """Haar-random SU(2) from a uniformly random unit quaternion (four i.i.d.
    normals, normalised; Marsaglia 1972 / Muller 1959).  Returns 8 doubles:
    row-major [[a+ib, c+id], [-c+id, a-ib]]."""
    v = rng.standard_normal(4)
    a, b, c, d = v / np.linalg.norm(v)
    return (a, b, c, d, -c, d, a, -b)


def random_regular3(n: int, rng: np.random.Generator) -> List[Tuple[int, int]]:
    """Random simple 3-regular graph by the configuration model with
    rejection (retry until no self-loop or repeated edge).  n must be even."""
    if n % 2 or n < 4:
        raise ValueError("3-regular graph needs an even n >= 4")
    while True:
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return [(int(a), int(b)) for a, b in pairs]


# ----------------------------------------------------------------------------- workloads

def random_layers(n: int = 6, depth: int = 20, seed: int = 0, p1: float = 1e-3,
                  p2: float = 1e-2) -> Circuit:
    """Each layer: H or RZ(theta ~ U[0, 2pi)) on every qubit (fair coin per
    qubit), then CX on a uniformly random perfect matching with random
    orientation; depolarizing after every gate."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"random_layers_n{n}_d{depth}")
    for _ in range(depth):
        for q in range(n):
            if rng.random() < 0.5:
                c.add(H, q, channel=_noise_for(H, p1, p2))
            else:
                c.add(RZ, q, params=(rng.uniform(0, 2 * math.pi),), channel=_noise_for(RZ, p1, p2))
        perm = rng.permutation(n)
        for k in range(n // 2):
            a, b = int(perm[2 * k]), int(perm[2 * k + 1])
            if rng.random() < 0.5:
                a, b = b, a
            c.add(CX, a, b, channel=_noise_for(CX, p1, p2))
    return c


def brickwork(n: int = 20, depth: int = 40, seed: int = 0, p1: float = 1e-3,
              p2: float = 1e-2) -> Circuit:
    """Haar SU(2) on every qubit, then CZ on (0,1),(2,3),... in even layers and
    (1,2),(3,4),... in odd layers."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"brickwork_n{n}_d{depth}")
    for layer in range(depth):
        for q in range(n):
            c.add(U1Q, q, params=haar_su2(rng), channel=_noise_for(U1Q, p1, p2))
        for a in range(layer % 2, n - 1, 2):
            c.add(CZ, a, a + 1, channel=_noise_for(CZ, p1, p2))
    return c


def qaoa_3regular(n: int = 28, layers: int = 4, seed: int = 0, p1: float = 5e-4,
                  p2: float = 5e-3) -> Circuit:
    """QAOA-style circuit on a seeded random 3-regular graph: H on all qubits,
    then per layer RZZ(gamma_l) on every edge (edge-list order) and
    RX(beta_l) on every qubit; gamma, beta ~ U[0, pi)."""
    rng = np.random.default_rng(seed)
    edges = random_regular3(n, rng)
    gammas = rng.uniform(0, math.pi, layers)
    betas = rng.uniform(0, math.pi, layers)
    c = Circuit(n, name=f"qaoa3reg_n{n}_p{layers}")
    for q in range(n):
        c.add(H, q, channel=_noise_for(H, p1, p2))
    for layer in range(layers):
        for a, b in edges:
            c.add(RZZ, a, b, params=(gammas[layer],), channel=_noise_for(RZZ, p1, p2))
        for q in range(n):
            c.add(RX, q, params=(betas[layer],), channel=_noise_for(RX, p1, p2))
    return c


def repetition_memory(d: int = 3, rounds: int = 3, seed: int = 0, p1: float = 1e-2,
                      p2: float = 2e-2, pm: float = 1e-2, kind: int = RESET) -> Circuit:
    """Bit-flip repetition-code memory, a small stand-in for the surface-code
    memory circuits with d rounds of mid-circuit measurements of Sec. III-B2:
    data qubits 0..d-1 start in a seeded product state (RY angles), ancilla
    d+i collects the parity of data i and i+1 with two CX per round and is then
    reset (or measured, `kind`), with a measurement-flip channel after it.
    One round's ancilla operations are adjacent: one non-invertible layer."""
    rng = np.random.default_rng(seed)
    n = 2 * d - 1
    c = Circuit(n, name=f"repetition_d{d}_r{rounds}")
    for q in range(d):
        c.add(RY, q, params=(float(rng.uniform(0, math.pi)),), channel=_noise_for(RY, p1, p2))
    for _ in range(rounds):
        for i in range(d - 1):
            c.add(CX, i, d + i, channel=_noise_for(CX, p1, p2))
            c.add(CX, i + 1, d + i, channel=_noise_for(CX, p1, p2))
        for i in range(d - 1):
            c.add(kind, d + i, channel=measurement_flip(pm) if pm > 0 else None)
        for q in range(d):
            c.add(RX, q, params=(float(rng.uniform(0, 0.3)),), channel=_noise_for(RX, p1, p2))
    return c


def mcm_brickwork(n: int = 24, depth: int = 12, layers: int = 3, per_layer: int = 2, seed: int = 0,
                  p1: float = 1e-3, p2: float = 1e-2, kind: int = RESET) -> Circuit:
    """Brickwork (Haar SU(2) + CZ) with `layers` layers of mid-circuit resets
    (or measurements) spread evenly through the depth, each on `per_layer`
    seeded distinct qubits."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"mcm_brickwork_n{n}_d{depth}_l{layers}x{per_layer}")
    at = {int(round((k + 1) * depth / (layers + 1))) for k in range(layers)}
    for layer in range(depth):
        if layer in at:
            for q in sorted(int(v) for v in rng.choice(n, per_layer, replace=False)):
                c.add(kind, q)
        for q in range(n):
            c.add(U1Q, q, params=haar_su2(rng), channel=_noise_for(U1Q, p1, p2))
        for a in range(layer % 2, n - 1, 2):
            c.add(CZ, a, a + 1, channel=_noise_for(CZ, p1, p2))
    return c


def ghz(n: int, p1: float = 0.0, p2: float = 0.0) -> Circuit:
    """H on qubit 0 then a CX chain 0->1->...->n-1."""
    c = Circuit(n, name=f"ghz_n{n}")
    c.add(H, 0, channel=_noise_for(H, p1, p2))
    for q in range(n - 1):
        c.add(CX, q, q + 1, channel=_noise_for(CX, p1, p2))
    return c


def product_rx(thetas: Sequence[float], p: float) -> Circuit:
    """RX(theta_q) on each qubit followed by 1q depolarizing p."""
    c = Circuit(len(thetas), name=f"product_rx_n{len(thetas)}")
    for q, t in enumerate(thetas):
        c.add(RX, q, params=(t,), channel=depolarizing_1q(p) if p > 0 else None)
    return c


def random_mixed(n: int, n_gates: int, seed: int, p1: float = 1e-2, p2: float = 3e-2,
                 kinds: Sequence[int] = tuple(range(16))) -> Circuit:
    """Random gate soup over every supported gate kind (for commutation and
    parity tests): random qubits, random angles, Haar 1q/2q unitaries."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"mixed_n{n}_g{n_gates}_s{seed}")
    for _ in range(n_gates):
        kind = int(rng.choice(kinds))
        if kind in TWO_QUBIT and n < 2:
            kind = H
        if kind in TWO_QUBIT:
            a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        else:
            a, b = int(rng.integers(n)), -1
        if kind in (RX, RY, RZ, RZZ):
            params = (rng.uniform(0, 2 * math.pi),)
        elif kind == U1Q:
            params = haar_su2(rng)
        elif kind == U2Q:
            m = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
            qm, r = np.linalg.qr(m)
            qm = qm * (np.diag(r) / np.abs(np.diag(r)))
            params = tuple(v for z in qm.reshape(-1) for v in (z.real, z.imag))
        else:
            params = ()
        c.add(kind, a, b, params=params, channel=_noise_for(kind, p1, p2))
    return c


def job_mix(count: int = 2048, seed: int = 0, n_lo: int = 12, n_hi: int = 18,
            d_lo: int = 20, d_hi: int = 80) -> List[Circuit]:
    """Batched workload: brickwork and QAOA circuits of n ~ U{n_lo..n_hi}
    (QAOA needs an even n), depth ~ U{d_lo..d_hi}; job j is seeded with j."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        depth = int(rng.integers(d_lo, d_hi + 1))
        if rng.random() < 0.5:
            jobs.append(brickwork(n, depth, seed=seed * 100003 + j))
        else:
            n -= n % 2
            jobs.append(qaoa_3regular(n, max(1, depth // 4), seed=seed * 100003 + j,
                                      p1=1e-3, p2=1e-2))
    return jobs


def served_stream(count: int, seed: int = 0, n_lo: int = 10, n_hi: int = 30,
                  d_lo: int = 20, d_hi: int = 100):
    """Serving workload: (circuit, shots) pairs with n ~ U{n_lo..n_hi}, depth
    ~ U{d_lo..d_hi}, p ~ logU[1e-4, 1e-2], shots ~ logU[1e5, 1e6]."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        depth = int(rng.integers(d_lo, d_hi + 1))
        p = float(10 ** rng.uniform(-4, -2))
        shots = int(10 ** rng.uniform(5, 6))
        if rng.random() < 0.5:
            circ = brickwork(n, depth, seed=j, p1=p / 10, p2=p)
        else:
            n -= n % 2
            circ = qaoa_3regular(n, max(1, depth // 4), seed=j, p1=p / 10, p2=p)
        out.append((circ, shots))
    return out


WORKLOADS = {
    "random_layers_6q": lambda: random_layers(6, 20, 0, 1e-3, 1e-2),
    "brickwork_20q": lambda: brickwork(20, 40, 0, 1e-3, 1e-2),
    "qaoa_28q": lambda: qaoa_3regular(28, 4, 0, 5e-4, 5e-3),
    # same recipe at 26 qubits (512 MiB complex64 state): the profiling case
    "qaoa_26q": lambda: qaoa_3regular(26, 4, 0, 5e-4, 5e-3),
    # config 2's recipe at 24 qubits (128 MiB complex64 state, above L2)
    "brickwork_24q": lambda: brickwork(24, 40, 0, 1e-3, 1e-2),
}
