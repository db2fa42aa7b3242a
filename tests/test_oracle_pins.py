"""Pins for the CPU oracle against things other than itself: published
known-answer vectors, numpy's Philox, textbook gate matrices and scipy's expm,
brute-force full-matrix simulation, a numpy density-matrix simulation, exact
enumeration of error realizations, closed forms (GHZ Pauli frames, product
states), the paper's commutation rules as matrix identities, and independent
re-derivations of the pruning rule and the tree's branch slots."""
import math
import os

import numpy as np
import pytest

import oracle
import tusq_workloads as W
from tests import bruteforce as BF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- Philox

def _numpy_philox(ctr, key):
    """numpy's Philox is Philox4x64-10 and increments its 256-bit counter
    before producing each block, so start one below the wanted counter."""
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr)) - 1
    v %= 1 << 256
    bg = np.random.Philox(counter=[(v >> (64 * i)) & (2 ** 64 - 1) for i in range(4)],
                          key=[int(k) for k in key])
    return [int(x) for x in bg.random_raw(4)]


def test_philox_known_answers():
    rows = [l for l in open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) >= 2
    for row in rows:
        lhs, rhs = row.split(":")
        words = [int(w, 16) for w in lhs.split()]
        want = [int(w, 16) for w in rhs.split()]
        got = [int(x) for x in oracle.philox4x64_10(words[:4], words[4:6])]
        assert got == want


def test_philox_matches_numpy_random_inputs():
    rng = np.random.default_rng(7)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2 ** 63, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2)]
        assert [int(x) for x in oracle.philox4x64_10(ctr, key)] == _numpy_philox(ctr, key)


def test_er_draw_definition():
    # draw(seed, s, c) = word (c mod 4) of Philox at counter (s, c // 4, 0, 0), key (seed, 0)
    for seed, s, c in [(0, 0, 0), (0, 5, 7), (123, 99999, 181), (2 ** 40, 3, 4)]:
        assert oracle.draw_er(seed, s, c) == _numpy_philox([s, c // 4, 0, 0], [seed, 0])[c % 4]
    assert oracle.draw_prune(9, 4) == _numpy_philox([4, 0, 0, 0], [9, 2])[0]


# --------------------------------------------------------------- gate matrices

@pytest.mark.parametrize("kind", range(16))
def test_gate_matrices_textbook(kind):
    rng = np.random.default_rng(kind)
    if kind in (W.RX, W.RY, W.RZ, W.RZZ):
        params = (rng.uniform(-7, 7),)
    elif kind == W.U1Q:
        params = W.haar_su2(rng)
    elif kind == W.U2Q:
        params = W.random_mixed(2, 1, 3, kinds=(W.U2Q,)).gates[0][3]
    else:
        params = ()
    M = oracle.gate_matrix(kind, params)
    np.testing.assert_allclose(M, BF.textbook_matrix(kind, params), atol=1e-14)
    np.testing.assert_allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-14)


# ------------------------------------------------- statevector vs brute force

@pytest.mark.parametrize("seed", range(6))
def test_simulate_matches_full_matrices(seed):
    n = 2 + seed % 4
    circ = W.random_mixed(n, 25, seed)
    rng = np.random.default_rng(seed)
    events = sorted({(int(rng.integers(0, circ.n_gates + 1)), int(rng.integers(n)),
                      int(rng.integers(1, 4))) for _ in range(4)})
    # one event per (slot, qubit): drop duplicates on the same pair
    seen, ev = set(), []
    for e in events:
        if e[:2] not in seen:
            seen.add(e[:2])
            ev.append(e)
    probs, psi = oracle.simulate(circ, ev, want_state=True)
    ref = BF.state_of_instance(circ, ev)
    np.testing.assert_allclose(psi, ref, atol=1e-12)
    np.testing.assert_allclose(probs, np.abs(ref) ** 2, atol=1e-12)
    assert abs(np.sum(probs) - 1) < 1e-12


def test_p0_is_noiseless_svs():
    circ = W.random_layers(5, 8, seed=3, p1=0.0, p2=0.0)
    probs, pl = oracle.run(circ, 1000, 0)
    assert len(pl.inst) == 1 and pl.inst[0] == () and pl.weights[0] == 1.0
    np.testing.assert_allclose(probs, np.abs(BF.state_of_instance(circ, [])) ** 2, atol=1e-13)


# --------------------------------------------------------------- density matrix

@pytest.mark.parametrize("maker", [
    lambda: W.random_layers(3, 3, seed=1, p1=0.05, p2=0.1),
    lambda: W.random_mixed(3, 10, seed=4, p1=0.05, p2=0.1),
    lambda: W.brickwork(4, 2, seed=2, p1=0.03, p2=0.08),
])
def test_dm_matches_numpy_density_matrix(maker):
    circ = maker()
    np.testing.assert_allclose(oracle.dm_run(circ), BF.dm_bruteforce(circ), atol=1e-13)


def test_exact_enumeration_mixture_equals_dm():
    # Sec. II: a Pauli channel is the weighted average of the fixed-Pauli
    # circuits, so summing every ER's exact probability times its statevector
    # output reproduces the density matrix, up to rounding.
    circ = W.Circuit(3)
    circ.add(W.H, 0, channel=W.depolarizing_1q(0.2))
    circ.add(W.CX, 0, 1, channel=W.depolarizing_2q(0.15))
    circ.add(W.RY, 2, params=(0.7,), channel=W.pauli_twirled_decoherence(1.0, 5.0, 3.0))
    circ.add(W.CZ, 1, 2, channel=W.depolarizing_2q(0.1))
    circ.add(W.RX, 1, params=(1.3,), channel=W.depolarizing_1q(0.3))
    total = np.zeros(8)
    for prob, ev in BF.enumerate_ers(circ):
        total += oracle.simulate(circ, ev, weight=prob)[0]
    np.testing.assert_allclose(total, oracle.dm_run(circ), atol=1e-12)
    np.testing.assert_allclose(total, BF.dm_bruteforce(circ), atol=1e-12)


def test_sampled_mixture_statistically_matches_dm():
    # 6-qubit random-layer workload, 10,000 shots, no pruning: every outcome
    # lies within 6 sigma of the density matrix (each leaf term is in [0, 1]).
    circ = W.random_layers(6, 20, 0, 1e-3, 1e-2)
    S = 10_000
    q, _ = oracle.run(circ, S, seed=0, prune=False)
    qdm = oracle.dm_run(circ)
    assert np.all(np.abs(q - qdm) <= 6 * np.sqrt(qdm / S) + 1e-12)
    assert abs(q.sum() - 1) < 1e-12


def test_seed_average_shrinks_error():
    circ = W.random_layers(4, 6, 1, 2e-2, 5e-2)
    qdm = oracle.dm_run(circ)
    S = 2000
    single = [np.abs(oracle.run(circ, S, seed=s, prune=False)[0] - qdm).sum() for s in range(16)]
    avg = np.mean([oracle.run(circ, S, seed=s, prune=False)[0] for s in range(16)], axis=0)
    err_avg = np.abs(avg - qdm).sum()
    assert err_avg < 0.5 * np.mean(single)     # ~1/4 expected for 16 seeds


# ------------------------------------------------------------------ closed forms

def _frame_xmask(circ, events):
    """Propagate a Pauli frame (x, z bit per qubit) through H and CX."""
    x = [0] * circ.n_qubits
    z = [0] * circ.n_qubits
    for j in range(circ.n_gates + 1):
        for (s, q, p) in events:
            if s == j:
                x[q] ^= p in (1, 2)
                z[q] ^= p in (2, 3)
        if j == circ.n_gates:
            break
        kind, a, b, _ = circ.gates[j]
        if kind == W.H:
            x[a], z[a] = z[a], x[a]
        elif kind == W.CX:
            x[b] ^= x[a]
            z[a] ^= z[b]
    return sum(bit << q for q, bit in enumerate(x))


@pytest.mark.parametrize("seed", range(5))
def test_ghz_instances_are_xor_shifted(seed):
    n = 5
    circ = W.ghz(n, p1=0.1, p2=0.1)
    rng = np.random.default_rng(seed)
    chans = [j for j, c in enumerate(circ.channels) if c is not None]
    events = []
    for j in rng.choice(chans, 3, replace=False):
        code = int(rng.integers(1, 16 if circ.gates[j][0] == W.CX else 4))
        for q, pp in BF.channel_paulis(circ, int(j), code):
            if pp:
                events.append((int(j) + 1, q, pp))
    events.sort()
    probs, _ = oracle.simulate(circ, events)
    m = _frame_xmask(circ, events)
    ideal = np.zeros(1 << n)
    ideal[0] = ideal[(1 << n) - 1] = 0.5
    np.testing.assert_allclose(probs, ideal[np.arange(1 << n) ^ m], atol=1e-13)


def test_product_state_depolarizing_closed_form():
    # P(bit q = 1) = (1 - 2p/3) sin^2(t/2) + (2p/3) cos^2(t/2); the output is the
    # product of the marginals.
    thetas = [0.3, 1.1, 2.0, 2.9]
    p = 0.12
    circ = W.product_rx(thetas, p)
    marg = [(1 - 2 * p / 3) * math.sin(t / 2) ** 2 + (2 * p / 3) * math.cos(t / 2) ** 2 for t in thetas]
    want = np.array([np.prod([marg[q] if (x >> q) & 1 else 1 - marg[q] for q in range(4)])
                     for x in range(16)])
    total = np.zeros(16)
    for prob, ev in BF.enumerate_ers(circ):
        total += oracle.simulate(circ, ev, weight=prob)[0]
    np.testing.assert_allclose(total, want, atol=1e-13)
    np.testing.assert_allclose(oracle.dm_run(circ), want, atol=1e-13)


def test_twirl_formulas():
    codes, probs = W.pauli_twirled_decoherence(1.0, 4.0, 2.0)
    a = (1 - math.exp(-0.25)) / 4
    assert codes == (1, 2, 3)
    assert probs[0] == pytest.approx(a) and probs[1] == pytest.approx(a)
    assert probs[2] == pytest.approx((1 - math.exp(-0.5)) / 2 - a)


# ------------------------------------------------------------------ commutation

def _close_up_to_phase(A, B):
    k = np.argmax(np.abs(B))
    ph = A.flat[k] / B.flat[k]
    return abs(abs(ph) - 1) < 1e-12 and np.allclose(A, ph * B, atol=1e-12)


def test_commutation_rules_are_matrix_identities():
    P = BF.PAULI
    CXm = BF.textbook_matrix(W.CX)
    kr = np.kron
    # rule 2: a Pauli passes a Pauli gate unchanged (up to phase)
    for a in (1, 2, 3):
        for g in (1, 2, 3):
            assert _close_up_to_phase(P[g] @ P[a], P[a] @ P[g])
    # rule 3: X/Y/Z pass R_X/R_Y/R_Z of any angle
    for a, kind in ((1, W.RX), (2, W.RY), (3, W.RZ)):
        R = BF.textbook_matrix(kind, (0.77,))
        assert np.allclose(R @ P[a], P[a] @ R)
    # rule 4: X on control -> X on control and target; X on target stays
    assert _close_up_to_phase(CXm @ kr(P[1], P[0]), kr(P[1], P[1]) @ CXm)
    assert _close_up_to_phase(CXm @ kr(P[0], P[1]), kr(P[0], P[1]) @ CXm)
    # rule 5: Z on target -> Z on both; Z on control stays
    assert _close_up_to_phase(CXm @ kr(P[0], P[3]), kr(P[3], P[3]) @ CXm)
    assert _close_up_to_phase(CXm @ kr(P[3], P[0]), kr(P[3], P[0]) @ CXm)
    # rule 6: Y on control -> Y_c X_t; Y on target -> Z_c Y_t
    assert _close_up_to_phase(CXm @ kr(P[2], P[0]), kr(P[2], P[1]) @ CXm)
    assert _close_up_to_phase(CXm @ kr(P[0], P[2]), kr(P[3], P[2]) @ CXm)
    # Fig. 4(C): X through R_Z(t) would turn it into R_Z(-t)
    Rz = BF.textbook_matrix(W.RZ, (0.9,))
    assert np.allclose(Rz @ P[1], P[1] @ BF.textbook_matrix(W.RZ, (-0.9,)))
    assert not np.allclose(Rz @ P[1], P[1] @ Rz)


def _fig4b_circuit():
    c = W.Circuit(2)
    c.add(W.H, 0, channel=W.depolarizing_1q(0.01))
    c.add(W.CX, 0, 1, channel=W.depolarizing_2q(0.01))
    return c


@pytest.mark.parametrize("mode", [1, 2])
def test_fig4b_x_through_cnot(mode):
    c = _fig4b_circuit()
    a = oracle.commute_one(c, [(0, 1)], mode)           # (X, II)
    b = oracle.commute_one(c, [(1, 4 * 1 + 1)], mode)   # (I, XX)
    assert a == b == ((2, 0, 1), (2, 1, 1))
    # X on control + X on target cancel back to a lone X after H ... and Z
    # on the control passes the CNOT unchanged
    assert oracle.commute_one(c, [(0, 3)], mode) == ((2, 0, 3),)
    # the same ER in "off" mode keeps the raw slot
    assert oracle.commute_one(c, [(0, 1)], 0) == ((1, 0, 1),)


def test_fig4c_x_not_pushed_through_rz():
    c = W.Circuit(1)
    c.add(W.H, 0, channel=W.depolarizing_1q(0.01))
    c.add(W.RZ, 0, params=(0.4,))
    c.add(W.H, 0)
    assert oracle.commute_one(c, [(0, 1)], 2) == ((1, 0, 1),)     # blocked before RZ
    assert oracle.commute_one(c, [(0, 3)], 1) == ((2, 0, 3),)     # Z passes RZ, stops at H (paper mode)
    assert oracle.commute_one(c, [(0, 3)], 2) == ((3, 0, 1),)     # Clifford mode: Z -> X through H


def test_rule1_merge_and_cancel():
    c = W.Circuit(1)
    c.add(W.RX, 0, params=(0.3,), channel=W.depolarizing_1q(0.1))
    c.add(W.RX, 0, params=(0.5,), channel=W.depolarizing_1q(0.1))
    assert oracle.commute_one(c, [(0, 1), (1, 1)], 2) == ()              # X X = I
    # X after the first RX commutes through the second and merges with Z: Y
    assert oracle.commute_one(c, [(0, 1), (1, 3)], 2) == ((2, 0, 2),)


def test_rzz_whole_factor_passes():
    c = W.Circuit(2)
    c.add(W.H, 0, channel=W.depolarizing_1q(0.1))
    c.add(W.H, 1, channel=W.depolarizing_1q(0.1))
    c.add(W.RZZ, 0, 1, params=(0.6,))
    c.add(W.U1Q, 0, params=W.haar_su2(np.random.default_rng(0)))
    c.add(W.U1Q, 1, params=W.haar_su2(np.random.default_rng(1)))
    # X alone anticommutes with ZZ: blocked before the RZZ (slot 2)
    assert oracle.commute_one(c, [(0, 1)], 2) == ((2, 0, 1),)
    # X (x) X commutes with ZZ: passes whole, stops at the U1Q gates
    assert oracle.commute_one(c, [(0, 1), (1, 1)], 2) == ((3, 0, 1), (4, 1, 1))
    # X (x) Z: the Z factor passes alone, the X factor is blocked
    assert oracle.commute_one(c, [(0, 1), (1, 3)], 2) == ((2, 0, 1), (4, 1, 3))
    # paper mode has no RZZ rule
    assert oracle.commute_one(c, [(0, 1), (1, 1)], 1) == ((2, 0, 1), (2, 1, 1))


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("mode", [1, 2])
def test_commutation_is_lossless_bruteforce(seed, mode):
    n = 3 + seed % 2
    circ = W.random_mixed(n, 14, seed, p1=0.2, p2=0.3)
    pl_raw = oracle.plan(circ, 300, seed, commute_mode=0, prune=False)
    chans = [j for j, c in enumerate(circ.channels) if c is not None]
    for er in pl_raw.raw[:40]:
        raw_ev = []
        for (c, code) in er:
            j = chans[c]
            for q, pp in BF.channel_paulis(circ, j, code):
                if pp:
                    raw_ev.append((j + 1, q, pp))
        com_ev = oracle.commute_one(circ, er, mode)
        assert _close_up_to_phase(BF.state_of_instance(circ, com_ev),
                                  BF.state_of_instance(circ, sorted(raw_ev)))


def test_commutation_invariance_of_whole_output():
    circ = W.random_layers(5, 10, 2, 2e-2, 5e-2)
    outs = [oracle.run(circ, 3000, 11, commute_mode=m, prune=False)[0] for m in (0, 1, 2)]
    np.testing.assert_allclose(outs[0], outs[1], atol=1e-12)
    np.testing.assert_allclose(outs[0], outs[2], atol=1e-12)


# --------------------------------------------------------------- sampling/tally

def test_sampled_frequencies_match_channel_probabilities():
    c = W.Circuit(2)
    c.add(W.H, 0, channel=((1, 2, 3), (0.05, 0.02, 0.11)))
    c.add(W.CX, 0, 1, channel=((1, 6, 15), (0.04, 0.07, 0.01)))
    S = 200_000
    pl = oracle.plan(c, S, seed=5, commute_mode=0, prune=False)
    counts = {er: int(cnt) for er, cnt in zip(pl.raw, pl.raw_count)}
    assert sum(counts.values()) == S
    # marginal frequencies of each channel's outcomes vs their probabilities
    for ch, (codes, probs) in enumerate([c.channels[0], c.channels[1]]):
        obs = {k: 0 for k in codes}
        for er, cnt in counts.items():
            for (cc, code) in er:
                if cc == ch:
                    obs[code] += cnt
        for k, p in zip(codes, probs):
            sd = math.sqrt(S * p * (1 - p))
            assert abs(obs[k] - S * p) < 5 * sd


def test_tally_sorted_and_counts_sum():
    circ = W.random_layers(6, 20, 0)
    pl = oracle.plan(circ, 10_000, 0, commute_mode=2, prune=False)
    assert int(pl.raw_count.sum()) == 10_000 and int(pl.key_count.sum()) == 10_000
    assert len(set(pl.raw)) == len(pl.raw)
    assert len(set(pl.keys)) == len(pl.keys)


# --------------------------------------------------------------------- pruning

def _key_lt(a, b):
    """Event-list order: event by event, an ended list sorts after any event."""
    for x, y in zip(a, b):
        if x != y:
            return x < y
    return len(a) > len(b)


def _prune_rederive(keys, counts, S, seed, alpha, beta):
    counts = [int(c) for c in counts]
    cmax = max(counts)
    sig = [i for i, c in enumerate(counts) if c >= alpha * cmax]
    insig = [i for i, c in enumerate(counts) if not c >= alpha * cmax]
    cins = sum(counts[i] for i in insig)
    npick = min(beta, len(insig))
    arr = list(insig)
    for i in range(npick):
        r = _numpy_philox([i, 0, 0, 0], [seed, 2])[0]
        j = i + r % (len(arr) - i)
        arr[i], arr[j] = arr[j], arr[i]
    picked = arr[:npick]
    cpick = sum(counts[i] for i in picked)
    w = {i: counts[i] / S for i in sig}
    for i in picked:
        w[i] = (counts[i] / S) * (cins / cpick)
    return sorted(w), w, len(sig), npick


@pytest.mark.parametrize("alpha,beta", [(0.01, 100), (0.05, 7), (0.0, 5), (1.0, 3)])
def test_pruning_rule_rederived(alpha, beta):
    circ = W.random_layers(6, 20, 0)
    S, seed = 10_000, 3
    full = oracle.plan(circ, S, seed, commute_mode=2, prune=False)
    pr = oracle.plan(circ, S, seed, commute_mode=2, prune=True, alpha=alpha, beta=beta)
    kept, w, nsig, npick = _prune_rederive(full.keys, full.key_count, S, seed, alpha, beta)
    assert pr.n_sig == nsig and pr.n_pick == npick
    # Eq. S_final: significant ones plus min(beta, |C_I|)
    assert len(pr.inst) == nsig + min(beta, pr.n_insig)
    assert list(pr.inst) == [full.keys[i] for i in kept]
    assert list(pr.weights) == [w[i] for i in kept]          # bit-exact FP64
    assert abs(pr.weights.sum() - 1) < 1e-12


# ----------------------------------------------------------- DFS order, branch slots

def test_dfs_order_and_branch_slots_and_edge_count():
    circ = W.random_layers(5, 6, 4, 3e-2, 6e-2)
    G = circ.n_gates
    pl = oracle.plan(circ, 4000, 1, commute_mode=2, prune=False)
    inst = pl.inst
    for a, b in zip(inst, inst[1:]):
        assert _key_lt(a, b)
    # branch slot = smaller slot of the first differing events (ended = G + 1)
    for i, (a, b) in enumerate(zip(inst, inst[1:])):
        k = 0
        while k < min(len(a), len(b)) and a[k] == b[k]:
            k += 1
        sa = a[k][0] if k < len(a) else G + 1
        sb = b[k][0] if k < len(b) else G + 1
        assert pl.lcp[i] == min(sa, sb)
    # explicit trie over token sequences: (events at slot j, then gate j) for
    # every slot; DFTT applies G gates on the first path and 2 (G - t) per
    # branch, i.e. 2|E_gates| - G (Sec. III-B1, T_dftt = 2|E|).
    prefixes = set()
    for ev in inst:
        toks = []
        for j in range(G):
            toks.extend(("e",) + e for e in ev if e[0] == j)
            toks.append(("g", j))
            prefixes.add(tuple(toks))
    n_gate_edges = len(prefixes)
    t_dftt = G + sum(2 * (G - t) for t in pl.lcp)
    assert t_dftt == 2 * n_gate_edges - G
