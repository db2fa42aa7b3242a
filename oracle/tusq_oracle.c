/*
 * tusq_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately simple CPU reference for the TUSQ noisy
 * statevector path (arXiv 2508.04880).  Everything is complex128 / FP64.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's shared object; the CUDA library never does, and the
 * two share no code, headers or tables.
 *
 * What it computes (paper sections in brackets):
 *   - Pauli-channel noise as a classical mixture of fixed-Pauli circuits
 *     [Sec. II, depolarizing channel as a weighted average of I/X/Y/Z circuits].
 *   - Error-realization (ER) sampling for every shot and ER tallying
 *     [Sec. III-A1].  The random numbers come from Philox4x64-10
 *     (Salmon, Moraes, Dror, Shaw, SC'11), implemented here from its
 *     published definition.
 *   - ER commutation [Sec. III-A2, rules 1-6 in Sec. III-A3], done as a
 *     naive rewrite to a fixpoint (each noisy Pauli is moved one gate at a
 *     time while a rule allows it), not with the paper's per-qubit stacks.
 *   - Optional readout fold of the Paulis left after the last gate: Z
 *     dropped, Y turned into X, since only |psi_x|^2 is observed [Sec. II]
 *     (pinned in tests/test_terminal_fold.py).
 *   - Pruning with alpha / beta and reweighting [Sec. III-A4, Eq. S_final].
 *   - The DFS order of the instance tree and the branch slot between
 *     neighbouring leaves [Sec. III-B].
 *   - Per-instance statevector simulation from |0...0>, with no tree and no
 *     uncomputation, accumulating w_i |psi_x|^2 [Sec. II, Eq. 1].
 *   - A density-matrix simulator rho -> U rho U^dag and
 *     rho -> sum_k p_k P_k rho P_k for n <= 6 [Sec. II], and
 *     rho -> sum_m K_m rho K_m^dag for the non-invertible RESET / MEASURE.
 *   - Non-invertible operations [Sec. III-B2] unravelled into their Kraus
 *     branches: every selected instance is expanded into its 2^R branch
 *     records, each simulated from |0...0> with the unnormalised K_m psi
 *     (pinned against the density matrix in tests/test_noninvertible.py).
 *
 * Conventions (the paper fixes none of them): qubit q is bit q of the
 * amplitude index; for a two-qubit gate on (q0, q1) the local index is
 * 2*bit(q0) + bit(q1); RX/RY/RZ(t) = exp(-i t sigma / 2);
 * RZZ(t) = exp(-i t Z(x)Z / 2); Pauli codes I=0 X=1 Y=2 Z=3 and a two-qubit
 * Pauli is 4*P(q0) + P(q1).
 *
 * Parity pins for each function live in tests/test_oracle_*.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cx;

/* Gate kinds; the numbering is the interface numbering of the circuit format. */
enum {
    OK_H = 0, OK_X, OK_Y, OK_Z, OK_S, OK_SDG, OK_T, OK_TDG,
    OK_RX, OK_RY, OK_RZ, OK_U1Q, OK_CX, OK_CZ, OK_RZZ, OK_U2Q,
    OK_RESET, OK_MEASURE, OK_NKINDS
};
#define OR_OUTCOME1 4 /* event code: the non-invertible gate at this slot takes Kraus branch 1 */
#define OR_PSTRIDE 32 /* doubles of parameters per gate in the flat arrays */

static int two_qubit(int kind)
{
    return kind == OK_CX || kind == OK_CZ || kind == OK_RZZ || kind == OK_U2Q;
}

static int noninvertible(int kind) { return kind == OK_RESET || kind == OK_MEASURE; }

/* Kraus operator K_m of a non-invertible one-qubit operation [Sec. III-B2]:
 * reset to |0> has K_m = |0><m|, a Z measurement K_m = |m><m|;
 * sum_m K_m^dag K_m = I for both. */
static void kraus_2x2(int kind, int m, cx k[4])
{
    k[0] = k[1] = k[2] = k[3] = 0;
    if (kind == OK_RESET) k[m] = 1;          /* row 0, column m */
    else k[3 * m] = 1;                        /* (m, m) */
}

/* ------------------------------------------------------------------ matrices */

static void pauli_2x2(int p, cx m[4])
{
    m[0] = m[1] = m[2] = m[3] = 0;
    if (p == 0) { m[0] = 1; m[3] = 1; }
    if (p == 1) { m[1] = 1; m[2] = 1; }
    if (p == 2) { m[1] = -I; m[2] = I; }
    if (p == 3) { m[0] = 1; m[3] = -1; }
}

/* Row-major matrix of a gate; returns its dimension (2 or 4), 0 if unknown. */
int or_gate_matrix(int kind, const double *prm, double *out_re_im)
{
    cx m[16];
    int d = two_qubit(kind) ? 4 : 2;
    double c, s, r = 1.0 / sqrt(2.0);
    memset(m, 0, sizeof m);
    switch (kind) {
    case OK_H: m[0] = r; m[1] = r; m[2] = r; m[3] = -r; break;
    case OK_X: pauli_2x2(1, m); break;
    case OK_Y: pauli_2x2(2, m); break;
    case OK_Z: pauli_2x2(3, m); break;
    case OK_S: m[0] = 1; m[3] = I; break;
    case OK_SDG: m[0] = 1; m[3] = -I; break;
    case OK_T: m[0] = 1; m[3] = cexp(I * M_PI / 4); break;
    case OK_TDG: m[0] = 1; m[3] = cexp(-I * M_PI / 4); break;
    case OK_RX:
        c = cos(prm[0] / 2); s = sin(prm[0] / 2);
        m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case OK_RY:
        c = cos(prm[0] / 2); s = sin(prm[0] / 2);
        m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    case OK_RZ:
        m[0] = cexp(-I * prm[0] / 2); m[3] = cexp(I * prm[0] / 2); break;
    case OK_U1Q:
        for (int k = 0; k < 4; k++) m[k] = prm[2 * k] + I * prm[2 * k + 1];
        break;
    case OK_CX: m[0] = 1; m[5] = 1; m[11] = 1; m[14] = 1; break;
    case OK_CZ: m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; break;
    case OK_RZZ:
        m[0] = cexp(-I * prm[0] / 2); m[5] = cexp(I * prm[0] / 2);
        m[10] = cexp(I * prm[0] / 2); m[15] = cexp(-I * prm[0] / 2); break;
    case OK_U2Q:
        for (int k = 0; k < 16; k++) m[k] = prm[2 * k] + I * prm[2 * k + 1];
        break;
    default: return 0;
    }
    for (int k = 0; k < d * d; k++) {
        out_re_im[2 * k] = creal(m[k]);
        out_re_im[2 * k + 1] = cimag(m[k]);
    }
    return d;
}

static int gate_cx(int kind, const double *prm, cx *m)
{
    double ri[32];
    int d = or_gate_matrix(kind, prm, ri);
    for (int k = 0; k < d * d; k++) m[k] = ri[2 * k] + I * ri[2 * k + 1];
    return d;
}

/* ------------------------------------------------------ statevector updates */

/* psi <- M psi on qubit q (Eq. 1 with k = 1). */
static void apply_1q(cx *psi, int n, int q, const cx m[4])
{
    int64_t dim = (int64_t)1 << n, bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static) if (n >= 16)
    for (int64_t i = 0; i < dim; i++) {
        if (i & bit) continue;
        cx a = psi[i], b = psi[i | bit];
        psi[i] = m[0] * a + m[1] * b;
        psi[i | bit] = m[2] * a + m[3] * b;
    }
}

/* psi <- M psi on (q0, q1), local index 2*bit(q0) + bit(q1) (Eq. 1, k = 2). */
static void apply_2q(cx *psi, int n, int q0, int q1, const cx m[16])
{
    int64_t dim = (int64_t)1 << n, b0 = (int64_t)1 << q0, b1 = (int64_t)1 << q1;
#pragma omp parallel for schedule(static) if (n >= 16)
    for (int64_t i = 0; i < dim; i++) {
        if ((i & b0) || (i & b1)) continue;
        int64_t idx[4] = {i, i | b1, i | b0, i | b0 | b1};
        cx v[4], w[4];
        for (int k = 0; k < 4; k++) v[k] = psi[idx[k]];
        for (int r = 0; r < 4; r++) {
            w[r] = 0;
            for (int c = 0; c < 4; c++) w[r] += m[4 * r + c] * v[c];
        }
        for (int k = 0; k < 4; k++) psi[idx[k]] = w[k];
    }
}

static void apply_gate(cx *psi, int n, int kind, int q0, int q1, const double *prm)
{
    cx m[16];
    gate_cx(kind, prm, m);
    if (two_qubit(kind)) apply_2q(psi, n, q0, q1, m);
    else apply_1q(psi, n, q0, m);
}

static void apply_pauli(cx *psi, int n, int q, int p)
{
    cx m[4];
    if (p == 0) return;
    pauli_2x2(p, m);
    apply_1q(psi, n, q, m);
}

/*
 * Simulate one fixed-Pauli circuit instance from |0...0>: for every slot
 * j = 0..G, the instance's Paulis at slot j, then gate j (slot G has no gate).
 * Events must be sorted by slot.  The final state goes to psi_out (2^n
 * complex as re,im pairs) if given, and w * |psi_x|^2 is added to acc if given.
 */
int or_simulate(int n, int G, const int *kinds, const int *q0, const int *q1,
                const double *params, int n_ev, const int *ev_slot,
                const int *ev_q, const int *ev_p, double w, double *acc,
                double *psi_out)
{
    int64_t dim = (int64_t)1 << n;
    cx *psi = calloc((size_t)dim, sizeof(cx));
    if (!psi) return -1;
    psi[0] = 1;
    int e = 0;
    for (int j = 0; j <= G; j++) {
        int branch = 0;
        while (e < n_ev && ev_slot[e] == j) {
            if (ev_p[e] == OR_OUTCOME1) {
                if (j == G || !noninvertible(kinds[j]) || ev_q[e] != q0[j]) { free(psi); return -3; }
                branch = 1;
            } else {
                apply_pauli(psi, n, ev_q[e], ev_p[e]);
            }
            e++;
        }
        if (j < G && noninvertible(kinds[j])) {
            /* the unnormalised Kraus branch: its norm carries the branch probability */
            cx k[4];
            kraus_2x2(kinds[j], branch, k);
            apply_1q(psi, n, q0[j], k);
        } else if (j < G) {
            apply_gate(psi, n, kinds[j], q0[j], q1[j], params + (int64_t)OR_PSTRIDE * j);
        }
    }
    if (e != n_ev) { free(psi); return -2; } /* unsorted or out-of-range slot */
    if (acc) {
#pragma omp parallel for schedule(static) if (n >= 16)
        for (int64_t i = 0; i < dim; i++) {
            double a = cabs(psi[i]);
            acc[i] += w * a * a;
        }
    }
    if (psi_out)
        for (int64_t i = 0; i < dim; i++) {
            psi_out[2 * i] = creal(psi[i]);
            psi_out[2 * i + 1] = cimag(psi[i]);
        }
    free(psi);
    return 0;
}

/* Simulate instances [first, first + count) of a flattened instance list
 * (events of instance i are [off[i], off[i+1])) and accumulate their
 * weighted output probabilities into acc. */
int or_run_instances(int n, int G, const int *kinds, const int *q0, const int *q1,
                     const double *params, const int64_t *off, const int *ev_slot,
                     const int *ev_q, const int *ev_p, const double *weights,
                     int64_t first, int64_t count, double *acc)
{
    for (int64_t i = first; i < first + count; i++) {
        int64_t a = off[i], b = off[i + 1];
        int rc = or_simulate(n, G, kinds, q0, q1, params, (int)(b - a), ev_slot + a,
                             ev_q + a, ev_p + a, weights[i], acc, NULL);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------ density matrix (n<=6) */

/* rho <- M rho M^dag for a gate given as a full 2^n x 2^n operator built by
 * applying M to every column, then conj(M) to every row. */
static void dm_apply_gate_cols_rows(cx *rho, int n, int kind, int q0, int q1, const cx *m)
{
    int64_t dim = (int64_t)1 << n;
    cx *col = malloc(sizeof(cx) * dim);
    cx mc[16];
    int d = two_qubit(kind) ? 4 : 2;
    for (int k = 0; k < d * d; k++) mc[k] = conj(m[k]);
    for (int64_t c = 0; c < dim; c++) {
        for (int64_t r = 0; r < dim; r++) col[r] = rho[r * dim + c];
        if (d == 4) apply_2q(col, n, q0, q1, m); else apply_1q(col, n, q0, m);
        for (int64_t r = 0; r < dim; r++) rho[r * dim + c] = col[r];
    }
    for (int64_t r = 0; r < dim; r++) {
        cx *row = rho + r * dim;
        if (d == 4) apply_2q(row, n, q0, q1, mc); else apply_1q(row, n, q0, mc);
    }
    free(col);
}

/* Density-matrix simulation of the whole noisy circuit: after gate j, if it
 * has a channel, rho <- (1 - sum p) rho + sum_k p_k P_k rho P_k (Sec. II).
 * probs_out receives diag(rho).  Only for n <= 6 (4096 x 4096 at most ...). */
int or_dm_run(int n, int G, const int *kinds, const int *q0, const int *q1,
              const double *params, const int *ch_of_gate, const int *ch_nterms,
              const int *ch_codes, const double *ch_probs, double *probs_out)
{
    if (n > 8) return -1;
    int64_t dim = (int64_t)1 << n, sz = dim * dim;
    cx *rho = calloc((size_t)sz, sizeof(cx));
    cx *acc = calloc((size_t)sz, sizeof(cx));
    cx *tmp = calloc((size_t)sz, sizeof(cx));
    rho[0] = 1;
    for (int j = 0; j < G; j++) {
        cx m[16];
        if (noninvertible(kinds[j])) {
            /* rho <- sum_m K_m rho K_m^dag [Sec. III-B2] */
            for (int64_t i = 0; i < sz; i++) acc[i] = 0;
            for (int b = 0; b < 2; b++) {
                kraus_2x2(kinds[j], b, m);
                memcpy(tmp, rho, sizeof(cx) * sz);
                dm_apply_gate_cols_rows(tmp, n, kinds[j], q0[j], -1, m);
                for (int64_t i = 0; i < sz; i++) acc[i] += tmp[i];
            }
            memcpy(rho, acc, sizeof(cx) * sz);
        } else {
            gate_cx(kinds[j], params + (int64_t)OR_PSTRIDE * j, m);
            dm_apply_gate_cols_rows(rho, n, kinds[j], q0[j], q1[j], m);
        }
        int c = ch_of_gate[j];
        if (c < 0) continue;
        double ptot = 0;
        for (int k = 0; k < ch_nterms[c]; k++) ptot += ch_probs[15 * c + k];
        for (int64_t i = 0; i < sz; i++) acc[i] = (1.0 - ptot) * rho[i];
        for (int k = 0; k < ch_nterms[c]; k++) {
            int code = ch_codes[15 * c + k];
            memcpy(tmp, rho, sizeof(cx) * sz);
            int pa, pb;
            if (two_qubit(kinds[j])) { pa = code >> 2; pb = code & 3; }
            else { pa = code; pb = 0; }
            cx pm[4];
            /* P rho P for a Hermitian Pauli: apply P to columns then rows. */
            if (pa) { pauli_2x2(pa, pm); dm_apply_gate_cols_rows(tmp, n, OK_X, q0[j], -1, pm); }
            if (pb) { pauli_2x2(pb, pm); dm_apply_gate_cols_rows(tmp, n, OK_X, q1[j], -1, pm); }
            for (int64_t i = 0; i < sz; i++) acc[i] += ch_probs[15 * c + k] * tmp[i];
        }
        memcpy(rho, acc, sizeof(cx) * sz);
    }
    for (int64_t i = 0; i < dim; i++) probs_out[i] = creal(rho[i * dim + i]);
    free(rho); free(acc); free(tmp);
    return 0;
}

/* ------------------------------------------------------------- Philox4x64-10 */

static uint64_t mulhilo64(uint64_t a, uint64_t b, uint64_t *hi)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    return (uint64_t)p;
}

/* Philox4x64 with 10 rounds (Salmon et al., SC'11): each round multiplies
 * words 0 and 2 by the two Philox multipliers, swaps and xors in the key;
 * the key is bumped by the two Weyl constants between rounds. */
void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t hi0, hi1;
        uint64_t lo0 = mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0);
        uint64_t lo1 = mulhilo64(0xCA5A826395121157ULL, c2, &hi1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 64-bit draw for (shot s, channel c) under a seed: word (c mod 4) of
 * Philox4x64-10 at counter (s, floor(c/4), 0, 0), key (seed, 0). */
static uint64_t draw_er(uint64_t seed, uint64_t s, uint64_t c)
{
    uint64_t ctr[4] = {s, c / 4, 0, 0}, key[2] = {seed, 0}, out[4];
    or_philox4x64_10(ctr, key, out);
    return out[c % 4];
}

/* The 64-bit draw number i of the pruning pick stream: word 0 of
 * Philox4x64-10 at counter (i, 0, 0, 0), key (seed, 2). */
static uint64_t draw_prune(uint64_t seed, uint64_t i)
{
    uint64_t ctr[4] = {i, 0, 0, 0}, key[2] = {seed, 2}, out[4];
    or_philox4x64_10(ctr, key, out);
    return out[0];
}

/* Integer threshold of a cumulative probability: floor(x * 2^64), clamped. */
static uint64_t cdf_threshold(double x)
{
    if (x >= 1.0) return UINT64_MAX;
    if (x <= 0.0) return 0;
    return (uint64_t)(x * 18446744073709551616.0);
}

/* ------------------------------------------------------- shot sampling */

/* Shots drawn from an output distribution.  The paper samples the output
 * state vector of each kept instance s_i times (Sec. III-A1); here the
 * shots are drawn from the tally-weighted mixture the traversal returns.
 * Each outcome gets the fixed-point weight w_x = floor(p_x * 2^56) (0 for
 * p_x <= 0), C_x = w_0 + ... + w_x is the integer cumulative weight and
 * W = C_(2^n - 1).  Shot s takes r = word 0 of Philox4x64-10 at counter
 * (s, 0, 0, 0), key (seed, 3), the target t = floor(r * W / 2^64) (< W) and
 * lands on the first x with C_x > t.  counts[x] = shots landing on x.
 * Returns -1 when W = 0 (nothing to sample). */
uint64_t or_draw_sample(uint64_t seed, uint64_t s)
{
    uint64_t ctr[4] = {s, 0, 0, 0}, key[2] = {seed, 3}, out[4];
    or_philox4x64_10(ctr, key, out);
    return out[0];
}

int or_sample(int n, const double *probs, uint64_t shots, uint64_t seed, uint64_t *counts)
{
    uint64_t dim = (uint64_t)1 << n;
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * dim);
    if (!C) return -2;
    uint64_t acc = 0;
    for (uint64_t x = 0; x < dim; x++) {
        double p = probs[x];
        uint64_t w = p > 0.0 ? (uint64_t)(p * 72057594037927936.0) : 0;   /* 2^56 */
        acc += w;
        C[x] = acc;
        counts[x] = 0;
    }
    if (acc == 0) { free(C); return -1; }
    for (uint64_t s = 0; s < shots; s++) {
        uint64_t r = or_draw_sample(seed, s);
        uint64_t t = (uint64_t)(((unsigned __int128)r * acc) >> 64);
        /* first x with C[x] > t (C is non-decreasing and C[dim-1] = acc > t) */
        uint64_t lo = 0, hi = dim - 1;
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > t) hi = mid; else lo = mid + 1;
        }
        counts[lo]++;
    }
    free(C);
    return 0;
}

/* --------------------------------------------------------------- the plan */

typedef struct { int slot, q, p; } ev_t;

typedef struct {
    int n, G, C;
    const int *kinds, *q0, *q1, *ch_gate;
    uint64_t shots;
    /* raw tally (sorted) */
    int64_t n_raw;
    int64_t *raw_off;
    int *raw_ch, *raw_code;
    uint64_t *raw_count;
    /* commuted tally (sorted) */
    int64_t n_key;
    int64_t *key_off;
    ev_t *key_ev;
    uint64_t *key_count;
    /* selected instances in DFS order */
    int64_t n_inst;
    int64_t *inst_off;
    ev_t *inst_ev;
    uint64_t *inst_count;
    double *inst_w;
    int *lcp;
    int64_t n_sig, n_insig, n_pick;
    uint64_t c_max, c_insig, c_pick;
} or_plan;

/* Comparison of two event lists: event by event (slot, qubit, pauli); a list
 * that has ended compares greater than any event (the end sentinel sorts
 * last). */
static int cmp_events(const ev_t *a, int na, const ev_t *b, int nb)
{
    for (int i = 0;; i++) {
        if (i == na && i == nb) return 0;
        if (i == na) return 1;
        if (i == nb) return -1;
        if (a[i].slot != b[i].slot) return a[i].slot < b[i].slot ? -1 : 1;
        if (a[i].q != b[i].q) return a[i].q < b[i].q ? -1 : 1;
        if (a[i].p != b[i].p) return a[i].p < b[i].p ? -1 : 1;
    }
}

/* Raw ERs compare as lists of (channel, code) with the same end rule. */
static int cmp_raw(const int *ca, const int *pa, int na, const int *cb, const int *pb, int nb)
{
    for (int i = 0;; i++) {
        if (i == na && i == nb) return 0;
        if (i == na) return 1;
        if (i == nb) return -1;
        if (ca[i] != cb[i]) return ca[i] < cb[i] ? -1 : 1;
        if (pa[i] != pb[i]) return pa[i] < pb[i] ? -1 : 1;
    }
}

/* qsort needs the arrays through file-scope pointers. */
static const int64_t *g_off;
static const int *g_ch, *g_code;
static const ev_t *g_ev;

static int qs_raw(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    int r = cmp_raw(g_ch + g_off[a], g_code + g_off[a], (int)(g_off[a + 1] - g_off[a]),
                    g_ch + g_off[b], g_code + g_off[b], (int)(g_off[b + 1] - g_off[b]));
    if (r) return r;
    return a < b ? -1 : (a > b);
}

static int qs_key(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    int r = cmp_events(g_ev + g_off[a], (int)(g_off[a + 1] - g_off[a]),
                       g_ev + g_off[b], (int)(g_off[b + 1] - g_off[b]));
    if (r) return r;
    return a < b ? -1 : (a > b);
}

/* ---------------------------------------------------- commutation (naive) */

/* Pauli product with the phase dropped (rule 1): as bit pairs X=01 Z=10,
 * Y=11 in (x, z) form the product is the xor. */
static int pauli_mul(int a, int b)
{
    static const int to_xz[4] = {0, 1, 3, 2}; /* I X Y Z -> x + 2z */
    static const int from_xz[4] = {0, 1, 3, 2};
    return from_xz[to_xz[a] ^ to_xz[b]];
}

/* Does the (up to) two-qubit Pauli pa (x) pb pass gate j, and what does it
 * become?  Decided numerically from the gate's matrix:
 *   - Clifford kinds allowed by the mode: P' = U P U^dag must be a Pauli up to
 *     phase; it is found by comparing against all candidates.
 *   - rotation kinds (RX, RY, RZ, T, TDG, RZZ): P passes unchanged iff it
 *     commutes with the rotation's generator (so that the gate's angle is not
 *     changed, Sec. III-A2 and Fig. 4(C)).
 *   - everything else blocks.
 * Mode 1 ("paper") allows the rule set of Sec. III-A3: Pauli gates (rule 2),
 * same-axis rotations RX/RY/RZ (rule 3), CX (rules 4-6).  Mode 2 adds the
 * remaining parameter-free Cliffords (H, S, SDG, CZ) and the commuting rule
 * for T, TDG and RZZ. */
static int pass_gate(int mode, int kind, int pa, int pb, int *oa, int *ob)
{
    int clifford = 0, rotation = 0;
    cx gen[16];
    switch (kind) {
    case OK_X: case OK_Y: case OK_Z: case OK_CX: clifford = 1; break;
    case OK_H: case OK_S: case OK_SDG: case OK_CZ: clifford = (mode >= 2); break;
    case OK_RX: rotation = 1; pauli_2x2(1, gen); break;
    case OK_RY: rotation = 1; pauli_2x2(2, gen); break;
    case OK_RZ: rotation = 1; pauli_2x2(3, gen); break;
    case OK_T: case OK_TDG: rotation = (mode >= 2); pauli_2x2(3, gen); break;
    case OK_RZZ:
        rotation = (mode >= 2);
        memset(gen, 0, sizeof gen);
        gen[0] = 1; gen[5] = -1; gen[10] = -1; gen[15] = 1;
        break;
    default: break;
    }
    int d = two_qubit(kind) ? 4 : 2;
    cx P[16];
    /* Full Pauli on the gate's support, local index 2*bit(q0)+bit(q1). */
    if (d == 2) pauli_2x2(pa, P);
    else {
        cx A[4], B[4];
        pauli_2x2(pa, A); pauli_2x2(pb, B);
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++)
                P[4 * r + c] = A[2 * (r >> 1) + (c >> 1)] * B[2 * (r & 1) + (c & 1)];
    }
    if (rotation) {
        double err = 0;
        for (int r = 0; r < d; r++)
            for (int c = 0; c < d; c++) {
                cx s1 = 0, s2 = 0;
                for (int k = 0; k < d; k++) {
                    s1 += P[d * r + k] * gen[d * k + c];
                    s2 += gen[d * r + k] * P[d * k + c];
                }
                err += cabs(s1 - s2);
            }
        if (err > 1e-9) return 0;
        *oa = pa; *ob = pb;
        return 1;
    }
    if (!clifford) return 0;
    cx U[16], T1[16], Q[16];
    double zero[OR_PSTRIDE] = {0};
    gate_cx(kind, zero, U);
    /* Q = U P U^dag */
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            cx s = 0;
            for (int k = 0; k < d; k++) s += U[d * r + k] * P[d * k + c];
            T1[d * r + c] = s;
        }
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            cx s = 0;
            for (int k = 0; k < d; k++) s += T1[d * r + k] * conj(U[d * c + k]);
            Q[d * r + c] = s;
        }
    int ncand = (d == 2) ? 4 : 16;
    for (int cand = 0; cand < ncand; cand++) {
        int ca = (d == 2) ? cand : cand >> 2, cb = (d == 2) ? 0 : cand & 3;
        cx C[16];
        if (d == 2) pauli_2x2(ca, C);
        else {
            cx A[4], B[4];
            pauli_2x2(ca, A); pauli_2x2(cb, B);
            for (int r = 0; r < 4; r++)
                for (int c = 0; c < 4; c++)
                    C[4 * r + c] = A[2 * (r >> 1) + (c >> 1)] * B[2 * (r & 1) + (c & 1)];
        }
        /* proportional with a unit-modulus factor? */
        cx ph = 0;
        for (int k = 0; k < d * d; k++)
            if (cabs(C[k]) > 0.5) { ph = Q[k] / C[k]; break; }
        if (fabs(cabs(ph) - 1.0) > 1e-9) continue;
        double err = 0;
        for (int k = 0; k < d * d; k++) err += cabs(Q[k] - ph * C[k]);
        if (err < 1e-9) { *oa = ca; *ob = cb; return 1; }
    }
    return 0;
}

typedef struct { int q, p, slot; } npauli_t; /* a noisy Pauli sitting before gate `slot` */

/* Next gate index >= from that acts on qubit q (G if none), by a plain scan. */
static int next_gate_on(const or_plan *P, int q, int from)
{
    for (int j = from; j < P->G; j++)
        if (P->q0[j] == q || (two_qubit(P->kinds[j]) && P->q1[j] == q)) return j;
    return P->G;
}

/* Remove element i of v (order is not kept; the list is sorted at the end). */
static void drop(npauli_t *v, int *nv, int i) { v[i] = v[--*nv]; }

/* Commute one raw ER to its canonical event list (Sec. III-A2/3).  The noisy
 * Paulis start right after their channel's gate; then, until nothing changes:
 * each Pauli is placed at the next gate on its wire, Paulis waiting at the
 * same gate on the same wire are multiplied together (rule 1, identities
 * dropped), and at the lowest-index gate where something can move, the Paulis
 * waiting on its support are pushed through it: the whole factor if it
 * passes, otherwise each single-qubit factor that passes on its own (factors
 * are never split further).  Mode 0 keeps the raw positions. */
static int commute_er(const or_plan *P, int mode, const int *chs, const int *codes, int ne,
                      ev_t **out)
{
    int vcap = 2 * ne + 8;
    npauli_t *v = malloc(sizeof(npauli_t) * vcap);
    int nv = 0;
    for (int i = 0; i < ne; i++) {
        int j = P->ch_gate[chs[i]];
        if (two_qubit(P->kinds[j])) {
            int pa = codes[i] >> 2, pb = codes[i] & 3;
            if (pa) v[nv++] = (npauli_t){P->q0[j], pa, j + 1};
            if (pb) v[nv++] = (npauli_t){P->q1[j], pb, j + 1};
        } else {
            v[nv++] = (npauli_t){P->q0[j], codes[i], j + 1};
        }
    }
    int changed = (mode > 0);
    while (changed) {
        changed = 0;
        for (int i = 0; i < nv; i++) v[i].slot = next_gate_on(P, v[i].q, v[i].slot);
        /* rule 1 */
        for (int i = 0; i < nv; i++)
            for (int k = i + 1; k < nv; k++)
                if (v[k].q == v[i].q && v[k].slot == v[i].slot) {
                    v[i].p = pauli_mul(v[i].p, v[k].p);
                    drop(v, &nv, k);
                    k--;
                    changed = 1;
                }
        for (int i = 0; i < nv; i++)
            if (v[i].p == 0) { drop(v, &nv, i); i--; changed = 1; }
        if (changed) continue;
        /* one push, at the lowest gate index where one is possible */
        int best_j = P->G, best_ia = -1, best_ib = -1, ra = 0, rb = 0;
        for (int i = 0; i < nv; i++) {
            int j = v[i].slot;
            if (j >= best_j) continue;
            int ia = -1, ib = -1;
            for (int k = 0; k < nv; k++) {
                if (v[k].slot != j) continue;
                if (v[k].q == P->q0[j]) ia = k;
                else if (two_qubit(P->kinds[j]) && v[k].q == P->q1[j]) ib = k;
            }
            int pa = ia >= 0 ? v[ia].p : 0, pb = ib >= 0 ? v[ib].p : 0;
            int oa, ob, sa, sb, move_a = 0, move_b = 0, xa = 0, xb = 0;
            if (pass_gate(mode, P->kinds[j], pa, pb, &oa, &ob)) {
                move_a = (ia >= 0); move_b = (ib >= 0); xa = oa; xb = ob;
            } else if (two_qubit(P->kinds[j])) {
                if (pa && pass_gate(mode, P->kinds[j], pa, 0, &oa, &ob)) {
                    move_a = 1; xa = pauli_mul(xa, oa); xb = pauli_mul(xb, ob);
                }
                if (pb && pass_gate(mode, P->kinds[j], 0, pb, &sa, &sb)) {
                    move_b = 1; xa = pauli_mul(xa, sa); xb = pauli_mul(xb, sb);
                }
            }
            if (!move_a && !move_b) continue;
            best_j = j;
            best_ia = move_a ? ia : -1;
            best_ib = move_b ? ib : -1;
            ra = xa; rb = xb;
        }
        if (best_j == P->G) break;
        int j = best_j;
        if (best_ia >= 0 && best_ib >= 0) {
            int hi = best_ia > best_ib ? best_ia : best_ib, lo = best_ia + best_ib - hi;
            drop(v, &nv, hi);
            drop(v, &nv, lo);
        } else {
            drop(v, &nv, best_ia >= 0 ? best_ia : best_ib);
        }
        if (nv + 2 > vcap) {
            vcap *= 2;
            v = realloc(v, sizeof(npauli_t) * vcap);
        }
        if (ra) v[nv++] = (npauli_t){P->q0[j], ra, j + 1};
        if (rb) v[nv++] = (npauli_t){P->q1[j], rb, j + 1};
        changed = 1;
    }
    if (mode > 0)
        for (int i = 0; i < nv; i++) v[i].slot = next_gate_on(P, v[i].q, v[i].slot);
    /* sort by (slot, qubit) with a plain insertion sort */
    for (int i = 1; i < nv; i++) {
        npauli_t t = v[i];
        int k = i - 1;
        while (k >= 0 && (v[k].slot > t.slot || (v[k].slot == t.slot && v[k].q > t.q))) {
            v[k + 1] = v[k];
            k--;
        }
        v[k + 1] = t;
    }
    *out = malloc(sizeof(ev_t) * (nv + 1));
    for (int i = 0; i < nv; i++) (*out)[i] = (ev_t){v[i].slot, v[i].q, v[i].p};
    free(v);
    return nv;
}

/* Kraus branches of the non-invertible gates [Sec. III-B2]: each selected
 * instance is replaced by its 2^R branch records (m_1 .. m_R over the R
 * RESET / MEASURE gates in gate order), written as outcome events
 * (j_r, q_r, OR_OUTCOME1) for the gates with m_r = 1; every record keeps the
 * instance's count and weight (the unnormalised branch states carry the
 * branch probabilities).  The list is then sorted back into DFS order.
 * Returns -1 when the expansion would exceed 2^24 instances. */
static int expand_kraus(or_plan *P)
{
    int R = 0;
    for (int j = 0; j < P->G; j++) R += noninvertible(P->kinds[j]);
    if (R == 0) return 0;
    if (R > 24 || (P->n_inst << R) > ((int64_t)1 << 24)) return -1;
    int *js = malloc(sizeof(int) * R);
    R = 0;
    for (int j = 0; j < P->G; j++) if (noninvertible(P->kinds[j])) js[R++] = j;
    int64_t nb = (int64_t)1 << R, nout = P->n_inst * nb;
    int64_t cap = (P->inst_off[P->n_inst] + (int64_t)R * P->n_inst) * nb + 1;
    int64_t *off = malloc(sizeof(int64_t) * (nout + 1));
    ev_t *ev = malloc(sizeof(ev_t) * cap);
    uint64_t *cnt = malloc(sizeof(uint64_t) * (nout + 1));
    double *w = malloc(sizeof(double) * (nout + 1));
    int64_t k = 0, e = 0;
    for (int64_t i = 0; i < P->n_inst; i++)
        for (int64_t b = 0; b < nb; b++) {
            off[k] = e;
            int64_t start = e;
            for (int64_t x = P->inst_off[i]; x < P->inst_off[i + 1]; x++) ev[e++] = P->inst_ev[x];
            for (int r = 0; r < R; r++)
                if (b >> r & 1) ev[e++] = (ev_t){js[r], P->q0[js[r]], OR_OUTCOME1};
            /* insertion sort of this list by (slot, qubit, code) */
            for (int64_t x = start + 1; x < e; x++) {
                ev_t t = ev[x];
                int64_t y = x - 1;
                while (y >= start && cmp_events(&t, 1, &ev[y], 1) < 0) { ev[y + 1] = ev[y]; y--; }
                ev[y + 1] = t;
            }
            cnt[k] = P->inst_count[i];
            w[k] = P->inst_w[i];
            k++;
        }
    off[nout] = e;
    int64_t *ord = malloc(sizeof(int64_t) * nout);
    for (int64_t i = 0; i < nout; i++) ord[i] = i;
    g_off = off; g_ev = ev;
    qsort(ord, nout, sizeof(int64_t), qs_key);
    free(P->inst_off); free(P->inst_ev); free(P->inst_count); free(P->inst_w); free(P->lcp);
    P->inst_off = malloc(sizeof(int64_t) * (nout + 1));
    P->inst_ev = malloc(sizeof(ev_t) * (e + 1));
    P->inst_count = malloc(sizeof(uint64_t) * (nout + 1));
    P->inst_w = malloc(sizeof(double) * (nout + 1));
    P->lcp = malloc(sizeof(int) * (nout + 1));
    int64_t f = 0;
    for (int64_t i = 0; i < nout; i++) {
        int64_t o = ord[i];
        P->inst_off[i] = f;
        memcpy(P->inst_ev + f, ev + off[o], sizeof(ev_t) * (off[o + 1] - off[o]));
        f += off[o + 1] - off[o];
        P->inst_count[i] = cnt[o];
        P->inst_w[i] = w[o];
    }
    P->inst_off[nout] = f;
    P->n_inst = nout;
    free(js); free(off); free(ev); free(cnt); free(w); free(ord);
    return 0;
}

void or_plan_free(void *h)
{
    or_plan *P = h;
    if (!P) return;
    free(P->raw_off); free(P->raw_ch); free(P->raw_code); free(P->raw_count);
    free(P->key_off); free(P->key_ev); free(P->key_count);
    free(P->inst_off); free(P->inst_ev); free(P->inst_count); free(P->inst_w); free(P->lcp);
    free(P);
}

/*
 * The whole Error Characterization Module (Sec. III-A) plus the DFS order
 * (Sec. III-B):
 *  1. sample every channel for every shot (threshold rule on Philox draws);
 *  2. tally identical ERs (sort + run-length count);
 *  3. commute each distinct ER, re-tally the resulting event lists;
 *  4. prune: significant iff count >= alpha * c_max (FP64 comparison); pick
 *     min(beta, |C_I|) insignificant instances uniformly without replacement
 *     (partial Fisher-Yates over C_I in key order, j = i + r mod (|C_I| - i));
 *     weights w = c / S for significant ones and
 *     (c / S) * (C_insig / sum of picked counts) for picked ones;
 *     with prune == 0 every instance is kept with w = c / S;
 *  5. sort the kept instances by key and compute the branch slot between
 *     neighbours: the smaller slot of the first differing events (an ended
 *     list counts as slot G + 1).
 */
void *or_plan_build(int n, int G, const int *kinds, const int *q0, const int *q1,
                    int C, const int *ch_gate, const int *ch_nterms, const int *ch_codes,
                    const double *ch_probs, uint64_t shots, uint64_t seed,
                    int commute_mode, int prune, double alpha, int64_t beta, int terminal_fold)
{
    or_plan *P = calloc(1, sizeof(or_plan));
    P->n = n; P->G = G; P->C = C; P->kinds = kinds; P->q0 = q0; P->q1 = q1;
    P->ch_gate = ch_gate; P->shots = shots;

    /* thresholds T[c][k]: outcome = first k with r < T[c][k]; k = 0 is I */
    uint64_t *thr = malloc(sizeof(uint64_t) * 16 * (C > 0 ? C : 1));
    for (int c = 0; c < C; c++) {
        int K = ch_nterms[c];
        double s = 0;
        for (int k = 0; k < K; k++) s += ch_probs[15 * c + k];
        double cdf = 1.0 - s;
        thr[16 * c] = cdf_threshold(cdf);
        for (int k = 1; k <= K; k++) {
            cdf += ch_probs[15 * c + k - 1];
            thr[16 * c + k] = (k == K) ? UINT64_MAX : cdf_threshold(cdf);
        }
    }
    /* 1. sample */
    int64_t cap = 1024, used = 0;
    int *ech = malloc(sizeof(int) * cap), *ecode = malloc(sizeof(int) * cap);
    int64_t *soff = malloc(sizeof(int64_t) * (shots + 1));
    for (uint64_t s = 0; s < shots; s++) {
        soff[s] = used;
        for (int c = 0; c < C; c++) {
            uint64_t r = draw_er(seed, s, (uint64_t)c);
            int K = ch_nterms[c], k = 0;
            while (k < K && !(r < thr[16 * c + k])) k++;
            if (k == 0) continue;
            if (used == cap) {
                cap *= 2;
                ech = realloc(ech, sizeof(int) * cap);
                ecode = realloc(ecode, sizeof(int) * cap);
            }
            ech[used] = c;
            ecode[used] = ch_codes[15 * c + k - 1];
            used++;
        }
    }
    soff[shots] = used;
    free(thr);
    /* 2. tally */
    int64_t *ord = malloc(sizeof(int64_t) * (shots ? shots : 1));
    for (uint64_t s = 0; s < shots; s++) ord[s] = (int64_t)s;
    g_off = soff; g_ch = ech; g_code = ecode;
    qsort(ord, shots, sizeof(int64_t), qs_raw);
    P->raw_off = malloc(sizeof(int64_t) * (shots + 1));
    P->raw_ch = malloc(sizeof(int) * (used + 1));
    P->raw_code = malloc(sizeof(int) * (used + 1));
    P->raw_count = malloc(sizeof(uint64_t) * (shots + 1));
    int64_t nr = 0, ne = 0;
    for (uint64_t i = 0; i < shots; i++) {
        int64_t s = ord[i];
        int len = (int)(soff[s + 1] - soff[s]);
        if (nr > 0) {
            int64_t a = P->raw_off[nr - 1];
            if (cmp_raw(P->raw_ch + a, P->raw_code + a, (int)(ne - a), ech + soff[s],
                        ecode + soff[s], len) == 0) {
                P->raw_count[nr - 1]++;
                continue;
            }
        }
        P->raw_off[nr] = ne;
        memcpy(P->raw_ch + ne, ech + soff[s], sizeof(int) * len);
        memcpy(P->raw_code + ne, ecode + soff[s], sizeof(int) * len);
        ne += len;
        P->raw_count[nr] = 1;
        nr++;
    }
    P->raw_off[nr] = ne;
    P->n_raw = nr;
    free(ord); free(soff); free(ech); free(ecode);

    /* 3. commute every distinct ER, then re-tally */
    int64_t ecap = 2 * ne + 64;
    ev_t *kev = malloc(sizeof(ev_t) * ecap);
    int64_t *koff = malloc(sizeof(int64_t) * (nr + 1));
    int64_t kused = 0;
    for (int64_t i = 0; i < nr; i++) {
        koff[i] = kused;
        int len = (int)(P->raw_off[i + 1] - P->raw_off[i]);
        ev_t *one;
        int m = commute_er(P, commute_mode, P->raw_ch + P->raw_off[i],
                           P->raw_code + P->raw_off[i], len, &one);
        if (terminal_fold) {
            /* readout fold (Sec. II, output = |psi_x|^2): after the last
             * gate Z leaves every |psi_x|^2 unchanged and Y = iXZ acts on
             * them as X does, so Z events at slot G go and Y becomes X */
            int kept = 0;
            for (int e = 0; e < m; e++) {
                ev_t t = one[e];
                if (t.slot == G) {
                    if (t.p == 3) continue;
                    t.p = 1;
                }
                one[kept++] = t;
            }
            m = kept;
        }
        if (kused + m > ecap) {
            ecap = 2 * (kused + m);
            kev = realloc(kev, sizeof(ev_t) * ecap);
        }
        memcpy(kev + kused, one, sizeof(ev_t) * m);
        free(one);
        kused += m;
    }
    koff[nr] = kused;
    int64_t *kord = malloc(sizeof(int64_t) * (nr ? nr : 1));
    for (int64_t i = 0; i < nr; i++) kord[i] = i;
    g_off = koff; g_ev = kev;
    qsort(kord, nr, sizeof(int64_t), qs_key);
    P->key_off = malloc(sizeof(int64_t) * (nr + 1));
    P->key_ev = malloc(sizeof(ev_t) * (kused + 1));
    P->key_count = malloc(sizeof(uint64_t) * (nr + 1));
    int64_t nk = 0, ke = 0;
    for (int64_t i = 0; i < nr; i++) {
        int64_t r = kord[i];
        int len = (int)(koff[r + 1] - koff[r]);
        if (nk > 0) {
            int64_t a = P->key_off[nk - 1];
            if (cmp_events(P->key_ev + a, (int)(ke - a), kev + koff[r], len) == 0) {
                P->key_count[nk - 1] += P->raw_count[r];
                continue;
            }
        }
        P->key_off[nk] = ke;
        memcpy(P->key_ev + ke, kev + koff[r], sizeof(ev_t) * len);
        ke += len;
        P->key_count[nk] = P->raw_count[r];
        nk++;
    }
    P->key_off[nk] = ke;
    P->n_key = nk;
    free(kord); free(koff); free(kev);

    /* 4. prune */
    char *keep = calloc((size_t)(nk ? nk : 1), 1);
    double *w = calloc((size_t)(nk ? nk : 1), sizeof(double));
    uint64_t cmax = 0;
    for (int64_t i = 0; i < nk; i++) if (P->key_count[i] > cmax) cmax = P->key_count[i];
    P->c_max = cmax;
    if (!prune) {
        for (int64_t i = 0; i < nk; i++) { keep[i] = 1; w[i] = (double)P->key_count[i] / (double)shots; }
        P->n_sig = nk;
    } else {
        int64_t *insig = malloc(sizeof(int64_t) * (nk ? nk : 1));
        int64_t ni = 0;
        uint64_t cins = 0;
        for (int64_t i = 0; i < nk; i++) {
            if ((double)P->key_count[i] >= alpha * (double)cmax) {
                keep[i] = 1;
                w[i] = (double)P->key_count[i] / (double)shots;
                P->n_sig++;
            } else {
                insig[ni++] = i;
                cins += P->key_count[i];
            }
        }
        P->n_insig = ni;
        P->c_insig = cins;
        int64_t npick = beta < ni ? beta : ni;
        for (int64_t i = 0; i < npick; i++) {
            uint64_t r = draw_prune(seed, (uint64_t)i);
            int64_t j = i + (int64_t)(r % (uint64_t)(ni - i));
            int64_t t = insig[i]; insig[i] = insig[j]; insig[j] = t;
        }
        uint64_t cpick = 0;
        for (int64_t i = 0; i < npick; i++) cpick += P->key_count[insig[i]];
        for (int64_t i = 0; i < npick; i++) {
            int64_t k = insig[i];
            keep[k] = 1;
            w[k] = ((double)P->key_count[k] / (double)shots) * ((double)cins / (double)cpick);
        }
        P->n_pick = npick;
        P->c_pick = cpick;
        free(insig);
    }
    /* 5. kept instances in key order (already sorted) and branch slots */
    int64_t nin = 0, iev = 0;
    for (int64_t i = 0; i < nk; i++) if (keep[i]) { nin++; iev += P->key_off[i + 1] - P->key_off[i]; }
    P->n_inst = nin;
    P->inst_off = malloc(sizeof(int64_t) * (nin + 1));
    P->inst_ev = malloc(sizeof(ev_t) * (iev + 1));
    P->inst_count = malloc(sizeof(uint64_t) * (nin + 1));
    P->inst_w = malloc(sizeof(double) * (nin + 1));
    P->lcp = malloc(sizeof(int) * (nin + 1));
    int64_t m = 0, e = 0;
    for (int64_t i = 0; i < nk; i++) {
        if (!keep[i]) continue;
        int64_t len = P->key_off[i + 1] - P->key_off[i];
        P->inst_off[m] = e;
        memcpy(P->inst_ev + e, P->key_ev + P->key_off[i], sizeof(ev_t) * len);
        e += len;
        P->inst_count[m] = P->key_count[i];
        P->inst_w[m] = w[i];
        m++;
    }
    P->inst_off[m] = e;
    if (expand_kraus(P) != 0) {
        free(keep); free(w);
        or_plan_free(P);
        return NULL;
    }
    nin = P->n_inst;
    for (int64_t i = 0; i + 1 < nin; i++) {
        const ev_t *a = P->inst_ev + P->inst_off[i], *b = P->inst_ev + P->inst_off[i + 1];
        int na = (int)(P->inst_off[i + 1] - P->inst_off[i]);
        int nb = (int)(P->inst_off[i + 2] - P->inst_off[i + 1]);
        int k = 0;
        while (k < na && k < nb && a[k].slot == b[k].slot && a[k].q == b[k].q && a[k].p == b[k].p) k++;
        int sa = k < na ? a[k].slot : G + 1, sb = k < nb ? b[k].slot : G + 1;
        P->lcp[i] = sa < sb ? sa : sb;
    }
    free(keep); free(w);
    return P;
}

/* sizes: n_raw, raw events, n_key, key events, n_inst, inst events, n_sig,
 * n_insig, n_pick, c_max, c_insig, c_pick */
void or_plan_sizes(const void *h, int64_t out[12])
{
    const or_plan *P = h;
    out[0] = P->n_raw; out[1] = P->raw_off[P->n_raw];
    out[2] = P->n_key; out[3] = P->key_off[P->n_key];
    out[4] = P->n_inst; out[5] = P->inst_off[P->n_inst];
    out[6] = P->n_sig; out[7] = P->n_insig; out[8] = P->n_pick;
    out[9] = (int64_t)P->c_max; out[10] = (int64_t)P->c_insig; out[11] = (int64_t)P->c_pick;
}

void or_plan_raw(const void *h, int64_t *off, int *ch, int *code, uint64_t *count)
{
    const or_plan *P = h;
    memcpy(off, P->raw_off, sizeof(int64_t) * (P->n_raw + 1));
    memcpy(ch, P->raw_ch, sizeof(int) * P->raw_off[P->n_raw]);
    memcpy(code, P->raw_code, sizeof(int) * P->raw_off[P->n_raw]);
    memcpy(count, P->raw_count, sizeof(uint64_t) * P->n_raw);
}

static void unpack_events(const ev_t *ev, int64_t n, int *slot, int *q, int *p)
{
    for (int64_t i = 0; i < n; i++) { slot[i] = ev[i].slot; q[i] = ev[i].q; p[i] = ev[i].p; }
}

void or_plan_keys(const void *h, int64_t *off, int *slot, int *q, int *p, uint64_t *count)
{
    const or_plan *P = h;
    memcpy(off, P->key_off, sizeof(int64_t) * (P->n_key + 1));
    unpack_events(P->key_ev, P->key_off[P->n_key], slot, q, p);
    memcpy(count, P->key_count, sizeof(uint64_t) * P->n_key);
}

void or_plan_instances(const void *h, int64_t *off, int *slot, int *q, int *p,
                       uint64_t *count, double *w, int *lcp)
{
    const or_plan *P = h;
    memcpy(off, P->inst_off, sizeof(int64_t) * (P->n_inst + 1));
    unpack_events(P->inst_ev, P->inst_off[P->n_inst], slot, q, p);
    memcpy(count, P->inst_count, sizeof(uint64_t) * P->n_inst);
    memcpy(w, P->inst_w, sizeof(double) * P->n_inst);
    if (P->n_inst > 1) memcpy(lcp, P->lcp, sizeof(int) * (P->n_inst - 1));
}

/* Commute one raw ER (list of channel indices and outcome codes) and return
 * its event list; used by tests of individual rules. */
int or_commute_one(int n, int G, const int *kinds, const int *q0, const int *q1,
                   const int *ch_gate, int mode, int ne, const int *chs, const int *codes,
                   int *slot, int *q, int *p, int cap)
{
    or_plan P;
    memset(&P, 0, sizeof P);
    P.n = n; P.G = G; P.kinds = kinds; P.q0 = q0; P.q1 = q1; P.ch_gate = ch_gate;
    ev_t *tmp;
    int m = commute_er(&P, mode, chs, codes, ne, &tmp);
    if (m > cap) { free(tmp); return -1; }
    if (m > 0) unpack_events(tmp, m, slot, q, p);
    free(tmp);
    return m;
}

/* The raw sampling draw, exposed for tests of the threshold rule. */
uint64_t or_draw_er(uint64_t seed, uint64_t shot, uint64_t channel)
{
    return draw_er(seed, shot, channel);
}

uint64_t or_draw_prune(uint64_t seed, uint64_t i) { return draw_prune(seed, i); }
