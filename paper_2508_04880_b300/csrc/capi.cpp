// extern "C" entry points for circuits and plans (host only).
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace tusq {
int build_plan(const tusq_circuit &circ, const tusq_plan_opts &opts, uint64_t shots,
               uint64_t seed, tusq_plan_t &P);
int build_plan_from_instances(const tusq_circuit &circ, uint64_t n_inst, const uint64_t *ev_off,
                              const int32_t *ev_slot, const int32_t *ev_qubit,
                              const int32_t *ev_pauli, const double *weights, tusq_plan_t &P);
int build_plan_shard(const tusq_plan_t &src, int rank, int world, tusq_plan_t &P);

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace tusq

using namespace tusq;

#define TUSQ_FAIL(code, msg) do { set_error(msg); return (code); } while (0)

extern "C" {

const char *tusq_last_error(void) { return g_last_error.c_str(); }

int tusq_circuit_create(int n_qubits, tusq_circuit **out) {
    if (!out) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_create: out is NULL");
    if (n_qubits < 1 || n_qubits > kMaxQubits)
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_create: n_qubits must be in [1, 34]");
    tusq_circuit *c = new (std::nothrow) tusq_circuit;
    if (!c) TUSQ_FAIL(TUSQ_ENOMEM, "tusq_circuit_create: out of host memory");
    c->n = n_qubits;
    *out = c;
    return TUSQ_OK;
}

static int expected_params(int kind) {
    switch (kind) {
    case TUSQ_RX: case TUSQ_RY: case TUSQ_RZ: case TUSQ_RZZ: return 1;
    case TUSQ_U1Q: return 8;
    case TUSQ_U2Q: return 32;
    default: return 0;
    }
}

int tusq_circuit_add_gate(tusq_circuit *c, int kind, int q0, int q1, const double *params,
                          int n_params) {
    if (!c) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: circuit is NULL");
    if (kind < TUSQ_H || kind > TUSQ_MEASURE) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: unknown gate kind");
    if (q0 < 0 || q0 >= c->n) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: q0 out of range");
    bool two = is_two_qubit(kind);
    if (two && (q1 < 0 || q1 >= c->n || q1 == q0))
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: q1 out of range or equal to q0");
    int np = expected_params(kind);
    if (n_params != np || (np > 0 && !params))
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: wrong number of parameters for this kind");
    Gate g;
    g.kind = kind;
    g.q0 = q0;
    g.q1 = two ? q1 : -1;
    for (int i = 0; i < np; ++i) {
        if (!std::isfinite(params[i])) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: non-finite parameter");
        g.p[i] = params[i];
    }
    if (kind == TUSQ_U1Q || kind == TUSQ_U2Q) {
        int d = kind == TUSQ_U1Q ? 2 : 4;
        double err = 0;
        for (int r = 0; r < d; ++r)
            for (int s = 0; s < d; ++s) {
                std::complex<double> acc = 0;
                for (int k = 0; k < d; ++k) {
                    std::complex<double> a(g.p[2 * (d * r + k)], g.p[2 * (d * r + k) + 1]);
                    std::complex<double> b(g.p[2 * (d * s + k)], g.p[2 * (d * s + k) + 1]);
                    acc += a * std::conj(b);
                }
                err += std::abs(acc - (r == s ? 1.0 : 0.0));
            }
        if (err > 1e-9) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_add_gate: matrix is not unitary");
    }
    c->gates.push_back(g);
    c->ch_of_gate.push_back(-1);
    return (int)c->gates.size() - 1;
}

int tusq_circuit_set_channel(tusq_circuit *c, int gate_index, int n_terms, const uint8_t *codes,
                             const double *probs) {
    if (!c) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_set_channel: circuit is NULL");
    if (gate_index < 0 || gate_index >= (int)c->gates.size())
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_set_channel: gate index out of range");
    if (n_terms < 0 || n_terms > 15 || (n_terms > 0 && (!codes || !probs)))
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_set_channel: bad term list");
    int maxcode = is_two_qubit(c->gates[gate_index].kind) ? 15 : 3;
    Channel ch;
    ch.gate = gate_index;
    ch.nterms = n_terms;
    double s = 0;
    for (int k = 0; k < n_terms; ++k) {
        if (codes[k] < 1 || codes[k] > maxcode)
            TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_set_channel: Pauli code out of range for this gate");
        if (!(probs[k] >= 0.0) || !std::isfinite(probs[k]))
            TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_set_channel: negative or non-finite probability");
        ch.codes[k] = codes[k];
        ch.probs[k] = probs[k];
        s += probs[k];
    }
    if (s > 1.0 + 1e-12) TUSQ_FAIL(TUSQ_EINVAL, "tusq_circuit_set_channel: probabilities sum above 1");
    int &slot = c->ch_of_gate[gate_index];
    if (n_terms == 0) {
        slot = -1;
        return TUSQ_OK;
    }
    if (slot >= 0) c->channels[slot] = ch;
    else {
        slot = (int)c->channels.size();
        c->channels.push_back(ch);
    }
    return TUSQ_OK;
}

void tusq_circuit_free(tusq_circuit *c) { delete c; }

int tusq_plan(const tusq_circuit *c, const tusq_plan_opts *opts, uint64_t shots, uint64_t seed,
              tusq_plan_t **out) {
    if (!c || !out) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan: NULL argument");
    if (shots == 0) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan: shots must be positive");
    tusq_plan_opts o{0.01, 100, 1, TUSQ_COMMUTE_CLIFFORD, 0};
    if (opts) o = *opts;
    if (o.commute_mode < 0 || o.commute_mode > 2) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan: bad commute_mode");
    if (!(o.alpha >= 0.0) || o.alpha > 1.0) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan: alpha must be in [0, 1]");
    if (c->gates.size() >= (1u << 22) - 1) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan: too many gates");
    tusq_plan_t *p = new (std::nothrow) tusq_plan_t;
    if (!p) TUSQ_FAIL(TUSQ_ENOMEM, "tusq_plan: out of host memory");
    try {
        int rc = build_plan(*c, o, shots, seed, *p);
        if (rc) { delete p; return rc; }
    } catch (const std::bad_alloc &) {
        delete p;
        TUSQ_FAIL(TUSQ_ENOMEM, "tusq_plan: out of host memory");
    }
    *out = p;
    return TUSQ_OK;
}

int tusq_plan_from_instances(const tusq_circuit *c, uint64_t n_inst, const uint64_t *ev_off,
                             const int32_t *ev_slot, const int32_t *ev_qubit,
                             const int32_t *ev_pauli, const double *weights, tusq_plan_t **out) {
    if (!c || !out || !ev_off || (n_inst && !weights))
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_from_instances: NULL argument");
    if (n_inst && ev_off[n_inst] > ev_off[0] && (!ev_slot || !ev_qubit || !ev_pauli))
        TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_from_instances: NULL event arrays");
    tusq_plan_t *p = new (std::nothrow) tusq_plan_t;
    if (!p) TUSQ_FAIL(TUSQ_ENOMEM, "tusq_plan_from_instances: out of host memory");
    int rc;
    try {
        rc = build_plan_from_instances(*c, n_inst, ev_off, ev_slot, ev_qubit, ev_pauli, weights, *p);
    } catch (const std::bad_alloc &) {
        delete p;
        TUSQ_FAIL(TUSQ_ENOMEM, "tusq_plan_from_instances: out of host memory");
    }
    if (rc) { delete p; return rc; }
    *out = p;
    return TUSQ_OK;
}

int tusq_plan_stats(const tusq_plan_t *p, tusq_plan_stats_t *out) {
    if (!p || !out) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_stats: NULL argument");
    *out = p->stats;
    return TUSQ_OK;
}

int tusq_plan_export(const tusq_plan_t *p, uint64_t *n_inst, const uint64_t **ev_off,
                     const int32_t **ev_slot, const int32_t **ev_qubit, const int32_t **ev_pauli,
                     const uint64_t **counts, const double **weights, const int32_t **lcp) {
    if (!p) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_export: plan is NULL");
    if (n_inst) *n_inst = p->n_inst();
    if (ev_off) *ev_off = p->ev_off.data();
    if (ev_slot) *ev_slot = p->ev_slot.data();
    if (ev_qubit) *ev_qubit = p->ev_qubit.data();
    if (ev_pauli) *ev_pauli = p->ev_pauli.data();
    if (counts) *counts = p->counts.data();
    if (weights) *weights = p->weights.data();
    if (lcp) *lcp = p->lcp.data();
    return TUSQ_OK;
}

int tusq_plan_export_tally(const tusq_plan_t *p, int stage, uint64_t *n, const uint64_t **off,
                           const int32_t **a, const int32_t **b, const int32_t **c,
                           const uint64_t **counts) {
    if (!p) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_export_tally: plan is NULL");
    if (stage != 0 && stage != 1) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_export_tally: stage must be 0 or 1");
    const FlatList &L = stage == 0 ? p->raw : p->commuted;
    if (n) *n = L.size();
    if (off) *off = L.off.data();
    if (a) *a = L.a.data();
    if (b) *b = L.b.data();
    if (c) *c = L.c.data();
    if (counts) *counts = L.count.data();
    return TUSQ_OK;
}

int tusq_plan_shard(const tusq_plan_t *p, int rank, int world, tusq_plan_t **out) {
    if (!p || !out) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_shard: NULL argument");
    if (world < 1 || rank < 0 || rank >= world) TUSQ_FAIL(TUSQ_EINVAL, "tusq_plan_shard: bad rank/world");
    tusq_plan_t *s = new (std::nothrow) tusq_plan_t;
    if (!s) TUSQ_FAIL(TUSQ_ENOMEM, "tusq_plan_shard: out of host memory");
    try {
        build_plan_shard(*p, rank, world, *s);
    } catch (const std::bad_alloc &) {
        delete s;
        TUSQ_FAIL(TUSQ_ENOMEM, "tusq_plan_shard: out of host memory");
    }
    *out = s;
    return TUSQ_OK;
}

int tusq_plan_n_qubits(const tusq_plan_t *p) { return p ? p->n : TUSQ_EINVAL; }

void tusq_plan_free(tusq_plan_t *p) { delete p; }

}  // extern "C"
