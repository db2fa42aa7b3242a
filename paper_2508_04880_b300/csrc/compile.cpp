// Schedule compiler: turns a plan (DFS-ordered instances and branch slots)
// into the device program of one DFTT traversal (Sec. III-B): forward
// segments split at the branch slots that will be revisited, uncompute
// segments back to each branch slot, fused passes over qubit windows, and
// register stages inside each pass.  Non-invertible gates (RESET, MEASURE)
// are never uncomputed: a return across one restores the branch node's
// snapshot, or the DFTT+Caching state saved just before the layer (Sec.
// III-B2) followed by an uncompute up to the node, or re-derives the node
// forward from the deepest saved state above it (or |0..0>), whichever
// applies fewer ops.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <stdexcept>
#include <unordered_map>

#include "internal.h"
#include "program.h"

namespace tusq {

using cd = std::complex<double>;

namespace {

// ----------------------------------------------------------------- host ops

enum HType { H_MAT1 = 0, H_MAT2 = 1, H_DIAG = 2, H_DENSE = 3 };

struct HOp {
    int type = H_MAT1;
    int q0 = 0, q1 = -1;          // MAT2: basis index 2*bit(q0) + bit(q1)
    bool pauli = false;
    bool noninv = false;          // a Kraus branch of RESET / MEASURE: never inverted
    int key = 0;                  // canonical position: 2*slot for events, 2*slot+1 for gates
    int uid = 0;                  // identity within the instance (for set differences)
    std::vector<int> merged;      // uids of ops merged into this one (besides uid)
    cd m[16];
    double phi0 = 0;              // DIAG, in turns
    std::vector<std::pair<uint64_t, double>> terms;   // (global mask, turns)
    // H_DENSE: a run of thread-independent ops of one register stage as one
    // 32x32 matrix in the register basis (row-major, <i|U|j>), applied on the
    // tensor cores; phi0 / terms then hold the absorbed diagonal terms on
    // fixed (non-register) bits only, a per-thread constant phase
    std::vector<cd> du;
    uint64_t qmask() const {
        if (type == H_DIAG) {
            uint64_t m = 0;
            for (auto &t : terms) m |= t.first;
            return m;
        }
        return (1ULL << q0) | (q1 >= 0 ? (1ULL << q1) : 0);
    }
};

const double kPi = 3.14159265358979323846;

void gate_matrix(const Gate &g, cd *m) {
    const cd I(0, 1);
    double r = 1.0 / std::sqrt(2.0);
    for (int k = 0; k < 16; ++k) m[k] = 0;
    switch (g.kind) {
    case TUSQ_H: m[0] = r; m[1] = r; m[2] = r; m[3] = -r; break;
    case TUSQ_X: m[1] = 1; m[2] = 1; break;
    case TUSQ_Y: m[1] = -I; m[2] = I; break;
    case TUSQ_RX: {
        double c = std::cos(g.p[0] / 2), s = std::sin(g.p[0] / 2);
        m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    }
    case TUSQ_RY: {
        double c = std::cos(g.p[0] / 2), s = std::sin(g.p[0] / 2);
        m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    }
    case TUSQ_U1Q: for (int k = 0; k < 4; ++k) m[k] = cd(g.p[2 * k], g.p[2 * k + 1]); break;
    case TUSQ_CX: m[0] = 1; m[5] = 1; m[11] = 1; m[14] = 1; break;
    case TUSQ_U2Q: for (int k = 0; k < 16; ++k) m[k] = cd(g.p[2 * k], g.p[2 * k + 1]); break;
    case TUSQ_RESET: case TUSQ_MEASURE: m[0] = 1; break;   // Kraus branch 0: |0><0|
    default: throw std::logic_error("gate_matrix: not a dense kind");
    }
}

// Kraus branch 1 of a non-invertible gate: |0><1| (RESET) or |1><1| (MEASURE).
void kraus1(int kind, cd *m) {
    for (int k = 0; k < 4; ++k) m[k] = 0;
    if (kind == TUSQ_RESET) m[1] = 1;
    else m[3] = 1;
}

// Diagonal gates as exp(2 pi i (phi0 + sum_k phi_k parity(x & mask_k))).
void gate_diag(const Gate &g, HOp &op) {
    uint64_t a = 1ULL << g.q0, b = g.q1 >= 0 ? 1ULL << g.q1 : 0;
    switch (g.kind) {
    case TUSQ_Z: op.terms = {{a, 0.5}}; break;
    case TUSQ_S: op.terms = {{a, 0.25}}; break;
    case TUSQ_SDG: op.terms = {{a, -0.25}}; break;
    case TUSQ_T: op.terms = {{a, 0.125}}; break;
    case TUSQ_TDG: op.terms = {{a, -0.125}}; break;
    case TUSQ_RZ:      // diag(e^{-it/2}, e^{it/2})
        op.phi0 = -g.p[0] / (4 * kPi); op.terms = {{a, g.p[0] / (2 * kPi)}}; break;
    case TUSQ_CZ:      // pi * x_a x_b = (pi/2)(x_a + x_b - (x_a xor x_b))
        op.terms = {{a, 0.25}, {b, 0.25}, {a | b, -0.25}}; break;
    case TUSQ_RZZ:     // exp(-i t/2 (-1)^(x_a xor x_b))
        op.phi0 = -g.p[0] / (4 * kPi); op.terms = {{a | b, g.p[0] / (2 * kPi)}}; break;
    default: throw std::logic_error("gate_diag: not a diagonal kind");
    }
}

HOp gate_op(const Gate &g, int j) {
    HOp op;
    op.key = 2 * j + 1;
    op.q0 = g.q0;
    op.q1 = g.q1;
    if (is_diagonal(g.kind)) {
        op.type = H_DIAG;
        gate_diag(g, op);
    } else {
        op.type = is_two_qubit(g.kind) ? H_MAT2 : H_MAT1;
        gate_matrix(g, op.m);
        op.noninv = is_noninvertible(g.kind);
    }
    return op;
}

HOp pauli_op(int slot, int q, int p) {
    HOp op;
    op.key = 2 * slot;
    op.q0 = q;
    op.pauli = true;
    const cd I(0, 1);
    if (p == 3) {
        op.type = H_DIAG;
        op.terms = {{1ULL << q, 0.5}};
    } else {
        op.type = H_MAT1;
        for (auto &z : op.m) z = 0;
        if (p == 1) { op.m[1] = 1; op.m[2] = 1; }
        else { op.m[1] = -I; op.m[2] = I; }
    }
    return op;
}

HOp inverse(const HOp &o) {
    if (o.noninv) throw std::logic_error("compile: uncompute across a non-invertible gate");
    HOp r = o;
    if (o.type == H_DIAG) {
        r.phi0 = -o.phi0;
        for (auto &t : r.terms) t.second = -t.second;
    } else {
        int d = o.type == H_MAT1 ? 2 : 4;
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) r.m[d * i + k] = std::conj(o.m[d * k + i]);
    }
    return r;
}

// --------------------------------------------------------- pass scheduling

struct Pass {
    std::vector<int> win;          // global qubits, ascending
    std::vector<HOp> ops;          // in application order
};

// Greedy list scheduling over the dependence DAG of `ops` (two ops depend
// on each other if they share a qubit, unless both are diagonal).  A group
// has a window of at most `cap` bits (qubits_of gives the bits of a
// non-diagonal op; diagonal ops fit any window) and takes every op that
// becomes ready and fits.  When nothing more fits, the window grows by the
// bits of one blocked ready op: the choice that lets the most ops into the
// group (found by trying each candidate; the trial is undone afterwards).
template <class QubitsOf>
std::vector<std::vector<int>> schedule(const std::vector<HOp> &ops, int cap, uint64_t forced,
                                       QubitsOf qubits_of, std::vector<uint64_t> *wins,
                                       bool lookahead = true) {
    const int m = (int)ops.size();
    std::vector<std::vector<int>> succ(m);
    std::vector<int> indeg(m, 0);
    std::vector<uint64_t> wq(m);
    for (int b = 0; b < m; ++b) wq[b] = ops[b].type == H_DIAG ? 0 : qubits_of(ops[b]);
    // dependences by qubit: an op follows the last non-diagonal op on each of
    // its qubits; a non-diagonal op also follows the diagonal ops on its
    // qubits since then (diagonal ops commute with each other)
    {
        std::vector<int> last_nd(64, -1);
        std::vector<std::vector<int>> diag_since(64);
        std::vector<int> mark(m, -1);
        auto edge = [&](int a, int b) {
            if (a < 0 || mark[a] == b) return;
            mark[a] = b;
            succ[a].push_back(b);
            indeg[b]++;
        };
        for (int b = 0; b < m; ++b) {
            const uint64_t qm = ops[b].qmask();
            const bool diag = ops[b].type == H_DIAG;
            for (int q = 0; q < 64; ++q) {
                if (!(qm >> q & 1)) continue;
                edge(last_nd[q], b);
                if (!diag)
                    for (int a : diag_since[q]) edge(a, b);
            }
            for (int q = 0; q < 64; ++q) {
                if (!(qm >> q & 1)) continue;
                if (diag) diag_since[q].push_back(b);
                else { last_nd[q] = b; diag_since[q].clear(); }
            }
        }
    }
    std::vector<int> ready;       // ready and not yet scheduled (blocked by the window)
    for (int b = 0; b < m; ++b)
        if (indeg[b] == 0) ready.push_back(b);
    // schedule everything that fits W, starting from `ready`; returns the
    // scheduled ops in application order and leaves the blocked ones in
    // ready.  With `undo`, every in-degree decrement is logged so that a
    // trial can be rolled back.
    std::vector<int> work, blocked;
    auto closure = [&](uint64_t W, std::vector<int> &rdy, std::vector<int> *out, std::vector<int> *undo) {
        int count = 0;
        work.clear();
        blocked.clear();
        std::sort(rdy.begin(), rdy.end());
        work.insert(work.end(), rdy.begin(), rdy.end());
        size_t h = 0;
        while (h < work.size()) {
            int b = work[h++];
            if ((wq[b] & ~W) != 0) { blocked.push_back(b); continue; }
            ++count;
            if (out) out->push_back(b);
            for (int s : succ[b]) {
                if (undo) undo->push_back(s);
                if (--indeg[s] == 0) work.push_back(s);
            }
        }
        if (!undo) rdy = blocked;
        return count;
    };
    int left = m;
    std::vector<std::vector<int>> groups;
    std::vector<int> undo;
    while (left > 0) {
        uint64_t W = forced;
        std::vector<int> g;
        left -= closure(W, ready, &g, nullptr);
        for (;;) {
            // candidate window extensions: the bits of each blocked ready op
            int best = -1;
            int best_gain = -1;
            uint64_t best_q = 0;
            std::vector<uint64_t> tried;
            for (int b : ready) {
                uint64_t q = wq[b] & ~W;
                if (__builtin_popcountll(W | q) > cap) continue;
                if (std::find(tried.begin(), tried.end(), q) != tried.end()) continue;
                tried.push_back(q);
                if (!lookahead) {   // list order: the first blocked op that fits
                    if (best < 0 || b < best) { best = b; best_q = q; }
                    continue;
                }
                undo.clear();
                std::vector<int> rdy2 = ready;
                int gain = closure(W | q, rdy2, nullptr, &undo);
                for (int s : undo) indeg[s]++;
                int nb = __builtin_popcountll(q);
                // most ops per added bit first, then fewer bits, then list order
                if (best < 0 || gain > best_gain ||
                    (gain == best_gain &&
                     nb < __builtin_popcountll(best_q))) {
                    best = b;
                    best_gain = gain;
                    best_q = q;
                }
            }
            if (best < 0) break;
            W |= best_q;
            left -= closure(W, ready, &g, nullptr);
        }
        if (g.empty()) throw std::logic_error("schedule: no progress (gate wider than window?)");
        groups.push_back(g);
        if (wins) wins->push_back(W);
    }
    return groups;
}

// Merge neighbouring diagonal ops (unless `diag` is false) and neighbouring
// 1q matrices on the same qubit inside one op list (application order).
std::vector<HOp> merge_ops(const std::vector<HOp> &in, bool diag = true) {
    std::vector<HOp> out;
    auto absorb = [](HOp &p, const HOp &o) {
        p.merged.push_back(o.uid);
        p.merged.insert(p.merged.end(), o.merged.begin(), o.merged.end());
        p.pauli = false;
        p.noninv = p.noninv || o.noninv;
    };
    for (const HOp &o : in) {
        if (!out.empty()) {
            HOp &p = out.back();
            if (diag && o.type == H_DIAG && p.type == H_DIAG &&
                p.terms.size() + o.terms.size() <= (size_t)kMaxDiagTerms) {
                p.phi0 += o.phi0;
                for (auto &t : o.terms) {
                    bool hit = false;
                    for (auto &u : p.terms)
                        if (u.first == t.first) { u.second += t.second; hit = true; break; }
                    if (!hit) p.terms.push_back(t);
                }
                absorb(p, o);
                continue;
            }
            if (o.type == H_MAT1 && p.type == H_MAT1 && o.q0 == p.q0) {
                cd r[4];
                for (int i = 0; i < 2; ++i)
                    for (int k = 0; k < 2; ++k)
                        r[2 * i + k] = o.m[2 * i] * p.m[k] + o.m[2 * i + 1] * p.m[2 + k];
                for (int k = 0; k < 4; ++k) p.m[k] = r[k];
                absorb(p, o);
                continue;
            }
        }
        out.push_back(o);
    }
    return out;
}

// Move each diagonal op of a pass to the register stage where its terms are
// cheapest.  A stage applies a term whose qubits are all outside its register
// bits as one parity per thread added to the thread's constant phase, but a
// term on register bits as a sweep over the thread's registers for its
// register-mask group (shared by the terms of one group in the same run).
// Diagonal ops commute with each other, so an op may sit in any stage from the
// one of the last non-diagonal op before it on one of its qubits to the one of
// the first non-diagonal op after it (stage lists are in application order).
// Rs[s] is stage s's register-bit mask over local bits; local[q] the local
// bit of global qubit q (-1 outside the window: a tile bit, never a register).
void place_diagonals(const std::vector<HOp> &ops, std::vector<std::vector<int>> &sched,
                     const std::vector<uint64_t> &Rs, const int *local) {
    const int S = (int)sched.size();
    const int m = (int)ops.size();
    if (S < 2) return;
    std::vector<int> stage_of(m, -1);
    for (int s = 0; s < S; ++s)
        for (int b : sched[s]) stage_of[b] = s;
    auto reg_mask = [&](uint64_t qmask, int s) {
        uint64_t mu = 0;
        for (uint64_t q = qmask; q; q &= q - 1) {
            const int l = local[__builtin_ctzll(q)];
            if (l >= 0 && (Rs[s] >> l & 1)) mu |= 1ULL << l;
        }
        return mu;
    };
    // per stage: the register-mask groups of its diagonal terms, and how many
    // diagonal ops it holds
    std::vector<std::vector<uint64_t>> groups(S);
    std::vector<int> ndiag(S, 0);
    auto account = [&](int b, int s, bool add) {
        ndiag[s] += add ? 1 : -1;
        auto &g = groups[s];
        for (const auto &t : ops[b].terms) {
            const uint64_t mu = reg_mask(t.first, s);
            if (!mu) continue;
            if (add) g.push_back(mu);
            else g.erase(std::find(g.begin(), g.end(), mu));
        }
    };
    // estimated instructions per amplitude of adding op b to stage s
    constexpr double kFixedTerm = 0.25, kSharedGroup = 0.3, kNewGroup = 2.8, kNewStage = 0.5;
    auto cost = [&](int b, int s) {
        double c = ndiag[s] == 0 ? kNewStage : 0.0;
        std::vector<uint64_t> seen;
        for (const auto &t : ops[b].terms) {
            const uint64_t mu = reg_mask(t.first, s);
            if (!mu) {
                c += kFixedTerm;
                continue;
            }
            const bool shared = std::find(groups[s].begin(), groups[s].end(), mu) != groups[s].end() ||
                                std::find(seen.begin(), seen.end(), mu) != seen.end();
            c += shared ? kSharedGroup : kNewGroup;
            seen.push_back(mu);
        }
        return c;
    };
    for (int b = 0; b < m; ++b)
        if (ops[b].type == H_DIAG) account(b, stage_of[b], true);
    for (int b = 0; b < m; ++b) {
        if (ops[b].type != H_DIAG) continue;
        const uint64_t qm = ops[b].qmask();
        int lo = 0, hi = S - 1;
        for (int a = 0; a < m; ++a) {
            if (ops[a].type == H_DIAG || !(ops[a].qmask() & qm)) continue;
            if (a < b) lo = std::max(lo, stage_of[a]);
            else hi = std::min(hi, stage_of[a]);
        }
        const int s0 = stage_of[b];
        if (lo >= hi) continue;
        account(b, s0, false);
        int best = s0;
        double best_cost = cost(b, s0);
        for (int s = lo; s <= hi; ++s) {
            if (s == s0) continue;
            const double c = cost(b, s);
            if (c < best_cost - 1e-9) {   // strictly cheaper: ties keep the scheduled stage
                best = s;
                best_cost = c;
            }
        }
        account(b, best, true);
        if (best == s0) continue;
        auto &from = sched[s0];
        from.erase(std::find(from.begin(), from.end(), b));
        // a later non-diagonal op on its qubits in the new stage (best == hi):
        // before the stage's ops; otherwise after them (best == lo may hold an
        // earlier one)
        bool later_here = false;
        for (int a : sched[best])
            if (a > b && ops[a].type != H_DIAG && (ops[a].qmask() & qm)) later_here = true;
        if (later_here) sched[best].insert(sched[best].begin(), b);
        else sched[best].push_back(b);
        stage_of[b] = best;
    }
}

// ------------------------------------------------------------- encoding

inline uint32_t swz(uint32_t e, bool c128) { return tile_swizzle(e, c128); }

// Structure of a matrix op: real entries, or [[c, -is], [-is, c]] (RX-type;
// tangent form SUB_RXT when |c| >= |s|, else SUB_RXS).
uint32_t mat1_sub(const cd *m) {
    bool real = true;
    for (int k = 0; k < 4; ++k) real = real && m[k].imag() == 0.0;
    if (real) return SUB_REAL;
    if (m[0] == m[3] && m[0].imag() == 0.0 && m[1] == m[2] && m[1].real() == 0.0) {
        const double c = m[0].real(), sn = -m[1].imag();
        return std::fabs(c) >= std::fabs(sn) ? SUB_RXT : SUB_RXS;
    }
    return SUB_GENERAL;
}

// The four matrix entries the kernels read for a 2x2 of form `sub`: the
// matrix itself, or for the tangent forms the parameter in entry 0 (t = s/c
// or k = c/s) with the factor taken out (c, or -is) multiplied into *K.
void encode_mat1(const cd *m, uint32_t sub, cd *out, cd &K) {
    if (sub == SUB_RXT || sub == SUB_RXS) {
        const double c = m[0].real(), sn = -m[1].imag();
        out[1] = out[2] = out[3] = 0;
        if (sub == SUB_RXT) {
            out[0] = sn / c;
            K *= c;
        } else {
            out[0] = c / sn;
            K *= cd(0, -sn);
        }
        return;
    }
    for (int k = 0; k < 4; ++k) out[k] = m[k];
}

// A 4x4 that exchanges two basis states and fixes the others (CX in some
// basis order): returns true with the two states.
bool mat2_swap(const cd *m, int &s0, int &s1) {
    int perm[4];
    for (int r = 0; r < 4; ++r) {
        perm[r] = -1;
        for (int c = 0; c < 4; ++c) {
            if (m[4 * r + c] == cd(1, 0)) {
                if (perm[r] >= 0) return false;
                perm[r] = c;
            } else if (m[4 * r + c] != cd(0, 0)) {
                return false;
            }
        }
        if (perm[r] < 0) return false;
    }
    int moved[4], nm = 0;
    for (int r = 0; r < 4; ++r)
        if (perm[r] != r) moved[nm++] = r;
    if (nm != 2 || perm[moved[0]] != moved[1] || perm[moved[1]] != moved[0]) return false;
    s0 = moved[0];
    s1 = moved[1];
    return true;
}

// SIMT cost of an op in FP32 instructions per amplitude (register-stage
// estimate used to decide which thread-independent runs go to the tensor
// cores): a general 2x2 is 8, a real one 4, the tangent forms 2, a 4x4 16, a
// basis swap 6, each register-mask group of a diagonal run 2.
double simt_cost(const HOp &o, const uint64_t *greg, int v) {
    if (o.type == H_MAT1) {
        const uint32_t sub = mat1_sub(o.m);
        return sub == SUB_GENERAL ? 8.0 : sub == SUB_REAL ? 4.0 : 2.0;
    }
    if (o.type == H_MAT2) {
        int s0, s1;
        return mat2_swap(o.m, s0, s1) ? 6.0 : 16.0;
    }
    uint32_t groups = 0;
    for (auto &t : o.terms) {
        int mu = 0;
        for (int i = 0; i < v; ++i)
            if (t.first & greg[i]) mu |= 1 << i;
        groups |= 1u << mu;
    }
    return 2.0 * __builtin_popcount(groups & ~1u) + 0.5;
}

uint64_t to_fixed(double turns, bool c128) {
    double f = turns - std::floor(turns);
    if (c128) {
        long double v = (long double)f * 9223372036854775808.0L;   // 2^63
        return (uint64_t)llroundl(v) & 0x7FFFFFFFFFFFFFFFULL;
    }
    return (uint64_t)llround(f * 2147483648.0) & 0x7FFFFFFFULL;     // 2^31
}

struct Encoder {
    Program &prog;
    int n;
    bool c128;
    int V;
    int Lmax;
    bool lookahead = true;
    bool place_diag = true;     // move diagonal ops to their cheapest register stage
    int tc_mode = TUSQ_TC_NONE;
    // dense ops' matrices already in the pool: hash of U's bits -> pool
    // indices, and each entry's unitarity (a traversal re-applies the same
    // stages for many leaves, so most dense ops repeat an earlier U)
    std::unordered_map<uint64_t, std::vector<uint32_t>> dense_index;
    std::vector<uint8_t> dense_unitary;
    bool keep_dense_u = false;

    // Program bytes of one op in shared memory.
    uint32_t op_bytes(const HOp &o) const {
        const uint32_t mb = c128 ? 256u : 128u;
        if (o.type == H_DIAG) return (uint32_t)sizeof(DevOp) + 16 * (uint32_t)o.terms.size();
        if (o.type == H_DENSE) return (uint32_t)sizeof(DevOp) + 16 * (uint32_t)o.terms.size();
        return (uint32_t)sizeof(DevOp) + mb;
    }

    // Tensor-core form of one register stage (Sec. II, Eq. 1: consecutive
    // gates on the same 2^k amplitudes multiply into one matrix).  R is the
    // stage's register mask over local bits, win the pass window.  Matrix ops
    // act on register bits with one matrix for every thread; a diagonal op is
    // thread-independent when none of its terms mixes register and fixed
    // bits -- its register-only terms join the matrix, its fixed-only terms
    // are a per-thread constant phase that commutes with the whole stage and
    // rides along on the dense op.  A diagonal op with a mixed term stays a
    // SIMT op and ends the run.  Runs whose SIMT cost reaches kDenseMinCost
    // become one H_DENSE op.
    std::vector<HOp> densify(const std::vector<HOp> &ops, uint64_t R, const std::vector<int> &win) const {
        const int L = (int)win.size();
        const int v = std::min(V, L);
        int local[64];
        for (int i = 0; i < 64; ++i) local[i] = -1;
        for (int i = 0; i < L; ++i) local[win[i]] = i;
        int regidx[64];
        for (int i = 0; i < 64; ++i) regidx[i] = -1;
        uint64_t greg[8] = {0};
        uint64_t rg = 0;
        {
            int k = 0;
            for (int b = 0; b < L; ++b)
                if (R >> b & 1) {
                    regidx[b] = k;
                    greg[k] = 1ULL << win[b];
                    rg |= greg[k];
                    ++k;
                }
        }
        std::vector<HOp> out, run;
        auto flush = [&]() {
            double cost = 0;
            for (const HOp &o : run) cost += simt_cost(o, greg, v);
            if (run.empty() || cost < kDenseMinCost) {
                out.insert(out.end(), run.begin(), run.end());
                run.clear();
                return;
            }
            HOp d;
            d.type = H_DENSE;
            d.key = run.front().key;
            d.uid = run.front().uid;
            d.du.assign(32 * 32, cd(0, 0));
            for (int i = 0; i < 32; ++i) d.du[33 * i] = 1.0;
            // unitary unless a Kraus branch (RESET / MEASURE) is in the run
            d.noninv = false;
            for (const HOp &o : run) d.noninv = d.noninv || o.noninv;
            // U <- M_o U for each op in order, applied by its structure: a 2x2
            // mixes row pairs, a 4x4 row quads, a diagonal scales rows (each
            // new entry sums the same products in the same order as the full
            // 32x32 product would)
            for (const HOp &o : run) {
                if (&o != &run.front()) {
                    d.merged.push_back(o.uid);
                }
                d.merged.insert(d.merged.end(), o.merged.begin(), o.merged.end());
                std::vector<cd> &u = d.du;
                if (o.type == H_MAT1) {
                    const int b = regidx[local[o.q0]];
                    for (int r = 0; r < 32; ++r) {
                        if (r >> b & 1) continue;
                        const int r1 = r | 1 << b;
                        for (int c = 0; c < 32; ++c) {
                            const cd x = u[32 * r + c], y = u[32 * r1 + c];
                            u[32 * r + c] = o.m[0] * x + o.m[1] * y;
                            u[32 * r1 + c] = o.m[2] * x + o.m[3] * y;
                        }
                    }
                } else if (o.type == H_MAT2) {
                    const int ra = regidx[local[o.q0]], rb = regidx[local[o.q1]];
                    const int both = (1 << ra) | (1 << rb);
                    for (int base = 0; base < 32; ++base) {
                        if (base & both) continue;
                        // the quad's rows in ascending order, with their 4x4 indices
                        int rows[4], li[4];
                        int nq = 0;
                        for (int r = base; r < 32; ++r)
                            if ((r & ~both) == base) {
                                rows[nq] = r;
                                li[nq] = 2 * (r >> ra & 1) + (r >> rb & 1);
                                ++nq;
                            }
                        for (int c = 0; c < 32; ++c) {
                            cd x[4];
                            for (int q = 0; q < 4; ++q) x[q] = u[32 * rows[q] + c];
                            for (int q = 0; q < 4; ++q) {
                                cd acc = 0;
                                for (int k = 0; k < 4; ++k) acc += o.m[4 * li[q] + li[k]] * x[k];
                                u[32 * rows[q] + c] = acc;
                            }
                        }
                    }
                } else {
                    // register-only terms into the matrix; fixed-only ones ride along
                    d.phi0 += o.phi0;
                    for (int r = 0; r < 32; ++r) {
                        double turns = 0;
                        for (auto &t : o.terms) {
                            if ((t.first & rg) == 0) continue;
                            int mu = 0;
                            for (int i = 0; i < v; ++i)
                                if (t.first & greg[i]) mu |= 1 << i;
                            if (__builtin_popcount(r & mu) & 1) turns += t.second;
                        }
                        const cd ph = std::polar(1.0, 2 * kPi * turns);
                        for (int c = 0; c < 32; ++c) u[32 * r + c] = ph * u[32 * r + c];
                    }
                    for (auto &t : o.terms)
                        if ((t.first & rg) == 0) d.terms.push_back(t);
                }
            }
            out.push_back(d);
            run.clear();
        };
        for (const HOp &o : ops) {
            bool indep = true;
            if (o.type == H_DIAG)
                for (auto &t : o.terms)
                    if ((t.first & rg) && (t.first & ~rg)) { indep = false; break; }
            if (indep) {
                run.push_back(o);
            } else {
                flush();
                out.push_back(o);
            }
        }
        flush();
        return out;
    }

    // Encode one pass (window + ops already in application order) into
    // PassDescs: several when the register stages exceed kMaxStages or the
    // program (ops, matrix slots, diagonal terms) exceeds the shared-memory
    // budget; only the last one carries `flags`.  last_uids receives the uids
    // of the ops in that last PassDesc.
    void emit(const std::vector<int> &win, const std::vector<HOp> &ops_in, uint32_t flags,
              double leaf_w, int snap, std::vector<int> &pass_ids, std::vector<int> *last_uids) {
        if (last_uids) last_uids->clear();
        const int L = (int)win.size();
        int local[64];
        for (int i = 0; i < 64; ++i) local[i] = -1;
        for (int i = 0; i < L; ++i) local[win[i]] = i;
        // diagonal gates stay separate ops until their stages are chosen
        std::vector<HOp> ops = merge_ops(ops_in, false);
        // stage scheduling over local bits
        auto lq = [&](const HOp &o) -> uint64_t {
            if (o.type == H_DIAG) return 0;
            uint64_t m = 1ULL << local[o.q0];
            if (o.type == H_MAT2) m |= 1ULL << local[o.q1];
            return m;
        };
        const int v = std::min(V, L);
        // program budget: a pass that may carry dense ops keeps room for the B
        // region (one dense op's B parts) at the top of its program area
        const bool may_dense = tc_mode != TUSQ_TC_NONE && !c128 && L == kDenseTileBits && v == kRegBitsC64;
        const uint32_t dense_region = may_dense ? 4u * (uint32_t)dense_b_words(tc_mode) : 0u;
        const uint32_t budget = kMaxPassProgramBytes - dense_region;
        std::vector<uint64_t> swin;
        std::vector<std::vector<int>> sched;
        if (!ops.empty()) sched = schedule(ops, v, 0, lq, &swin, lookahead);
        // each stage's register bits: its window filled up to v with the
        // highest unused local bits (the encoding below uses the same rule)
        std::vector<uint64_t> Rfill(sched.size());
        for (size_t s = 0; s < sched.size(); ++s) {
            uint64_t R = swin[s];
            for (int b = L - 1; b >= 0 && __builtin_popcountll(R) < v; --b) R |= 1ULL << b;
            Rfill[s] = R;
        }
        if (place_diag) place_diagonals(ops, sched, Rfill, local);
        // inside a stage, order the ops so that every diagonal op that is ready
        // at the same time is applied together (alternately all ready diagonal
        // ops, then all ready matrix ops), and merge neighbours: each diagonal
        // run costs a pass over the thread's registers per register-mask group
        struct Piece { uint64_t R; std::vector<HOp> ops; };
        std::vector<Piece> pieces;
        for (size_t s = 0; s < sched.size(); ++s) {
            const std::vector<int> &g = sched[s];
            const int m = (int)g.size();
            std::vector<int> indeg(m, 0);
            std::vector<std::vector<int>> succ(m);
            for (int b = 0; b < m; ++b)
                for (int a = 0; a < b; ++a) {
                    const HOp &x = ops[g[a]], &y = ops[g[b]];
                    if (x.type == H_DIAG && y.type == H_DIAG) continue;
                    if (x.qmask() & y.qmask()) { succ[a].push_back(b); indeg[b]++; }
                }
            std::vector<HOp> ordered;
            std::vector<char> done(m, 0);
            int left = m;
            bool diag_phase = true;
            while (left > 0) {
                bool progress = true;
                int taken = 0;
                while (progress) {
                    progress = false;
                    for (int b = 0; b < m; ++b) {
                        if (done[b] || indeg[b] != 0) continue;
                        if ((ops[g[b]].type == H_DIAG) != diag_phase) continue;
                        done[b] = 1;
                        --left;
                        ++taken;
                        ordered.push_back(ops[g[b]]);
                        for (int c : succ[b]) indeg[c]--;
                        progress = true;
                    }
                }
                diag_phase = !diag_phase;
                (void)taken;
            }
            std::vector<HOp> merged = merge_ops(ordered);
            // the register bits the stage will use (filled up to v with the
            // highest unused local bits, as the encoding below does)
            const uint64_t Rs = Rfill[s];
            if (may_dense) merged = densify(merged, Rs, win);
            // cut into pieces of at most kMaxStageOps ops and at most the
            // per-pass program budget (same register bits)
            Piece cur{Rs, {}};
            uint32_t cur_bytes = 0;
            for (const HOp &o : merged) {
                const uint32_t ob = op_bytes(o);
                if (!cur.ops.empty() && ((int)cur.ops.size() >= kMaxStageOps || cur_bytes + ob > budget)) {
                    pieces.push_back(cur);
                    cur.ops.clear();
                    cur_bytes = 0;
                }
                cur.ops.push_back(o);
                cur_bytes += ob;
            }
            if (!cur.ops.empty()) pieces.push_back(cur);
        }
        const uint32_t mat_bytes = c128 ? 256 : 128;
        auto piece_bytes = [&](const Piece &pc) {
            uint32_t b = 0;
            for (const HOp &o : pc.ops) b += op_bytes(o);
            return b;
        };
        size_t p0 = 0;
        do {
            // as many pieces as the stage and program limits allow
            size_t p1 = p0;
            uint32_t bytes = 0;
            while (p1 < pieces.size() && (int)(p1 - p0) < kMaxStages) {
                uint32_t b = piece_bytes(pieces[p1]);
                if (p1 > p0 && bytes + b > budget) break;
                bytes += b;
                ++p1;
            }
            PassDesc pd;
            std::memset(&pd, 0, sizeof pd);
            pd.L = L;
            pd.n_stages = (int)(p1 - p0);
            bool last = (p1 >= pieces.size());
            pd.flags = last ? flags : PF_WRITE;
            pd.leaf_w = leaf_w;
            pd.snap = snap;
            pd.src_snap = -1;
            pd.op0 = (uint32_t)prog.ops.size();
            pd.mat0 = (uint32_t)(prog.mats.size() / 32);
            pd.term0 = (uint32_t)prog.term_mask.size();
            for (int i = 0; i < L; ++i) pd.win[i] = (uint8_t)win[i];
            int ncw = 0;
            for (int q = 0; q < n; ++q)
                if (local[q] < 0) pd.cw[ncw++] = (uint8_t)q;
            pd.n_cw = ncw;
            pd.cwmask = 0;
            for (int b = 0; b < ncw; ++b) pd.cwmask |= 1ULL << pd.cw[b];
            pd.ntiles = 1ULL << ncw;
            // load rows: complex64 threads move adjacent pairs (local bit 0 in
            // the registers, 16-byte accesses), so row i starts at local index
            // i << (L - v + 1); complex128 threads move single amplitudes,
            // row i at i << (L - v)
            const int rsh = c128 ? L - v : L - v + 1;
            const int nrow = c128 ? (1 << v) : (1 << (v - 1));
            for (int i = 0; i < nrow; ++i) {
                uint32_t e = (uint32_t)i << rsh;
                uint64_t g = 0;
                for (int b = 0; b < L; ++b)
                    if (e >> b & 1) g |= 1ULL << win[b];
                pd.grow[i] = g;
                pd.srow[i] = (uint16_t)swz(e, c128);
            }
            cd Kpass = 1.0;   // the scalar the tangent forms of this launch take out
            for (size_t s = p0; s < p1; ++s) {
                StageDesc &sd = pd.st[s - p0];
                uint64_t R = pieces[s].R;
                // fill up to v register bits with the highest unused local bits
                for (int b = L - 1; b >= 0 && __builtin_popcountll(R) < v; --b) R |= 1ULL << b;
                int nr = 0, nc = 0;
                for (int b = 0; b < L; ++b) {
                    if (R >> b & 1) sd.rbits[nr++] = (uint8_t)b;
                    else sd.cpos[nc++] = (uint8_t)b;
                }
                for (int i = 0; i < v; ++i) sd.greg[i] = 1ULL << win[sd.rbits[i]];
                for (int i = 0; i < nc; ++i) sd.cglob[i] = (uint8_t)win[sd.cpos[i]];
                for (int r = 0; r < (1 << v); ++r) {
                    uint32_t e = 0;
                    for (int i = 0; i < v; ++i)
                        if (r >> i & 1) e |= 1u << sd.rbits[i];
                    sd.sr[r] = (uint16_t)swz(e, c128);
                }
                int regidx[64];
                for (int i = 0; i < 64; ++i) regidx[i] = -1;
                for (int i = 0; i < v; ++i) regidx[sd.rbits[i]] = i;
                sd.op_begin = (uint32_t)prog.ops.size();
                const std::vector<HOp> &pops = pieces[s].ops;
                for (size_t oi = 0; oi < pops.size(); ++oi) {
                    const HOp &o = pops[oi];
                    if (last && last_uids) {
                        last_uids->push_back(o.uid);
                        last_uids->insert(last_uids->end(), o.merged.begin(), o.merged.end());
                    }
                    DevOp d;
                    std::memset(&d, 0, sizeof d);
                    // a run of 2x2s of one form on distinct register bits becomes
                    // one product op (one dispatch in the kernels); 2x2s on
                    // distinct qubits commute, so the run's order is kept
                    size_t run_end = oi + 1;
                    uint32_t run_bits = 0;
                    if (o.type == H_MAT1) {
                        const uint32_t sub0 = mat1_sub(o.m);
                        run_bits = 1u << regidx[local[o.q0]];
                        while (run_end < pops.size() && pops[run_end].type == H_MAT1 &&
                               mat1_sub(pops[run_end].m) == sub0 &&
                               !(run_bits >> regidx[local[pops[run_end].q0]] & 1u)) {
                            run_bits |= 1u << regidx[local[pops[run_end].q0]];
                            ++run_end;
                        }
                    }
                    if (o.type == H_MAT1 && run_end - oi >= 2) {
                        d.type = OP_MAT1;
                        d.a = (int32_t)run_bits;
                        d.sub = mat1_sub(o.m);
                        d.code = CODE_PROD + d.sub;
                        d.mat = (uint32_t)(prog.mats.size() / 32);
                        cd pm[32];
                        for (auto &z : pm) z = 0;
                        for (size_t k = oi; k < run_end; ++k) {
                            const int b = regidx[local[pops[k].q0]];
                            encode_mat1(pops[k].m, d.sub, pm + 4 * b, Kpass);
                            if (k > oi && last && last_uids) {
                                last_uids->push_back(pops[k].uid);
                                last_uids->insert(last_uids->end(), pops[k].merged.begin(), pops[k].merged.end());
                            }
                        }
                        for (int q = 0; q < 32; ++q) {
                            prog.mats.push_back(pm[q].real());
                            prog.mats.push_back(pm[q].imag());
                        }
                        prog.ops.push_back(d);
                        oi = run_end - 1;
                        continue;
                    }
                    if (o.type == H_MAT1) {
                        d.type = OP_MAT1;
                        d.a = regidx[local[o.q0]];
                        d.sub = mat1_sub(o.m);
                        d.code = CODE_MAT1 + 5 * d.sub + (uint32_t)d.a;
                        d.mat = (uint32_t)(prog.mats.size() / 32);
                        cd em[4];
                        encode_mat1(o.m, d.sub, em, Kpass);
                        for (int k = 0; k < 16; ++k) {
                            cd z = k < 4 ? em[k] : cd(0, 0);
                            prog.mats.push_back(z.real());
                            prog.mats.push_back(z.imag());
                        }
                    } else if (o.type == H_MAT2) {
                        int ra = regidx[local[o.q0]], rb = regidx[local[o.q1]];
                        // device basis: k = bit_lo + 2 bit_hi over register bits lo < hi;
                        // gate basis: l = 2 bit(q0) + bit(q1)
                        int lo = std::min(ra, rb), hi = std::max(ra, rb);
                        d.type = OP_MAT2;
                        d.a = lo;
                        d.b = hi;
                        d.mat = (uint32_t)(prog.mats.size() / 32);
                        auto l_of = [&](int k) {
                            int blo = k & 1, bhi = k >> 1;
                            int b0 = (ra == lo) ? blo : bhi, b1 = (rb == lo) ? blo : bhi;
                            return 2 * b0 + b1;
                        };
                        cd dm[16];
                        for (int r = 0; r < 4; ++r)
                            for (int c = 0; c < 4; ++c) {
                                dm[4 * r + c] = o.m[4 * l_of(r) + l_of(c)];
                                prog.mats.push_back(dm[4 * r + c].real());
                                prog.mats.push_back(dm[4 * r + c].imag());
                            }
                        int s0 = 0, s1 = 0;
                        d.sub = mat2_swap(dm, s0, s1) ? SUB_SWAP : SUB_GENERAL;
                        d.sw0 = (int16_t)s0;
                        d.sw1 = (int16_t)s1;
                        d.code = (d.sub == SUB_SWAP ? CODE_SWAP : CODE_MAT2) + pair_code(lo, hi);
                    } else if (o.type == H_DENSE) {
                        d.type = OP_DENSE;
                        d.code = CODE_DENSE;
                        d.sub = (uint32_t)tc_mode;
                        // one pool entry per distinct B (the operand the kernel reads;
                        // U itself in prog.dense_u when kept)
                        const size_t words = dense_b_words(tc_mode);
                        std::vector<float> bw(words);
                        encode_dense_b(o.du.data(), tc_mode, bw.data());
                        uint64_t h = 1469598103934665603ull;   // FNV-1a over B's bits
                        {
                            const unsigned char *ub = reinterpret_cast<const unsigned char *>(bw.data());
                            for (size_t k = 0; k < words * sizeof(float); ++k) h = (h ^ ub[k]) * 1099511628211ull;
                        }
                        auto &cands = dense_index[h];
                        int32_t idx = -1;
                        for (uint32_t c : cands)
                            if (std::memcmp(prog.dense_pool.data() + words * c, bw.data(), words * sizeof(float)) == 0) {
                                idx = (int32_t)c;
                                break;
                            }
                        if (idx < 0) {
                            idx = (int32_t)dense_unitary.size();
                            cands.push_back((uint32_t)idx);
                            // unitary (no Kraus branch in the run): the kernel may
                            // restore each vector's norm after the product
                            dense_unitary.push_back(o.noninv ? 0 : 1);
                            if (keep_dense_u)
                                for (size_t k = 0; k < 1024; ++k) {
                                    prog.dense_u.push_back(o.du[k].real());
                                    prog.dense_u.push_back(o.du[k].imag());
                                }
                            prog.dense_pool.insert(prog.dense_pool.end(), bw.begin(), bw.end());
                        }
                        d.mat = (uint32_t)idx;
                        d.b = dense_unitary[idx];
                        // the absorbed fixed-bit terms: a per-thread constant phase
                        d.phi0 = to_fixed(o.phi0, false);
                        d.term_begin = (uint32_t)prog.term_mask.size();
                        d.csr[0] = 0;
                        for (int mu = 1; mu <= 33; ++mu) d.csr[mu] = (uint16_t)o.terms.size();
                        d.mu_mask = 0;
                        for (auto &t : o.terms) {
                            prog.term_mask.push_back(t.first);
                            prog.term_phi.push_back(to_fixed(t.second, false));
                        }
                    } else {
                        d.type = OP_DIAG;
                        d.code = CODE_DIAG;
                        d.phi0 = to_fixed(o.phi0, c128);
                        // register mask of each term, sort by it
                        std::vector<std::pair<int, std::pair<uint64_t, double>>> t;
                        for (auto &term : o.terms) {
                            int mu = 0;
                            for (int i = 0; i < v; ++i)
                                if (term.first & sd.greg[i]) mu |= 1 << i;
                            t.push_back({mu, term});
                        }
                        std::stable_sort(t.begin(), t.end(), [](auto &x, auto &y) { return x.first < y.first; });
                        d.term_begin = (uint32_t)prog.term_mask.size();
                        int k = 0;
                        for (int mu = 0; mu <= 32; ++mu) {
                            while (k < (int)t.size() && t[k].first < mu) ++k;
                            d.csr[mu] = (uint16_t)k;
                        }
                        d.csr[33] = (uint16_t)t.size();
                        for (int mu = 1; mu < 32; ++mu)
                            if (d.csr[mu + 1] > d.csr[mu]) d.mu_mask |= 1u << mu;
                        for (auto &x : t) {
                            prog.term_mask.push_back(x.second.first);
                            prog.term_phi.push_back(to_fixed(x.second.second, c128));
                        }
                    }
                    prog.ops.push_back(d);
                }
                sd.op_count = (uint32_t)(prog.ops.size() - sd.op_begin);
            }
            // dense ops: each names the next one's pool index (cyclically)
            {
                std::vector<uint32_t> dk;
                for (uint32_t k = pd.op0; k < (uint32_t)prog.ops.size(); ++k)
                    if (prog.ops[k].type == OP_DENSE) dk.push_back(k);
                for (size_t i = 0; i < dk.size(); ++i)
                    prog.ops[dk[i]].a = (int32_t)prog.ops[dk[(i + 1) % dk.size()]].mat;
                if (!dk.empty()) pd.flags |= PF_DENSE | ((uint32_t)tc_mode << kDenseModeShift);
            }
            if (Kpass != cd(1.0, 0.0)) {
                // the scalar goes on the first stage that multiplies by a
                // per-thread phase anyway (it has a diagonal op), else on the last
                int ks = -1;
                for (int st = 0; st < pd.n_stages && ks < 0; ++st)
                    for (uint32_t k = 0; k < pd.st[st].op_count; ++k)
                        if (prog.ops[pd.st[st].op_begin + k].type == OP_DIAG) { ks = st; break; }
                if (ks < 0) ks = pd.n_stages - 1;
                pd.st[ks].kre = Kpass.real();
                pd.st[ks].kim = Kpass.imag();
                pd.st[ks].kflag = 1;
            }
            pd.nops = (uint32_t)prog.ops.size() - pd.op0;
            pd.nmat = (uint32_t)(prog.mats.size() / 32) - pd.mat0;
            pd.nterm = (uint32_t)prog.term_mask.size() - pd.term0;
            pd.prog_bytes = pd.nops * (uint32_t)sizeof(DevOp) + pd.nmat * mat_bytes + pd.nterm * 16;
            if (pd.flags & PF_DENSE) pd.prog_bytes += dense_region;
            // the kernels reserve exactly this much shared memory for a program
            if (pd.prog_bytes > kMaxPassProgramBytes)
                throw std::logic_error("encoder: pass program exceeds the shared-memory budget");
            pass_ids.push_back((int)prog.passes.size());
            prog.passes.push_back(pd);
            p0 = p1;
        } while (p0 < pieces.size());
    }
};

// ---------------------------------------------------------------- traversal

struct Compiler {
    const tusq_plan_t &P;
    const CompileOpts &co;
    Program &prog;
    Encoder enc;
    int G, n, L;
    uint64_t forced;
    std::vector<HOp> gate_ops;

    // DFTT+Caching (Sec. III-B2): the states just before a layer of
    // non-invertible gates on the current root-to-leaf path, shallowest
    // first.  `shared` entries reuse a branch node's snapshot slot.
    struct CacheEnt { int slot, snap; bool shared; };
    std::vector<CacheEnt> cache;
    std::vector<int> cache_free;        // unused cache slots
    std::vector<char> layer_start;      // gate j opens a non-invertible layer
    int K = 0;                          // cache capacity

    Compiler(const tusq_plan_t &p, const CompileOpts &c, Program &pr)
        : P(p), co(c), prog(pr), enc{pr, p.n, c.precision == TUSQ_C128,
                                     c.precision == TUSQ_C128 ? kRegBitsC128 : kRegBitsC64, 0} {
        G = P.G;
        n = P.n;
        // at most 256 threads x 2^V registers per CTA: 2^13 (c64), 2^12 (c128)
        int lmax = co.precision == TUSQ_C128 ? 12 : 13;
        if (co.max_window > 0) lmax = std::min(co.max_window, lmax);
        L = std::min(lmax, n);
        enc.Lmax = L;
        enc.lookahead = co.schedule == 0;
        enc.tc_mode = co.precision == TUSQ_C64 ? co.tc_mode : TUSQ_TC_NONE;
        enc.keep_dense_u = co.keep_dense_u;
        // the lowest qubits stay in every window (contiguous 128-byte runs),
        // leaving room for any two-qubit gate
        int nf = std::min(co.precision == TUSQ_C128 ? 3 : 4, std::max(L - 2, 0));
        forced = (nf >= 64) ? ~0ULL : ((1ULL << nf) - 1);
        for (int j = 0; j < G; ++j) gate_ops.push_back(gate_op(P.gates[j], j));
        layer_start.assign(G + 1, 0);
        int layers = 0;
        for (int j = 0; j < G; ++j)
            if (is_noninvertible(P.gates[j].kind) && (j == 0 || !is_noninvertible(P.gates[j - 1].kind))) {
                layer_start[j] = 1;
                ++layers;
            }
        if (co.traversal != TUSQ_FROM_SCRATCH && layers > 0)
            K = co.cache_states < 0 ? std::min(layers, kDefaultCacheStates) : co.cache_states;
        for (int k = K; k-- > 0;) cache_free.push_back(co.snapshots + k);
    }

    // Cache entries below slot t are off the next path: free their slots.
    void pop_cache_below(int t) {
        while (!cache.empty() && cache.back().slot > t) {
            if (!cache.back().shared) cache_free.push_back(cache.back().snap);
            cache.pop_back();
        }
    }

    // A slot for the state before the layer at `slot`: a free one, else the
    // shallowest entry's (the cache keeps the K closest to the leaf).
    int cache_take(int slot) {
        if (K == 0) return -1;
        if (cache_free.empty()) {
            size_t k = 0;
            while (k < cache.size() && cache[k].shared) ++k;
            if (k == cache.size()) return -1;
            cache_free.push_back(cache[k].snap);
            cache.erase(cache.begin() + k);
        }
        int idx = cache_free.back();
        cache_free.pop_back();
        cache.push_back(CacheEnt{slot, idx, false});
        return idx;
    }

    // Instance i's ops with canonical position in [2*a, 2*b) i.e. events at
    // slots a..b-1 and gates a..b-1, in canonical order.
    std::vector<HOp> segment(uint64_t i, int a, int b) {
        std::vector<HOp> out;
        uint64_t e = P.ev_off[i], e1 = P.ev_off[i + 1];
        while (e < e1 && P.ev_slot[e] < a) ++e;
        for (int j = a; j < b; ++j) {
            bool branch1 = false;     // the non-invertible gate j takes Kraus branch 1
            for (; e < e1 && P.ev_slot[e] == j; ++e) {
                if (P.ev_pauli[e] == TUSQ_OUTCOME1) { branch1 = true; continue; }
                HOp o = pauli_op(j, P.ev_qubit[e], P.ev_pauli[e]);
                o.uid = -(int)(e - P.ev_off[i]) - 1;
                out.push_back(o);
            }
            if (j < G) {
                HOp o = gate_ops[j];
                if (branch1) kraus1(P.gates[j].kind, o.m);
                o.uid = j;
                out.push_back(o);
            }
        }
        return out;
    }

    void count(const std::vector<HOp> &ops) {
        for (auto &o : ops) {
            if (o.pauli) prog.pauli_apps++;
            else prog.gate_apps++;
        }
    }

    void push_passes(const std::vector<int> &ids) {
        prog.passes_count += ids.size();
        for (int id : ids) prog.steps.push_back(Step{ST_PASS, id, 0, -1, 0});
    }

    // Schedule a list of ops into passes; the last launch gets `last_flags`.
    // last_uids receives the uids of the ops applied by that last launch.
    void emit_ops(const std::vector<HOp> &ops, uint32_t last_flags, double w, int snap,
                  std::vector<int> *last_uids) {
        count(ops);
        std::vector<uint64_t> wins;
        auto gq = [](const HOp &o) { return o.type == H_DIAG ? 0ULL : o.qmask(); };
        std::vector<std::vector<int>> groups;
        if (!ops.empty()) groups = schedule(ops, L, forced, gq, &wins, co.schedule == 0);
        if (groups.empty()) {
            // nothing to apply: an empty pass carries the flags
            std::vector<int> win;
            for (int b = 0; b < L; ++b) win.push_back(b);
            std::vector<int> ids;
            enc.emit(win, {}, last_flags, w, snap, ids, last_uids);
            push_passes(ids);
            return;
        }
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            uint64_t W = wins[gi];
            for (int b = 0; __builtin_popcountll(W) < L && b < n; ++b) W |= 1ULL << b;
            std::vector<int> win;
            for (int b = 0; b < n; ++b)
                if (W >> b & 1) win.push_back(b);
            std::vector<HOp> pops;
            for (int oi : groups[gi]) pops.push_back(ops[oi]);
            bool last = (gi + 1 == groups.size());
            std::vector<int> ids;
            enc.emit(win, pops, last ? last_flags : PF_WRITE, w, snap, ids, last ? last_uids : nullptr);
            push_passes(ids);
        }
    }

    void run() {
        const uint64_t N = P.n_inst();
        prog.steps.push_back(Step{ST_INIT, 0, 0, -1, 0});
        if (N == 0) return;
        // LIFO of the branch nodes on the current root-to-leaf path that will
        // be returned to: their slot, stack depth, snapshot slot (-1: none)
        // and whether their norm/checksum was recorded.
        struct Rec { int slot, depth, snap; bool recorded; };
        std::vector<Rec> stack;
        const bool scratch = co.traversal == TUSQ_FROM_SCRATCH;
        const bool snap_policy = co.traversal == TUSQ_DFTT_SNAPSHOT;
        const bool track = !scratch && (co.checks || snap_policy);
        // reused[i]: the branch node of pair (i, i+1) is returned to again,
        // i.e. the next branch slot that is not larger is equal to it
        // (next smaller-or-equal element, by a monotonic stack).
        std::vector<char> reused(N > 1 ? N - 1 : 0, 0);
        {
            std::vector<uint64_t> mono;
            for (uint64_t i = N > 1 ? N - 1 : 0; i-- > 0;) {
                while (!mono.empty() && P.lcp[mono.back()] > P.lcp[i]) mono.pop_back();
                reused[i] = !mono.empty() && P.lcp[mono.back()] == P.lcp[i];
                mono.push_back(i);
            }
        }
        for (uint64_t i = 0; i < N; ++i) {
            int t_in = (i == 0 || scratch) ? 0 : P.lcp[i - 1];
            // future branch slots on this path: running minima of the next
            // branch slots, above t_in
            std::vector<int> chain;
            if (track) {
                int m = G + 2;
                for (uint64_t k = i; k + 1 < N; ++k) {
                    int t = P.lcp[k];
                    if (t <= t_in) break;
                    if (t < m) { chain.push_back(t); m = t; }
                }
                std::reverse(chain.begin(), chain.end());
            }
            // split points: the future branch nodes and, with a cache, the
            // nodes just before each non-invertible layer
            std::vector<int> splits(chain.begin(), chain.end());
            // without the branch stack, still end a pass at the next branch
            // node, so that the leaf pass that skips its write holds no op
            // above the node the uncompute returns to
            if (!track && !scratch && co.leaf_peek && i + 1 < N && P.lcp[i] > t_in && P.lcp[i] <= G)
                splits.push_back(P.lcp[i]);
            if (K > 0)
                for (int j = t_in + 1; j < G; ++j)
                    if (layer_start[j]) splits.push_back(j);
            std::sort(splits.begin(), splits.end());
            std::vector<int> bounds;
            bounds.push_back(t_in);
            for (int s : splits) if (s > bounds.back()) bounds.push_back(s);
            bounds.push_back(G + 1);
            std::vector<int> leaf_ops;     // uids the unwritten leaf launch applied
            bool last_inst = (i + 1 == N);
            for (size_t s = 0; s + 1 < bounds.size(); ++s) {
                std::vector<HOp> ops = segment(i, bounds[s], bounds[s + 1]);
                bool final_seg = (s + 2 == bounds.size());
                if (!final_seg) {
                    // the pass that ends at a future branch node records it
                    // (and snapshots it while slots last); one that ends just
                    // before a non-invertible layer puts the state in the cache
                    const int node = bounds[s + 1];
                    const bool is_branch = std::binary_search(chain.begin(), chain.end(), node);
                    const bool is_layer = K > 0 && node < G && layer_start[node];
                    int depth = (int)stack.size();
                    int snap = is_branch && depth < co.snapshots ? depth : -1;
                    bool rec = is_branch && co.checks && !(snap_policy && snap >= 0);
                    int wsnap = snap;
                    if (is_layer) {
                        if (snap >= 0) cache.push_back(CacheEnt{node, snap, true});
                        else wsnap = cache_take(node);
                    }
                    uint32_t fl = PF_WRITE | (rec ? PF_REDUCE : 0u) | (wsnap >= 0 ? PF_SNAPSHOT : 0u);
                    emit_ops(ops, fl, 0.0, wsnap, nullptr);
                    if (rec) prog.steps.push_back(Step{ST_RECORD, 0, depth, snap, 0});
                    if (is_branch) {
                        stack.push_back(Rec{node, depth, snap, rec});
                        prog.max_depth = std::max(prog.max_depth, depth + 1);
                    }
                } else {
                    bool peek = co.leaf_peek && !scratch && !last_inst;
                    uint32_t fl = PF_LEAF | (peek ? 0u : PF_WRITE);
                    if (scratch || last_inst) fl &= ~PF_WRITE;   // nothing reads the state afterwards
                    emit_ops(ops, fl, P.weights[i], -1, &leaf_ops);
                    prog.leaf_passes++;
                    if (!peek) leaf_ops.clear();
                    if (scratch || last_inst) leaf_ops.clear();
                }
            }
            if (last_inst) break;
            int t = scratch ? 0 : P.lcp[i];
            if (scratch || (co.root_reset && t == 0)) {
                prog.steps.push_back(Step{ST_INIT, 0, 0, -1, 0});
                prog.resets++;
                stack.clear();
                pop_cache_below(t);
                // the branch slots are free again: drop the entries sharing them
                cache.erase(std::remove_if(cache.begin(), cache.end(), [](const CacheEnt &c) { return c.shared; }),
                            cache.end());
                continue;
            }
            while (!stack.empty() && stack.back().slot > t) stack.pop_back();
            if (track && (stack.empty() || stack.back().slot != t))
                throw std::logic_error("compile: branch slot was not materialised");
            return_to(i, t, leaf_ops, stack, snap_policy);
            pop_cache_below(t);
            // a node that no later pair branches at is done with; its
            // snapshot slot goes back to the branch stack
            if (track && !reused[i]) {
                const int freed = stack.back().snap;
                stack.pop_back();
                if (freed >= 0)
                    cache.erase(std::remove_if(cache.begin(), cache.end(),
                                               [&](const CacheEnt &c) { return c.shared && c.snap == freed; }),
                                cache.end());
            }
        }
    }

    // Uncompute back to the branch node on top of the stack, with the drift
    // check when the node was recorded.
    template <class Stack>
    void undo_to_branch(const std::vector<HOp> &undo, Stack &stack) {
        if (!co.checks || stack.empty() || !stack.back().recorded) {
            emit_ops(undo, PF_WRITE, 0.0, -1, nullptr);
            return;
        }
        int depth = stack.back().depth;
        int snap = stack.back().snap;
        emit_ops(undo, PF_WRITE | PF_REDUCE, 0.0, -1, nullptr);
        int chk = prog.n_checks++;
        prog.steps.push_back(Step{ST_CHECK, 0, depth, snap, chk});
        if (snap >= 0) prog.steps.push_back(Step{ST_RESTORE, 0, depth, snap, chk});
    }

    template <class Stack>
    void return_to(uint64_t i, int t, const std::vector<int> &leaf_ops, Stack &stack, bool snap_policy) {
        const int G = this->G;
        const bool own_snap = !stack.empty() && stack.back().slot == t && stack.back().snap >= 0;
        if (snap_policy && own_snap) {
            // the branch node's own snapshot: a restore, which fuse_restores
            // folds into the next pass's tile loads
            prog.steps.push_back(Step{ST_RESTORE, 0, stack.back().depth, stack.back().snap, -1});
            prog.restores++;
            return;
        }
        // instance i's ops at slots >= t, last applied first, not counting
        // those of the leaf pass that skipped its write
        std::vector<HOp> all = segment(i, t, G + 1);
        std::vector<const HOp *> todo;
        int j1 = G;              // first non-invertible gate among them
        for (auto it = all.rbegin(); it != all.rend(); ++it) {
            bool skipped = false;
            for (int u : leaf_ops)
                if (u == it->uid) { skipped = true; break; }
            if (skipped) continue;
            todo.push_back(&*it);
            if (it->noninv) j1 = std::min(j1, it->uid);
        }
        if (todo.empty()) return;     // the state never left the branch node
        if (j1 == G) {
            std::vector<HOp> undo;
            for (const HOp *o : todo) undo.push_back(inverse(*o));
            undo_to_branch(undo, stack);
            return;
        }
        // The way back crosses a non-invertible layer (Sec. III-B2).
        if (own_snap) {
            prog.steps.push_back(Step{ST_RESTORE, 0, stack.back().depth, stack.back().snap, -1});
            prog.restores++;
            return;
        }
        // (a) the cached state before that layer, then uncompute up to t
        int L1 = j1;
        while (L1 > 0 && is_noninvertible(P.gates[L1 - 1].kind)) --L1;
        int snap_c = -1;
        size_t cost_c = 0;
        if (L1 >= t)
            for (const CacheEnt &c : cache)
                if (c.slot == L1) { snap_c = c.snap; cost_c = segment(i, t, L1).size(); }
        // (b) re-derive forward from the deepest saved state at or above t
        // (a snapshotted branch node or a cached one), else from |0..0>
        int s_d = 0, snap_d = -1;
        for (const auto &r : stack)
            if (r.snap >= 0 && r.slot <= t && r.slot > s_d) { s_d = r.slot; snap_d = r.snap; }
        for (const CacheEnt &c : cache)
            if (c.slot <= t && (c.slot > s_d || (snap_d < 0 && c.slot == s_d))) { s_d = c.slot; snap_d = c.snap; }
        const size_t cost_d = segment(i, s_d, t).size();
        if (snap_c >= 0 && cost_c <= cost_d) {
            prog.steps.push_back(Step{ST_RESTORE, 0, 0, snap_c, -1});
            prog.cache_restores++;
            std::vector<HOp> seg = segment(i, t, L1), undo;
            for (auto it = seg.rbegin(); it != seg.rend(); ++it) undo.push_back(inverse(*it));
            if (!undo.empty()) undo_to_branch(undo, stack);
            return;
        }
        if (snap_d >= 0) prog.steps.push_back(Step{ST_RESTORE, 0, 0, snap_d, -1});
        else prog.steps.push_back(Step{ST_INIT, 0, 0, -1, 0});
        prog.rederives++;
        std::vector<HOp> fwd = segment(i, s_d, t);
        if (!fwd.empty()) emit_ops(fwd, PF_WRITE, 0.0, -1, nullptr);
    }

};

}  // namespace

void fuse_restores(Program &prog) {
    std::vector<Step> out;
    out.reserve(prog.steps.size());
    for (size_t k = 0; k < prog.steps.size(); ++k) {
        const Step &s = prog.steps[k];
        if (s.type == ST_RESTORE && s.check < 0 && s.snap >= 0 && k + 1 < prog.steps.size() &&
            prog.steps[k + 1].type == ST_PASS) {
            PassDesc &d = prog.passes[prog.steps[k + 1].pass];
            const bool writes = (d.flags & PF_WRITE) != 0;
            // A pass that does not write the state (a leaf peek) may read the
            // snapshot too when nothing reads the state buffer before it is
            // overwritten: the next step restores, resets, or there is none.
            // The pass may write the snapshot slot it reads: a CTA loads its
            // whole tile before writing that tile back, and tiles are disjoint.
            const Step *after = k + 2 < prog.steps.size() ? &prog.steps[k + 2] : nullptr;
            const bool state_dead = !after || after->type == ST_INIT ||
                                    (after->type == ST_RESTORE && after->check < 0);
            if ((writes || state_dead) && d.src_snap < 0) {
                d.src_snap = s.snap;
                continue;
            }
        }
        out.push_back(s);
    }
    prog.steps.swap(out);
}

void compile_program(const tusq_plan_t &P, const CompileOpts &co, Program &prog) {
    prog = Program{};
    prog.n = P.n;
    prog.precision = co.precision;
    prog.reg_bits = co.precision == TUSQ_C128 ? kRegBitsC128 : kRegBitsC64;
    prog.n_snapshots = co.snapshots;
    Compiler c(P, co, prog);
    c.run();
    // cache slots follow the branch-snapshot slots actually used
    const int B = std::min(co.snapshots, prog.max_depth);
    int top = B;
    auto remap = [&](int32_t &x) {
        if (x >= co.snapshots) {
            x = x - co.snapshots + B;
            top = std::max(top, x + 1);
        }
    };
    for (PassDesc &d : prog.passes)
        if (d.flags & PF_SNAPSHOT) remap(d.snap);
    for (Step &st : prog.steps)
        if (st.type == ST_RESTORE && st.snap >= 0) remap(st.snap);
    prog.n_snap_slots = top;
    // every snapshot slot a step or pass names must exist in the buffer the
    // runtime allocates (n_snap_slots states)
    for (const PassDesc &d : prog.passes)
        if ((d.flags & PF_SNAPSHOT) && (d.snap < 0 || d.snap >= top))
            throw std::logic_error("compile: pass snapshot slot out of range");
    for (const Step &st : prog.steps)
        if ((st.type == ST_RESTORE && (st.snap < 0 || st.snap >= top)) || (st.type == ST_CHECK && st.snap >= top))
            throw std::logic_error("compile: step snapshot slot out of range");
    prog.matsf.assign(prog.mats.begin(), prog.mats.end());
}

}  // namespace tusq
