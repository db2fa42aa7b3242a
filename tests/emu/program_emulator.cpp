// Host interpreter of the engine's compiled device program -- TEST ONLY.
//
// Built by tests/test_schedule_emulated.py into a separate shared object
// (never part of libtusq.so, never called by the library or the bench).
// It executes the schedule compiler's output with the semantics of the CUDA
// kernels -- tiles gathered through the window, register stages gathered
// through their register bits, 2x2 / 4x4 / diagonal-run ops, the leaf,
// snapshot, record and check steps -- in FP64 on the host, so that the
// compiler's traversal, fusion and layout logic can be checked against the
// oracle without a GPU.  The diagonal runs are evaluated both from the
// per-register fixed-point angles (a Walsh-Hadamard form of the register-mask
// groups whose phases the kernels apply group by group) and directly from the
// global index; any mismatch is reported.  Tensor-core dense ops apply the
// FP64 matrix U the compiler stored in the program's dense_u.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "../../paper_2508_04880_b300/csrc/internal.h"
#include "../../paper_2508_04880_b300/csrc/program.h"

namespace tusq {
void compile_program(const tusq_plan_t &P, const CompileOpts &co, Program &prog);
}
using namespace tusq;
using cd = std::complex<double>;

// The planner's device sampling lives in the CUDA library; this host-only
// build of the planner never asks for it.
int tusq::sample_ers_device(const std::vector<Channel> &, uint64_t, uint64_t, std::vector<uint32_t> &,
                            std::vector<uint64_t> &, std::vector<uint64_t> &, std::vector<uint32_t> &) {
    set_error("device sampling is not part of the host interpreter");
    return TUSQ_EINVAL;
}

static double g_diag_mismatch = 0;

static cd unit_of(uint64_t fixed, bool c128) {
    double turns = c128 ? (double)(fixed & 0x7FFFFFFFFFFFFFFFULL) * std::ldexp(1.0, -63)
                        : (double)(fixed & 0x7FFFFFFFULL) * std::ldexp(1.0, -31);
    return std::polar(1.0, 2 * M_PI * turns);
}

static void run_pass(const Program &pg, const PassDesc &d, std::vector<cd> &state,
                     std::vector<cd> *snap, std::vector<double> &acc, double red[3], int V, bool c128) {
    const int L = d.L;
    const int v = std::min(V, L);
    const uint64_t T = 1ULL << (L - v);
    std::vector<cd> tile(1ULL << L);
    for (uint64_t t = 0; t < d.ntiles; ++t) {
        uint64_t tb = 0;
        for (int b = 0; b < d.n_cw; ++b)
            if (t >> b & 1) tb |= 1ULL << d.cw[b];
        auto gidx = [&](uint64_t e) {
            uint64_t g = tb;
            for (int b = 0; b < L; ++b)
                if (e >> b & 1) g |= 1ULL << d.win[b];
            return g;
        };
        for (uint64_t e = 0; e < tile.size(); ++e) tile[e] = state[gidx(e)];
        for (int s = 0; s < d.n_stages; ++s) {
            const StageDesc &sd = d.st[s];
            for (uint64_t tid = 0; tid < T; ++tid) {
                uint64_t eb = 0;
                for (int b = 0; b < L - v; ++b)
                    if (tid >> b & 1) eb |= 1ULL << sd.cpos[b];
                std::vector<uint64_t> es(1 << v);
                for (int r = 0; r < (1 << v); ++r) {
                    uint64_t e = eb;
                    for (int i = 0; i < v; ++i)
                        if (r >> i & 1) e |= 1ULL << sd.rbits[i];
                    es[r] = e;
                }
                std::vector<cd> a(1 << v);
                for (int r = 0; r < (1 << v); ++r) a[r] = tile[es[r]];
                for (uint32_t k = 0; k < sd.op_count; ++k) {
                    const DevOp &op = pg.ops[sd.op_begin + k];
                    const double *m = &pg.mats[32 * (size_t)op.mat];
                    auto M = [&](int q) { return cd(m[2 * q], m[2 * q + 1]); };
                    // a 2x2 of form `sub` on register bit `bit`, entries from slot
                    // offset e0; the tangent forms carry one parameter in entry e0
                    // (their factor is the stage scalar)
                    auto two_by_two = [&](int bit, int e0) {
                        for (int r = 0; r < (1 << v); ++r) {
                            if (r >> bit & 1) continue;
                            cd x = a[r], y = a[r | 1 << bit];
                            const cd I(0, 1);
                            if (op.sub == SUB_RXT) {
                                const double t = M(e0).real();
                                a[r] = x - I * t * y;
                                a[r | 1 << bit] = y - I * t * x;
                            } else if (op.sub == SUB_RXS) {
                                const double k = M(e0).real();
                                a[r] = y + I * k * x;
                                a[r | 1 << bit] = x + I * k * y;
                            } else {
                                a[r] = M(e0) * x + M(e0 + 1) * y;
                                a[r | 1 << bit] = M(e0 + 2) * x + M(e0 + 3) * y;
                            }
                        }
                    };
                    if (op.type == OP_DENSE) {
                        // U from the FP64 pool (row-major 32x32); its absorbed
                        // fixed-bit terms follow as a per-thread constant phase
                        const double *u = &pg.dense_u[2048 * (size_t)op.mat];
                        std::vector<cd> y(1 << v, cd(0));
                        for (int r = 0; r < (1 << v); ++r)
                            for (int c2 = 0; c2 < (1 << v); ++c2)
                                y[r] += cd(u[2 * (32 * r + c2)], u[2 * (32 * r + c2) + 1]) * a[c2];
                        a = y;
                    }
                    if (op.type == OP_DENSE && op.csr[1] == op.csr[0] && op.phi0 == 0) {
                    } else if (op.type == OP_MAT1 && op.code >= CODE_PROD) {
                        // product op: bit b's 2x2 at matrix entries 4b..4b+3
                        for (int bit = 0; bit < v; ++bit)
                            if (op.a >> bit & 1) two_by_two(bit, 4 * bit);
                    } else if (op.type == OP_MAT1) {
                        two_by_two(op.a, 0);
                    } else if (op.type == OP_MAT2) {
                        for (int r = 0; r < (1 << v); ++r) {
                            if ((r >> op.a & 1) || (r >> op.b & 1)) continue;
                            int idx[4] = {r, r | 1 << op.a, r | 1 << op.b, r | 1 << op.a | 1 << op.b};
                            cd in[4], out[4];
                            for (int q = 0; q < 4; ++q) in[q] = a[idx[q]];
                            for (int q = 0; q < 4; ++q) {
                                out[q] = 0;
                                for (int c = 0; c < 4; ++c) out[q] += M(4 * q + c) * in[c];
                            }
                            for (int q = 0; q < 4; ++q) a[idx[q]] = out[q];
                        }
                    } else {
                        // per-register angle: A + (sum C - WHT(C)[r]) / 2 in fixed point
                        uint64_t gfix = tb;
                        for (int b = 0; b < L - v; ++b)
                            if (tid >> b & 1) gfix |= 1ULL << d.win[sd.cpos[b]];
                        const uint64_t mask = c128 ? ~0ULL : 0xFFFFFFFFULL;
                        uint64_t A = op.phi0;
                        std::vector<uint64_t> C(1 << v, 0);
                        for (int mu = 0; mu < (1 << v) + 0; ++mu)
                            for (int q = op.csr[mu]; q < op.csr[mu + 1]; ++q) {
                                uint64_t ph = pg.term_phi[op.term_begin + q];
                                bool c = __builtin_popcountll(gfix & pg.term_mask[op.term_begin + q]) & 1;
                                if (mu == 0) { if (c) A += ph; continue; }
                                A += c ? ph : 0;
                                C[mu] += c ? (0 - ph) : ph;
                            }
                        uint64_t sum = 0;
                        for (auto x : C) sum += x;
                        std::vector<uint64_t> F = C;
                        for (int h = 1; h < (1 << v); h <<= 1)
                            for (int i = 0; i < (1 << v); ++i) {
                                if (i & h) continue;
                                uint64_t x = F[i], y = F[i | h];
                                F[i] = (x + y) & mask;
                                F[i | h] = (x - y) & mask;
                            }
                        for (int r = 0; r < (1 << v); ++r) {
                            uint64_t ang = (A + ((((sum - F[r]) & mask)) >> 1)) & mask;
                            cd ph = unit_of(ang, c128);
                            // direct evaluation from the global index
                            uint64_t g = gidx(es[r]);
                            uint64_t dir = op.phi0;
                            for (int q = op.csr[0]; q < op.csr[33]; ++q)
                                if (__builtin_popcountll(g & pg.term_mask[op.term_begin + q]) & 1)
                                    dir += pg.term_phi[op.term_begin + q];
                            g_diag_mismatch = std::max(g_diag_mismatch, std::abs(unit_of(dir & mask, c128) - ph));
                            a[r] *= ph;
                        }
                    }
                }
                if (sd.kflag)
                    for (int r = 0; r < (1 << v); ++r) a[r] *= cd(sd.kre, sd.kim);
                for (int r = 0; r < (1 << v); ++r) tile[es[r]] = a[r];
            }
        }
        for (uint64_t e = 0; e < tile.size(); ++e) {
            uint64_t g = gidx(e);
            cd z = tile[e];
            if (d.flags & PF_WRITE) state[g] = z;
            if ((d.flags & PF_SNAPSHOT) && snap) (*snap)[g] = z;
            if (d.flags & PF_LEAF) acc[g] += d.leaf_w * std::norm(z);
            if (d.flags & PF_REDUCE) {
                red[0] += std::norm(z);
                double h = ((g * 0x9E3779B97F4A7C15ULL) >> 63) ? -1.0 : 1.0;
                red[1] += h * z.real();
                red[2] += h * z.imag();
            }
        }
    }
}

extern "C" int emu_run(const tusq_plan_t *p, const tusq_run_opts *o, double *probs, double *info_out) {
    const bool c128 = o->precision == TUSQ_C128;
    const size_t state_bytes = (size_t)(c128 ? 16 : 8) << p->n;
    CompileOpts co;
    co.precision = o->precision;
    co.max_window = o->max_window;
    co.traversal = o->traversal;
    co.leaf_peek = o->leaf_peek;
    co.root_reset = o->root_reset;
    co.schedule = o->schedule;
    co.checks = o->drift_tol >= 0 && o->traversal != TUSQ_FROM_SCRATCH;
    bool snaps = co.checks || o->traversal == TUSQ_DFTT_SNAPSHOT;
    co.snapshots = snaps ? (int)std::min<uint64_t>(o->snapshot_bytes / state_bytes, 64) : 0;
    co.cache_states = o->cache_states;
    co.tc_mode = o->tc_mode;
    co.keep_dense_u = true;     // the interpreter applies each dense op's U
    Program pg;
    compile_program(*p, co, pg);
    const uint64_t dim = 1ULL << p->n;
    std::vector<cd> state(dim);
    std::vector<std::vector<cd>> snapv(std::max(pg.n_snap_slots, 0), std::vector<cd>(dim));
    std::vector<double> acc(dim, 0.0);
    std::vector<double> rec(4 * (pg.max_depth + 1), 0.0);
    std::vector<int> flag(pg.n_checks + 1, 0);
    double red[3] = {0, 0, 0};
    double max_drift = 0;
    int restores = 0;
    g_diag_mismatch = 0;
    for (const Step &s : pg.steps) {
        if (s.type == ST_INIT) {
            std::fill(state.begin(), state.end(), cd(0));
            state[0] = 1;
        } else if (s.type == ST_PASS) {
            const PassDesc &d = pg.passes[s.pass];
            red[0] = red[1] = red[2] = 0;
            run_pass(pg, d, state, (d.flags & PF_SNAPSHOT) ? &snapv[d.snap] : nullptr, acc, red,
                     pg.reg_bits, c128);
        } else if (s.type == ST_RECORD) {
            rec[4 * s.depth] = red[0];
            rec[4 * s.depth + 1] = red[1];
            rec[4 * s.depth + 2] = red[2];
        } else if (s.type == ST_CHECK) {
            double dn = std::fabs(std::sqrt(red[0]) - std::sqrt(rec[4 * s.depth]));
            double dc = std::hypot(red[1] - rec[4 * s.depth + 1], red[2] - rec[4 * s.depth + 2]);
            double drift = std::max(dn, dc);
            max_drift = std::max(max_drift, drift);
            flag[s.check] = drift > o->drift_tol && s.snap >= 0;
        } else if (s.type == ST_RESTORE) {
            if (s.check < 0 || flag[s.check]) {
                state = snapv[s.snap];
                ++restores;
            }
        }
    }
    for (uint64_t i = 0; i < dim; ++i) probs[i] = acc[i];
    info_out[0] = max_drift;
    info_out[1] = restores;
    info_out[2] = g_diag_mismatch;
    info_out[3] = (double)pg.passes_count;
    return 0;
}
