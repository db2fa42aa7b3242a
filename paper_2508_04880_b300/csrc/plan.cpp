// Host-side Error Characterization Module (Sec. III-A) and instance tree
// (Sec. III-B): ER sampling, tallying, commutation, pruning, DFS order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace tusq {

bool is_two_qubit(int kind) {
    return kind == TUSQ_CX || kind == TUSQ_CZ || kind == TUSQ_RZZ || kind == TUSQ_U2Q;
}

bool is_diagonal(int kind) {
    switch (kind) {
    case TUSQ_Z: case TUSQ_S: case TUSQ_SDG: case TUSQ_T: case TUSQ_TDG:
    case TUSQ_RZ: case TUSQ_CZ: case TUSQ_RZZ: return true;
    default: return false;
    }
}

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------ Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of two 64x64
// multiplications with the Philox multipliers, a word permutation and a key
// xor; the key advances by the Weyl constants between rounds.
struct U4 { uint64_t v[4]; };

inline U4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1) {
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    constexpr uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    return U4{{c0, c1, c2, c3}};
}

uint64_t threshold_of(double x) {
    if (x >= 1.0) return UINT64_MAX;
    if (x <= 0.0) return 0;
    return (uint64_t)(x * 18446744073709551616.0);
}

// An ER / event list packed as 32-bit words for hashing and ordering:
// raw ER word = channel << 4 | code; commuted word = (slot << 8 | qubit) << 2 | (pauli - 1)
// (slot < 2^22, qubit < 2^6); word order equals (slot, qubit, pauli) order.
using Key = std::vector<uint32_t>;

struct KeyHash {
    size_t operator()(const Key &k) const {
        uint64_t h = 0x243F6A8885A308D3ULL ^ k.size();
        for (uint32_t w : k) {
            h ^= w;
            h *= 0x100000001B3ULL;
            h ^= h >> 29;
        }
        return (size_t)h;
    }
};

// Event-list order with the end of a list sorting after every event.
bool key_less(const Key &a, const Key &b) {
    size_t n = std::min(a.size(), b.size());
    for (size_t i = 0; i < n; ++i)
        if (a[i] != b[i]) return a[i] < b[i];
    return a.size() > b.size();
}

inline uint32_t pack_event(int slot, int q, int p) {
    return ((uint32_t)slot << 8 | (uint32_t)q) << 2 | (uint32_t)(p - 1);
}
inline Event unpack_event(uint32_t w) {
    return Event{(int32_t)(w >> 10), (int32_t)((w >> 2) & 0xFF), (int32_t)(w & 3) + 1};
}

// Pauli in (x, z) bit form: I=(0,0) X=(1,0) Y=(1,1) Z=(0,1).
inline int px(int p) { return p == 1 || p == 2; }
inline int pz(int p) { return p == 2 || p == 3; }
inline int mkp(int x, int z) { return x ? (z ? 2 : 1) : (z ? 3 : 0); }

// Does the Pauli (pa on q0, pb on q1) pass gate `kind` under `mode`, and what
// does it become?  Cliffords act by their symplectic update on (x, z);
// rotations let through the Paulis that commute with their generator.
bool pass_gate(int mode, int kind, int pa, int pb, int &oa, int &ob) {
    int xa = px(pa), za = pz(pa), xb = px(pb), zb = pz(pb);
    bool cliff2 = mode >= TUSQ_COMMUTE_CLIFFORD;
    switch (kind) {
    case TUSQ_X: case TUSQ_Y: case TUSQ_Z:            // rule 2
        oa = pa; ob = 0; return true;
    case TUSQ_RX: if (za) return false; oa = pa; ob = 0; return true;   // rule 3
    case TUSQ_RY: if (xa != za) return false; oa = pa; ob = 0; return true;
    case TUSQ_RZ: if (xa) return false; oa = pa; ob = 0; return true;
    case TUSQ_CX:                                       // rules 4-6
        oa = mkp(xa, za ^ zb); ob = mkp(xb ^ xa, zb); return true;
    case TUSQ_H: if (!cliff2) return false; oa = mkp(za, xa); ob = 0; return true;
    case TUSQ_S: case TUSQ_SDG: if (!cliff2) return false; oa = mkp(xa, za ^ xa); ob = 0; return true;
    case TUSQ_T: case TUSQ_TDG: if (!cliff2 || xa) return false; oa = pa; ob = 0; return true;
    case TUSQ_CZ: if (!cliff2) return false; oa = mkp(xa, za ^ xb); ob = mkp(xb, zb ^ xa); return true;
    case TUSQ_RZZ: if (!cliff2 || (xa ^ xb)) return false; oa = pa; ob = pb; return true;
    default: return false;
    }
}

inline int pmul(int a, int b) { return mkp(px(a) ^ px(b), pz(a) ^ pz(b)); }

// Frontier form of the per-qubit-stack algorithm (Sec. III-A3): one pending
// Pauli per qubit; at each gate the pending factor on its support is pushed
// through whole if it passes, else each single-qubit factor that passes on
// its own; blocked factors are emitted just before the gate; the channel
// outcome after the gate is multiplied into the pending Paulis (rule 1).
// Whatever is pending at the end is emitted at slot G.
struct Commuter {
    const std::vector<Gate> *gates;
    const std::vector<Channel> *chans;
    int n, G, mode;

    void raw_paulis(uint32_t w, int &q0, int &pa, int &q1, int &pb) const {
        const Channel &ch = (*chans)[w >> 4];
        const Gate &g = (*gates)[ch.gate];
        int code = (int)(w & 15);
        if (is_two_qubit(g.kind)) { q0 = g.q0; pa = code >> 2; q1 = g.q1; pb = code & 3; }
        else { q0 = g.q0; pa = code; q1 = -1; pb = 0; }
    }

    Key run(const Key &er) const {
        Key out;
        if (er.empty()) return out;
        if (mode == TUSQ_COMMUTE_OFF) {
            for (uint32_t w : er) {
                int q0, pa, q1, pb;
                raw_paulis(w, q0, pa, q1, pb);
                int slot = (*chans)[w >> 4].gate + 1;
                if (pa) out.push_back(pack_event(slot, q0, pa));
                if (pb) out.push_back(pack_event(slot, q1, pb));
            }
            std::sort(out.begin(), out.end());
            return out;
        }
        int pend[kMaxQubits] = {0};
        int npend = 0;
        size_t next = 0;
        int j = (*chans)[er[0] >> 4].gate;   // nothing is pending before this gate's channel
        for (; j < G; ++j) {
            const Gate &g = (*gates)[j];
            bool two = is_two_qubit(g.kind);
            int pa = pend[g.q0], pb = two ? pend[g.q1] : 0;
            if (pa || pb) {
                int oa = 0, ob = 0, ra = 0, rb = 0;
                int emit_a = 0, emit_b = 0;
                if (pass_gate(mode, g.kind, pa, pb, oa, ob)) {
                    ra = oa; rb = ob;
                } else {
                    if (pa) {
                        if (pass_gate(mode, g.kind, pa, 0, oa, ob)) { ra = pmul(ra, oa); rb = pmul(rb, ob); }
                        else emit_a = pa;
                    }
                    if (pb) {
                        if (pass_gate(mode, g.kind, 0, pb, oa, ob)) { ra = pmul(ra, oa); rb = pmul(rb, ob); }
                        else emit_b = pb;
                    }
                }
                if (emit_a) out.push_back(pack_event(j, g.q0, emit_a));
                if (emit_b) out.push_back(pack_event(j, g.q1, emit_b));
                npend -= (pa != 0) + (pb != 0);
                pend[g.q0] = ra;
                if (two) pend[g.q1] = rb;
                npend += (ra != 0) + (two && rb != 0);
            }
            // rule 1: merge this gate's channel outcome
            while (next < er.size() && (*chans)[er[next] >> 4].gate == j) {
                int q0, a, q1, b;
                raw_paulis(er[next], q0, a, q1, b);
                if (a) { npend -= pend[q0] != 0; pend[q0] = pmul(pend[q0], a); npend += pend[q0] != 0; }
                if (b) { npend -= pend[q1] != 0; pend[q1] = pmul(pend[q1], b); npend += pend[q1] != 0; }
                ++next;
            }
            if (npend == 0 && next == er.size()) break;
            if (npend == 0) j = (*chans)[er[next] >> 4].gate - 1;   // skip to the next channel
        }
        for (int q = 0; q < n; ++q)
            if (pend[q]) out.push_back(pack_event(G, q, pend[q]));
        std::sort(out.begin(), out.end());
        return out;
    }
};

// Readout fold of the Paulis left after the last gate: only |psi_x|^2 is
// observed, so a Z there changes nothing and a Y acts like an X.
void fold_terminal(Key &k, int G) {
    size_t o = 0;
    for (uint32_t w : k) {
        Event e = unpack_event(w);
        if (e.slot == G) {
            if (!px(e.pauli)) continue;
            w = pack_event(G, e.qubit, 1);
        }
        k[o++] = w;
    }
    k.resize(o);
}

struct Kept {
    const Key *key;
    uint64_t count;
    double weight;
};
void finish_tree(tusq_plan_t &P, const std::vector<Kept> &kept);

// Kraus-branch expansion for the non-invertible gates (Sec. III-B2): every
// kept instance stands for 2^R leaves, one per branch record (m_1..m_R),
// with the instance's count and weight; the record is written as outcome
// events (slot j_r, qubit q_r, TUSQ_OUTCOME1) for the gates with m_r = 1.
// The leaves are re-sorted into DFS order.
constexpr uint64_t kMaxLeaves = 1ull << 24;

int expand_outcomes(const tusq_plan_t &P, std::vector<Kept> &kept, std::vector<Key> &store) {
    std::vector<uint32_t> outs;
    for (int j = 0; j < P.G; ++j)
        if (is_noninvertible(P.gates[j].kind)) outs.push_back(pack_event(j, P.gates[j].q0, TUSQ_OUTCOME1));
    const int R = (int)outs.size();
    if (R == 0) return TUSQ_OK;
    if (R > 24 || (kept.size() << R) > kMaxLeaves) {
        set_error("tusq_plan: " + std::to_string(kept.size()) + " instances x 2^" + std::to_string(R) +
                  " Kraus branches exceed 2^24 leaves");
        return TUSQ_EINVAL;
    }
    store.clear();
    store.reserve(kept.size() << R);
    std::vector<std::pair<uint64_t, uint64_t>> origin;   // (kept index, record)
    for (uint64_t i = 0; i < kept.size(); ++i)
        for (uint64_t m = 0; m < (1ull << R); ++m) {
            Key k = *kept[i].key;
            for (int r = 0; r < R; ++r)
                if (m >> r & 1) k.push_back(outs[r]);
            std::sort(k.begin(), k.end());
            store.push_back(std::move(k));
            origin.emplace_back(i, m);
        }
    std::vector<uint64_t> ord(store.size());
    for (uint64_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](uint64_t a, uint64_t b) { return key_less(store[a], store[b]); });
    std::vector<Kept> out;
    out.reserve(ord.size());
    for (uint64_t o : ord) {
        const Kept &src = kept[origin[o].first];
        out.push_back(Kept{&store[o], src.count, src.weight});
    }
    kept.swap(out);
    return TUSQ_OK;
}

void noninv_stats(tusq_plan_t &P) {
    P.stats.n_noninvertible = 0;
    P.stats.n_noninv_layers = 0;
    for (int j = 0; j < P.G; ++j)
        if (is_noninvertible(P.gates[j].kind)) {
            P.stats.n_noninvertible++;
            if (j == 0 || !is_noninvertible(P.gates[j - 1].kind)) P.stats.n_noninv_layers++;
        }
}

void parallel_for(int nthreads, uint64_t n, const std::function<void(int, uint64_t, uint64_t)> &f) {
    if (nthreads <= 1 || n < 1024) { f(0, 0, n); return; }
    std::vector<std::thread> th;
    uint64_t chunk = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t a = t * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back(f, t, a, b);
    }
    for (auto &x : th) x.join();
}

}  // namespace

// Build the plan.  Every step is deterministic and independent of the
// thread count: per-thread tallies are merged into one map and sorted.
int build_plan(const tusq_circuit &circ, const tusq_plan_opts &opts, uint64_t shots,
               uint64_t seed, tusq_plan_t &P) {
    P.n = circ.n;
    P.G = (int)circ.gates.size();
    P.gates = circ.gates;
    P.shots = shots;
    P.seed = seed;
    P.opts = opts;
    std::vector<Channel> chans = circ.ordered();
    const int C = (int)chans.size();
    for (auto &ch : chans) {
        double s = 0;
        for (int k = 0; k < ch.nterms; ++k) s += ch.probs[k];
        double cdf = 1.0 - s;
        ch.thr[0] = threshold_of(cdf);
        for (int k = 1; k <= ch.nterms; ++k) {
            cdf += ch.probs[k - 1];
            ch.thr[k] = (k == ch.nterms) ? UINT64_MAX : threshold_of(cdf);
        }
    }
    int nth = opts.n_threads > 0 ? opts.n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    tusq_plan_stats_t &st = P.stats;
    std::memset(&st, 0, sizeof st);
    st.shots = shots;
    st.n_channels = C;
    st.n_gates = P.G;

    // 1 + 2. sample every channel of every shot and tally identical ERs.
    double t0 = now_s();
    std::unordered_map<Key, uint64_t, KeyHash> raw;
    uint64_t n_ideal = 0;
    double t1 = t0;
    if (opts.device_sampling) {
        // the draws on the device; shots grouped by the hash of their ER
        // words, word lists compared within a hash group (exact tally)
        std::vector<uint32_t> cnt, words;
        std::vector<uint64_t> hash, off;
        int rc = sample_ers_device(chans, shots, seed, cnt, hash, off, words);
        if (rc) return rc;
        t1 = now_s();
        std::unordered_map<uint64_t, uint32_t> head;
        head.reserve(shots / 2 + 1);
        std::vector<uint64_t> rep, rcnt;
        std::vector<int64_t> nxt;
        auto same = [&](uint64_t a, uint64_t b) {
            return cnt[a] == cnt[b] && std::memcmp(&words[off[a]], &words[off[b]], sizeof(uint32_t) * cnt[a]) == 0;
        };
        for (uint64_t s = 0; s < shots; ++s) {
            if (cnt[s] == 0) { ++n_ideal; continue; }
            auto ins = head.try_emplace(hash[s], (uint32_t)rep.size());
            if (ins.second) { rep.push_back(s); rcnt.push_back(1); nxt.push_back(-1); continue; }
            int64_t u = ins.first->second;
            for (;;) {
                if (same(rep[u], s)) { rcnt[u]++; break; }
                if (nxt[u] < 0) {
                    nxt[u] = (int64_t)rep.size();
                    rep.push_back(s); rcnt.push_back(1); nxt.push_back(-1);
                    break;
                }
                u = nxt[u];
            }
        }
        raw.reserve(rep.size() + 1);
        for (size_t u = 0; u < rep.size(); ++u)
            raw.emplace(Key(words.begin() + off[rep[u]], words.begin() + off[rep[u]] + cnt[rep[u]]), rcnt[u]);
    } else {
    std::vector<std::unordered_map<Key, uint64_t, KeyHash>> maps(nth);
    std::vector<uint64_t> ideal(nth, 0);
    parallel_for(nth, shots, [&](int t, uint64_t a, uint64_t b) {
        auto &m = maps[t];
        Key er;
        for (uint64_t s = a; s < b; ++s) {
            er.clear();
            U4 blk{};
            for (int c = 0; c < C; ++c) {
                if ((c & 3) == 0) blk = philox(s, (uint64_t)c >> 2, 0, 0, seed, 0);
                uint64_t r = blk.v[c & 3];
                const Channel &ch = chans[c];
                if (r < ch.thr[0]) continue;
                int k = 1;
                while (k < ch.nterms && !(r < ch.thr[k])) ++k;
                er.push_back((uint32_t)c << 4 | ch.codes[k - 1]);
            }
            if (er.empty()) ideal[t]++;
            else m[er]++;
        }
    });
    t1 = now_s();
    for (int t = 0; t < nth; ++t) {
        n_ideal += ideal[t];
        if (raw.empty()) raw.swap(maps[t]);
        else for (auto &kv : maps[t]) raw[kv.first] += kv.second;
        maps[t].clear();
    }
    }
    if (n_ideal) raw[Key{}] += n_ideal;
    std::vector<const std::pair<const Key, uint64_t> *> rorder;
    rorder.reserve(raw.size());
    for (auto &kv : raw) rorder.push_back(&kv);
    std::sort(rorder.begin(), rorder.end(), [](auto *x, auto *y) { return key_less(x->first, y->first); });
    P.raw = FlatList{};
    for (auto *kv : rorder) {
        for (uint32_t w : kv->first) { P.raw.a.push_back(w >> 4); P.raw.b.push_back(w & 15); P.raw.c.push_back(0); }
        P.raw.off.push_back(P.raw.a.size());
        P.raw.count.push_back(kv->second);
    }
    st.n_raw_unique = rorder.size();
    double t2 = now_s();

    // 3. commute every distinct ER (in parallel), then re-tally.
    Commuter cm{&circ.gates, &chans, circ.n, P.G, opts.commute_mode};
    std::vector<Key> ckeys(rorder.size());
    parallel_for(nth, rorder.size(), [&](int, uint64_t a, uint64_t b) {
        for (uint64_t i = a; i < b; ++i) {
            ckeys[i] = cm.run(rorder[i]->first);
            if (opts.terminal_fold) fold_terminal(ckeys[i], P.G);
        }
    });
    std::unordered_map<Key, uint64_t, KeyHash> com;
    com.reserve(rorder.size());
    for (size_t i = 0; i < rorder.size(); ++i) com[ckeys[i]] += rorder[i]->second;
    std::vector<const std::pair<const Key, uint64_t> *> korder;
    korder.reserve(com.size());
    for (auto &kv : com) korder.push_back(&kv);
    std::sort(korder.begin(), korder.end(), [](auto *x, auto *y) { return key_less(x->first, y->first); });
    P.commuted = FlatList{};
    for (auto *kv : korder) {
        for (uint32_t w : kv->first) {
            Event e = unpack_event(w);
            P.commuted.a.push_back(e.slot); P.commuted.b.push_back(e.qubit); P.commuted.c.push_back(e.pauli);
        }
        P.commuted.off.push_back(P.commuted.a.size());
        P.commuted.count.push_back(kv->second);
    }
    st.n_commuted_unique = korder.size();
    double t3 = now_s();

    // 4. prune (Sec. III-A4).
    const uint64_t nk = korder.size();
    std::vector<char> keep(nk, 0);
    std::vector<double> w(nk, 0.0);
    uint64_t cmax = 0;
    for (auto *kv : korder) cmax = std::max(cmax, kv->second);
    if (!opts.prune) {
        for (uint64_t i = 0; i < nk; ++i) { keep[i] = 1; w[i] = (double)korder[i]->second / (double)shots; }
        st.n_significant = nk;
    } else {
        std::vector<uint64_t> insig;
        uint64_t cins = 0;
        for (uint64_t i = 0; i < nk; ++i) {
            uint64_t c = korder[i]->second;
            if ((double)c >= opts.alpha * (double)cmax) {
                keep[i] = 1;
                w[i] = (double)c / (double)shots;
                st.n_significant++;
            } else {
                insig.push_back(i);
                cins += c;
            }
        }
        st.n_insignificant = insig.size();
        uint64_t npick = std::min<uint64_t>(opts.beta, insig.size());
        for (uint64_t i = 0; i < npick; ++i) {
            uint64_t r = philox(i, 0, 0, 0, seed, 2).v[0];
            uint64_t j = i + r % (insig.size() - i);
            std::swap(insig[i], insig[j]);
        }
        uint64_t cpick = 0;
        for (uint64_t i = 0; i < npick; ++i) cpick += korder[insig[i]]->second;
        for (uint64_t i = 0; i < npick; ++i) {
            uint64_t k = insig[i];
            keep[k] = 1;
            w[k] = ((double)korder[k]->second / (double)shots) * ((double)cins / (double)cpick);
        }
        st.n_picked = npick;
    }
    // 5. kept instances in key order, branch slots, tree statistics.
    std::vector<Kept> kept;
    for (uint64_t i = 0; i < nk; ++i)
        if (keep[i]) kept.push_back(Kept{&korder[i]->first, korder[i]->second, w[i]});
    st.n_ecm_instances = kept.size();
    noninv_stats(P);
    std::vector<Key> expanded;
    int erc = expand_outcomes(P, kept, expanded);
    if (erc) return erc;
    finish_tree(P, kept);
    double t4 = now_s();
    st.seconds_sample = t1 - t0;
    st.seconds_tally = t2 - t1;
    st.seconds_commute = t3 - t2;
    st.seconds_prune_tree = t4 - t3;
    return TUSQ_OK;
}

// Plan from a caller-supplied instance list (no ECM).
int build_plan_from_instances(const tusq_circuit &circ, uint64_t n_inst, const uint64_t *ev_off,
                              const int32_t *ev_slot, const int32_t *ev_qubit,
                              const int32_t *ev_pauli, const double *weights, tusq_plan_t &P) {
    P.n = circ.n;
    P.G = (int)circ.gates.size();
    P.gates = circ.gates;
    P.shots = 0;
    std::memset(&P.stats, 0, sizeof P.stats);
    P.stats.n_gates = P.G;
    std::vector<Key> keys(n_inst);
    for (uint64_t i = 0; i < n_inst; ++i) {
        if (ev_off[i + 1] < ev_off[i]) { set_error("tusq_plan_from_instances: ev_off not ascending"); return TUSQ_EINVAL; }
        if (!(weights[i] >= 0.0)) { set_error("tusq_plan_from_instances: negative weight"); return TUSQ_EINVAL; }
        for (uint64_t e = ev_off[i]; e < ev_off[i + 1]; ++e) {
            int s = ev_slot[e], q = ev_qubit[e], p = ev_pauli[e];
            if (s < 0 || s > P.G || q < 0 || q >= P.n || p < 1 || p > TUSQ_OUTCOME1) {
                set_error("tusq_plan_from_instances: event out of range");
                return TUSQ_EINVAL;
            }
            if (p == TUSQ_OUTCOME1 && (s == P.G || !is_noninvertible(P.gates[s].kind) || P.gates[s].q0 != q)) {
                set_error("tusq_plan_from_instances: outcome event not at a RESET / MEASURE gate on its qubit");
                return TUSQ_EINVAL;
            }
            uint32_t w = pack_event(s, q, p);
            // (slot, qubit) strictly ascending, except that an outcome event
            // may follow a Pauli on the same (slot, qubit)
            if (!keys[i].empty() && !((keys[i].back() >> 2) < (w >> 2) ||
                                      ((keys[i].back() >> 2) == (w >> 2) && p == TUSQ_OUTCOME1 &&
                                       (keys[i].back() & 3) != 3))) {
                set_error("tusq_plan_from_instances: events not sorted by (slot, qubit) or duplicated");
                return TUSQ_EINVAL;
            }
            keys[i].push_back(w);
        }
    }
    std::vector<uint64_t> ord(n_inst);
    for (uint64_t i = 0; i < n_inst; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](uint64_t a, uint64_t b) { return key_less(keys[a], keys[b]); });
    std::vector<Kept> kept;
    for (uint64_t i = 0; i < n_inst; ++i) {
        if (i && keys[ord[i]] == keys[ord[i - 1]]) {
            set_error("tusq_plan_from_instances: two identical instances");
            return TUSQ_EINVAL;
        }
        kept.push_back(Kept{&keys[ord[i]], 0, weights[ord[i]]});
    }
    P.stats.n_ecm_instances = n_inst;
    noninv_stats(P);
    finish_tree(P, kept);
    return TUSQ_OK;
}

// Contiguous chunk `rank` of `world` of a plan's DFS order, balanced by the
// DFTT gate work of each leaf (the first leaf of a chunk pays its whole
// path, later ones the part below their branch slot).
int build_plan_shard(const tusq_plan_t &src, int rank, int world, tusq_plan_t &P) {
    const uint64_t N = src.n_inst();
    std::vector<double> cost(N);
    for (uint64_t i = 0; i < N; ++i) cost[i] = 1.0 + (i ? (double)(src.G - src.lcp[i - 1]) : (double)src.G);
    double total = 0;
    for (double c : cost) total += c;
    // chunk r = leaves whose cumulative cost midpoint falls in [r, r+1) * total / world
    uint64_t a = N, b = N;
    double acc = 0;
    for (uint64_t i = 0; i < N; ++i) {
        double mid = acc + 0.5 * cost[i];
        int r = (int)std::min<double>(world - 1, std::floor(mid * world / total));
        if (r == rank && a == N) a = i;
        if (r > rank && b == N) { b = i; break; }
        acc += cost[i];
    }
    if (a == N) b = N;
    P.n = src.n;
    P.G = src.G;
    P.gates = src.gates;
    P.shots = src.shots;
    P.seed = src.seed;
    P.opts = src.opts;
    std::memset(&P.stats, 0, sizeof P.stats);
    P.stats.shots = src.shots;
    P.stats.n_gates = src.G;
    std::vector<Key> keys;
    for (uint64_t i = a; i < b; ++i) {
        Key k;
        for (uint64_t e = src.ev_off[i]; e < src.ev_off[i + 1]; ++e)
            k.push_back(pack_event(src.ev_slot[e], src.ev_qubit[e], src.ev_pauli[e]));
        keys.push_back(k);
    }
    std::vector<Kept> kept;
    for (uint64_t i = a; i < b; ++i) kept.push_back(Kept{&keys[i - a], src.counts[i], src.weights[i]});
    P.stats.n_ecm_instances = kept.size();
    noninv_stats(P);
    finish_tree(P, kept);
    return TUSQ_OK;
}

namespace {

// Kept instances in DFS order -> flat event lists, branch slots between
// neighbours and the tree statistics of Sec. III-B1.
void finish_tree(tusq_plan_t &P, const std::vector<Kept> &kept) {
    tusq_plan_stats_t &st = P.stats;
    P.ev_off.assign(1, 0);
    P.ev_slot.clear(); P.ev_qubit.clear(); P.ev_pauli.clear();
    P.counts.clear(); P.weights.clear(); P.lcp.clear();
    const Key *prev = nullptr;
    for (const Kept &kp : kept) {
        const Key &k = *kp.key;
        for (uint32_t wd : k) {
            Event e = unpack_event(wd);
            P.ev_slot.push_back(e.slot); P.ev_qubit.push_back(e.qubit); P.ev_pauli.push_back(e.pauli);
        }
        P.ev_off.push_back(P.ev_slot.size());
        P.counts.push_back(kp.count);
        P.weights.push_back(kp.weight);
        if (prev) {
            size_t m = 0;
            while (m < prev->size() && m < k.size() && (*prev)[m] == k[m]) ++m;
            int sa = m < prev->size() ? unpack_event((*prev)[m]).slot : P.G + 1;
            int sb = m < k.size() ? unpack_event(k[m]).slot : P.G + 1;
            P.lcp.push_back(std::min(sa, sb));
        }
        prev = &k;
    }
    const uint64_t N = P.counts.size();
    st.n_instances = N;
    uint64_t edges = N ? (uint64_t)P.G : 0, pa_dftt = 0, pa_scratch = 0;
    for (int32_t t : P.lcp) edges += (uint64_t)(P.G - t);
    st.tree_gate_edges = edges;
    st.dftt_gate_apps = N ? 2 * edges - P.G : 0;
    st.scratch_gate_apps = N * (uint64_t)P.G;
    for (uint64_t i = 0; i < N; ++i) {
        // forward from the previous branch slot, uncompute back to the next
        // one (Kraus-branch choices are not Pauli applications)
        int tin = i ? P.lcp[i - 1] : 0, tout = (i + 1 < N) ? P.lcp[i] : P.G + 1;
        for (uint64_t e = P.ev_off[i]; e < P.ev_off[i + 1]; ++e) {
            if (P.ev_pauli[e] == TUSQ_OUTCOME1) continue;
            pa_scratch++;
            if (P.ev_slot[e] >= tin) pa_dftt++;
            if (P.ev_slot[e] >= tout) pa_dftt++;
        }
    }
    st.dftt_pauli_apps = pa_dftt;
    st.scratch_pauli_apps = pa_scratch;
}

}  // namespace
}  // namespace tusq

std::vector<tusq::Channel> tusq_circuit::ordered() const {
    std::vector<tusq::Channel> out;
    for (size_t j = 0; j < gates.size(); ++j)
        if (ch_of_gate[j] >= 0) {
            tusq::Channel c = channels[ch_of_gate[j]];
            c.gate = (int)j;
            out.push_back(c);
        }
    return out;
}
