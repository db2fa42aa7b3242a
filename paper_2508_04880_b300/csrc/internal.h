// Internal structures of the tusq library (host side).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tusq.h"

namespace tusq {

constexpr int kMaxQubits = 34;

struct Gate {
    int kind = 0, q0 = 0, q1 = -1;
    double p[32] = {0};
};

struct Channel {
    int gate = 0;
    int nterms = 0;
    uint8_t codes[15] = {0};
    double probs[15] = {0};
    uint64_t thr[16] = {0};   // outcome k is the first k with r < thr[k]
};

bool is_two_qubit(int kind);
bool is_diagonal(int kind);
inline bool is_noninvertible(int kind) { return kind == TUSQ_RESET || kind == TUSQ_MEASURE; }

struct Event {
    int32_t slot, qubit, pauli;
    bool operator==(const Event &o) const { return slot == o.slot && qubit == o.qubit && pauli == o.pauli; }
    bool operator!=(const Event &o) const { return !(*this == o); }
    bool operator<(const Event &o) const {
        if (slot != o.slot) return slot < o.slot;
        if (qubit != o.qubit) return qubit < o.qubit;
        return pauli < o.pauli;
    }
};

// Flat list of variable-length records (off has n + 1 entries).
struct FlatList {
    std::vector<uint64_t> off{0};
    std::vector<int32_t> a, b, c;
    std::vector<uint64_t> count;
    uint64_t size() const { return off.size() - 1; }
};

void set_error(const std::string &msg);

// Samples every channel of every shot on the current CUDA device (the ER
// draws of Sec. III-A1): per shot the number of ER words and their hash, the
// offsets of each shot's words and the words (channel << 4 | code).
int sample_ers_device(const std::vector<Channel> &chans, uint64_t shots, uint64_t seed, std::vector<uint32_t> &cnt,
                      std::vector<uint64_t> &hash, std::vector<uint64_t> &off, std::vector<uint32_t> &words);

}  // namespace tusq

struct tusq_circuit {
    int n = 0;
    std::vector<tusq::Gate> gates;
    std::vector<int> ch_of_gate;        // -1 if gate has no channel
    std::vector<tusq::Channel> channels;  // in gate order (rebuilt by ordered())
    std::vector<tusq::Channel> ordered() const;
};

struct tusq_plan_t {
    int n = 0, G = 0;
    std::vector<tusq::Gate> gates;
    uint64_t shots = 0, seed = 0;
    tusq_plan_opts opts{};
    tusq::FlatList raw;        // stage 0
    tusq::FlatList commuted;   // stage 1
    // kept instances in DFS order
    std::vector<uint64_t> ev_off{0};
    std::vector<int32_t> ev_slot, ev_qubit, ev_pauli;
    std::vector<uint64_t> counts;
    std::vector<double> weights;
    std::vector<int32_t> lcp;
    tusq_plan_stats_t stats{};
    uint64_t n_inst() const { return counts.size(); }
};
