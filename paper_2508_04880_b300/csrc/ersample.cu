// ER sampling on the device (Sec. III-A1: every channel of every shot is
// sampled before any state-vector work; the paper does this on the CPU).
//
// Shot s, channel c (gate order) draws r = word (c mod 4) of Philox4x64-10 at
// counter (s, floor(c / 4), 0, 0), key (seed, 0), and takes outcome k = the
// first k with r < thr_c[k] (thr_c[0] = identity).  The host planner draws the
// same way, so both give the same error realizations.
//
// Two kernels, one thread per shot: the first counts each shot's
// non-identity outcomes and hashes its ER words (channel << 4 | Pauli code);
// after the host turns the counts into offsets, the second writes the words.
// The host then tallies by hash, comparing word lists for exactness.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"
#include "philox.cuh"

namespace tusq {

namespace {

struct DevChannel {
    uint64_t thr[16];
    uint8_t codes[16];
    int32_t nterms;
    int32_t pad;
};

__device__ __forceinline__ uint64_t er_mix(uint64_t h, uint32_t w) {
    h ^= w;
    h *= 0x100000001B3ull;
    return h ^ (h >> 29);
}

// Calls f(word) for every non-identity outcome of shot s, in channel order.
template <class F>
__device__ __forceinline__ void shot_ers(const DevChannel *ch, const uint64_t *thr0, int C, uint64_t s, uint64_t seed,
                                         F f) {
    uint64_t blk[4];
    for (int c = 0; c < C; ++c) {
        if ((c & 3) == 0) philox4x64_10(s, (uint64_t)c >> 2, 0, 0, seed, 0, blk);
        const uint64_t r = blk[c & 3];
        if (r < thr0[c]) continue;
        const DevChannel &d = ch[c];
        int k = 1;
        while (k < d.nterms && !(r < d.thr[k])) ++k;
        f(((uint32_t)c << 4) | d.codes[k - 1]);
    }
}

__global__ void __launch_bounds__(256) er_count(const DevChannel *ch, const uint64_t *thr0, int C, uint64_t shots,
                                                uint64_t seed, uint32_t *cnt, uint64_t *hash) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t n = 0;
        uint64_t h = 0x243F6A8885A308D3ull;
        shot_ers(ch, thr0, C, s, seed, [&](uint32_t w) {
            ++n;
            h = er_mix(h, w);
        });
        cnt[s] = n;
        hash[s] = h ^ n;
    }
}

__global__ void __launch_bounds__(256) er_write(const DevChannel *ch, const uint64_t *thr0, int C, uint64_t shots,
                                                uint64_t seed, const uint64_t *off, uint32_t *words) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t *out = words + off[s];
        shot_ers(ch, thr0, C, s, seed, [&](uint32_t w) { *out++ = w; });
    }
}

// Device scratch of one sampling call on a private non-blocking stream:
// stream-ordered allocations and copies, so that planning the next job does
// not synchronise with a traversal running on another stream.
struct Scratch {
    cudaStream_t st = nullptr;
    std::vector<void *> bufs;
    ~Scratch() {
        for (void *b : bufs) cudaFreeAsync(b, st);
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    }
    cudaError_t alloc(void **p, size_t bytes) {
        cudaError_t e = cudaMallocAsync(p, bytes, st);
        if (e == cudaSuccess) bufs.push_back(*p);
        return e;
    }
};

}  // namespace

#define E_TRY(x)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) {                                                                 \
            set_error(std::string("tusq_plan (device sampling): ") + #x + ": " + cudaGetErrorString(e_)); \
            return TUSQ_ECUDA;                                                                   \
        }                                                                                        \
    } while (0)

// Samples every channel of every shot on the current device.  Returns per
// shot the number of ER words and their hash, the offsets of each shot's
// words and the words themselves (channel << 4 | code, channel order).
int sample_ers_device(const std::vector<Channel> &chans, uint64_t shots, uint64_t seed, std::vector<uint32_t> &cnt,
                      std::vector<uint64_t> &hash, std::vector<uint64_t> &off, std::vector<uint32_t> &words) {
    const int C = (int)chans.size();
    std::vector<DevChannel> hc(C > 0 ? C : 1);
    std::vector<uint64_t> hthr0(C > 0 ? C : 1, UINT64_MAX);
    for (int c = 0; c < C; ++c) {
        DevChannel d{};
        for (int k = 0; k < 16; ++k) d.thr[k] = chans[c].thr[k];
        for (int k = 0; k < 15; ++k) d.codes[k] = chans[c].codes[k];
        d.nterms = chans[c].nterms;
        hc[c] = d;
        hthr0[c] = chans[c].thr[0];
    }
    cnt.assign(shots, 0);
    hash.assign(shots, 0);
    off.assign(shots + 1, 0);
    words.clear();
    if (shots == 0) return TUSQ_OK;
    Scratch sc;
    E_TRY(cudaStreamCreateWithFlags(&sc.st, cudaStreamNonBlocking));
    void *dch = nullptr, *dthr0 = nullptr, *dcnt = nullptr, *dhash = nullptr, *doff = nullptr, *dwords = nullptr;
    E_TRY(sc.alloc(&dch, sizeof(DevChannel) * hc.size()));
    E_TRY(sc.alloc(&dthr0, sizeof(uint64_t) * hthr0.size()));
    E_TRY(sc.alloc(&dcnt, sizeof(uint32_t) * shots));
    E_TRY(sc.alloc(&dhash, sizeof(uint64_t) * shots));
    E_TRY(cudaMemcpyAsync(dch, hc.data(), sizeof(DevChannel) * hc.size(), cudaMemcpyHostToDevice, sc.st));
    E_TRY(cudaMemcpyAsync(dthr0, hthr0.data(), sizeof(uint64_t) * hthr0.size(), cudaMemcpyHostToDevice, sc.st));
    int dev = 0, nsm = 148;
    E_TRY(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (shots + 255) / 256;
    const unsigned grid = (unsigned)(want < (uint64_t)nsm * 32 ? want : (uint64_t)nsm * 32);
    er_count<<<grid, 256, 0, sc.st>>>((const DevChannel *)dch, (const uint64_t *)dthr0, C, shots, seed,
                                      (uint32_t *)dcnt, (uint64_t *)dhash);
    E_TRY(cudaGetLastError());
    E_TRY(cudaMemcpyAsync(cnt.data(), dcnt, sizeof(uint32_t) * shots, cudaMemcpyDeviceToHost, sc.st));
    E_TRY(cudaMemcpyAsync(hash.data(), dhash, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, sc.st));
    E_TRY(cudaStreamSynchronize(sc.st));
    for (uint64_t s = 0; s < shots; ++s) off[s + 1] = off[s] + cnt[s];
    words.resize(off[shots]);
    if (!words.empty()) {
        E_TRY(sc.alloc(&doff, sizeof(uint64_t) * shots));
        E_TRY(sc.alloc(&dwords, sizeof(uint32_t) * words.size()));
        E_TRY(cudaMemcpyAsync(doff, off.data(), sizeof(uint64_t) * shots, cudaMemcpyHostToDevice, sc.st));
        er_write<<<grid, 256, 0, sc.st>>>((const DevChannel *)dch, (const uint64_t *)dthr0, C, shots, seed,
                                          (const uint64_t *)doff, (uint32_t *)dwords);
        E_TRY(cudaGetLastError());
        E_TRY(cudaMemcpyAsync(words.data(), dwords, sizeof(uint32_t) * words.size(), cudaMemcpyDeviceToHost,
                              sc.st));
        E_TRY(cudaStreamSynchronize(sc.st));
    }
    return TUSQ_OK;
}

}  // namespace tusq
