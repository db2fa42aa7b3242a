// Shot sampling of the output distribution on the device (sm_103a).
//
// The paper samples the output state vector of each kept instance s_i times
// (Sec. III-A1); the traversal here returns the exact tally-weighted
// distribution, and this entry point draws shots from it.  Every outcome gets
// the integer weight w_x = floor(p_x 2^56) (0 for p_x <= 0 or NaN), the
// cumulative weights C_x = w_0 + ... + w_x are formed by an exact integer
// prefix sum (so the result does not depend on the summation order), and
// shot s lands on the first x with C_x > floor(r_s W / 2^64), W = C_last,
// r_s = word 0 of Philox4x64-10 at counter (s, 0, 0, 0), key (seed, 3).
//
// Kernels: (1) weights and per-block inclusive scans (one CTA per 4096
// outcomes, warp shuffles), (2) a scan of the block totals in one CTA,
// (3) block offsets added back, (4) one thread per shot: Philox draw, binary
// search over C, atomic increment of the outcome's count.  Passes 1 and 3
// are HBM streams over 2^n x (8 + 8) bytes; pass 4 is latency-bound
// (log2(2^n) dependent loads per shot).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "internal.h"
#include "philox.cuh"

namespace tusq {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 16;
constexpr int kScanChunk = kScanThreads * kScanPerThread;   // outcomes per CTA

__device__ __forceinline__ uint64_t philox_word0(uint64_t c0, uint64_t k0, uint64_t k1) {
    uint64_t out[4];
    philox4x64_10(c0, 0, 0, 0, k0, k1, out);
    return out[0];
}

__device__ __forceinline__ uint64_t weight_of(double p) {
    return p > 0.0 ? __double2ull_rz(p * 72057594037927936.0) : 0ull;   // 2^56
}

// Inclusive scan of a CTA's values (one per thread) with warp shuffles.
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t v, uint64_t *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (warp > 0) v += warp_tot[warp - 1];
    return v;
}

// (1) C[x] = cumulative weight within the CTA's chunk; totals[b] = chunk sum.
__global__ void __launch_bounds__(kScanThreads) scan_chunks(const double *probs, uint64_t dim, uint64_t *C,
                                                            uint64_t *totals) {
    __shared__ uint64_t warp_tot[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanPerThread;
    uint64_t w[kScanPerThread];
    uint64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanPerThread; ++i) {
        const uint64_t x = base + i;
        run += x < dim ? weight_of(probs[x]) : 0ull;
        w[i] = run;
    }
    const uint64_t incl = block_inclusive_scan(run, warp_tot);
    const uint64_t off = incl - run;
#pragma unroll
    for (int i = 0; i < kScanPerThread; ++i) {
        const uint64_t x = base + i;
        if (x < dim) C[x] = w[i] + off;
    }
    if (threadIdx.x == blockDim.x - 1) totals[blockIdx.x] = incl;
}

// (2) exclusive scan of the chunk totals in place (one CTA, serial over
// tiles of blockDim.x totals); the grand total goes to *total.
__global__ void __launch_bounds__(kScanThreads) scan_totals(uint64_t *totals, uint64_t n, uint64_t *total) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t b = 0; b < n; b += blockDim.x) {
        const uint64_t i = b + threadIdx.x;
        const uint64_t v = i < n ? totals[i] : 0ull;
        const uint64_t incl = block_inclusive_scan(v, warp_tot);
        const uint64_t c = carry;
        if (i < n) totals[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// (3) add each chunk's offset.
__global__ void __launch_bounds__(kScanThreads) add_offsets(uint64_t *C, uint64_t dim, const uint64_t *offsets) {
    const uint64_t off = offsets[blockIdx.x];
    if (off == 0) return;
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
#pragma unroll
    for (int i = 0; i < kScanPerThread; ++i) {
        const uint64_t x = base + (uint64_t)i * kScanThreads + threadIdx.x;
        if (x < dim) C[x] += off;
    }
}

// (4) one thread per shot.
__global__ void __launch_bounds__(256) draw_shots(const uint64_t *C, uint64_t dim, const uint64_t *total,
                                                  uint64_t shots, uint64_t seed, unsigned long long *counts) {
    const uint64_t W = *total;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = philox_word0(s, seed, 3);
        const uint64_t t = __umul64hi(r, W);
        uint64_t lo = 0, hi = dim - 1;
        while (lo < hi) {
            const uint64_t mid = lo + ((hi - lo) >> 1);
            if (C[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        atomicAdd(counts + lo, 1ull);
    }
}

}  // namespace

}  // namespace tusq

using namespace tusq;

#define S_TRY(x)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) {                                                        \
            set_error(std::string("tusq_sample: ") + #x + ": " + cudaGetErrorString(e_)); \
            return TUSQ_ECUDA;                                                          \
        }                                                                               \
    } while (0)

extern "C" int tusq_sample(const double *probs_dev, int n_qubits, uint64_t shots, uint64_t seed,
                           uint64_t *counts_dev, void *cuda_stream) {
    if (!probs_dev || !counts_dev || n_qubits < 0 || n_qubits > kMaxQubits) {
        set_error("tusq_sample: NULL buffer or n_qubits outside 0..34");
        return TUSQ_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint64_t dim = 1ull << n_qubits;
    const uint64_t nchunks = (dim + kScanChunk - 1) / kScanChunk;
    uint64_t *scratch = nullptr;
    const size_t bytes = sizeof(uint64_t) * (dim + nchunks + 1);
    S_TRY(cudaMemsetAsync(counts_dev, 0, sizeof(uint64_t) * dim, st));
    if (shots == 0) return TUSQ_OK;
    S_TRY(cudaMallocAsync((void **)&scratch, bytes, st));
    uint64_t *C = scratch, *totals = scratch + dim, *total = totals + nchunks;
    scan_chunks<<<(unsigned)nchunks, kScanThreads, 0, st>>>(probs_dev, dim, C, totals);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        scan_totals<<<1, kScanThreads, 0, st>>>(totals, nchunks, total);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        add_offsets<<<(unsigned)nchunks, kScanThreads, 0, st>>>(C, dim, totals);
        e = cudaGetLastError();
    }
    uint64_t W = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&W, total, sizeof W, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && W == 0) {
        cudaFreeAsync(scratch, st);
        set_error("tusq_sample: the distribution has no positive weight");
        return TUSQ_EINVAL;
    }
    if (e == cudaSuccess) {
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t want = (shots + 255) / 256;
        const unsigned grid = (unsigned)(want < (uint64_t)nsm * 16 ? want : (uint64_t)nsm * 16);
        draw_shots<<<grid, 256, 0, st>>>(C, dim, total, shots, seed, (unsigned long long *)counts_dev);
        e = cudaGetLastError();
    }
    cudaError_t f = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) {
        set_error(std::string("tusq_sample: ") + cudaGetErrorString(e));
        return TUSQ_ECUDA;
    }
    if (f != cudaSuccess) {
        set_error(std::string("tusq_sample: cudaFreeAsync: ") + cudaGetErrorString(f));
        return TUSQ_ECUDA;
    }
    return TUSQ_OK;
}
