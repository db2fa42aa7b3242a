// Measured arithmetic peaks of the current device for the rooflines of the
// SIMT paths (tusq_measure_alu_peaks): FP32 and FP64 fused multiply-add
// throughput of a kernel with eight independent FMA chains per thread, a
// grid of 8 CTAs of 256 threads per SM, timed with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace tusq {

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T *sink, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)-1.2345) sink[threadIdx.x] = s;   // never true; keeps the chains alive
}

template <typename T>
static int rate(int nsm, int iters, cudaStream_t st, double *tflops) {
    T *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync(&sink, 256 * sizeof(T), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int grid = nsm * 8;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
        e = cudaEventRecord(e0, st);
        fma_rate_kernel<T><<<grid, 256, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (sink) cudaFreeAsync(sink, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_error(std::string("tusq_measure_alu_peaks: ") + cudaGetErrorString(e));
        return TUSQ_ECUDA;
    }
    const double fmas = (double)grid * 256 * iters * 16 * 8;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return TUSQ_OK;
}

}  // namespace tusq

extern "C" int tusq_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops, void *cuda_stream) {
    if (!fp32_tflops || !fp64_tflops) {
        tusq::set_error("tusq_measure_alu_peaks: NULL argument");
        return TUSQ_EINVAL;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = tusq::rate<float>(nsm, 2048, st, fp32_tflops);
    if (rc == TUSQ_OK) rc = tusq::rate<double>(nsm, 64, st, fp64_tflops);
    return rc;
}
