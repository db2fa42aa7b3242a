// Diagnostic entry of the tensor-core dense stage (tusq_dense_check): one
// CTA runs the dense-stage device path of the pass kernel on 256 vectors.
#include <cuda_runtime.h>

#include <complex>
#include <vector>

#include "dense.cuh"
#include "internal.h"

namespace tusq {

template <int MODE>
__global__ void __launch_bounds__(256, 1) dense_check_kernel(const float2 *x, float2 *y, const float *b,
                                                             uint32_t b_bytes, unsigned int *err, int renorm) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    unsigned char *abase = smem;                 // 64 KiB: A staging (the pass kernel's tile)
    const uint32_t bsm = smem_u32(smem + 65536); // the B region after it
    if (tid == 0) abort_flag = 0;
    dense_copy_b(bsm, b, b_bytes, tid, blockDim.x);
    float2 a[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = x[32 * tid + i];
    dense_setup(&tmem_slot, &mbar, tid);
    DenseCtx c{tmem_slot, smem_u32(&mbar), 0u, err, &abort_flag, 0, bsm};
    dense_apply<MODE>(a, abase, nullptr, c, tid, renorm != 0);
#pragma unroll
    for (int i = 0; i < 32; ++i) y[32 * tid + i] = a[i];
    dense_teardown(c.tmem, tid);
}

template <int MODE>
static cudaError_t launch_check(const float2 *x, float2 *y, const float *b, uint32_t bb, unsigned int *err,
                                cudaStream_t st) {
    const int renorm = 0;     // the diagnostic checks the raw tensor-core product
    // the 64 KiB area the pass kernel lends a dense op (its tile), then the
    // B region (at most 32 KiB) and slack up to 128 KiB: a descriptor read
    // with the leading and stride offsets exchanged would still stay inside
    // this CTA's allocation
    const size_t smem = 65536 + 65536;
    cudaError_t e = cudaFuncSetAttribute(dense_check_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dense_check_kernel<MODE><<<1, 256, smem, st>>>(x, y, b, bb, err, renorm);
    return cudaGetLastError();
}

}  // namespace tusq

using namespace tusq;

extern "C" int tusq_dense_check(int tc_mode, const double *u_host, const float *x_dev, float *y_dev,
                                void *cuda_stream) {
    if (tc_mode != TUSQ_TC_TF32X3 && tc_mode != TUSQ_TC_BF16X3 && tc_mode != TUSQ_TC_TF32) {
        set_error("tusq_dense_check: tc_mode must be TUSQ_TC_TF32X3, TUSQ_TC_BF16X3 or TUSQ_TC_TF32");
        return TUSQ_EINVAL;
    }
    if (!u_host || !x_dev || !y_dev) {
        set_error("tusq_dense_check: null pointer");
        return TUSQ_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<std::complex<double>> u(1024);
    for (int k = 0; k < 1024; ++k) u[k] = std::complex<double>(u_host[2 * k], u_host[2 * k + 1]);
    std::vector<float> b(dense_b_words(tc_mode));
    encode_dense_b(u.data(), tc_mode, b.data());
    const uint32_t bb = (uint32_t)(b.size() * 4);
    float *bd = nullptr;
    unsigned int *err = nullptr;
    int rc = TUSQ_OK;
    cudaError_t e = cudaMallocAsync(&bd, bb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bd, b.data(), bb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        const float2 *x = reinterpret_cast<const float2 *>(x_dev);
        float2 *y = reinterpret_cast<float2 *>(y_dev);
        if (tc_mode == TUSQ_TC_TF32X3) e = launch_check<TUSQ_TC_TF32X3>(x, y, bd, bb, err, st);
        else if (tc_mode == TUSQ_TC_BF16X3) e = launch_check<TUSQ_TC_BF16X3>(x, y, bd, bb, err, st);
        else e = launch_check<TUSQ_TC_TF32>(x, y, bd, bb, err, st);
    }
    unsigned int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (bd) cudaFreeAsync(bd, st);
    if (err) cudaFreeAsync(err, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        set_error(std::string("tusq_dense_check: ") + cudaGetErrorString(e));
        rc = TUSQ_ECUDA;
    } else if (herr) {
        set_error("tusq_dense_check: the wait for the tensor cores ran out");
        rc = TUSQ_ETIMEOUT;
    }
    return rc;
}
