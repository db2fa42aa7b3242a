// Join of a parallel-subtree traversal (Sec. III-B: subtrees of the
// instance tree traversed in parallel): the FP64 outputs of chunks 2..k are
// added into the first chunk's output, in chunk order, so the result does
// not depend on which chunk finishes first.  One streaming pass over
// (k + 1) x 2^n x 8 bytes, grid sized in multiples of the SM count.
#include <cuda_runtime.h>
#include <stdint.h>

namespace tusq {

namespace {

constexpr int kMaxParts = 16;

struct PartPtrs {
    const double *p[kMaxParts];
};

__global__ void __launch_bounds__(256) sum_parts_kernel(double *out, PartPtrs parts, int k, uint64_t dim) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        double v = out[i];
        for (int r = 0; r < k; ++r) v += parts.p[r][i];
        out[i] = v;
    }
}

}  // namespace

cudaError_t launch_sum_parts(double *out, const double *const *parts, int k, uint64_t dim, int nsm,
                             cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    if (k > kMaxParts) return cudaErrorInvalidValue;
    PartPtrs pp{};
    for (int r = 0; r < k; ++r) pp.p[r] = parts[r];
    uint64_t want = (dim + 255) / 256;
    const uint64_t cap = (uint64_t)nsm * 8;
    const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
    sum_parts_kernel<<<grid, 256, 0, st>>>(out, pp, k, dim);
    return cudaGetLastError();
}

}  // namespace tusq
