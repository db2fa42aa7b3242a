// Host side of the tensor-core dense stage: the B operand of a 32x32 complex
// matrix U in the shared-memory layout the kernels hand to tcgen05.mma (see
// dense.cuh for the real embedding and the chunked K-major layout), split
// into hi and lo parts in TF32 or BF16.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "program.h"

namespace tusq {

namespace {

// FP32 -> TF32 (10 mantissa bits kept), rounding to nearest with ties away
// from zero, the result in an FP32 container.
float tf32_round(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & ~0x1FFFu;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// FP32 -> BF16 bits, rounding to nearest even.
uint16_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

}  // namespace

// Number of FP32 words of the B parts of one dense op in tensor-core mode
// `mode` (a multiple of 32, i.e. whole matrix-pool slots).
size_t dense_b_words(int mode) {
    const size_t part = mode == TUSQ_TC_BF16X3 ? 8192 : 16384;   // bytes
    const int parts = mode == TUSQ_TC_TF32 ? 1 : 2;
    return parts * part / 4;
}

// u: row-major 32x32, u[i*32 + j] = <i|U|j> in the register basis.
void encode_dense_b(const std::complex<double> *u, int mode, float *out) {
    const bool bf = mode == TUSQ_TC_BF16X3;
    const size_t part_bytes = bf ? 8192 : 16384;
    const int epc = bf ? 8 : 4;                 // elements per 16-byte chunk
    const int es = bf ? 2 : 4;                  // element bytes
    const int parts = mode == TUSQ_TC_TF32 ? 1 : 2;
    unsigned char *base = reinterpret_cast<unsigned char *>(out);
    std::memset(base, 0, parts * part_bytes);
    for (int n = 0; n < 64; ++n)
        for (int k = 0; k < 64; ++k) {
            const std::complex<double> z = u[(n >> 1) * 32 + (k >> 1)];
            // [[Re, -Im], [Im, Re]] blocks
            double b;
            if ((n & 1) == 0) b = (k & 1) == 0 ? z.real() : -z.imag();
            else b = (k & 1) == 0 ? z.imag() : z.real();
            const size_t off = (size_t)(k / epc) * 1024 + (size_t)n * 16 + (size_t)(k % epc) * es;
            if (bf) {
                const uint16_t h = bf16_bits((float)b);
                const uint16_t l = bf16_bits((float)(b - (double)bf16_value(h)));
                std::memcpy(base + off, &h, 2);
                std::memcpy(base + part_bytes + off, &l, 2);
            } else {
                const float h = tf32_round((float)b);
                std::memcpy(base + off, &h, 4);
                if (parts == 2) {
                    const float l = tf32_round((float)(b - (double)h));
                    std::memcpy(base + part_bytes + off, &l, 4);
                }
            }
        }
}

}  // namespace tusq
