// Tensor-core dense stage (sm_103a, tcgen05): y = U x for every thread's
// vector x of 32 complex64 amplitudes, U a 32x32 complex matrix that does
// not depend on the thread (Sec. II, Eq. 1: a fused block of gates is one
// 2^k x 2^k matrix acting on groups of 2^k amplitudes).
//
// Real embedding with interleaved components: x as 64 reals
// (Re x_0, Im x_0, Re x_1, ...), y likewise, and the 64x64 real matrix
//   B[2i][2j] = Re U_ij   B[2i][2j+1] = -Im U_ij
//   B[2i+1][2j] = Im U_ij B[2i+1][2j+1] = Re U_ij
// so that y[n] = sum_k B[n][k] x[k]: a GEMM D = A B^T with A = 256 rows
// (one per thread) x K = 64, B = N 64 x K 64, both K-major.
//
// Shared-memory operand layout (no swizzle, K-major canonical form): the K
// extent is cut into 16-byte chunks (4 TF32 or 8 BF16 values); chunk c of
// row r sits at base + c * (rows * 16) + r * 16 (rows = 128 for A, 64 for B).  In the matrix descriptor
// the leading-dimension byte offset is the chunk stride (rows * 16) and the
// stride-dimension byte offset is the distance between 8-row groups (128).
//
// Precision modes (split products, FP32 accumulation in TMEM):
//   TF32X3: x = x_hi + x_lo, B = B_hi + B_lo in TF32; D = hi.hi + hi.lo + lo.hi
//   BF16X3: the same split in BF16 (kind::f16 with BF16 inputs)
//   TF32:   one TF32 product (about 1e-3 relative error; error studies only)
// The product lo.lo and the roundings of the splits are left out.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.h"

namespace tusq {

// Byte sizes of one operand part.
constexpr uint32_t dense_a_part_bytes(int mode) { return mode == TUSQ_TC_BF16X3 ? 16384u : 32768u; }  // 128 rows
constexpr uint32_t dense_b_part_bytes(int mode) { return mode == TUSQ_TC_BF16X3 ? 8192u : 16384u; }   // 64 rows
// Number of B parts stored (hi, and lo for the split modes).
constexpr int dense_b_parts(int mode) { return mode == TUSQ_TC_TF32 ? 1 : 2; }

#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Matrix descriptor of a K-major operand without swizzle.
__device__ __forceinline__ uint64_t dense_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: FP32 accumulator, A and B K-major, M = 128, N = 64;
// operand format 2 = TF32 (kind::tf32) or 1 = BF16 (kind::f16).
__device__ __forceinline__ uint32_t dense_idesc(bool bf16) {
    const uint32_t fmt = bf16 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void dense_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          bool accumulate, bool bf16) {
    const uint32_t acc = accumulate ? 1u : 0u;
    if (bf16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

// TF32 value (round to nearest, ties away) in an FP32 container.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// State of the tensor-core path in one CTA.
struct DenseCtx {
    uint32_t tmem;          // TMEM base address (lane 0, first of 128 columns)
    uint32_t mbar;          // shared address of the MMA-completion mbarrier
    uint32_t phase;         // parity of the mbarrier phase to wait for next
    unsigned int *err;      // device error word (bit 0: a bounded wait ran out)
    int *abort;             // shared flag: stop the CTA's work after a timeout
    int skip_issue;         // test hook: never issue the MMAs (the wait runs out)
    uint32_t bsm = 0;       // shared address of the B region (one dense op's B parts)
};

// Wait for the mbarrier phase with a bound of ~1 s of SM clock; on timeout
// set the error word and the CTA's abort flag and return false.  Callers
// read the abort flag only after a barrier that follows this wait.
__device__ __forceinline__ bool dense_wait(DenseCtx &c) {
    const long long t0 = clock64();
    uint32_t done = 0;
    for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(c.mbar), "r"(c.phase)
            : "memory");
        if (done) break;
        if (clock64() - t0 > (2ll << 30)) {
            atomicOr(c.err, 1u);
            *c.abort = 1;
            return false;
        }
    }
    c.phase ^= 1u;
    return true;
}

// FP32 words of one dense op's B operand parts (device side of dense_b_words).
__device__ __forceinline__ uint32_t dense_b_words_dev(uint32_t mode) {
    return (uint32_t)dense_b_parts((int)mode) * dense_b_part_bytes((int)mode) / 4u;
}

// Write part `part` (0 hi, 1 lo) of one thread's vector as row `row` of an A
// operand part at `abase`: 16-byte chunks of K at chunk * 2048 + row * 16.
template <int MODE>
__device__ __forceinline__ void dense_stage_part(const float2 (&a)[32], unsigned char *abase, int row, int part) {
    if constexpr (MODE == TUSQ_TC_BF16X3) {
        // 8 chunks of 8 BF16
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = a[4 * c + q];
                __nv_bfloat16 x = __float2bfloat16_rn(v.x), y = __float2bfloat16_rn(v.y);
                if (part) {
                    x = __float2bfloat16_rn(v.x - __bfloat162float(x));
                    y = __float2bfloat16_rn(v.y - __bfloat162float(y));
                }
                w[q] = (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
            }
            *reinterpret_cast<uint4 *>(abase + c * 2048 + row * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        // 16 chunks of 4 TF32
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float2 v0 = a[2 * c], v1 = a[2 * c + 1];
            float h0 = to_tf32(v0.x), h1 = to_tf32(v0.y), h2 = to_tf32(v1.x), h3 = to_tf32(v1.y);
            if (part) {
                h0 = to_tf32(v0.x - h0);
                h1 = to_tf32(v0.y - h1);
                h2 = to_tf32(v1.x - h2);
                h3 = to_tf32(v1.y - h3);
            }
            *reinterpret_cast<float4 *>(abase + c * 2048 + row * 16) = make_float4(h0, h1, h2, h3);
        }
    }
}

// Copy one dense op's B operand parts (`bytes`, hi then lo) from global
// memory to the CTA's B region at shared address bsm: 16-byte cp.async
// copies spread over the CTA's threads, one commit group per thread.
__device__ __forceinline__ void dense_copy_b(uint32_t bsm, const float *src, uint32_t bytes, int tid,
                                             int nthr) {
    for (uint32_t i = tid; i < bytes / 16u; i += nthr)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(bsm + 16u * i), "l"(src + 4u * i)
                     : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// y = U x on every thread's 32 registers, all 256 threads of the CTA taking
// part (every call site is reached by the whole CTA).  `abase`: 64 KiB of
// shared memory free for the call (the pass tile, whose amplitudes are held
// in registers meanwhile), which takes the A operand of all 256 rows: thread
// t writes row t & 127 of half t >> 7, and each half is an M = 128, N = 64,
// K = 64 product per split term into its own 64 TMEM columns.  This op's B
// parts are already on their way to the B region (c.bsm: copied by an
// earlier dense_copy_b); once its products are done the region is free and
// `bnext` (the next dense op's B parts, or null when the region already
// holds them) is copied in behind the read-out.
//   BF16X3: A hi of both halves (2 x 16 KiB) then A lo (2 x 16 KiB); one
//           round, products hi.hi + hi.lo + lo.hi;
//   TF32:   A of both halves (2 x 32 KiB); one round;
//   TF32X3: A hi of both halves (2 x 32 KiB): hi.hi + hi.lo, then A lo over
//           it: + lo.hi -- two rounds.
template <int MODE>
__device__ __forceinline__ void dense_apply(float2 (&a)[32], unsigned char *abase, const float *bnext,
                                            DenseCtx &c, int tid, bool renorm) {
    constexpr bool kBF = MODE == TUSQ_TC_BF16X3;
    constexpr uint32_t kApart = dense_a_part_bytes(MODE);     // one half (128 rows) of one part
    constexpr uint32_t kBpart = dense_b_part_bytes(MODE);
    constexpr uint32_t kBbytes = (uint32_t)dense_b_parts(MODE) * kBpart;
    constexpr int kSteps = kBF ? 4 : 8;            // K = 64 in steps of 16 (BF16) or 8 (TF32)
    constexpr int kRounds = MODE == TUSQ_TC_TF32X3 ? 2 : 1;
    const uint32_t a_s = smem_u32(abase), b_s = c.bsm;
    const int warp = tid >> 5, half = tid >> 7, row = tid & 127;
    // *c.abort only changes inside dense_wait, and every read of it follows
    // the barrier after that wait, so all threads see the same value
    if (*c.abort) return;
    // |x|^2 of the thread's vector: a unitary U keeps it, and the tensor
    // cores' FP32 accumulation shrinks it by a few units in the last place
    // per product (a bias, not noise), so the result is scaled back to it
    float nx = 0.f;
    if (renorm) {
#pragma unroll
        for (int i = 0; i < 32; ++i) nx = fmaf(a[i].x, a[i].x, fmaf(a[i].y, a[i].y, nx));
    }
    __syncthreads();                               // every thread has gathered its amplitudes
    dense_stage_part<MODE>(a, abase + half * kApart, row, 0);
    if constexpr (kBF) dense_stage_part<MODE>(a, abase + 2 * kApart + half * kApart, row, 1);
    for (int rd = 0; rd < kRounds; ++rd) {
        if (rd > 0) dense_stage_part<MODE>(a, abase + half * kApart, row, 1);   // TF32X3: A lo over A hi
        asm volatile("cp.async.wait_all;" ::: "memory");            // this op's B parts
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !c.skip_issue) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = dense_idesc(kBF);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t d = c.tmem + 64u * h;
                const uint32_t ah = a_s + h * kApart;
                if constexpr (MODE == TUSQ_TC_BF16X3) {
                    // (A part offset, B part): hi.hi, hi.lo, lo.hi
                    const uint32_t ao[3] = {0u, 0u, 2 * kApart}, bp[3] = {0u, 1u, 0u};
#pragma unroll
                    for (int t = 0; t < 3; ++t)
#pragma unroll
                        for (int s = 0; s < kSteps; ++s)
                            dense_mma(d, dense_desc(ah + ao[t] + s * 4096u, 2048u, 128u),
                                      dense_desc(b_s + bp[t] * kBpart + s * 2048u, 1024u, 128u), idesc,
                                      t > 0 || s > 0, true);
                } else if (MODE == TUSQ_TC_TF32X3 && rd == 0) {
#pragma unroll
                    for (int t = 0; t < 2; ++t)
#pragma unroll
                        for (int s = 0; s < kSteps; ++s)
                            dense_mma(d, dense_desc(ah + s * 4096u, 2048u, 128u),
                                      dense_desc(b_s + t * kBpart + s * 2048u, 1024u, 128u), idesc,
                                      t > 0 || s > 0, false);
                } else {
                    // TF32 (one product), or TF32X3's lo.hi added to the first round's
#pragma unroll
                    for (int s = 0; s < kSteps; ++s)
                        dense_mma(d, dense_desc(ah + s * 4096u, 2048u, 128u), dense_desc(b_s + s * 2048u, 1024u, 128u),
                                  idesc, rd > 0 || s > 0, false);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c.mbar)
                         : "memory");
        }
        dense_wait(c);                             // on timeout: error word and abort flag
        __syncthreads();
        if (*c.abort) return;                      // uniform: read after the barrier
    }
    // the products are done: the B region is free for the next dense op's parts
    if (bnext) dense_copy_b(b_s, bnext, kBbytes, tid, blockDim.x);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
        uint32_t r[64];
        const uint32_t taddr = c.tmem + ((uint32_t)((warp & 3) * 32) << 16) + 64u * half;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
            "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
            "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
              "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
              "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]),
              "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]),
              "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
              "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
              "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]),
              "=r"(r[63])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) a[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    }
    if (renorm) {
        float ny = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) ny = fmaf(a[i].x, a[i].x, fmaf(a[i].y, a[i].y, ny));
        const float sc = ny > 0.f ? sqrtf(nx / ny) : 1.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) a[i] = make_float2(a[i].x * sc, a[i].y * sc);
    }
    // the next write of the TMEM columns (the next dense op's products) is
    // issued after a CTA barrier, which this fence orders the read-out before
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Set-up by the whole CTA: warp 0 allocates 128 TMEM columns (address
// written to *tmem_slot), thread 0 initialises the mbarrier.
__device__ __forceinline__ void dense_setup(uint32_t *tmem_slot, uint64_t *mbar, int tid) {
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Tear-down by the whole CTA after its last dense op: its B copies are
// waited for and warp 0 frees the TMEM.
__device__ __forceinline__ void dense_teardown(uint32_t tmem, int tid) {
    asm volatile("cp.async.wait_all;" ::: "memory");   // a prefetched B the CTA did not use
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
    }
}

#endif  // __CUDACC__

}  // namespace tusq
