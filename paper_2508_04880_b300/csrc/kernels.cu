// CUDA kernels of the DFTT engine (sm_103a).
//
// pass_kernel: one full-state pass.  The state is cut into tiles of 2^L
// amplitudes that share every index bit outside a window of L qubits
// (the window always contains the lowest qubits, so each tile is a set of
// contiguous 128-byte runs).  A CTA loads a tile into shared memory with
// coalesced 16-byte loads, runs its register stages -- each thread gathers
// 2^V amplitudes that differ in the stage's V register bits, applies the
// stage's gates in registers (2x2, 4x4, diagonal phase runs), scatters them
// back -- and writes the tile back, optionally also to a snapshot, adding
// w|psi|^2 into the FP64 output (leaf) and producing partial sums of the
// norm and a checksum (drift check).  Shared-memory addresses are
// XOR-swizzled (tile_swizzle) so that every stage layout spreads over banks.
//
// B300 has little FP64 throughput, so complex64 passes keep FP64 out of the
// per-amplitude work: matrices come from an FP32 pool, partial sums are
// FP32 within a tile, and the leaf update costs one FP64 add per amplitude.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dense.cuh"
#include "program.h"

namespace tusq {

template <typename R> struct C2T;
template <> struct C2T<float> { using type = float2; };
template <> struct C2T<double> { using type = double2; };

template <typename C2> __device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    C2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * b + c
template <typename C2> __device__ __forceinline__ C2 cmad(C2 a, C2 b, C2 c) {
    C2 r;
    r.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    r.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
    return r;
}

// A pass's program as copied into shared memory next to the tile: its ops,
// matrix slots (16 complex entries each, FP32 for complex64) and diagonal
// terms (mask, fixed-point phase), indexed relative to the pass's first one.
template <typename R> struct SProg {
    using C2 = typename C2T<R>::type;
    const DevOp *ops;
    const C2 *mats;
    const uint64_t *terms;
    uint32_t op0, mat0, term0;
    __device__ __forceinline__ C2 mat(uint32_t slot, int k) const { return mats[16 * (slot - mat0) + k]; }
};

// 2x2 on register bit B; SUB picks the form (general, real, RX-type).
// Every product that reads the old pair is formed first, then the final
// fused multiply-adds overwrite the pair in place.
template <int V, int B, int SUB, typename C2>
__device__ __forceinline__ void apply1(C2 (&a)[1 << V], C2 m0, C2 m1, C2 m2, C2 m3) {
#pragma unroll
    for (int r = 0; r < (1 << V); ++r) {
        if (r & (1 << B)) continue;
        C2 &x = a[r];
        C2 &y = a[r | (1 << B)];
        if constexpr (SUB == SUB_REAL) {
            const auto t0 = m1.x * y.x, t1 = m1.x * y.y, t2 = m2.x * x.x, t3 = m2.x * x.y;
            x.x = fma(m0.x, x.x, t0);
            x.y = fma(m0.x, x.y, t1);
            y.x = fma(m3.x, y.x, t2);
            y.y = fma(m3.x, y.y, t3);
        } else if constexpr (SUB == SUB_RXT) {
            // [[1, -it], [-it, 1]], t = m0.x (the factor c is in the stage scalar)
            const auto t = m0.x;
            const auto xr = x.x, xi = x.y, yr = y.x, yi = y.y;
            x.x = fma(t, yi, xr);
            x.y = fma(-t, yr, xi);
            y.x = fma(t, xi, yr);
            y.y = fma(-t, xr, yi);
        } else if constexpr (SUB == SUB_RXS) {
            // [[ik, 1], [1, ik]], k = m0.x (the factor -is is in the stage scalar)
            const auto k = m0.x;
            const auto xr = x.x, xi = x.y, yr = y.x, yi = y.y;
            x.x = fma(-k, xi, yr);
            x.y = fma(k, xr, yi);
            y.x = fma(-k, yi, xr);
            y.y = fma(k, yr, xi);
        } else {
            const C2 xo = x, yo = y;
            const C2 u = cmad(m0, xo, cmul(m1, yo));
            const C2 w = cmad(m2, xo, cmul(m3, yo));
            x = u;
            y = w;
        }
    }
}

// 4x4 on register bits A < B, basis k = bit_A + 2 bit_B.
template <int V, int A, int B, typename C2>
__device__ __forceinline__ void apply2(C2 (&a)[1 << V], const C2 (&m)[16]) {
#pragma unroll
    for (int r = 0; r < (1 << V); ++r) {
        if (r & ((1 << A) | (1 << B))) continue;
        const int i0 = r, i1 = r | (1 << A), i2 = r | (1 << B), i3 = r | (1 << A) | (1 << B);
        C2 v0 = a[i0], v1 = a[i1], v2 = a[i2], v3 = a[i3];
        a[i0] = cmad(m[0], v0, cmad(m[1], v1, cmad(m[2], v2, cmul(m[3], v3))));
        a[i1] = cmad(m[4], v0, cmad(m[5], v1, cmad(m[6], v2, cmul(m[7], v3))));
        a[i2] = cmad(m[8], v0, cmad(m[9], v1, cmad(m[10], v2, cmul(m[11], v3))));
        a[i3] = cmad(m[12], v0, cmad(m[13], v1, cmad(m[14], v2, cmul(m[15], v3))));
    }
}

// Exchange of basis states s0, s1 of every quad on register bits A < B.
template <int V, int A, int B, typename C2>
__device__ __forceinline__ void swap2(C2 (&a)[1 << V], int s0, int s1) {
#pragma unroll
    for (int r = 0; r < (1 << V); ++r) {
        if (r & ((1 << A) | (1 << B))) continue;
        const int idx[4] = {r, r | (1 << A), r | (1 << B), r | (1 << A) | (1 << B)};
        C2 v[4] = {a[idx[0]], a[idx[1]], a[idx[2]], a[idx[3]]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            C2 o = v[q];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (p == q) continue;
                const bool take = (q == s0 && p == s1) || (q == s1 && p == s0);
                o.x = take ? v[p].x : o.x;
                o.y = take ? v[p].y : o.y;
            }
            a[idx[q]] = o;
        }
    }
}

// A product op: 2x2s of form SUB on the register bits in `bits`, bit b's
// matrix at m[4b..4b+3].
template <int V, int SUB, typename C2>
__device__ __forceinline__ void apply_prod(C2 (&a)[1 << V], uint32_t bits, const C2 *m) {
    if (bits & 1u) apply1<V, 0, SUB>(a, m[0], m[1], m[2], m[3]);
    if constexpr (V > 1) if (bits & 2u) apply1<V, 1, SUB>(a, m[4], m[5], m[6], m[7]);
    if constexpr (V > 2) if (bits & 4u) apply1<V, 2, SUB>(a, m[8], m[9], m[10], m[11]);
    if constexpr (V > 3) if (bits & 8u) apply1<V, 3, SUB>(a, m[12], m[13], m[14], m[15]);
    if constexpr (V > 4) if (bits & 16u) apply1<V, 4, SUB>(a, m[16], m[17], m[18], m[19]);
}

// A matrix op, dispatched once on its host-decoded code (form and register
// bits); each case loads only the matrix entries its form uses.
template <int V, typename R>
__device__ __forceinline__ void apply_matrix_op(typename C2T<R>::type (&a)[1 << V], const DevOp &op,
                                                const SProg<R> &P) {
    using C2 = typename C2T<R>::type;
    const C2 *m = P.mats + 16 * (op.mat - P.mat0);
#define TUSQ_M1(B)                                                                               \
    case CODE_MAT1 + 5 * SUB_GENERAL + B:                                                        \
        if constexpr (V > B) apply1<V, B, SUB_GENERAL>(a, m[0], m[1], m[2], m[3]);              \
        break;                                                                                   \
    case CODE_MAT1 + 5 * SUB_REAL + B:                                                           \
        if constexpr (V > B) apply1<V, B, SUB_REAL>(a, m[0], m[1], m[2], m[3]);                 \
        break;                                                                                   \
    case CODE_MAT1 + 5 * SUB_RXT + B:                                                            \
        if constexpr (V > B) apply1<V, B, SUB_RXT>(a, m[0], m[1], m[2], m[3]);                  \
        break;                                                                                   \
    case CODE_MAT1 + 5 * SUB_RXS + B:                                                            \
        if constexpr (V > B) apply1<V, B, SUB_RXS>(a, m[0], m[1], m[2], m[3]);                  \
        break;
#define TUSQ_M2(X, Y)                                                                            \
    case CODE_MAT2 + pair_code(X, Y):                                                            \
        if constexpr (V > Y) {                                                                   \
            C2 mm[16];                                                                           \
            _Pragma("unroll") for (int q = 0; q < 16; ++q) mm[q] = m[q];                        \
            apply2<V, X, Y>(a, mm);                                                              \
        }                                                                                        \
        break;                                                                                   \
    case CODE_SWAP + pair_code(X, Y):                                                            \
        if constexpr (V > Y) swap2<V, X, Y>(a, op.sw0, op.sw1);                                  \
        break;
    switch (op.code) {
    case CODE_PROD + SUB_GENERAL: apply_prod<V, SUB_GENERAL>(a, (uint32_t)op.a, m); break;
    case CODE_PROD + SUB_REAL: apply_prod<V, SUB_REAL>(a, (uint32_t)op.a, m); break;
    case CODE_PROD + SUB_RXT: apply_prod<V, SUB_RXT>(a, (uint32_t)op.a, m); break;
    case CODE_PROD + SUB_RXS: apply_prod<V, SUB_RXS>(a, (uint32_t)op.a, m); break;
        TUSQ_M1(0) TUSQ_M1(1) TUSQ_M1(2) TUSQ_M1(3) TUSQ_M1(4)
        TUSQ_M2(0, 1) TUSQ_M2(0, 2) TUSQ_M2(0, 3) TUSQ_M2(0, 4) TUSQ_M2(1, 2)
        TUSQ_M2(1, 3) TUSQ_M2(1, 4) TUSQ_M2(2, 3) TUSQ_M2(2, 4) TUSQ_M2(3, 4)
    default: break;
    }
#undef TUSQ_M1
#undef TUSQ_M2
}

// Fixed-point phase -> (cos, sin) of 2 pi * phase.
template <typename R> struct Phase;
template <> struct Phase<float> {
    using U = uint32_t;
    // 2^-31-turn units; the low 31 bits, read as a signed 32-bit fraction of a
    // turn, give the exact angle reduced to [-1/2, 1/2) turn.  It is rounded
    // to 2^-23 turn and converted to float by the 1.5 * 2^23 exponent trick
    // (integer and FP32 adds, no conversion instruction) before the fast
    // hardware sine and cosine (absolute error about 4e-7 there).
    __device__ static float2 unit(U p) {
        const int32_t t = (int32_t)((p << 1) + 256u) >> 9;              // [-2^22, 2^22)
        const float f = __int_as_float(0x4B400000 + t) - 12582912.0f;   // exactly t
        float sn, cs;
        __sincosf(f * 7.490140565847857e-07f, &sn, &cs);                 // 2 pi / 2^23
        return make_float2(cs, sn);
    }
};
template <> struct Phase<double> {
    using U = uint64_t;
    static constexpr U kMask = 0x7FFFFFFFFFFFFFFFull;
    __device__ static double2 unit(U p) {
        double t = (double)(p & kMask) * 1.0842021724855044e-19;  // 2^-63 turns
        double s, c;
        sincospi(2.0 * t, &s, &c);
        return make_double2(c, s);
    }
};

// Multiply the registers r with parity(r & MU) = 1 by w (MU a constant).
template <int V, int MU, typename C2>
__device__ __forceinline__ void phase_group(C2 (&a)[1 << V], C2 w) {
#pragma unroll
    for (int r = 0; r < (1 << V); ++r)
        if (__builtin_popcount(r & MU) & 1) a[r] = cmul(a[r], w);
}

template <int V, typename C2>
__device__ __forceinline__ void phase_group_dispatch(C2 (&a)[1 << V], int mu, C2 w) {
#define TUSQ_G(M) \
    case M: if constexpr ((M >> V) == 0) phase_group<V, M>(a, w); break;
    switch (mu) {
        TUSQ_G(1) TUSQ_G(2) TUSQ_G(3) TUSQ_G(4) TUSQ_G(5) TUSQ_G(6) TUSQ_G(7) TUSQ_G(8)
        TUSQ_G(9) TUSQ_G(10) TUSQ_G(11) TUSQ_G(12) TUSQ_G(13) TUSQ_G(14) TUSQ_G(15) TUSQ_G(16)
        TUSQ_G(17) TUSQ_G(18) TUSQ_G(19) TUSQ_G(20) TUSQ_G(21) TUSQ_G(22) TUSQ_G(23) TUSQ_G(24)
        TUSQ_G(25) TUSQ_G(26) TUSQ_G(27) TUSQ_G(28) TUSQ_G(29) TUSQ_G(30) TUSQ_G(31)
    default: break;
    }
#undef TUSQ_G
}

// Diagonal run on the 2^V registers of one thread.  gfix is the global
// index of the thread's register 0 (register bits cleared).  A term with
// register mask mu and fixed-bit parity p adds phi (p xor parity(r & mu))
// to register r's angle, i.e. p phi to a per-thread constant and
// (p ? -phi : phi) parity(r & mu) to the rest.  The terms of one mu are
// summed (exactly, in fixed-point turns) into C_mu, and the registers of odd
// parity against mu are multiplied by exp(2 pi i C_mu); only the non-empty
// groups (mu_mask) are visited.  The per-thread constant multiplies all of a
// thread's registers alike, so it commutes with every in-register op of the
// stage: it is added to `acc` and applied once when the stage ends.
template <typename R, int V>
__device__ __forceinline__ void apply_diag(typename C2T<R>::type (&a)[1 << V], const DevOp &op,
                                           const SProg<R> &P, uint64_t gfix, typename Phase<R>::U &acc) {
    using U = typename Phase<R>::U;
    U A = (U)op.phi0;
    const ulonglong2 *tm = reinterpret_cast<const ulonglong2 *>(P.terms) + (op.term_begin - P.term0);
    for (int k = op.csr[0]; k < op.csr[1]; ++k) {
        const ulonglong2 t = tm[k];
        if (__popcll(gfix & t.x) & 1) A += (U)t.y;
    }
    uint32_t mm = op.mu_mask;
    while (mm) {
        const int mu = __ffs(mm) - 1;
        mm &= mm - 1;
        U cm = 0;
        for (int k = op.csr[mu]; k < op.csr[mu + 1]; ++k) {
            const ulonglong2 t = tm[k];
            const U ph = (U)t.y;
            const bool c = __popcll(gfix & t.x) & 1;
            A += c ? ph : (U)0;
            cm += c ? (U)(0 - ph) : ph;
        }
        phase_group_dispatch<V>(a, mu, Phase<R>::unit(cm));
    }
    acc += A;
}

// Sign +-1 of the checksum weight of global index x (a 32-bit integer hash
// of x folded to 32 bits; C. Wellons' "lowbias32" mixer).
__device__ __forceinline__ float check_sign(uint64_t x) {
    uint32_t h = (uint32_t)x ^ ((uint32_t)(x >> 32) * 0x9E3779B9u);
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return (h >> 31) ? -1.0f : 1.0f;
}

// FP32 -> FP64 by bit manipulation on the integer pipes (the conversion
// instruction runs on B300's scarce FP64 units).  Exact for normal
// non-negative inputs; zero and subnormal inputs give 0.
__device__ __forceinline__ double f32_to_f64_nonneg(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const uint64_t bits = ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// Leaf update of one output element: acc += w p (p, w in FP32 for complex64).
__device__ __forceinline__ double leaf_add(double acc, float wp) { return acc + f32_to_f64_nonneg(wp); }

// Copy a pass's program (ops, matrix slots, diagonal terms) into shared
// memory at pbase; the caller synchronises before use.
template <typename R>
__device__ __forceinline__ SProg<R> load_program(const PassDesc &d, unsigned char *pbase, const DevOp *ops,
                                                 const double *mats, const float *matsf,
                                                 const uint64_t *tmask, const uint64_t *tphi, int tid,
                                                 int nthr) {
    using C2 = typename C2T<R>::type;
    constexpr bool kC128 = sizeof(R) == 8;
    DevOp *sops = reinterpret_cast<DevOp *>(pbase);
    C2 *smats = reinterpret_cast<C2 *>(pbase + (size_t)d.nops * sizeof(DevOp));
    uint64_t *sterms = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(smats) +
                                                    (size_t)d.nmat * 16 * sizeof(C2));
    const int4 *src = reinterpret_cast<const int4 *>(ops + d.op0);
    int4 *dst = reinterpret_cast<int4 *>(sops);
    for (uint32_t i = tid; i < d.nops * (uint32_t)(sizeof(DevOp) / 16); i += nthr) dst[i] = src[i];
    const int4 *msrc = kC128 ? reinterpret_cast<const int4 *>(mats + 32 * (size_t)d.mat0)
                             : reinterpret_cast<const int4 *>(matsf + 32 * (size_t)d.mat0);
    int4 *mdst = reinterpret_cast<int4 *>(smats);
    for (uint32_t i = tid; i < d.nmat * (uint32_t)(16 * sizeof(C2) / 16); i += nthr) mdst[i] = msrc[i];
    for (uint32_t i = tid; i < d.nterm; i += nthr) {
        sterms[2 * i] = tmask[d.term0 + i];
        sterms[2 * i + 1] = tphi[d.term0 + i];
    }
    return SProg<R>{sops, smats, sterms, d.op0, d.mat0, d.term0};
}

// The register stages of one pass on one tile in shared memory (tile bits
// tb); threads beyond 2^(L-V) only take part in the barriers.
template <typename R, int V, int TC = 0>
__device__ __forceinline__ void run_stages(typename C2T<R>::type *tile, const PassDesc &d, const SProg<R> &P,
                                           int tid, uint64_t tb, DenseCtx *dc = nullptr,
                                           const float *dpool = nullptr) {
    using C2 = typename C2T<R>::type;
    constexpr int NR = 1 << V;
    constexpr bool kC128 = sizeof(R) == 8;
    const int L = d.L;
    const bool active = tid < (1 << (L - V));
    for (int s = 0; s < d.n_stages; ++s) {
        const StageDesc &sd = d.st[s];
        if (active) {
            // thread bits -> the stage's non-register local bits: insert a zero
            // at each register bit (ascending)
            uint32_t e = (uint32_t)tid;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const uint32_t rb = sd.rbits[i];
                e = ((e >> rb) << (rb + 1)) | (e & ((1u << rb) - 1u));
            }
            const uint32_t sb = tile_swizzle(e, kC128);
            C2 a[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) a[r] = tile[sb ^ sd.sr[r]];
            bool have_gfix = false;
            uint64_t gfix = 0;
            typename Phase<R>::U acc = 0;     // the stage's per-thread constant phase
            for (uint32_t k = 0; k < sd.op_count; ++k) {
                const DevOp &op = P.ops[sd.op_begin - P.op0 + k];
                if (TC != 0 && op.code == CODE_DENSE) {
                    // tensor cores: the stage's thread-independent run as one 32x32
                    // matrix (every thread of the CTA takes part); its fixed-bit
                    // terms join the per-thread constant phase
                    if constexpr (TC != 0 && sizeof(R) == 4 && V == 5) {
                        if (op.csr[1] > op.csr[0] || op.phi0 != 0) {
                            if (!have_gfix) {
                                gfix = tb;
                                for (int i = 0; i < L - V; ++i)
                                    if (tid >> i & 1) gfix |= 1ull << sd.cglob[i];
                                have_gfix = true;
                            }
                            apply_diag<R, V>(a, op, P, gfix, acc);
                        }
                        // op.a: the pass's next dense op (cyclically, the next tile's
                        // first), whose B parts follow into the B region
                        const float *bnext = op.a != (int32_t)op.mat
                                                 ? dpool + (size_t)op.a * dense_b_words_dev(op.sub)
                                                 : nullptr;
                        unsigned char *stg = reinterpret_cast<unsigned char *>(tile);
                        const bool renorm = op.b != 0;    // U is unitary
                        dense_apply<TC>(a, stg, bnext, *dc, tid, renorm);   // op.sub == TC
                    }
                } else if (op.code != CODE_DIAG) {
                    apply_matrix_op<V, R>(a, op, P);
                } else {
                    if (!have_gfix) {
                        // global index of this thread's register 0
                        // global index of register 0: the tile bits and, for each
                        // thread bit set, its global position
                        gfix = tb;
                        for (int i = 0; i < L - V; ++i)
                            if (tid >> i & 1) gfix |= 1ull << sd.cglob[i];
                        have_gfix = true;
                    }
                    apply_diag<R, V>(a, op, P, gfix, acc);
                }
            }
            if (have_gfix || sd.kflag) {
                // the per-thread constant phase and/or the pass's scalar
                C2 u;
                if (have_gfix) {
                    u = Phase<R>::unit(acc);
                } else {
                    u.x = 1;
                    u.y = 0;
                }
                if (sd.kflag) {
                    C2 k;
                    k.x = (R)sd.kre;
                    k.y = (R)sd.kim;
                    u = cmul(u, k);
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) a[r] = cmul(a[r], u);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) tile[sb ^ sd.sr[r]] = a[r];
        }
        __syncthreads();
    }
}

// The tiles first, first + stride, ... of one pass for this CTA: load (from
// src), register stages, store and epilogue (state, snapshot, FP64 leaf
// accumulation, partial sums of the norm and checksum into partial_out[0..2]
// when the pass reduces).  The pass's program is in shared memory (P); the
// first statement of the tile loop waits for it.
template <typename R, int V, int TC>
__device__ __forceinline__ void pass_body(const PassDesc &d, const void *srcv, void *statev, void *snapv, double *acc,
                                          double *partial_out, const SProg<R> &P, unsigned char *smem_raw,
                                          uint64_t first, uint64_t stride, DenseCtx &dctx,
                                          const float *dpool = nullptr) {
    using C2 = typename C2T<R>::type;
    constexpr int NR = 1 << V;
    constexpr bool kC128 = sizeof(R) == 8;
    // complex64 threads move adjacent pairs in the load/store phases
    constexpr int NROW = kC128 ? NR : NR / 2;
    const int L = d.L;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    C2 *tile = reinterpret_cast<C2 *>(smem_raw);
    C2 *state = reinterpret_cast<C2 *>(statev);
    const C2 *srcp = reinterpret_cast<const C2 *>(srcv);   // tile loads (state or a snapshot)
    C2 *snap = reinterpret_cast<C2 *>(snapv);
    const uint32_t flags = d.flags;
    (void)nthr;

    // this thread's part of a load row (local index tid, or 2 tid for pairs)
    const uint32_t erow = kC128 ? (uint32_t)tid : (uint32_t)tid << 1;
    uint64_t gthr = 0;
    for (int b = 0; b < L; ++b)
        if (erow >> b & 1) gthr |= 1ull << d.win[b];
    const uint32_t sthr = tile_swizzle(erow, kC128);
    const float wleaf = (float)d.leaf_w;
    __syncthreads();


    double red_n = 0.0, red_r = 0.0, red_i = 0.0;

    // tile bits of this CTA's first tile and of the grid stride, deposited
    // into the tile-index positions; later tiles follow by a masked add
    // (carries skip the positions outside the mask)
    uint64_t tb = 0, tstride = 0;
    for (int b = 0; b < d.n_cw; ++b) {
        if (first >> b & 1) tb |= 1ull << d.cw[b];
        if (stride >> b & 1) tstride |= 1ull << d.cw[b];
    }
    for (uint64_t t = first; t < d.ntiles; t += stride, tb = ((tb | ~d.cwmask) + tstride) & d.cwmask) {
        const uint64_t gbase = tb | gthr;
        // load the tile: every row load in flight before the shared stores
        if constexpr (kC128) {
            C2 buf[NROW];
#pragma unroll
            for (int i = 0; i < NROW; ++i) buf[i] = srcp[gbase | d.grow[i]];
#pragma unroll
            for (int i = 0; i < NROW; ++i) tile[sthr ^ d.srow[i]] = buf[i];
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(srcp);
            float4 *dst = reinterpret_cast<float4 *>(tile);
            float4 buf[NROW];
#pragma unroll
            for (int i = 0; i < NROW; ++i) buf[i] = src[(gbase | d.grow[i]) >> 1];
#pragma unroll
            for (int i = 0; i < NROW; ++i) dst[(sthr ^ d.srow[i]) >> 1] = buf[i];
        }
        __syncthreads();
        run_stages<R, V, TC>(tile, d, P, tid, tb, TC != 0 ? &dctx : nullptr, dpool);
        if constexpr (TC != 0)
            if (*dctx.abort) break;      // a tensor-core wait ran out: stop (uniform after the stage barrier)
        // store + epilogue
        float pn = 0.f, pr = 0.f, pi = 0.f;
        double dn = 0.0, dr = 0.0, di = 0.0;
        if constexpr (kC128) {
#pragma unroll
            for (int i = 0; i < NROW; ++i) {
                const uint64_t g = gbase | d.grow[i];
                C2 v = tile[sthr ^ d.srow[i]];
                if (flags & PF_WRITE) state[g] = v;
                if (flags & PF_SNAPSHOT) snap[g] = v;
                if (flags & PF_LEAF) acc[g] = fma(d.leaf_w, v.x * v.x + v.y * v.y, acc[g]);
                if (flags & PF_REDUCE) {
                    const double h = check_sign(g);
                    dn += v.x * v.x + v.y * v.y;
                    dr += h * v.x;
                    di += h * v.y;
                }
            }
        } else {
            const float4 *ts = reinterpret_cast<const float4 *>(tile);
            if (flags & PF_LEAF) {
                // every accumulator load in flight before the updates
                double2 *accp = reinterpret_cast<double2 *>(acc);
                double2 ab[NROW];
#pragma unroll
                for (int i = 0; i < NROW; ++i) ab[i] = accp[(gbase | d.grow[i]) >> 1];
#pragma unroll
                for (int i = 0; i < NROW; ++i) {
                    const float4 v = ts[(sthr ^ d.srow[i]) >> 1];
                    ab[i].x = leaf_add(ab[i].x, wleaf * fmaf(v.x, v.x, v.y * v.y));
                    ab[i].y = leaf_add(ab[i].y, wleaf * fmaf(v.z, v.z, v.w * v.w));
                    accp[(gbase | d.grow[i]) >> 1] = ab[i];
                }
            }
            if (flags & (PF_WRITE | PF_SNAPSHOT | PF_REDUCE)) {
#pragma unroll
                for (int i = 0; i < NROW; ++i) {
                    const uint64_t g = gbase | d.grow[i];
                    const float4 v = ts[(sthr ^ d.srow[i]) >> 1];
                    if (flags & PF_WRITE) reinterpret_cast<float4 *>(state)[g >> 1] = v;
                    if (flags & PF_SNAPSHOT) reinterpret_cast<float4 *>(snap)[g >> 1] = v;
                    if (flags & PF_REDUCE) {
                        const float h0 = check_sign(g), h1 = check_sign(g | 1);
                        pn = fmaf(v.x, v.x, fmaf(v.y, v.y, pn));
                        pn = fmaf(v.z, v.z, fmaf(v.w, v.w, pn));
                        pr = fmaf(h0, v.x, fmaf(h1, v.z, pr));
                        pi = fmaf(h0, v.y, fmaf(h1, v.w, pi));
                    }
                }
            }
        }
        if (flags & PF_REDUCE) {
            red_n += (double)pn + dn;
            red_r += (double)pr + dr;
            red_i += (double)pi + di;
        }
        __syncthreads();
    }
    if (flags & PF_REDUCE) {
        // fixed-order block reduction: warp shuffles, then thread 0
        __shared__ double wsum[3][32];
        for (int off = 16; off > 0; off >>= 1) {
            red_n += __shfl_down_sync(0xffffffffu, red_n, off);
            red_r += __shfl_down_sync(0xffffffffu, red_r, off);
            red_i += __shfl_down_sync(0xffffffffu, red_i, off);
        }
        const int warp = tid >> 5, lane = tid & 31, nw = (nthr + 31) >> 5;
        if (lane == 0) { wsum[0][warp] = red_n; wsum[1][warp] = red_r; wsum[2][warp] = red_i; }
        __syncthreads();
        if (tid == 0) {
            double a0 = 0, a1 = 0, a2 = 0;
            for (int w = 0; w < nw; ++w) { a0 += wsum[0][w]; a1 += wsum[1][w]; a2 += wsum[2][w]; }
            partial_out[0] = a0;
            partial_out[1] = a1;
            partial_out[2] = a2;
        }
    }
}

// The B region is the top of a dense pass's program area (at pbase): the
// pass's first dense op's B parts are copied there before its first tile,
// each later op's by the one before (global reads of the pass's ops, so the
// copy may start before the program is in shared memory).
__device__ __forceinline__ void dense_pass_prefetch(const PassDesc &d, const DevOp *ops, const float *dpool,
                                                    unsigned char *pbase, DenseCtx &dc, int tid, int nthr) {
    for (uint32_t k = 0; k < d.nops; ++k) {
        const DevOp &op = ops[d.op0 + k];
        if (op.code != CODE_DENSE) continue;
        const uint32_t words = dense_b_words_dev(op.sub);
        dc.bsm = smem_u32(pbase + d.prog_bytes - 4u * words);
        dense_copy_b(dc.bsm, dpool + (size_t)op.mat * words, 4u * words, tid, nthr);
        break;
    }
}

// TC: the tc mode of the instantiation for passes with tensor-core dense ops
// (complex64, V = 5; one per mode); TC = 0 carries none of that code.
template <typename R, int V, int TC = 0>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) pass_kernel(const __grid_constant__ PassArgs args) {
    using C2 = typename C2T<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PassDesc &d = args.d;
    const int tid = threadIdx.x;
    // the pass's program into shared memory (ops, matrices, diagonal terms)
    const SProg<R> P = load_program<R>(d, smem_raw + (sizeof(C2) << d.L), args.ops, args.mats, args.matsf,
                                       args.tmask, args.tphi, tid, blockDim.x);
    // tensor-core dense ops: 128 TMEM columns and a completion mbarrier
    DenseCtx dctx{0u, 0u, 0u, args.err, nullptr, args.dense_skip};
    if constexpr (TC != 0) {
        __shared__ uint32_t s_tmem;
        __shared__ __align__(8) uint64_t s_mbar;
        __shared__ int s_abort;
        // once a tensor-core wait of this traversal has run out, its later
        // dense passes do nothing (the result is void and reported as a timeout)
        if (*args.err) return;
        if (tid == 0) s_abort = 0;
        dense_pass_prefetch(d, args.ops, args.dpool, smem_raw + (sizeof(C2) << d.L), dctx, tid, blockDim.x);
        dense_setup(&s_tmem, &s_mbar, tid);
        dctx.tmem = s_tmem;
        dctx.mbar = smem_u32(&s_mbar);
        dctx.abort = &s_abort;
    }

    pass_body<R, V, TC>(d, args.src, args.state, args.snap, args.acc, args.partials + 3 * blockIdx.x, P,
                           smem_raw, blockIdx.x, gridDim.x, dctx, args.dpool);
    if constexpr (TC != 0) dense_teardown(dctx.tmem, tid);
}

// state <- |0..0>
template <typename C2>
__global__ void init_kernel(C2 *state, uint64_t dim) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        C2 z;
        z.x = (i == 0) ? 1 : 0;
        z.y = 0;
        state[i] = z;
    }
}

// Per-check record: norm2, cs_re, cs_im.  A record stores the sums at a
// branch node on the way down; a check recomputes them after the
// uncompute and stores max(|sqrt(n2) - sqrt(n2_ref)|, |cs - cs_ref|).
__global__ void finalize_kernel(const double *partials, int nparts, double *records, int depth,
                                int is_check, double *drift_log, int check, int *restore_flag,
                                int has_snapshot, double tol, unsigned long long *counters,
                                double record_bias) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double n2 = 0, cr = 0, ci = 0;
    for (int b = 0; b < nparts; ++b) {
        n2 += partials[3 * b];
        cr += partials[3 * b + 1];
        ci += partials[3 * b + 2];
    }
    double *rec = records + 4 * depth;
    if (!is_check) {
        rec[0] = n2 + record_bias;
        rec[1] = cr;
        rec[2] = ci;
        return;
    }
    double dn = fabs(sqrt(n2) - sqrt(fmax(rec[0], 0.0)));
    double dc = hypot(cr - rec[1], ci - rec[2]);
    double drift = fmax(dn, dc);
    drift_log[check] = drift;
    int bad = drift > tol;
    restore_flag[check] = bad && has_snapshot;
    if (bad) {
        if (has_snapshot) atomicAdd(counters + 0, 1ull);
        else atomicAdd(counters + 1, 1ull);
    }
}

// state <- snapshot; when check >= 0 only if that check flagged drift.
template <typename C2>
__global__ void restore_kernel(C2 *state, const C2 *snap, uint64_t dim, const int *restore_flag,
                               int check) {
    if (check >= 0 && !restore_flag[check]) return;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x)
        state[i] = snap[i];
}

// ------------------------------------------------------------ host launchers

// Allow the dynamic shared memory a pass tile needs (above the 48 KB
// default); returns the attribute call's own status.
template <typename R, int V, int TC = 0>
static cudaError_t allow_smem(size_t smem) {
    static size_t allowed = 48 * 1024;
    if (smem <= allowed) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(pass_kernel<R, V, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) allowed = smem;
    return e;
}

template <typename R, int V, int TC = 0>
static cudaError_t launch_pass_t(const PassArgs &a, int grid, cudaStream_t st) {
    const size_t smem = ((sizeof(R) * 2) << a.d.L) + a.d.prog_bytes;
    const int threads = 1 << (a.d.L - V);
    cudaError_t e = allow_smem<R, V, TC>(smem);
    if (e != cudaSuccess) return e;
    pass_kernel<R, V, TC><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R, int V, int TC = 0>
static int occupancy_t(int L, uint32_t prog_cap) {
    const size_t smem = ((sizeof(R) * 2) << L) + prog_cap;
    const int threads = 1 << (L - V);
    int nb = 0;
    if (allow_smem<R, V, TC>(smem) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_kernel<R, V, TC>, threads, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_pass(const PassArgs &a, int precision, int V, int grid, cudaStream_t st) {
    if (precision == TUSQ_C128) {
        switch (V) {
        case 1: return launch_pass_t<double, 1>(a, grid, st);
        case 2: return launch_pass_t<double, 2>(a, grid, st);
        case 3: return launch_pass_t<double, 3>(a, grid, st);
        default: return launch_pass_t<double, 4>(a, grid, st);
        }
    }
    switch (V) {
    case 1: return launch_pass_t<float, 1>(a, grid, st);
    case 2: return launch_pass_t<float, 2>(a, grid, st);
    case 3: return launch_pass_t<float, 3>(a, grid, st);
    case 4: return launch_pass_t<float, 4>(a, grid, st);
    default:
        switch (pass_dense_mode(a.d.flags)) {
        case TUSQ_TC_TF32X3: return launch_pass_t<float, 5, TUSQ_TC_TF32X3>(a, grid, st);
        case TUSQ_TC_BF16X3: return launch_pass_t<float, 5, TUSQ_TC_BF16X3>(a, grid, st);
        case TUSQ_TC_TF32: return launch_pass_t<float, 5, TUSQ_TC_TF32>(a, grid, st);
        default: return launch_pass_t<float, 5>(a, grid, st);
        }
    }
}

// Resident CTAs per SM for a pass configuration (for grid sizing); tc: the
// tc mode of the pass's tensor-core dense ops (0: none).
int pass_occupancy(int precision, int V, int L, int tc) {
    const uint32_t cap = kMaxPassProgramBytes;
    if (precision == TUSQ_C128) {
        switch (V) {
        case 1: return occupancy_t<double, 1>(L, cap);
        case 2: return occupancy_t<double, 2>(L, cap);
        case 3: return occupancy_t<double, 3>(L, cap);
        default: return occupancy_t<double, 4>(L, cap);
        }
    }
    switch (V) {
    case 1: return occupancy_t<float, 1>(L, cap);
    case 2: return occupancy_t<float, 2>(L, cap);
    case 3: return occupancy_t<float, 3>(L, cap);
    case 4: return occupancy_t<float, 4>(L, cap);
    default:
        switch (tc) {
        case TUSQ_TC_TF32X3: return occupancy_t<float, 5, TUSQ_TC_TF32X3>(L, cap);
        case TUSQ_TC_BF16X3: return occupancy_t<float, 5, TUSQ_TC_BF16X3>(L, cap);
        case TUSQ_TC_TF32: return occupancy_t<float, 5, TUSQ_TC_TF32>(L, cap);
        default: return occupancy_t<float, 5>(L, cap);
        }
    }
}

cudaError_t launch_init(void *state, int precision, uint64_t dim, int nsm, cudaStream_t st) {
    int grid = (int)((dim + 255) / 256);
    if (grid > nsm * 8) grid = nsm * 8;
    if (precision == TUSQ_C128) init_kernel<double2><<<grid, 256, 0, st>>>((double2 *)state, dim);
    else init_kernel<float2><<<grid, 256, 0, st>>>((float2 *)state, dim);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int nparts, double *records, int depth,
                            int is_check, double *drift_log, int check, int *restore_flag,
                            int has_snapshot, double tol, unsigned long long *counters,
                            double record_bias, cudaStream_t st) {
    finalize_kernel<<<1, 32, 0, st>>>(partials, nparts, records, depth, is_check, drift_log, check,
                                      restore_flag, has_snapshot, tol, counters, record_bias);
    return cudaGetLastError();
}

cudaError_t launch_restore(void *state, const void *snap, int precision, uint64_t dim,
                           const int *restore_flag, int check, int nsm, cudaStream_t st) {
    int grid = (int)((dim + 255) / 256);
    if (grid > nsm * 8) grid = nsm * 8;
    if (precision == TUSQ_C128)
        restore_kernel<double2><<<grid, 256, 0, st>>>((double2 *)state, (const double2 *)snap, dim,
                                                      restore_flag, check);
    else
        restore_kernel<float2><<<grid, 256, 0, st>>>((float2 *)state, (const float2 *)snap, dim,
                                                     restore_flag, check);
    return cudaGetLastError();
}

// ------------------------------------------------------------ batched jobs

// Largest job a CTA holds in shared memory: 2^13 complex64 or 2^12
// complex128 amplitudes (64 KiB).
template <typename R> constexpr int job_max_qubits() { return sizeof(R) == 4 ? 13 : 12; }

// Barrier of the k CTAs running one group job: every member adds one to the
// job's counter and waits until it reaches `target` (k times the barriers
// passed so far).  The wait is bounded (about 1 s of SM clock, or until
// another group gave up): it then sets the batch's error word and abort
// flag and returns false.
__device__ __forceinline__ bool group_barrier(const BatchArgs &B, unsigned int *bar, unsigned int target,
                                              int tid) {
    __shared__ int s_ok;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const long long t0 = clock64();
        int ok = 1;
        for (;;) {
            unsigned int v, ab;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(ab) : "l"(B.abort) : "memory");
            if (ab) { ok = 0; break; }
            if (clock64() - t0 > (2ll << 30)) {
                atomicOr(B.err, 1u);
                atomicExch(B.abort, 1u);
                ok = 0;
                break;
            }
            __nanosleep(128);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Member `rank` of the k-CTA group running job j: its share of every step --
// amplitudes rank*T + tid (+ k*T ...) of resets and restores, tiles rank,
// rank + k, ... of every pass (state and snapshots in global memory) -- with
// a group barrier after each step that writes the state.  Records and drift
// checks read the members' partial sums after the pass barrier; every member
// takes the same restore decision, only rank 0 writes records and counters.
// Returns false when a barrier gave up or a tensor-core wait ran out (TC: the
// tc mode of the job's dense ops, dc the CTA's tensor-core context).
template <typename R, int V, int TC>
__device__ bool run_group_job(const BatchArgs &B, int j, int rank, unsigned char *smem_raw, unsigned char *pbase,
                              DenseCtx &dc) {
    using C2 = typename C2T<R>::type;
    __shared__ int s_restore;
    const JobDesc &J = B.jobs[j];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int k = J.group_k;
    const uint64_t dim = 1ull << J.n;
    const uint64_t first = (uint64_t)rank * nthr + tid, step = (uint64_t)k * nthr;
    C2 *state = reinterpret_cast<C2 *>(J.state);
    const C2 *snaps = reinterpret_cast<const C2 *>(J.snaps);
    unsigned int nb = 0;
    const unsigned int width = (unsigned int)(k + (B.stall_test ? 1 : 0));
    for (uint64_t e = first; e < dim; e += step) J.acc[e] = 0.0;
    for (uint32_t s = 0; s < J.nsteps; ++s) {
        const Step &st = B.steps[J.step0 + s];
        if (st.type == ST_INIT) {
            for (uint64_t e = first; e < dim; e += step) {
                C2 z;
                z.x = (e == 0) ? 1 : 0;
                z.y = 0;
                state[e] = z;
            }
            if (!group_barrier(B, J.bar, width * ++nb, tid)) return false;
        } else if (st.type == ST_PASS) {
            const PassDesc &d = B.passes[st.pass];
            const SProg<R> P = load_program<R>(d, pbase, B.ops, B.mats, B.matsf, B.tmask, B.tphi, tid, nthr);
            if constexpr (TC != 0)
                if (d.flags & PF_DENSE) dense_pass_prefetch(d, B.ops, B.dpool, pbase, dc, tid, nthr);
            const void *src = d.src_snap >= 0 ? (const void *)(snaps + dim * d.src_snap) : (const void *)state;
            void *snap = (d.flags & PF_SNAPSHOT) ? (void *)(snaps + dim * d.snap) : nullptr;
            pass_body<R, V, TC>(d, src, state, snap, J.acc, J.partials + 3 * rank, P, smem_raw, (uint64_t)rank,
                                (uint64_t)k, dc, B.dpool);
            if constexpr (TC != 0) {
                // the next pass's program overwrites the B region: the copies
                // in flight (a prefetch for a next tile) land first
                asm volatile("cp.async.wait_all;" ::: "memory");
                if (*dc.abort) {      // uniform: set before a barrier inside the pass
                    if (tid == 0) atomicExch(B.abort, 1u);
                    return false;
                }
            }
            if (!group_barrier(B, J.bar, width * ++nb, tid)) return false;
        } else if (st.type == ST_RECORD || st.type == ST_CHECK) {
            if (tid == 0) {
                double n2 = 0, cr = 0, ci = 0;
                for (int m = 0; m < k; ++m) {
                    n2 += J.partials[3 * m];
                    cr += J.partials[3 * m + 1];
                    ci += J.partials[3 * m + 2];
                }
                double *rec = J.records + 4 * st.depth;
                if (st.type == ST_RECORD) {
                    if (rank == 0) {
                        rec[0] = n2;
                        rec[1] = cr;
                        rec[2] = ci;
                    }
                } else {
                    const double dn = fabs(sqrt(n2) - sqrt(fmax(rec[0], 0.0)));
                    const double dc = hypot(cr - rec[1], ci - rec[2]);
                    const double drift = fmax(dn, dc);
                    const bool bad = drift > B.drift_tol;
                    s_restore = bad && st.snap >= 0;
                    if (rank == 0) {
                        if (bad) atomicAdd(B.counters + (st.snap >= 0 ? 0 : 1), 1ull);
                        atomicMax(B.counters + 2, (unsigned long long)__double_as_longlong(drift));
                    }
                }
            }
            __syncthreads();
        } else if (st.type == ST_RESTORE) {
            if (st.check < 0 || s_restore) {
                const C2 *sn = snaps + dim * st.snap;
                for (uint64_t e = first; e < dim; e += step) state[e] = sn[e];
            }
            if (!group_barrier(B, J.bar, width * ++nb, tid)) return false;
        }
    }
    return true;
}

// job_body: one CTA's part of a batch launch.  First the CTA runs its
// share of the group jobs (more amplitudes than one CTA's shared memory
// holds) in the order the host assigned; then it takes single-CTA jobs from
// a work queue and runs each job's whole program -- resets, fused passes
// (register stages on the state held in shared memory), leaf accumulation
// into the job's FP64 output, snapshot writes and restores, drift records
// and checks -- without leaving the CTA.  Jobs of uneven size and depth
// share one launch.  TC: the tc mode of the batch's tensor-core dense ops
// (complex64 13-qubit tiles: 13-qubit single-CTA jobs and group jobs); each
// CTA of such a launch holds 128 TMEM columns from start to end.
template <typename R, int V, int TC>
__device__ __forceinline__ void job_body(const BatchArgs &B, DenseCtx &dctx) {
    using C2 = typename C2T<R>::type;
    constexpr bool kC128 = sizeof(R) == 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *tile = reinterpret_cast<C2 *>(smem_raw);
    unsigned char *pbase = smem_raw + (sizeof(C2) << job_max_qubits<R>());
    __shared__ int s_job;
    __shared__ int s_restore;
    __shared__ double s_red[3];
    __shared__ double s_wsum[3][8];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (uint32_t a = B.assign_off[blockIdx.x]; a < B.assign_off[blockIdx.x + 1]; ++a)
        if (!run_group_job<R, V, TC>(B, (int)B.assign[a].job, (int)B.assign[a].rank, smem_raw, pbase, dctx)) return;
    for (;;) {
        if (tid == 0) s_job = (int)atomicAdd(B.next_job, 1u);
        __syncthreads();
        const int q = s_job;
        __syncthreads();
        if (q >= B.n_small) break;
        const int j = (int)B.small_ids[q];
        const JobDesc &J = B.jobs[j];
        const int N = 1 << J.n;
        for (int e = tid; e < N; e += nthr) J.acc[e] = 0.0;
        for (uint32_t k = 0; k < J.nsteps; ++k) {
            const Step &st = B.steps[J.step0 + k];
            if (st.type == ST_INIT) {
                for (int e = tid; e < N; e += nthr) {
                    C2 z;
                    z.x = (e == 0) ? 1 : 0;
                    z.y = 0;
                    tile[tile_swizzle((uint32_t)e, kC128)] = z;
                }
                __syncthreads();
            } else if (st.type == ST_PASS) {
                const PassDesc &d = B.passes[st.pass];
                const SProg<R> P = load_program<R>(d, pbase, B.ops, B.mats, B.matsf, B.tmask, B.tphi, tid, nthr);
                if constexpr (TC != 0)
                    if (d.flags & PF_DENSE) dense_pass_prefetch(d, B.ops, B.dpool, pbase, dctx, tid, nthr);
                __syncthreads();
                run_stages<R, V, TC>(tile, d, P, tid, 0, TC != 0 ? &dctx : nullptr, B.dpool);
                if constexpr (TC != 0) {
                    // the next pass's program overwrites the B region
                    asm volatile("cp.async.wait_all;" ::: "memory");
                    if (*dctx.abort) {    // uniform: set before the last stage barrier
                        if (tid == 0) atomicExch(B.abort, 1u);
                        return;
                    }
                }
                const uint32_t flags = d.flags;
                double rn = 0, rr = 0, ri = 0;
                C2 *sn = (flags & PF_SNAPSHOT) ? reinterpret_cast<C2 *>(J.snaps) + (size_t)d.snap * N : nullptr;
                for (int e = tid; e < N; e += nthr) {
                    const C2 v = tile[tile_swizzle((uint32_t)e, kC128)];
                    if (flags & PF_SNAPSHOT) sn[e] = v;
                    if (flags & PF_LEAF) {
                        if constexpr (kC128) J.acc[e] = fma(d.leaf_w, v.x * v.x + v.y * v.y, J.acc[e]);
                        else J.acc[e] = leaf_add(J.acc[e], (float)d.leaf_w * fmaf(v.x, v.x, v.y * v.y));
                    }
                    if (flags & PF_REDUCE) {
                        const double h = check_sign((uint64_t)e);
                        rn += (double)v.x * v.x + (double)v.y * v.y;
                        rr += h * v.x;
                        ri += h * v.y;
                    }
                }
                if (flags & PF_REDUCE) {
                    for (int off = 16; off > 0; off >>= 1) {
                        rn += __shfl_down_sync(0xffffffffu, rn, off);
                        rr += __shfl_down_sync(0xffffffffu, rr, off);
                        ri += __shfl_down_sync(0xffffffffu, ri, off);
                    }
                    if ((tid & 31) == 0) {
                        s_wsum[0][tid >> 5] = rn;
                        s_wsum[1][tid >> 5] = rr;
                        s_wsum[2][tid >> 5] = ri;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        double a0 = 0, a1 = 0, a2 = 0;
                        for (int w = 0; w < (nthr + 31) / 32; ++w) {
                            a0 += s_wsum[0][w];
                            a1 += s_wsum[1][w];
                            a2 += s_wsum[2][w];
                        }
                        s_red[0] = a0;
                        s_red[1] = a1;
                        s_red[2] = a2;
                    }
                }
                __syncthreads();
            } else if (st.type == ST_RECORD) {
                if (tid == 0) {
                    J.records[4 * st.depth + 0] = s_red[0];
                    J.records[4 * st.depth + 1] = s_red[1];
                    J.records[4 * st.depth + 2] = s_red[2];
                }
                __syncthreads();
            } else if (st.type == ST_CHECK) {
                if (tid == 0) {
                    const double *rec = J.records + 4 * st.depth;
                    const double dn = fabs(sqrt(s_red[0]) - sqrt(fmax(rec[0], 0.0)));
                    const double dc = hypot(s_red[1] - rec[1], s_red[2] - rec[2]);
                    const double drift = fmax(dn, dc);
                    const bool bad = drift > B.drift_tol;
                    s_restore = bad && st.snap >= 0;
                    if (bad) atomicAdd(B.counters + (st.snap >= 0 ? 0 : 1), 1ull);
                    // running maximum of the drift (non-negative doubles order like their bits)
                    atomicMax(B.counters + 2, (unsigned long long)__double_as_longlong(drift));
                }
                __syncthreads();
            } else if (st.type == ST_RESTORE) {
                if (st.check < 0 || s_restore) {
                    const C2 *sn = reinterpret_cast<const C2 *>(J.snaps) + (size_t)st.snap * N;
                    for (int e = tid; e < N; e += nthr) tile[tile_swizzle((uint32_t)e, kC128)] = sn[e];
                }
                __syncthreads();
            }
        }
    }
}

// The persistent launch of a batch: job_body, with (TC) the CTA's 128 TMEM
// columns allocated before it and freed after it, whichever way it ends.
template <typename R, int V, int TC = 0>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) job_kernel(const __grid_constant__ BatchArgs B) {
    DenseCtx dctx{0u, 0u, 0u, B.err, nullptr, 0};
    if constexpr (TC != 0) {
        __shared__ uint32_t s_tmem;
        __shared__ __align__(8) uint64_t s_mbar;
        __shared__ int s_abort;
        if (threadIdx.x == 0) s_abort = 0;
        dense_setup(&s_tmem, &s_mbar, threadIdx.x);
        dctx.tmem = s_tmem;
        dctx.mbar = smem_u32(&s_mbar);
        dctx.abort = &s_abort;
    }
    job_body<R, V, TC>(B, dctx);
    if constexpr (TC != 0) dense_teardown(dctx.tmem, threadIdx.x);
}

template <typename R, int V, int TC = 0>
static cudaError_t launch_job_t(const BatchArgs &b, int grid, bool cooperative, cudaStream_t st) {
    const size_t smem = (sizeof(R) * 2 << job_max_qubits<R>()) + kMaxPassProgramBytes;
    cudaError_t e = cudaFuncSetAttribute(job_kernel<R, V, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // group jobs wait at barriers for CTAs of the same launch: the
    // cooperative attribute guarantees that the whole grid is resident
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = cooperative ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, job_kernel<R, V, TC>, b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// One launch over every job of a batch; `grid` CTAs drain the work queue.
// tc: the tc mode of the batch's dense ops (complex64), 0 for none.
cudaError_t launch_jobs(const BatchArgs &b, int precision, int tc, int grid, bool cooperative, cudaStream_t st) {
    if (precision == TUSQ_C128) return launch_job_t<double, kRegBitsC128>(b, grid, cooperative, st);
    switch (tc) {
    case TUSQ_TC_TF32X3: return launch_job_t<float, kRegBitsC64, TUSQ_TC_TF32X3>(b, grid, cooperative, st);
    case TUSQ_TC_BF16X3: return launch_job_t<float, kRegBitsC64, TUSQ_TC_BF16X3>(b, grid, cooperative, st);
    case TUSQ_TC_TF32: return launch_job_t<float, kRegBitsC64, TUSQ_TC_TF32>(b, grid, cooperative, st);
    default: return launch_job_t<float, kRegBitsC64>(b, grid, cooperative, st);
    }
}

int job_max_qubits_of(int precision) {
    return precision == TUSQ_C128 ? job_max_qubits<double>() : job_max_qubits<float>();
}

// Resident job CTAs per SM (tc: the instantiation of that tc mode).
template <typename R, int V, int TC = 0>
static int job_occupancy_t() {
    const size_t smem = (sizeof(R) * 2 << job_max_qubits<R>()) + kMaxPassProgramBytes;
    int nb = 0;
    if (cudaFuncSetAttribute(job_kernel<R, V, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, job_kernel<R, V, TC>, 256, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

int job_occupancy(int precision, int tc) {
    if (precision == TUSQ_C128) return job_occupancy_t<double, kRegBitsC128>();
    switch (tc) {
    case TUSQ_TC_TF32X3: return job_occupancy_t<float, kRegBitsC64, TUSQ_TC_TF32X3>();
    case TUSQ_TC_BF16X3: return job_occupancy_t<float, kRegBitsC64, TUSQ_TC_BF16X3>();
    case TUSQ_TC_TF32: return job_occupancy_t<float, kRegBitsC64, TUSQ_TC_TF32>();
    default: return job_occupancy_t<float, kRegBitsC64>();
    }
}

}  // namespace tusq
