// Blackwell tensor-core primitives (sm_100 family, here sm_103a) as inline
// PTX: TMEM allocation, tcgen05.mma issue and commit, mbarrier waits with an
// iteration bound, TMEM -> register loads, and shared-memory descriptors.
//
// Operand tiles live in shared memory in the K-major, no-swizzle canonical
// layout: 8-row x 16-byte core matrices; core matrices adjacent along K are
// LBO bytes apart, 8-row groups SBO bytes apart.  A 16-bit element (row, k)
// sits at (row/8)*SBO + (k/8)*LBO + (row%8)*16 + (k%8)*2; a 32-bit element at
// (row/8)*SBO + (k/4)*LBO + (row%8)*16 + (k%4)*4.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace occk {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- TMEM ------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst_smem)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- mbarrier --------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`, giving up after `limit` polls.  Returns
// false on timeout (the caller records an error and leaves cleanly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

// ---- MMA ---------------------------------------------------------------------
// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, cta_group::1.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
// Arrive on `bar` once every previously issued tcgen05.mma of this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

// ---- TMEM -> registers: 32 lanes (one warp's quarter) x 16 columns of 32 bit
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// ---- descriptors ---------------------------------------------------------------
// Shared-memory matrix descriptor, SWIZZLE_NONE, sm_100 version bit (46) set.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D = F32, A/B format (0 F16, 1 BF16, 2 TF32), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- operand formats of the mixed-precision forms ---------------------------------
// BF16 / FP16 / TF32: one product per K step.  BF16X3 / FP16X3: each FP32
// value x is split as hi = rn(x), lo = rn(x - hi) and the product is
// hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-2p of the product, is dropped).
// For FP16 the lo part is stored times 2^11 so that it stays a normal number;
// the cross terms then go to a second accumulator that is scaled back by 2^-11.
enum { Q_BF16 = 0, Q_FP16 = 1, Q_TF32 = 2, Q_BF16X3 = 3, Q_FP16X3 = 4 };
constexpr float kLo = 2048.f;

template <int P>
struct Fmt {
    static constexpr bool split = (P == Q_BF16X3 || P == Q_FP16X3);
    static constexpr bool dual = (P == Q_FP16X3);
    static constexpr int esz = (P == Q_TF32) ? 4 : 2;
    static constexpr int KSTEP = (P == Q_TF32) ? 8 : 16;   // K of one tcgen05.mma
    static constexpr uint32_t fmt = (P == Q_BF16 || P == Q_BF16X3) ? 1u : (P == Q_TF32 ? 2u : 0u);
};

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Convert 8 consecutive K values of one operand row into the format of P and
// store them at `dst` (16-bit formats: one 16-byte chunk, i.e. one core-matrix
// row; TF32: two chunks, the second `lbo` bytes further along K).  For the
// split formats the lo part goes to dst + part_bytes.
template <int P>
__device__ __forceinline__ void put8(uint8_t* dst, uint32_t part_bytes, uint32_t lbo, const float* v) {
    if constexpr (P == Q_TF32) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 q;
            q.x = tf32_bits(v[4 * h + 0]);
            q.y = tf32_bits(v[4 * h + 1]);
            q.z = tf32_bits(v[4 * h + 2]);
            q.w = tf32_bits(v[4 * h + 3]);
            *reinterpret_cast<uint4*>(dst + h * lbo) = q;
        }
    } else if constexpr (P == Q_BF16 || P == Q_BF16X3) {
        __nv_bfloat162 h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            if constexpr (Fmt<P>::split) {
                const float2 f = __bfloat1622float2(h[q]);
                l[q] = __floats2bfloat162_rn(v[2 * q] - f.x, v[2 * q + 1] - f.y);
            }
        }
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(h);
        if constexpr (Fmt<P>::split) *reinterpret_cast<uint4*>(dst + part_bytes) = *reinterpret_cast<uint4*>(l);
    } else {
        __half2 h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
            if constexpr (Fmt<P>::split) {
                const float2 f = __half22float2(h[q]);
                l[q] = __floats2half2_rn((v[2 * q] - f.x) * kLo, (v[2 * q + 1] - f.y) * kLo);
            }
        }
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(h);
        if constexpr (Fmt<P>::split) *reinterpret_cast<uint4*>(dst + part_bytes) = *reinterpret_cast<uint4*>(l);
    }
}

// Inverse of put8: the 8 FP32 values (hi + lo, lo scaled back for FP16) of
// one operand row chunk stored by put8<P> at `src`.
template <int P>
__device__ __forceinline__ void get8(const uint8_t* src, uint32_t part_bytes, uint32_t lbo, float* v) {
    if constexpr (P == Q_TF32) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 q = *reinterpret_cast<const uint4*>(src + h * lbo);
            v[4 * h + 0] = __uint_as_float(q.x);
            v[4 * h + 1] = __uint_as_float(q.y);
            v[4 * h + 2] = __uint_as_float(q.z);
            v[4 * h + 3] = __uint_as_float(q.w);
        }
    } else if constexpr (P == Q_BF16 || P == Q_BF16X3) {
        const uint4 qh = *reinterpret_cast<const uint4*>(src);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&qh);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            v[2 * q] = f.x;
            v[2 * q + 1] = f.y;
        }
        if constexpr (Fmt<P>::split) {
            const uint4 ql = *reinterpret_cast<const uint4*>(src + part_bytes);
            const __nv_bfloat162* l = reinterpret_cast<const __nv_bfloat162*>(&ql);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(l[q]);
                v[2 * q] += f.x;
                v[2 * q + 1] += f.y;
            }
        }
    } else {
        const uint4 qh = *reinterpret_cast<const uint4*>(src);
        const __half2* h = reinterpret_cast<const __half2*>(&qh);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __half22float2(h[q]);
            v[2 * q] = f.x;
            v[2 * q + 1] = f.y;
        }
        if constexpr (Fmt<P>::split) {
            const uint4 ql = *reinterpret_cast<const uint4*>(src + part_bytes);
            const __half2* l = reinterpret_cast<const __half2*>(&ql);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __half22float2(l[q]);
                v[2 * q] += f.x * (1.f / kLo);
                v[2 * q + 1] += f.y * (1.f / kLo);
            }
        }
    }
}

// ---- splitting FP32 into low-precision hi/lo parts --------------------------------
struct SplitBF16 {
    using T = __nv_bfloat16;
    static constexpr uint32_t fmt = 1;
    __device__ static void split(float x, T& hi, T& lo) {
        hi = __float2bfloat16_rn(x);
        lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
};
struct SplitFP16 {
    using T = __half;
    static constexpr uint32_t fmt = 0;
    __device__ static void split(float x, T& hi, T& lo) {
        hi = __float2half_rn(x);
        lo = __float2half_rn(x - __half2float(hi));
    }
};

}  // namespace tc
}  // namespace occk
