// Steps (a) and (e) of the mixed-precision forms on a pipelined tcgen05 GEMM.
//
// Operands are first converted, in one memory-bound pass each, into "panels"
// in global memory: 128 rows x 128 bytes of K (64 BF16/FP16 or 32 TF32
// elements), already in the K-major no-swizzle canonical layout of the tensor
// core, hi part followed by lo part for the split forms.  The GEMM then moves
// whole panels into a ring of shared-memory stages with bulk asynchronous
// copies (cp.async.bulk, completion counted on an mbarrier), so no thread
// touches operand bytes.  Warp roles per CTA (192 threads):
//   warp 0      producer: one lane issues the bulk copies of each stage
//   warp 1      MMA: one lane issues tcgen05.mma for each stage
//   warps 2..5  flush: add each stage's TMEM accumulator into FP32 registers
//               (two TMEM buffers alternate, so every accumulation chain is one
//               stage long -- the tensor core's FP32 accumulation drifts toward
//               zero over long chains), then write the output tile
// Every mbarrier wait is bounded; on timeout the CTA records the error word,
// raises an abort flag that the other roles poll, frees TMEM and returns.
//
//   (e) KB[rowoff + r][i] = sum_{lm, j} (W[lm][r][j] s_lm) (w_lm Mcal[lm][i][j] / s_lm)
//   (a) O[B][lm][i <= j] = (1 / s_lm) sum_r C_ri (W[lm][r][j] s_lm)
// with s_lm = sqrt((l+m)!(l-m)!) / h^l at the leaf level, which brings every
// component to O(1) for the 16-bit formats.
#include <cstdio>

#include "occk_internal.h"
#include "tc.cuh"

namespace occk {

int tc_mode(int prec);
int panel_elem_bytes(int prec);
int panel_bytes(int prec);

namespace {

using namespace tc;

constexpr uint32_t kLBO = 128, kSBO = 1024;
constexpr int kPart = 128 * 128;                 // bytes of one panel part
constexpr uint32_t kWait = 1u << 22;
template <int P>
struct Q : Fmt<P> {
    static constexpr int BK = 128 / Fmt<P>::esz;
    static constexpr int pbytes = kPart * (Fmt<P>::split ? 2 : 1);
    static constexpr int stages = Fmt<P>::split ? 3 : 4;
    static constexpr int smem = stages * 2 * pbytes;
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// Write 8 consecutive K values of one panel row (row r, elements k8..k8+7 of
// the panel) in the canonical layout, hi then lo part.
template <int P>
__device__ __forceinline__ void panel_put8(uint8_t* panel, int r, int k8, const float* v) {
    const uint32_t rowoff = (uint32_t)(r >> 3) * kSBO + (uint32_t)(r & 7) * 16u;
    put8<P>(panel + rowoff + (uint32_t)((k8 * Q<P>::esz) / 16) * kLBO, kPart, kLBO, v);
}

__device__ __forceinline__ size_t tri_ix(int i, int j, int n) {
    return (size_t)i * (size_t)(2 * n - i + 1) / 2 + (size_t)(j - i);
}

__device__ __forceinline__ int rank_of(int c) {
    int l = (int)sqrtf((float)c);
    while (l * l > c) --l;
    while ((l + 1) * (l + 1) <= c) ++l;
    return l;
}

// ---------------------------------------------------------------------------
// Panel builders (one block of 128 threads per panel, thread = panel row)
// ---------------------------------------------------------------------------
struct Plan {
    // step (e)
    const int* rtA;      // [nleaf] row tiles of W per leaf
    const long long* offA;   // [nleaf] first A panel of the leaf
    int KC, jc, it;      // K chunks (nc * jc), chunks per lm, i tiles
    // step (a)
    const int* kca;      // [nleaf] K chunks (rows of S_B / BK)
    const long long* offAa;  // [nleaf] first C panel
    const long long* offBa;  // [nleaf] first W panel
    int scaled;              // O and Mcal stored in scaled form
    float inv_h;             // 1 / leaf side
};

template <int P>
__global__ void k_panel_l2p_A(const int* __restrict__ leaf_rowoff, const float* __restrict__ W, int nocc, int nrow,
                              Plan pl, const float* __restrict__ lscale, uint8_t* __restrict__ panels) {
    const int kc = blockIdx.x, rt = blockIdx.y, B = blockIdx.z;
    if (rt >= pl.rtA[B]) return;
    constexpr int BK = Q<P>::BK;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int lm = kc / pl.jc, j0 = (kc % pl.jc) * BK;
    const float sc = lscale[lm];
    const int r = rt * 128 + threadIdx.x;
    const float* Wr = W + ((size_t)lm * nrow + rb0 + r) * nocc;
    uint8_t* panel = panels + (size_t)(pl.offA[B] + (long long)rt * pl.KC + kc) * Q<P>::pbytes;
    for (int k8 = 0; k8 < BK; k8 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + k8 + q;
            v[q] = (r < nr && j < nocc) ? Wr[j] * sc : 0.f;
        }
        panel_put8<P>(panel, threadIdx.x, k8, v);
    }
}

template <int P>
__global__ void k_panel_l2p_B(const float* __restrict__ Mbox, int nocc, int nc, int leaf_store0, Plan pl,
                              const float* __restrict__ lscale, uint8_t* __restrict__ panels) {
    const int kc = blockIdx.x, it = blockIdx.y, B = blockIdx.z;
    constexpr int BK = Q<P>::BK;
    const int lm = kc / pl.jc, j0 = (kc % pl.jc) * BK;
    const int l = rank_of(lm);
    const float w = (lm == l * l) ? 2.f : (((lm - l * l) & 1) ? 4.f : -4.f);
    // scaled storage holds Mcal~ = Mcal h^(l+1) / g, and Mcal / s_lm = Mcal~ / h
    const float sc = w * (pl.scaled ? pl.inv_h : 1.f / lscale[lm]);
    const size_t P2 = (size_t)nocc * (nocc + 1) / 2;
    const float* Ml = Mbox + ((size_t)(leaf_store0 + B) * nc + lm) * P2;
    const int i = it * 128 + threadIdx.x;
    uint8_t* panel = panels + (size_t)(((long long)B * pl.it + it) * pl.KC + kc) * Q<P>::pbytes;
    for (int k8 = 0; k8 < BK; k8 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + k8 + q;
            v[q] = (i < nocc && j < nocc) ? Ml[i <= j ? tri_ix(i, j, nocc) : tri_ix(j, i, nocc)] * sc : 0.f;
        }
        panel_put8<P>(panel, threadIdx.x, k8, v);
    }
}

template <int P>
__global__ void k_panel_a2_A(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos,
                             const float* __restrict__ Ct, int nocc, Plan pl, uint8_t* __restrict__ panels) {
    const int kc = blockIdx.x, it = blockIdx.y, B = blockIdx.z;
    if (kc >= pl.kca[B]) return;
    constexpr int BK = Q<P>::BK;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int i = it * 128 + threadIdx.x;
    uint8_t* panel = panels + (size_t)(pl.offAa[B] + (long long)it * pl.kca[B] + kc) * Q<P>::pbytes;
    for (int k8 = 0; k8 < BK; k8 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = kc * BK + k8 + q;
            v[q] = (r < nr && i < nocc) ? Ct[(size_t)leaf_aos[rb0 + r] * nocc + i] : 0.f;
        }
        panel_put8<P>(panel, threadIdx.x, k8, v);
    }
}

template <int P>
__global__ void k_panel_a2_B(const int* __restrict__ leaf_rowoff, const float* __restrict__ W, int nocc, int nrow,
                             int nc, Plan pl, const float* __restrict__ lscale, uint8_t* __restrict__ panels) {
    const int kc = blockIdx.x, B = blockIdx.z;
    const int lm = blockIdx.y / pl.it, jt = blockIdx.y % pl.it;
    if (kc >= pl.kca[B]) return;
    constexpr int BK = Q<P>::BK;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int j = jt * 128 + threadIdx.x;
    const float sc = lscale[lm];
    const float* Wl = W + ((size_t)lm * nrow + rb0) * nocc;
    uint8_t* panel =
        panels + (size_t)(pl.offBa[B] + ((long long)lm * pl.it + jt) * pl.kca[B] + kc) * Q<P>::pbytes;
    for (int k8 = 0; k8 < BK; k8 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = kc * BK + k8 + q;
            v[q] = (r < nr && j < nocc) ? Wl[(size_t)r * nocc + j] * sc : 0.f;
        }
        panel_put8<P>(panel, threadIdx.x, k8, v);
    }
}

// ---------------------------------------------------------------------------
// The pipelined GEMM on panels
// ---------------------------------------------------------------------------
struct PState {
    uint64_t full[4], empty[4], accf[2], acce[2];
    uint32_t tmem;
    int abort;
};

template <int P>
__device__ __forceinline__ void issue_panel_mmas(uint32_t a, uint32_t b, uint32_t d, uint32_t idesc) {
    constexpr int nks = Q<P>::BK / Q<P>::KSTEP;
    constexpr uint32_t kBuf = 128u;
#pragma unroll
    for (int ks = 0; ks < nks; ++ks) {
        const uint32_t adv = (uint32_t)ks * 2u * kLBO;
        const uint64_t ah = smem_desc(a + adv, kLBO, kSBO), bh = smem_desc(b + adv, kLBO, kSBO);
        const uint32_t acc = ks == 0 ? 0u : 1u;
        if constexpr (P == Q_TF32) {
            mma_tf32(d, ah, bh, idesc, acc);
        } else {
            mma_f16(d, ah, bh, idesc, acc);
            if constexpr (Q<P>::split) {
                const uint64_t al = smem_desc(a + kPart + adv, kLBO, kSBO), bl = smem_desc(b + kPart + adv, kLBO, kSBO);
                const uint32_t d2 = Q<P>::dual ? d + kBuf : d;
                mma_f16(d2, ah, bl, idesc, Q<P>::dual ? acc : 1u);
                mma_f16(d2, al, bh, idesc, 1u);
            }
        }
    }
}

// Runs the K loop of one 128 x 128 output tile and leaves the sum of this
// thread's row (flush warps only) in acc[128].  Returns false if aborted.
template <int P>
__device__ __forceinline__ bool pgemm_tile(const uint8_t* Apanels, const uint8_t* Bpanels, int nk, float* acc,
                                           int* err_word) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ PState st;
    constexpr int S = Q<P>::stages;
    constexpr uint32_t kBuf = Q<P>::dual ? 256u : 128u;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 2) {
        tmem_alloc(&st.tmem, 2 * kBuf);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&st.full[s], 1);
            mbar_init(&st.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&st.accf[b], 1);
            mbar_init(&st.acce[b], 128);
        }
        st.abort = 0;
        mbar_fence_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = st.tmem;
    const uint32_t sbase = smem_u32(smem);
    auto stageA = [&](int s) { return sbase + (uint32_t)(2 * s) * Q<P>::pbytes; };
    auto stageB = [&](int s) { return sbase + (uint32_t)(2 * s + 1) * Q<P>::pbytes; };
    if (warp == 0) {
        if (lane == 0) {
            for (int kc = 0; kc < nk && !*(volatile int*)&st.abort; ++kc) {
                const int s = kc % S;
                if (kc >= S && !mbar_wait_bounded(&st.empty[s], ((kc / S) - 1) & 1, kWait)) {
                    st.abort = 1;
                    break;
                }
                mbar_expect_tx(&st.full[s], 2u * Q<P>::pbytes);
                bulk_g2s(stageA(s), Apanels + (size_t)kc * Q<P>::pbytes, Q<P>::pbytes, &st.full[s]);
                bulk_g2s(stageB(s), Bpanels + (size_t)kc * Q<P>::pbytes, Q<P>::pbytes, &st.full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(128, 128, Q<P>::fmt);
            for (int kc = 0; kc < nk && !*(volatile int*)&st.abort; ++kc) {
                const int s = kc % S, b = kc & 1;
                if (!mbar_wait_bounded(&st.full[s], (kc / S) & 1, kWait)) {
                    st.abort = 1;
                    break;
                }
                if (kc >= 2 && !mbar_wait_bounded(&st.acce[b], ((kc >> 1) - 1) & 1, kWait)) {
                    st.abort = 1;
                    break;
                }
                fence_after_sync();
                issue_panel_mmas<P>(stageA(s), stageB(s), tmem + (uint32_t)b * kBuf, idesc);
                mma_commit(&st.empty[s]);
                mma_commit(&st.accf[b]);
            }
        }
    } else {
        const int q4 = warp & 3;   // TMEM lane quarter of this warp
        for (int kc = 0; kc < nk; ++kc) {
            const int b = kc & 1;
            if (*(volatile int*)&st.abort || !mbar_wait_bounded(&st.accf[b], (kc >> 1) & 1, kWait)) {
                st.abort = 1;
                break;
            }
            fence_after_sync();
            const uint32_t base = tmem + (uint32_t)b * kBuf + ((uint32_t)(q4 * 32) << 16);
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                float v[16];
                tmem_ld16(base + (uint32_t)(cc * 16), v);
                if constexpr (Q<P>::dual) {
                    float w[16];
                    tmem_ld16(base + 128u + (uint32_t)(cc * 16), w);
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] += w[q] * (1.f / kLo);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[cc * 16 + q] += v[q];
            }
            fence_before_sync();
            mbar_arrive(&st.acce[b]);
        }
    }
    fence_before_sync();
    __syncthreads();
    const bool ok = !*(volatile int*)&st.abort;
    if (!ok && t == 0) atomicExch(err_word, 1);
    if (warp == 2) tmem_dealloc(tmem, 2 * kBuf);
    return ok;
}

// blockIdx.z = leaf * nsplit + split: a split runs its share of the K panels
// and writes its own copy of KB (the K reduction adds the copies)
template <int P>
__global__ void __launch_bounds__(192, 1)
k_pgemm_l2p(const int* __restrict__ leaf_rowoff, int nocc, int nrow, int nsplit, Plan pl,
            const uint8_t* __restrict__ Apan, const uint8_t* __restrict__ Bpan, double* __restrict__ KB, int* err) {
    const int rt = blockIdx.x, it = blockIdx.y, B = blockIdx.z / nsplit, ks = blockIdx.z % nsplit;
    if (rt >= pl.rtA[B]) return;
    const int kc0 = (int)((long long)pl.KC * ks / nsplit), kc1 = (int)((long long)pl.KC * (ks + 1) / nsplit);
    const uint8_t* A = Apan + (size_t)(pl.offA[B] + (long long)rt * pl.KC + kc0) * Q<P>::pbytes;
    const uint8_t* Bp = Bpan + (size_t)(((long long)B * pl.it + it) * pl.KC + kc0) * Q<P>::pbytes;
    float acc[128];
#pragma unroll
    for (int q = 0; q < 128; ++q) acc[q] = 0.f;
    const bool ok = pgemm_tile<P>(A, Bp, kc1 - kc0, acc, err);
    const int warp = threadIdx.x >> 5;
    if (!ok || warp < 2) return;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r = rt * 128 + (warp & 3) * 32 + (threadIdx.x & 31);
    if (r >= nr) return;
    double* out = KB + (size_t)ks * nrow * nocc + (size_t)(rb0 + r) * nocc;
#pragma unroll
    for (int q = 0; q < 128; ++q) {
        const int i = it * 128 + q;
        if (i < nocc) out[i] = (double)acc[q];
    }
}

template <int P>
__global__ void __launch_bounds__(192, 1)
k_pgemm_a2(int nocc, int nc, int ntile, int leaf_store0, Plan pl, const uint8_t* __restrict__ Apan,
           const uint8_t* __restrict__ Bpan, const float* __restrict__ lscale, float* __restrict__ Obox, int* err) {
    const int B = blockIdx.y / nc, lm = blockIdx.y % nc;
    int tt = blockIdx.x, ti = 0;
    while (tt >= ntile - ti) {
        tt -= ntile - ti;
        ++ti;
    }
    const int tj = ti + tt;
    const int kca = pl.kca[B];
    const uint8_t* A = Apan + (size_t)(pl.offAa[B] + (long long)ti * kca) * Q<P>::pbytes;
    const uint8_t* Bp = Bpan + (size_t)(pl.offBa[B] + ((long long)lm * pl.it + tj) * kca) * Q<P>::pbytes;
    float acc[128];
#pragma unroll
    for (int q = 0; q < 128; ++q) acc[q] = 0.f;
    const bool ok = pgemm_tile<P>(A, Bp, kca, acc, err);
    const int warp = threadIdx.x >> 5;
    if (!ok || warp < 2) return;
    const int i = ti * 128 + (warp & 3) * 32 + (threadIdx.x & 31);
    if (i >= nocc) return;
    const size_t P2 = (size_t)nocc * (nocc + 1) / 2;
    float* O = Obox + ((size_t)(leaf_store0 + B) * nc + lm) * P2;
    const float inv = pl.scaled ? 1.f : 1.f / lscale[lm];   // scaled storage keeps O~ = O s_lm
#pragma unroll
    for (int q = 0; q < 128; ++q) {
        const int j = tj * 128 + q;
        if (j < nocc && j >= i) O[tri_ix(i, j, nocc)] = acc[q] * inv;
    }
}

// Plain GEMM D[M][N] = A[M][K] B[N][K]^T on FP32 row-major inputs, for
// checking the engine: generic panel builder and a plain epilogue.
template <int P>
__global__ void k_panel_rows(const float* __restrict__ X, int rows, int K, int KC, uint8_t* __restrict__ panels) {
    const int kc = blockIdx.x, rt = blockIdx.y;
    constexpr int BK = Q<P>::BK;
    const int r = rt * 128 + threadIdx.x;
    uint8_t* panel = panels + (size_t)((long long)rt * KC + kc) * Q<P>::pbytes;
    for (int k8 = 0; k8 < BK; k8 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kc * BK + k8 + q;
            v[q] = (r < rows && k < K) ? X[(size_t)r * K + k] : 0.f;
        }
        panel_put8<P>(panel, threadIdx.x, k8, v);
    }
}

template <int P>
__global__ void __launch_bounds__(192, 1)
k_pgemm_plain(int M, int N, int KC, const uint8_t* __restrict__ Apan, const uint8_t* __restrict__ Bpan,
              float* __restrict__ D, int* err) {
    const int mt = blockIdx.x, nt = blockIdx.y;
    float acc[128];
#pragma unroll
    for (int q = 0; q < 128; ++q) acc[q] = 0.f;
    const bool ok = pgemm_tile<P>(Apan + (size_t)mt * KC * Q<P>::pbytes, Bpan + (size_t)nt * KC * Q<P>::pbytes, KC,
                                  acc, err);
    const int warp = threadIdx.x >> 5;
    if (!ok || warp < 2) return;
    const int m = mt * 128 + (warp & 3) * 32 + (threadIdx.x & 31);
    if (m >= M) return;
#pragma unroll
    for (int q = 0; q < 128; ++q) {
        const int n = nt * 128 + q;
        if (n < N) D[(size_t)m * N + n] = acc[q];
    }
}

template <int P>
cudaError_t attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_pgemm_l2p<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q<P>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pgemm_a2<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q<P>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pgemm_plain<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q<P>::smem);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int P>
cudaError_t l2p_typed(const PanelArgs& a, cudaStream_t s) {
    cudaError_t e = attrs<P>();
    if (e != cudaSuccess) return e;
    Plan pl{a.rtA, a.offA, a.KC, a.jc, a.it, a.kca, a.offAa, a.offBa, a.scaled, a.inv_h_leaf};
    dim3 gA(a.KC, a.max_rt, a.nleaf), gB(a.KC, a.it, a.nleaf);
    k_panel_l2p_A<P><<<gA, 128, 0, s>>>(a.leaf_rowoff, a.W, a.nocc, a.nrow, pl, a.lscale, a.panA);
    k_panel_l2p_B<P><<<gB, 128, 0, s>>>(a.Mbox, a.nocc, a.nc, a.leaf_store0, pl, a.lscale, a.panB);
    dim3 g(a.max_rt, a.it, a.nleaf * a.nsplit);
    k_pgemm_l2p<P><<<g, 192, Q<P>::smem, s>>>(a.leaf_rowoff, a.nocc, a.nrow, a.nsplit, pl, a.panA, a.panB, a.KB,
                                              a.err);
    return cudaGetLastError();
}

template <int P>
cudaError_t a2_typed(const PanelArgs& a, cudaStream_t s) {
    cudaError_t e = attrs<P>();
    if (e != cudaSuccess) return e;
    Plan pl{a.rtA, a.offA, a.KC, a.jc, a.it, a.kca, a.offAa, a.offBa, a.scaled, a.inv_h_leaf};
    dim3 gA(a.max_kca, a.it, a.nleaf), gB(a.max_kca, a.it * a.nc, a.nleaf);
    k_panel_a2_A<P><<<gA, 128, 0, s>>>(a.leaf_rowoff, a.leaf_aos, a.Ct, a.nocc, pl, a.panA);
    k_panel_a2_B<P><<<gB, 128, 0, s>>>(a.leaf_rowoff, a.W, a.nocc, a.nrow, a.nc, pl, a.lscale, a.panB);
    dim3 g(a.it * (a.it + 1) / 2, a.nleaf * a.nc);
    k_pgemm_a2<P><<<g, 192, Q<P>::smem, s>>>(a.nocc, a.nc, a.it, a.leaf_store0, pl, a.panA, a.panB, a.lscale,
                                             a.Obox, a.err);
    return cudaGetLastError();
}

template <int P>
cudaError_t plain_typed(int M, int N, int K, const float* A, const float* B, float* D, uint8_t* panels, int* err,
                        cudaStream_t s) {
    cudaError_t e = attrs<P>();
    if (e != cudaSuccess) return e;
    const int KC = (K + Q<P>::BK - 1) / Q<P>::BK, mt = (M + 127) / 128, nt = (N + 127) / 128;
    uint8_t* pa = panels;
    uint8_t* pb = panels + (size_t)mt * KC * Q<P>::pbytes;
    k_panel_rows<P><<<dim3(KC, mt), 128, 0, s>>>(A, M, K, KC, pa);
    k_panel_rows<P><<<dim3(KC, nt), 128, 0, s>>>(B, N, K, KC, pb);
    k_pgemm_plain<P><<<dim3(mt, nt), 192, Q<P>::smem, s>>>(M, N, KC, pa, pb, D, err);
    return cudaGetLastError();
}

}  // namespace

int tc_mode(int prec) {
    switch (prec) {
        case OCCK_BF16: return Q_BF16;
        case OCCK_FP16: return Q_FP16;
        case OCCK_TF32: return Q_TF32;
        case OCCK_BF16X3: return Q_BF16X3;
        case OCCK_FP16X3: return Q_FP16X3;
        default: return -1;
    }
}

size_t tc_gemm_panel_bytes(int prec, int M, int N, int K) {
    const int esz = panel_elem_bytes(prec), pb = panel_bytes(prec);
    if (!esz) return 0;
    const size_t KC = (size_t)(K + 128 / esz - 1) / (128 / esz);
    return KC * ((size_t)(M + 127) / 128 + (size_t)(N + 127) / 128) * (size_t)pb;
}

cudaError_t tc_gemm(int prec, int M, int N, int K, const float* A, const float* B, float* D, uint8_t* panels,
                    int* err, cudaStream_t s) {
    switch (tc_mode(prec)) {
        case Q_BF16: return plain_typed<Q_BF16>(M, N, K, A, B, D, panels, err, s);
        case Q_FP16: return plain_typed<Q_FP16>(M, N, K, A, B, D, panels, err, s);
        case Q_TF32: return plain_typed<Q_TF32>(M, N, K, A, B, D, panels, err, s);
        case Q_BF16X3: return plain_typed<Q_BF16X3>(M, N, K, A, B, D, panels, err, s);
        case Q_FP16X3: return plain_typed<Q_FP16X3>(M, N, K, A, B, D, panels, err, s);
        default: return cudaErrorInvalidValue;
    }
}

int panel_elem_bytes(int prec) {
    switch (tc_mode(prec)) {
        case Q_TF32: return 4;
        case Q_BF16: case Q_FP16: case Q_BF16X3: case Q_FP16X3: return 2;
        default: return 0;
    }
}
int panel_bytes(int prec) {
    switch (tc_mode(prec)) {
        case Q_BF16: case Q_FP16: case Q_TF32: return kPart;
        case Q_BF16X3: case Q_FP16X3: return 2 * kPart;
        default: return 0;
    }
}

#define OCCK_Q_DISPATCH(prec, call)                                   \
    switch (tc_mode(prec)) {                                          \
        case Q_BF16: { constexpr int P = Q_BF16; return call; }       \
        case Q_FP16: { constexpr int P = Q_FP16; return call; }       \
        case Q_TF32: { constexpr int P = Q_TF32; return call; }       \
        case Q_BF16X3: { constexpr int P = Q_BF16X3; return call; }   \
        case Q_FP16X3: { constexpr int P = Q_FP16X3; return call; }   \
        default: return cudaErrorInvalidValue;                        \
    }

cudaError_t panel_l2p(int prec, const PanelArgs& a, cudaStream_t s) { OCCK_Q_DISPATCH(prec, l2p_typed<P>(a, s)); }
cudaError_t panel_a2(int prec, const PanelArgs& a, cudaStream_t s) { OCCK_Q_DISPATCH(prec, a2_typed<P>(a, s)); }

}  // namespace occk
