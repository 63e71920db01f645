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
#include <algorithm>
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

// Polls allowed to the MMA thread's wait for a stage's operands.  kWait in
// normal use; occk_debug_set_wait_limit lowers it so that a test can make
// that wait give up and exercise the abort path (the waits of the drain keep
// kWait).  One value per device, shared by every context in the process.
__device__ uint32_t g_mma_full_wait = kWait;

// Bounded wait that also gives up as soon as another role has raised *flag
// (a producer or epilogue waiting for a stage that an aborted MMA thread
// will never release).
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t* bar, uint32_t parity, uint32_t limit,
                                                    const int* flag) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(const volatile int*)flag) return false;
        if (it > 64) __nanosleep(32);
    }
    return false;
}
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
    uint32_t gp, gm;   // stages issued by the producer, consumed by the MMA thread
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
        st.gp = 0;
        st.gm = 0;
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
                if (kc >= S && !mbar_wait_abortable(&st.empty[s], ((kc / S) - 1) & 1, kWait, &st.abort)) {
                    st.abort = 1;
                    break;
                }
                mbar_expect_tx(&st.full[s], 2u * Q<P>::pbytes);
                bulk_g2s(stageA(s), Apanels + (size_t)kc * Q<P>::pbytes, Q<P>::pbytes, &st.full[s]);
                bulk_g2s(stageB(s), Bpanels + (size_t)kc * Q<P>::pbytes, Q<P>::pbytes, &st.full[s]);
                st.gp = (uint32_t)kc + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(128, 128, Q<P>::fmt);
            const uint32_t full_wait = g_mma_full_wait;
            for (int kc = 0; kc < nk && !*(volatile int*)&st.abort; ++kc) {
                const int s = kc % S, b = kc & 1;
                if (!mbar_wait_bounded(&st.full[s], (kc / S) & 1, full_wait)) {
                    st.abort = 1;
                    break;
                }
                if (kc >= 2 && !mbar_wait_abortable(&st.acce[b], ((kc >> 1) - 1) & 1, kWait, &st.abort)) {
                    st.abort = 1;
                    break;
                }
                fence_after_sync();
                issue_panel_mmas<P>(stageA(s), stageB(s), tmem + (uint32_t)b * kBuf, idesc);
                mma_commit(&st.empty[s]);
                mma_commit(&st.accf[b]);
                st.gm = (uint32_t)kc + 1;
            }
            // the last MMAs finish before TMEM is given back
            const uint32_t gl = st.gm;
            if (gl > 0) mbar_wait_bounded(&st.accf[(gl - 1) & 1], ((gl - 1) >> 1) & 1, kWait);
        }
    } else {
        const int q4 = warp & 3;   // TMEM lane quarter of this warp
        for (int kc = 0; kc < nk; ++kc) {
            const int b = kc & 1;
            if (*(volatile int*)&st.abort ||
                !mbar_wait_abortable(&st.accf[b], (kc >> 1) & 1, kWait, &st.abort)) {
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
    if (!ok && t == 0) {
        atomicExch(err_word, 1);
        // copies issued but never consumed: wait (bounded) until they land
        for (uint32_t g = st.gm; g < st.gp; ++g) mbar_wait_bounded(&st.full[g % S], (g / S) & 1, kWait);
    }
    __syncthreads();
    fence_after_sync();
    if (warp == 2) tmem_dealloc(tmem, 2 * kBuf);
    return ok;
}

// Persistent form of the panel GEMM: one CTA per SM walks a list of output
// tiles (it = blockIdx.x, + gridDim.x, ...); the stage ring, its mbarrier
// phases and the two TMEM accumulators carry on across tiles, so a tile with
// a short K (a leaf of a few dozen AOs) costs no set-up of its own.
// src(it, A, B, nk) gives a tile's panels; epi(it, row, col0, acc) stores
// columns col0 .. col0 + 128/(NF/4) - 1 of a row.  NF epilogue warps (4 or 8:
// with 8, two per TMEM lane quarter, each owning half of the columns).
struct PPState {
    uint64_t full[4], empty[4], accf[2], acce[2];
    uint32_t tmem;
    int abort;
    uint32_t gp, gm;   // stages issued by the producer, consumed by the MMA thread
};

template <int P, int NF, typename Src, typename Epi>
__device__ __forceinline__ void pgemm_persistent(long long nitems, Src src, Epi epi, int* err_word) {
    constexpr int NCOL = 128 / (NF / 4);   // output columns per epilogue thread
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ PPState st;
    constexpr int S = Q<P>::stages;
    constexpr uint32_t kBuf = Q<P>::dual ? 256u : 128u;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 2) {
        tmem_alloc(&st.tmem, 2 * kBuf);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int r = 0; r < S; ++r) {
            mbar_init(&st.full[r], 1);
            mbar_init(&st.empty[r], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&st.accf[b], 1);
            mbar_init(&st.acce[b], 32 * NF);
        }
        st.abort = 0;
        st.gp = 0;
        st.gm = 0;
        mbar_fence_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = st.tmem;
    const uint32_t sbase = smem_u32(smem);
    auto stageA = [&](int r) { return sbase + (uint32_t)(2 * r) * Q<P>::pbytes; };
    auto stageB = [&](int r) { return sbase + (uint32_t)(2 * r + 1) * Q<P>::pbytes; };
    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            for (long long it = blockIdx.x; it < nitems && !*(volatile int*)&st.abort; it += gridDim.x) {
                const uint8_t *A, *B;
                int nk;
                src(it, A, B, nk);
                for (int kc = 0; kc < nk; ++kc, ++g) {
                    const int r = (int)(g % S);
                    if (g >= (uint32_t)S &&
                        !mbar_wait_abortable(&st.empty[r], ((g / S) - 1) & 1, kWait, &st.abort)) {
                        st.abort = 1;
                        break;
                    }
                    mbar_expect_tx(&st.full[r], 2u * Q<P>::pbytes);
                    bulk_g2s(stageA(r), A + (size_t)kc * Q<P>::pbytes, Q<P>::pbytes, &st.full[r]);
                    bulk_g2s(stageB(r), B + (size_t)kc * Q<P>::pbytes, Q<P>::pbytes, &st.full[r]);
                    st.gp = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(128, 128, Q<P>::fmt);
            const uint32_t full_wait = g_mma_full_wait;
            uint32_t g = 0;
            for (long long it = blockIdx.x; it < nitems && !*(volatile int*)&st.abort; it += gridDim.x) {
                const uint8_t *A, *B;
                int nk;
                src(it, A, B, nk);
                for (int kc = 0; kc < nk; ++kc, ++g) {
                    const int r = (int)(g % S), b = (int)(g & 1);
                    if (!mbar_wait_bounded(&st.full[r], (g / S) & 1, full_wait) ||
                        (g >= 2 && !mbar_wait_abortable(&st.acce[b], ((g >> 1) - 1) & 1, kWait, &st.abort))) {
                        st.abort = 1;
                        break;
                    }
                    fence_after_sync();
                    issue_panel_mmas<P>(stageA(r), stageB(r), tmem + (uint32_t)b * kBuf, idesc);
                    mma_commit(&st.empty[r]);
                    mma_commit(&st.accf[b]);
                    st.gm = g + 1;
                }
            }
            const uint32_t gl = st.gm;   // the last MMAs finish before TMEM is given back
            if (gl > 0) mbar_wait_bounded(&st.accf[(gl - 1) & 1], ((gl - 1) >> 1) & 1, kWait);
        }
    } else {
        const int q4 = warp & 3;                      // TMEM lane quarter of this warp
        const int col0 = ((warp - 2) >> 2) * NCOL;    // its share of the columns
        uint32_t g = 0;
        float acc[NCOL];
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
            const uint8_t *A, *B;
            int nk;
            src(it, A, B, nk);
#pragma unroll
            for (int q = 0; q < NCOL; ++q) acc[q] = 0.f;
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc, ++g) {
                const int b = (int)(g & 1);
                if (*(volatile int*)&st.abort ||
                    !mbar_wait_abortable(&st.accf[b], (g >> 1) & 1, kWait, &st.abort)) {
                    st.abort = 1;
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t base = tmem + (uint32_t)b * kBuf + (uint32_t)col0 + ((uint32_t)(q4 * 32) << 16);
#pragma unroll
                for (int cc = 0; cc < NCOL / 16; ++cc) {
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
            if (!ok) break;
            epi(it, q4 * 32 + lane, col0, acc);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (t == 0 && st.abort) {
        atomicExch(err_word, 1);
        // copies issued but never consumed: wait (bounded) until they land
        for (uint32_t g = st.gm; g < st.gp; ++g) mbar_wait_bounded(&st.full[g % S], (g / S) & 1, kWait);
    }
    __syncthreads();
    fence_after_sync();
    if (warp == 2) tmem_dealloc(tmem, 2 * kBuf);
}

// Step (a), persistent: tiles ordered (triangular tile fastest, then lm,
// then leaf), so concurrently running CTAs share panels in L2.  Eight
// epilogue warps; dynamic shared memory: the stage ring plus eight 32 x 33
// FP32 staging tiles.
constexpr int kA2pThreads = 64 + 8 * 32;
template <int P>
constexpr int kA2pSmem = Q<P>::smem + 8 * 32 * 33 * 4;

template <int P>
__global__ void __launch_bounds__(kA2pThreads, 1)
k_pgemm_a2p(int nocc, int nc, int ntile, int leaf_store0, int nleaf, Plan pl, const uint8_t* __restrict__ Apan,
            const uint8_t* __restrict__ Bpan, const float* __restrict__ lscale, float* __restrict__ Obox, int* err) {
    const int ntt = ntile * (ntile + 1) / 2;
    const long long nitems = (long long)ntt * nleaf * nc;
    const size_t P2 = (size_t)nocc * (nocc + 1) / 2;
    auto decode = [&](long long it, int& ti, int& tj, int& B, int& lm) {
        int tt = (int)(it % ntt);
        const long long rest = it / ntt;
        lm = (int)(rest % nc);
        B = (int)(rest / nc);
        ti = 0;
        while (tt >= ntile - ti) {
            tt -= ntile - ti;
            ++ti;
        }
        tj = ti + tt;
    };
    auto src = [&](long long it, const uint8_t*& A, const uint8_t*& Bp, int& nk) {
        int ti, tj, B, lm;
        decode(it, ti, tj, B, lm);
        const int kca = pl.kca[B];
        A = Apan + (size_t)(pl.offAa[B] + (long long)ti * kca) * Q<P>::pbytes;
        Bp = Bpan + (size_t)(pl.offBa[B] + ((long long)lm * pl.it + tj) * kca) * Q<P>::pbytes;
        nk = kca;
    };
    // Epilogue through a per-warp 32 x 32 staging tile: a thread holds one
    // row of the output tile, but packed rows are contiguous in j, so each
    // warp writes its 32 rows 32 columns at a time, one row per store
    // instruction (128 contiguous bytes) instead of 32 rows per instruction.
    auto epi = [&](long long it, int row, int col0, const float* acc) {
        extern __shared__ __align__(1024) uint8_t smem[];
        int ti, tj, B, lm;
        decode(it, ti, tj, B, lm);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        float* tile = reinterpret_cast<float*>(smem + Q<P>::smem) + (warp - 2) * 32 * 33;
        float* O = Obox + ((size_t)(leaf_store0 + B) * nc + lm) * P2;
        const float inv = pl.scaled ? 1.f : 1.f / lscale[lm];   // scaled storage keeps O~ = O s_lm
        const int r0 = ti * 128 + (row & ~31);                  // first row of this warp
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
#pragma unroll
            for (int q = 0; q < 32; ++q) tile[lane * 33 + q] = acc[cc * 32 + q] * inv;
            __syncwarp();
            const int j = tj * 128 + col0 + cc * 32 + lane;
            for (int r = 0; r < 32; ++r) {
                const int i = r0 + r;
                if (i < nocc && j < nocc && j >= i) O[tri_ix(i, i, nocc) - (size_t)i + (size_t)j] = tile[r * 33 + lane];
            }
            __syncwarp();
        }
    };
    pgemm_persistent<P, 8>(nitems, src, epi, err);
}

// Step (e), persistent: one CTA per SM walks the output tiles (global row
// tile of the stacked leaves, 128-orbital tile, K split), the orbital tile
// fastest so that CTAs running together share a row tile's W panels in L2;
// the stage ring and the TMEM ping-pong carry on across tiles, so a tile's
// ring fill and its epilogue overlap the next tile's MMAs.  Eight epilogue
// warps stage their FP64 stores through per-warp 32 x 33 tiles (each store
// instruction writes 32 consecutive K entries of one row).
template <int P>
__global__ void __launch_bounds__(kA2pThreads, 1)
k_pgemm_l2p_pers(const int* __restrict__ leaf_rowoff, int nocc, int nrow, int nsplit, int nleaf, Plan pl,
                 const uint8_t* __restrict__ Apan, const uint8_t* __restrict__ Bpan, double* __restrict__ KB, int* err) {
    const long long nrt = (pl.offA[nleaf - 1] + (long long)pl.rtA[nleaf - 1] * pl.KC) / pl.KC;
    const long long nitems = nrt * pl.it * nsplit;
    // item -> (leaf B, row tile rt of B, orbital tile t, split ks)
    auto decode = [&](long long item, int& B, int& rt, int& t, int& ks) {
        ks = (int)(item % nsplit);
        const long long rest = item / nsplit;
        t = (int)(rest % pl.it);
        const long long g = rest / pl.it;                // global row tile
        int lo = 0, hi = nleaf - 1;                      // last leaf with offA / KC <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pl.offA[mid] / pl.KC <= g) lo = mid;
            else hi = mid - 1;
        }
        B = lo;
        rt = (int)(g - pl.offA[B] / pl.KC);
    };
    auto src = [&](long long item, const uint8_t*& A, const uint8_t*& Bp, int& nk) {
        int B, rt, t, ks;
        decode(item, B, rt, t, ks);
        const int kc0 = (int)((long long)pl.KC * ks / nsplit), kc1 = (int)((long long)pl.KC * (ks + 1) / nsplit);
        A = Apan + (size_t)(pl.offA[B] + (long long)rt * pl.KC + kc0) * Q<P>::pbytes;
        Bp = Bpan + (size_t)(((long long)B * pl.it + t) * pl.KC + kc0) * Q<P>::pbytes;
        nk = kc1 - kc0;
    };
    auto epi = [&](long long item, int row, int col0, const float* acc) {
        extern __shared__ __align__(1024) uint8_t smem[];
        int B, rt, t, ks;
        decode(item, B, rt, t, ks);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        float* tile = reinterpret_cast<float*>(smem + Q<P>::smem) + (warp - 2) * 32 * 33;
        const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
        const int r0 = rt * 128 + (row & ~31);                  // first row of this warp
        double* out = KB + (size_t)ks * nrow * nocc + (size_t)rb0 * nocc;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
#pragma unroll
            for (int q = 0; q < 32; ++q) tile[lane * 33 + q] = acc[cc * 32 + q];
            __syncwarp();
            const int i = t * 128 + col0 + cc * 32 + lane;
            for (int r = 0; r < 32; ++r)
                if (r0 + r < nr && i < nocc) out[(size_t)(r0 + r) * nocc + i] = (double)tile[r * 33 + lane];
            __syncwarp();
        }
    };
    pgemm_persistent<P, 8>(nitems, src, epi, err);
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
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!ok || warp < 2) return;
    // the stage ring is idle now: each flush warp transposes its 32 rows
    // through a 32 x 33 tile so that a store instruction writes 32 consecutive
    // K entries of one row
    extern __shared__ __align__(1024) uint8_t smem[];
    float* tile = reinterpret_cast<float*>(smem) + (warp - 2) * 32 * 33;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r0 = rt * 128 + (warp & 3) * 32;
    double* out = KB + (size_t)ks * nrow * nocc + (size_t)rb0 * nocc;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
#pragma unroll
        for (int q = 0; q < 32; ++q) tile[lane * 33 + q] = acc[cc * 32 + q];
        __syncwarp();
        const int i = it * 128 + cc * 32 + lane;
        for (int r = 0; r < 32; ++r)
            if (r0 + r < nr && i < nocc) out[(size_t)(r0 + r) * nocc + i] = (double)tile[r * 33 + lane];
        __syncwarp();
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
        e = cudaFuncSetAttribute(k_pgemm_a2p<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kA2pSmem<P>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pgemm_l2p_pers<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kA2pSmem<P>);
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
    // persistent: one CTA per SM over all (row tile, orbital tile, split)
    // items (the per-tile grid form, k_pgemm_l2p, is kept for reference)
    long long nrt = 0;
    {
        // total row tiles: from the host plan (rows of every leaf / 128)
        for (int B = 0; B < a.nleaf; ++B)
            nrt += (a.leaf_rowoff_host[B + 1] - a.leaf_rowoff_host[B] + 127) / 128;
    }
    const long long items = nrt * a.it * a.nsplit;
    const int grid = (int)std::min<long long>(items, std::max(a.sm_count, 1));
    if (grid > 0)
        k_pgemm_l2p_pers<P><<<grid, kA2pThreads, kA2pSmem<P>, s>>>(a.leaf_rowoff, a.nocc, a.nrow, a.nsplit,
                                                                 a.nleaf, pl, a.panA, a.panB, a.KB, a.err);
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
    const long long items = (long long)(a.it * (a.it + 1) / 2) * a.nleaf * a.nc;
    const int grid = (int)std::min<long long>(items, std::max(a.sm_count, 1));
    k_pgemm_a2p<P><<<grid, kA2pThreads, kA2pSmem<P>, s>>>(a.nocc, a.nc, a.it, a.leaf_store0, a.nleaf, pl, a.panA, a.panB,
                                                 a.lscale, a.Obox, a.err);
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

cudaError_t set_mma_wait_limit(long long polls) {
    const uint32_t v = polls < 0 ? kWait : (uint32_t)std::min<long long>(polls, 0xffffffffLL);
    return cudaMemcpyToSymbol(g_mma_full_wait, &v, sizeof(v));
}

cudaError_t panel_l2p(int prec, const PanelArgs& a, cudaStream_t s) { OCCK_Q_DISPATCH(prec, l2p_typed<P>(a, s)); }
cudaError_t panel_a2(int prec, const PanelArgs& a, cudaStream_t s) { OCCK_Q_DISPATCH(prec, a2_typed<P>(a, s)); }

}  // namespace occk
