// Steps (b) M2M, (c) M2L and (d) L2L of the mixed-precision forms on tcgen05.
//
// All three steps have the same shape (Eqs. fmm1-3 in real form): for a target
// box t and every stored occupied pair p,
//     Out[t][q][p] (+)= sum_{edges (t, s, op)} sum_c T_op[q][c] In[s][c][p].
// One work item is one target box and a tile of 128 pairs; on the tensor core
// it is a GEMM with M = 128 pairs, N = NP output components (nc rounded up to a
// power of two, at least 16) and K running over the edges' input components:
// A = In[s][c][p0..p0+127] (each thread loads its own pair row, coalesced
// along p, and converts it), B = the operator, prepared once per tree in the
// tensor core's layout and moved into shared memory with bulk asynchronous
// copies.  Persistent CTAs walk the items pair tile by pair tile, so the
// sources that neighbouring targets share are read from L2.
//
// Scaling.  Expansion components differ by many orders of magnitude (the
// (l+m)! normalisation of O_lm, powers of the box side), too many for FP16.
// On this path the multipoles and local expansions are kept in HBM in scaled
// form,
//     O~_lm = O_lm sqrt((l+m)!(l-m)!) / h^l,
//     Mcal~_lm = Mcal_lm h^(l+1) / sqrt((l+m)!(l-m)!),
// h the side of the box's level (step (a) produces O~ directly, step (e)
// consumes Mcal~), and each operator is prepared as
// T~[q][c] = s_out[q] T[q][c] / s_in[c].  Since |P_l^m| <= sqrt((l+m)!/(l-m)!)
// on the unit sphere and the binomial coefficients of the addition theorems
// are at most 2^(l+l'), all scaled operator entries are O(1) for boxes at least
// one box apart (M2L, |X - X'| >= 2h) and for parent-child shifts (M2M, L2L),
// and so are the scaled expansions.
//
// Accumulation restarts in TMEM at every stage (64 K values for 16-bit types,
// 32 for TF32) and the stages are summed in FP32 registers: the tensor core's
// own FP32 accumulation drifts toward zero over long chains.  Every mbarrier
// wait is bounded and is done by one thread, whose verdict the others read
// after a block barrier; on timeout the CTA raises the error word, waits
// (bounded) for its copies and MMAs in flight, frees TMEM and returns.
#include <cstdio>

#include "occk_internal.h"
#include "tc.cuh"

namespace occk {

int tc_mode(int prec);

namespace {

using namespace tc;

constexpr uint32_t kWaitT = 1u << 22;

constexpr int pow2ceil_i(int x) {
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

template <int P, int NP>
struct TT {
    using F = Fmt<P>;
    static constexpr int esz = F::esz;
    static constexpr int BK = 128 / esz;                 // K values of one stage
    static constexpr int KCH = NP < BK ? NP : BK;        // K values of one slot (one chunk of one edge)
    static constexpr int NCH = NP / KCH;                 // chunks per edge
    static constexpr int ES = BK / KCH;                  // slots per stage
    static constexpr int parts = F::split ? 2 : 1;
    static constexpr uint32_t A_part = 128u * KCH * esz;
    static constexpr uint32_t B_part = (uint32_t)NP * KCH * esz;
    static constexpr uint32_t A_slot = A_part * parts, B_slot = B_part * parts;
    static constexpr uint32_t A_stage = A_slot * ES, B_stage = B_slot * ES;
    static constexpr uint32_t LBO = 128;
    static constexpr uint32_t SBO = (uint32_t)KCH * esz * 8;   // stride of 8-row groups
    static constexpr int setN = F::dual ? 2 * NP : NP;          // TMEM columns of one accumulator set
    static constexpr int ACCB = (2 * setN <= 256) ? 2 : 1;      // accumulator sets (ping-pong if 2)
    static constexpr uint32_t tmem_cols = (uint32_t)pow2ceil_i(ACCB * setN < 32 ? 32 : ACCB * setN);
    static constexpr int smem = 2 * (int)(A_stage + B_stage);
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

// ---------------------------------------------------------------------------
// Operator panels: for operator o and chunk ch, NP rows (output components q)
// x KCH columns (input components c = ch*KCH + k), hi part then lo part, in
// the K-major canonical layout with SBO = KCH*esz*8.
// ---------------------------------------------------------------------------
template <int P, int NP>
__global__ void k_tr_op_panels(const double* __restrict__ ops, int nops, int nc, const int* __restrict__ opinfo,
                               const double* __restrict__ scd, int nlev, uint8_t* __restrict__ pan) {
    using C = TT<P, NP>;
    const int o = blockIdx.x, ch = blockIdx.y;
    if (o >= nops) return;
    const int kin = opinfo[4 * o + 0], lin = opinfo[4 * o + 1], kout = opinfo[4 * o + 2], lout = opinfo[4 * o + 3];
    const double* sin_ = scd + ((size_t)kin * nlev + lin) * nc;
    const double* sout = scd + ((size_t)kout * nlev + lout) * nc;
    const double* T = ops + (size_t)o * nc * nc;
    uint8_t* base = pan + ((size_t)o * C::NCH + ch) * C::B_slot;
    for (int x = threadIdx.x; x < NP * (C::KCH / 8); x += blockDim.x) {
        const int q = x / (C::KCH / 8), k8 = (x % (C::KCH / 8)) * 8;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = ch * C::KCH + k8 + u;
            v[u] = (q < nc && c < nc) ? (float)(sout[q] * T[(size_t)q * nc + c] / sin_[c]) : 0.f;
        }
        uint8_t* dst = base + (uint32_t)(q >> 3) * C::SBO + (uint32_t)(q & 7) * 16u +
                       (uint32_t)((k8 * C::esz) / 16) * C::LBO;
        put8<P>(dst, C::B_part, C::LBO, v);
    }
}

// The same scaled operators as plain row-major FP32 [nops][nc][nc], for the
// SIMT translations when they run on the scaled storage.
__global__ void k_tr_ops_scaled(const double* __restrict__ ops, int nops, int nc, const int* __restrict__ opinfo,
                                const double* __restrict__ scd, int nlev, float* __restrict__ out) {
    const int o = blockIdx.x;
    if (o >= nops) return;
    const int kin = opinfo[4 * o + 0], lin = opinfo[4 * o + 1], kout = opinfo[4 * o + 2], lout = opinfo[4 * o + 3];
    const double* sin_ = scd + ((size_t)kin * nlev + lin) * nc;
    const double* sout = scd + ((size_t)kout * nlev + lout) * nc;
    for (int x = threadIdx.x; x < nc * nc; x += blockDim.x) {
        const int q = x / nc, c = x % nc;
        out[(size_t)o * nc * nc + x] = (float)(sout[q] * ops[(size_t)o * nc * nc + x] / sin_[c]);
    }
}

struct TrKArgs {
    int mode;                 // 0 M2M (children), 1 M2L (interaction list), 2 L2L (parent)
    int P, nc, first_box, tgt0, ntgt, accumulate, nlev;
    const int* ptr; const int* list; const int* opidx; const int* parent; const int* box_level;
    const float* in; float* out;
    const uint8_t* pan;       // operator panels
    int* err;
};

template <int P, int NP>
__device__ __forceinline__ void issue_stage_mmas(uint32_t a, uint32_t b, int nvalid, uint32_t d) {
    using C = TT<P, NP>;
    using F = Fmt<P>;
    constexpr uint32_t idesc = instr_desc(128, NP, F::fmt);
    for (int k = 0; k < nvalid; ++k) {
        const uint32_t ak = a + (uint32_t)k * C::A_slot, bk = b + (uint32_t)k * C::B_slot;
#pragma unroll
        for (int ks = 0; ks < C::KCH / F::KSTEP; ++ks) {
            const uint32_t adv = (uint32_t)ks * 2u * C::LBO;
            const uint64_t ah = smem_desc(ak + adv, C::LBO, C::SBO), bh = smem_desc(bk + adv, C::LBO, C::SBO);
            const uint32_t acc = (k == 0 && ks == 0) ? 0u : 1u;
            if constexpr (P == Q_TF32) {
                mma_tf32(d, ah, bh, idesc, acc);
            } else {
                mma_f16(d, ah, bh, idesc, acc);
                if constexpr (F::split) {
                    const uint64_t al = smem_desc(ak + C::A_part + adv, C::LBO, C::SBO);
                    const uint64_t bl = smem_desc(bk + C::B_part + adv, C::LBO, C::SBO);
                    const uint32_t d2 = F::dual ? d + (uint32_t)NP : d;
                    mma_f16(d2, ah, bl, idesc, F::dual ? acc : 1u);
                    mma_f16(d2, al, bh, idesc, 1u);
                }
            }
        }
    }
}

constexpr int kMaxEdges = 256;   // edges of one target (an interaction list has at most 189)
// threads per pair row: each converts 1/TPR of a stage's K values and
// accumulates NP/TPR (at least 16) output columns
template <int NP>
constexpr int tpr() { return NP >= 64 ? 4 : 2; }

template <int P, int NP>
__global__ void __launch_bounds__(128 * tpr<NP>(), NP <= 32 ? 2 : 1)
k_tc_translate(TrKArgs a) {
    using C = TT<P, NP>;
    using F = Fmt<P>;
    constexpr int TPR = tpr<NP>();
    constexpr int kThreads = 128 * TPR;
    constexpr int NV = C::ES * C::KCH;          // K values of one stage
    constexpr int NVH = NV / TPR;               // ... converted by one thread
    constexpr int NPH = NP / TPR >= 16 ? NP / TPR : 16;   // output columns one thread accumulates
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bfull[2], mdone[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ long long s_xoff[kMaxEdges];     // element offset of each edge's source
    __shared__ int s_op[kMaxEdges];
    const int t = threadIdx.x, warp = t >> 5;
    const int row = t & 127, half = t >> 7;    // half: which share of the K values and columns
    const bool has_cols = half < NP / NPH;
    const int col0 = half * NPH;
    if (warp == 0) {
        tmem_alloc(&tmem_base, C::tmem_cols);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bfull[b], 1);
            mbar_init(&mdone[b], 1);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t sA = smem_u32(smem), sB = sA + 2u * C::A_stage;
    const int P2 = a.P;
    const int ntile = (P2 + 127) / 128;
    const long long nitems = (long long)a.ntgt * ntile;
    const size_t boxstride = (size_t)a.nc * (size_t)P2;
    // thread 0 only: outstanding copies and MMAs (1 + parity, 0 = none)
    uint32_t g = 0;                       // stages issued by this CTA so far
    int bpend0 = 0, bpend1 = 0, mpend0 = 0, mpend1 = 0;
    float acc[NPH];
    float v[NVH];

    for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int ptile = (int)(it / a.ntgt), tgt = a.tgt0 + (int)(it % a.ntgt);
        const int p = ptile * 128 + row;
        const bool live = p < P2;
        int e0 = 0, ne = 1;
        if (a.mode != 2) {
            e0 = a.ptr[tgt];
            ne = min(a.ptr[tgt + 1] - e0, kMaxEdges);
        }
        // edge table of this item, read once
        for (int k = t; k < ne; k += kThreads) {
            int src, op;
            if (a.mode == 0) {
                src = a.list[e0 + k];
                op = a.opidx[src];
            } else if (a.mode == 1) {
                src = a.list[e0 + k];
                op = a.opidx[e0 + k];
            } else {
                src = a.parent[tgt];
                op = a.opidx[tgt];
            }
            s_xoff[k] = (long long)(src - a.first_box) * (long long)boxstride;
            s_op[k] = op;
        }
        __syncthreads();
        const int nslot = ne * C::NCH, S = (nslot + C::ES - 1) / C::ES;
#pragma unroll
        for (int q = 0; q < NPH; ++q) acc[q] = 0.f;

        auto issue_B = [&](int s, int b) {
            const int nvalid = min(C::ES, nslot - s * C::ES);
            mbar_expect_tx(&bfull[b], (uint32_t)nvalid * C::B_slot);
            for (int k = 0; k < nvalid; ++k) {
                const int u = s * C::ES + k, e = u / C::NCH, ch = u % C::NCH;
                bulk_g2s(sB + (uint32_t)b * C::B_stage + (uint32_t)k * C::B_slot,
                         a.pan + ((size_t)s_op[e] * C::NCH + ch) * C::B_slot, C::B_slot, &bfull[b]);
            }
            const int pend = 1 + (int)(((g + (uint32_t)s) >> 1) & 1);
            if (b) bpend1 = pend; else bpend0 = pend;
        };
        // this thread's K values of stage s: [half*NVH, half*NVH + NVH), all
        // loads first (conversion and stores follow in store_stage)
        auto load_stage = [&](int s) {
#pragma unroll
            for (int k8 = 0; k8 < NVH; k8 += 8) {
                const int kidx = half * NVH + k8;
                const int k = kidx / C::KCH, cc = kidx % C::KCH;   // slot, first component in it
                const int u = s * C::ES + k;
                const int c0 = (u % C::NCH) * C::KCH + cc;
                if (live && u < nslot) {
                    const float* x = a.in + s_xoff[u / C::NCH] + (size_t)c0 * P2 + p;
                    if (c0 + 8 <= a.nc) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) v[k8 + q] = __ldg(x + (size_t)q * P2);
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) v[k8 + q] = c0 + q < a.nc ? __ldg(x + (size_t)q * P2) : 0.f;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[k8 + q] = 0.f;
                }
            }
        };
        auto store_stage = [&](int s, int b) {
            uint8_t* As = smem + (size_t)b * C::A_stage;
            const uint32_t rowoff = (uint32_t)(row >> 3) * C::SBO + (uint32_t)(row & 7) * 16u;
#pragma unroll
            for (int k8 = 0; k8 < NVH; k8 += 8) {
                const int kidx = half * NVH + k8;
                const int k = kidx / C::KCH, cc = kidx % C::KCH;
                if (s * C::ES + k < nslot)
                    put8<P>(As + (size_t)k * C::A_slot + rowoff + (uint32_t)((cc * C::esz) / 16) * C::LBO,
                            C::A_part, C::LBO, v + k8);
            }
        };
        auto flush = [&](int ab) {
            if (!has_cols) return;
            const uint32_t base = tmem + (uint32_t)(ab * C::setN + col0) + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
            for (int cc = 0; cc < NPH / 16; ++cc) {
                float r[16];
                tmem_ld16(base + (uint32_t)(cc * 16), r);
                if constexpr (F::dual) {
                    float w[16];
                    tmem_ld16(base + (uint32_t)NP + (uint32_t)(cc * 16), w);
#pragma unroll
                    for (int q = 0; q < 16; ++q) r[q] += w[q] * (1.f / kLo);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[cc * 16 + q] += r[q];
            }
        };
        auto wait_mma = [&](int b, uint32_t gs) {   // thread 0
            if (!mbar_wait_bounded(&mdone[b], (gs >> 1) & 1, kWaitT)) {
                abort_flag = 1;
            } else {
                if (b) mpend1 = 0; else mpend0 = 0;
            }
        };

        if (S > 0) {
            if (t == 0) issue_B(0, (int)(g & 1));
            load_stage(0);
        }
        bool aborted = false;
        for (int s = 0; s < S; ++s) {
            const uint32_t gs = g + (uint32_t)s;
            const int b = (int)(gs & 1);
            store_stage(s, b);
            fence_proxy_async();
            __syncthreads();
            if (*(volatile int*)&abort_flag) {
                aborted = true;
                break;
            }
            if (t == 0) {
                if (!mbar_wait_bounded(&bfull[b], (gs >> 1) & 1, kWaitT)) {
                    abort_flag = 1;
                } else {
                    if (b) bpend1 = 0; else bpend0 = 0;
                    fence_after_sync();
                    const int nvalid = min(C::ES, nslot - s * C::ES);
                    const int ab = C::ACCB == 2 ? b : 0;
                    issue_stage_mmas<P, NP>(sA + (uint32_t)b * C::A_stage, sB + (uint32_t)b * C::B_stage, nvalid,
                                            tmem + (uint32_t)(ab * C::setN));
                    mma_commit(&mdone[b]);
                    const int pend = 1 + (int)((gs >> 1) & 1);
                    if (b) mpend1 = pend; else mpend0 = pend;
                }
            }
            if (s + 1 < S) load_stage(s + 1);   // in flight during the MMA and the flush
            if constexpr (C::ACCB == 2) {
                if (s >= 1) {
                    if (t == 0 && !abort_flag) wait_mma(b ^ 1, gs - 1);
                    fence_before_sync();
                    __syncthreads();
                    if (*(volatile int*)&abort_flag) {
                        aborted = true;
                        break;
                    }
                    fence_after_sync();
                    flush(b ^ 1);
                    fence_before_sync();
                }
                if (s + 1 < S && t == 0 && !abort_flag) issue_B(s + 1, b ^ 1);
            } else {
                if (s + 1 < S && t == 0 && !abort_flag) issue_B(s + 1, b ^ 1);
                if (t == 0 && !abort_flag) wait_mma(b, gs);
                fence_before_sync();
                __syncthreads();
                if (*(volatile int*)&abort_flag) {
                    aborted = true;
                    break;
                }
                fence_after_sync();
                flush(0);
                fence_before_sync();
            }
        }
        if (!aborted && C::ACCB == 2 && S > 0) {
            const uint32_t gl = g + (uint32_t)(S - 1);
            const int bl = (int)(gl & 1);
            if (t == 0 && !abort_flag) wait_mma(bl, gl);
            fence_before_sync();
            __syncthreads();
            if (*(volatile int*)&abort_flag)
                aborted = true;
            else {
                fence_after_sync();
                flush(bl);
                fence_before_sync();
            }
        }
        if (aborted) break;
        g += (uint32_t)S;
        if (live && has_cols) {
            float* o = a.out + (size_t)(tgt - a.first_box) * boxstride + p;
            // every old value is read before the first store, so the reads
            // are all in flight together
            if (a.accumulate) {
#pragma unroll
                for (int q = 0; q < NPH; ++q)
                    if (col0 + q < a.nc) acc[q] += o[(size_t)(col0 + q) * P2];
            }
#pragma unroll
            for (int q = 0; q < NPH; ++q)
                if (col0 + q < a.nc) o[(size_t)(col0 + q) * P2] = acc[q];
        }
        __syncthreads();   // the edge table is rewritten by the next item
    }
    // leave: on an abort, wait (bounded) for this CTA's copies and MMAs in
    // flight before the shared memory and TMEM are given back
    if (t == 0 && abort_flag) {
        atomicExch(a.err, 1);
        if (bpend0) mbar_wait_bounded(&bfull[0], (uint32_t)(bpend0 - 1), kWaitT);
        if (bpend1) mbar_wait_bounded(&bfull[1], (uint32_t)(bpend1 - 1), kWaitT);
        if (mpend0) mbar_wait_bounded(&mdone[0], (uint32_t)(mpend0 - 1), kWaitT);
        if (mpend1) mbar_wait_bounded(&mdone[1], (uint32_t)(mpend1 - 1), kWaitT);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, C::tmem_cols);
}

// ---------------------------------------------------------------------------
// Slot pipeline.  With all three translations on the tensor core the
// multipoles and local expansions of the tree passes are kept in the tensor
// core's own operand layout ("slots"): for each box, pair tile (128 pairs)
// and chunk of KCH components, one A slot of 128 rows x KCH values in the
// K-major canonical layout, hi part then lo part.  A translation then moves
// only whole slots: one producer thread issues bulk asynchronous copies of
// the source slots and operator panels into a ring of shared-memory stages,
// one thread issues the MMAs, and eight warps (two per TMEM lane quarter,
// each owning half of the output columns) add each stage's accumulator into
// registers and finally write the target's slots (converting, and for L2L
// adding the old contents).  No thread touches an operand on the way in.
// Components past nc and rows past P are stored as zeros by every writer, so
// padded K columns never meet garbage.
// ---------------------------------------------------------------------------
struct SlotKArgs {
    int mode, P, ntile, first_box, tgt0, ntgt, accumulate;
    const int* ptr; const int* list; const int* opidx; const int* parent;
    const uint8_t* in; uint8_t* out; const uint8_t* pan; int* err;
};

template <int P, int NP>
struct SS {
    using C = TT<P, NP>;
    static constexpr int NS = NP >= 128 ? 3 : 4;                    // ring stages
    static constexpr uint32_t stage_bytes = C::A_stage + C::B_stage;
    static constexpr int smem = NS * (int)stage_bytes;
    static constexpr size_t tile_bytes = (size_t)C::NCH * C::A_slot;  // one pair tile of one box
    static constexpr uint32_t tmem_cols = (uint32_t)pow2ceil_i(2 * C::setN < 32 ? 32 : 2 * C::setN);
};

struct SlotState {
    uint64_t full[4], empty[4], accf[2], acce[2];
    uint32_t tmem;
    int abort;
    uint32_t gp, gm;   // stages issued by the producer, consumed by the MMA thread
};

__device__ __forceinline__ void slot_edge(const SlotKArgs& a, int tgt, int e0, int k, int& src, int& op) {
    if (a.mode == 0) {
        src = a.list[e0 + k];
        op = a.opidx[src];
    } else if (a.mode == 1) {
        src = a.list[e0 + k];
        op = a.opidx[e0 + k];
    } else {
        src = a.parent[tgt];
        op = a.opidx[tgt];
    }
}

__device__ __forceinline__ void slot_item(const SlotKArgs& a, long long it, int& pt, int& tgt, int& e0, int& ne) {
    pt = (int)(it / a.ntgt);
    tgt = a.tgt0 + (int)(it % a.ntgt);
    e0 = 0;
    ne = 1;
    if (a.mode != 2) {
        e0 = a.ptr[tgt];
        ne = a.ptr[tgt + 1] - e0;
    }
}

constexpr int kSlotThreads = 320;   // producer warp, MMA warp, 8 epilogue warps

template <int P, int NP>
__global__ void __launch_bounds__(kSlotThreads, 1)
k_tc_slot_translate(SlotKArgs a) {
    using C = TT<P, NP>;
    using S = SS<P, NP>;
    using F = Fmt<P>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ SlotState st;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 2) {
        tmem_alloc(&st.tmem, S::tmem_cols);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int r = 0; r < S::NS; ++r) {
            mbar_init(&st.full[r], 1);
            mbar_init(&st.empty[r], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&st.accf[b], 1);
            mbar_init(&st.acce[b], kSlotThreads - 64);
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
    auto ringA = [&](int r) { return sbase + (uint32_t)r * S::stage_bytes; };
    auto ringB = [&](int r) { return sbase + (uint32_t)r * S::stage_bytes + C::A_stage; };
    const long long nitems = (long long)a.ntgt * a.ntile;
    const size_t box_bytes = (size_t)a.ntile * S::tile_bytes;

    if (warp == 0) {
        if (lane == 0) {   // producer
            uint32_t g = 0;
            for (long long it = blockIdx.x; it < nitems && !*(volatile int*)&st.abort; it += gridDim.x) {
                int pt, tgt, e0, ne;
                slot_item(a, it, pt, tgt, e0, ne);
                const int nslot = ne * C::NCH, ns = (nslot + C::ES - 1) / C::ES;
                for (int s = 0; s < ns; ++s, ++g) {
                    const int r = (int)(g % S::NS);
                    if (g >= (uint32_t)S::NS && !mbar_wait_bounded(&st.empty[r], ((g / S::NS) - 1) & 1, kWaitT)) {
                        st.abort = 1;
                        break;
                    }
                    const int nvalid = min(C::ES, nslot - s * C::ES);
                    mbar_expect_tx(&st.full[r], (uint32_t)nvalid * (C::A_slot + C::B_slot));
                    for (int k = 0; k < nvalid; ++k) {
                        const int u = s * C::ES + k, e = u / C::NCH, ch = u % C::NCH;
                        int src, op;
                        slot_edge(a, tgt, e0, e, src, op);
                        bulk_g2s(ringA(r) + (uint32_t)k * C::A_slot,
                                 a.in + (size_t)(src - a.first_box) * box_bytes + (size_t)pt * S::tile_bytes +
                                     (size_t)ch * C::A_slot,
                                 C::A_slot, &st.full[r]);
                        bulk_g2s(ringB(r) + (uint32_t)k * C::B_slot, a.pan + ((size_t)op * C::NCH + ch) * C::B_slot,
                                 C::B_slot, &st.full[r]);
                    }
                    st.gp = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issue
            uint32_t g = 0;
            for (long long it = blockIdx.x; it < nitems && !*(volatile int*)&st.abort; it += gridDim.x) {
                int pt, tgt, e0, ne;
                slot_item(a, it, pt, tgt, e0, ne);
                const int nslot = ne * C::NCH, ns = (nslot + C::ES - 1) / C::ES;
                for (int s = 0; s < ns; ++s, ++g) {
                    const int r = (int)(g % S::NS), b = (int)(g & 1);
                    if (!mbar_wait_bounded(&st.full[r], (g / S::NS) & 1, kWaitT) ||
                        (g >= 2 && !mbar_wait_bounded(&st.acce[b], ((g >> 1) - 1) & 1, kWaitT))) {
                        st.abort = 1;
                        break;
                    }
                    fence_after_sync();
                    const int nvalid = min(C::ES, nslot - s * C::ES);
                    issue_stage_mmas<P, NP>(ringA(r), ringB(r), nvalid, tmem + (uint32_t)(b * C::setN));
                    mma_commit(&st.empty[r]);
                    mma_commit(&st.accf[b]);
                    st.gm = g + 1;
                }
                if (*(volatile int*)&st.abort) break;
            }
            // the last MMAs must be complete before TMEM is given back
            const uint32_t gl = st.gm;
            if (gl > 0) mbar_wait_bounded(&st.accf[(gl - 1) & 1], ((gl - 1) >> 1) & 1, kWaitT);
        }
    } else {   // warps 2..9: accumulate stages, write the target's slots
        // TMEM lane quarter of this warp (warp w may read lanes 32 (w % 4)..),
        // and which half of the output columns it owns (N >= 32)
        const int row = (warp & 3) * 32 + lane, half = (warp - 2) >> 2;
        constexpr int NPH = NP >= 32 ? NP / 2 : NP;
        const bool has_cols = half < NP / NPH;
        const int col0 = half * NPH;
        const uint32_t rowoff = (uint32_t)(row >> 3) * C::SBO + (uint32_t)(row & 7) * 16u;
        uint32_t g = 0;
        float acc[NPH];
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
            int pt, tgt, e0, ne;
            slot_item(a, it, pt, tgt, e0, ne);
            const int nslot = ne * C::NCH, ns = (nslot + C::ES - 1) / C::ES;
#pragma unroll
            for (int q = 0; q < NPH; ++q) acc[q] = 0.f;
            bool ok = true;
            for (int s = 0; s < ns; ++s, ++g) {
                const int b = (int)(g & 1);
                if (*(volatile int*)&st.abort || !mbar_wait_bounded(&st.accf[b], (g >> 1) & 1, kWaitT)) {
                    st.abort = 1;
                    ok = false;
                    break;
                }
                fence_after_sync();
                if (has_cols) {
                    const uint32_t base =
                        tmem + (uint32_t)(b * C::setN + col0) + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
                    for (int cc = 0; cc < NPH / 16; ++cc) {
                        float v[16];
                        tmem_ld16(base + (uint32_t)(cc * 16), v);
                        if constexpr (F::dual) {
                            float w[16];
                            tmem_ld16(base + (uint32_t)NP + (uint32_t)(cc * 16), w);
#pragma unroll
                            for (int q = 0; q < 16; ++q) v[q] += w[q] * (1.f / kLo);
                        }
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[cc * 16 + q] += v[q];
                    }
                }
                fence_before_sync();
                mbar_arrive(&st.acce[b]);
            }
            if (!ok) break;
            if (!has_cols) continue;
            uint8_t* dst = a.out + (size_t)(tgt - a.first_box) * box_bytes + (size_t)pt * S::tile_bytes + rowoff;
            auto chunk = [&](int k8) {   // 8 columns col0 + k8 .. : never straddle a K chunk
                const int c = col0 + k8, ch = c / C::KCH, cc = c % C::KCH;
                return dst + (size_t)ch * C::A_slot + (uint32_t)((cc * C::esz) / 16) * C::LBO;
            };
            if (a.accumulate) {   // every old value is read before the first store
#pragma unroll
                for (int k8 = 0; k8 < NPH; k8 += 8) {
                    float o[8];
                    get8<P>(chunk(k8), C::A_part, C::LBO, o);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[k8 + q] += o[q];
                }
            }
#pragma unroll
            for (int k8 = 0; k8 < NPH; k8 += 8) put8<P>(chunk(k8), C::A_part, C::LBO, acc + k8);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (t == 0 && st.abort) {
        atomicExch(a.err, 1);
        // copies issued but never consumed: wait (bounded) until they land
        for (uint32_t g = st.gm; g < st.gp; ++g) mbar_wait_bounded(&st.full[g % S::NS], (g / S::NS) & 1, kWaitT);
    }
    __syncthreads();
    fence_after_sync();
    if (warp == 2) tmem_dealloc(tmem, S::tmem_cols);
}

// FP32 [box][nc][P] <-> slots, one thread per (box, pair tile, row); padding
// (components past nc, rows past P) is written as zeros.
template <int P, int NP>
__global__ void k_slots_pack(const float* __restrict__ X, int nc, int Ppairs, int ntile, int box0,
                             uint8_t* __restrict__ slots) {
    using C = TT<P, NP>;
    using S = SS<P, NP>;
    const int pt = blockIdx.x, box = box0 + blockIdx.y, row = threadIdx.x;
    const int p = pt * 128 + row;
    const uint32_t rowoff = (uint32_t)(row >> 3) * C::SBO + (uint32_t)(row & 7) * 16u;
    uint8_t* dst = slots + (size_t)box * ntile * S::tile_bytes + (size_t)pt * S::tile_bytes + rowoff;
    const float* x = X + (size_t)box * nc * Ppairs + p;
    for (int ch = 0; ch < C::NCH; ++ch) {
        for (int k8 = 0; k8 < C::KCH; k8 += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = ch * C::KCH + k8 + q;
                v[q] = (p < Ppairs && c < nc) ? x[(size_t)c * Ppairs] : 0.f;
            }
            put8<P>(dst + (size_t)ch * C::A_slot + (uint32_t)((k8 * C::esz) / 16) * C::LBO, C::A_part, C::LBO, v);
        }
    }
}

template <int P, int NP>
__global__ void k_slots_unpack(const uint8_t* __restrict__ slots, int nc, int Ppairs, int ntile, int box0,
                               float* __restrict__ X) {
    using C = TT<P, NP>;
    using S = SS<P, NP>;
    const int pt = blockIdx.x, box = box0 + blockIdx.y, row = threadIdx.x;
    const int p = pt * 128 + row;
    if (p >= Ppairs) return;
    const uint32_t rowoff = (uint32_t)(row >> 3) * C::SBO + (uint32_t)(row & 7) * 16u;
    const uint8_t* src = slots + (size_t)box * ntile * S::tile_bytes + (size_t)pt * S::tile_bytes + rowoff;
    float* x = X + (size_t)box * nc * Ppairs + p;
    for (int ch = 0; ch < C::NCH; ++ch) {
        for (int k8 = 0; k8 < C::KCH; k8 += 8) {
            float v[8];
            get8<P>(src + (size_t)ch * C::A_slot + (uint32_t)((k8 * C::esz) / 16) * C::LBO, C::A_part, C::LBO, v);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = ch * C::KCH + k8 + q;
                if (c < nc) x[(size_t)c * Ppairs] = v[q];
            }
        }
    }
}

template <int P, int NP>
cudaError_t slot_translate_typed(const SlotArgs& h, int mode, int tgt0, int ntgt, const int* ptr, const int* list,
                                 const int* opidx, const uint8_t* in, uint8_t* out, int accumulate,
                                 cudaStream_t s) {
    using S = SS<P, NP>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_slot_translate<P, NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, S::smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (ntgt <= 0) return cudaSuccess;
    SlotKArgs a{};
    a.mode = mode; a.P = h.P; a.ntile = h.ntile; a.first_box = h.first_box; a.tgt0 = tgt0; a.ntgt = ntgt;
    a.accumulate = accumulate;
    a.ptr = ptr; a.list = list; a.opidx = opidx; a.parent = h.parent;
    a.in = in; a.out = out; a.pan = h.pan; a.err = h.err;
    const long long items = (long long)ntgt * h.ntile;
    const int grid = (int)(items < h.sm_count ? items : h.sm_count);   // one CTA per SM (TMEM, shared memory)
    k_tc_slot_translate<P, NP><<<grid, kSlotThreads, S::smem, s>>>(a);
    return cudaGetLastError();
}

template <int P, int NP>
cudaError_t tr_typed(const TrArgs& h, int mode, int tgt0, int ntgt, const int* ptr, const int* list,
                     const int* opidx, const float* in, float* out, int accumulate, cudaStream_t s) {
    using C = TT<P, NP>;
    static int bps = 0, smem_req = 0;
    if (!bps) {
        // CTAs per SM bounded by TMEM (512 columns); the dynamic shared memory
        // request is raised so that the hardware never places more than that
        const int tmem_bound = 512 / (int)C::tmem_cols;
        int occ = 0;
        cudaError_t e = cudaFuncSetAttribute(k_tc_translate<P, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_translate<P, NP>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tc_translate<P, NP>, 128 * tpr<NP>(), C::smem);
        if (e != cudaSuccess) return e;
        int req = C::smem;
        if (occ > tmem_bound) {
            req = (233472 / tmem_bound) - 2048;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tc_translate<P, NP>, 128 * tpr<NP>(), req);
            if (e != cudaSuccess) return e;
        }
        if (occ < 1) return cudaErrorInvalidConfiguration;
        bps = occ < tmem_bound ? occ : tmem_bound;
        smem_req = req;
    }
    if (ntgt <= 0) return cudaSuccess;
    TrKArgs a{};
    a.mode = mode;
    a.P = h.P; a.nc = h.nc; a.first_box = h.first_box; a.tgt0 = tgt0; a.ntgt = ntgt;
    a.accumulate = accumulate; a.nlev = h.nlev;
    a.ptr = ptr; a.list = list; a.opidx = opidx; a.parent = h.parent; a.box_level = h.box_level;
    a.in = in; a.out = out;
    a.pan = h.pan; a.err = h.err;
    const long long items = (long long)ntgt * ((h.P + 127) / 128);
    const long long cap = (long long)h.sm_count * bps;
    const int grid = (int)(items < cap ? items : cap);
    k_tc_translate<P, NP><<<grid, 128 * tpr<NP>(), smem_req, s>>>(a);
    return cudaGetLastError();
}

template <int P, int NP>
cudaError_t op_panels_typed(const double* ops, int nops, int nc, const int* opinfo, const double* scd, int nlev,
                            uint8_t* pan, cudaStream_t s) {
    if (nops <= 0) return cudaSuccess;
    k_tr_op_panels<P, NP><<<dim3(nops, TT<P, NP>::NCH), 256, 0, s>>>(ops, nops, nc, opinfo, scd, nlev, pan);
    return cudaGetLastError();
}

}  // namespace

int tr_np(int nc) {
    int np = 16;
    while (np < nc) np *= 2;
    return np <= 128 ? np : 0;
}

size_t tr_panel_bytes(int prec, int nc) {
    const int np = tr_np(nc);
    const int m = tc_mode(prec);
    if (!np || m < 0) return 0;
    const int esz = m == Q_TF32 ? 4 : 2;
    const int parts = (m == Q_BF16X3 || m == Q_FP16X3) ? 2 : 1;
    return (size_t)np * np * esz * parts;   // NCH chunks x NP x KCH = NP x NP elements per operator
}

#define OCCK_TR_DISPATCH(prec, np, call)                                                        \
    do {                                                                                        \
        switch (tc_mode(prec)) {                                                                \
            case Q_BF16: { constexpr int P = Q_BF16; OCCK_TR_NP(np, call); }                    \
            case Q_FP16: { constexpr int P = Q_FP16; OCCK_TR_NP(np, call); }                    \
            case Q_TF32: { constexpr int P = Q_TF32; OCCK_TR_NP(np, call); }                    \
            case Q_BF16X3: { constexpr int P = Q_BF16X3; OCCK_TR_NP(np, call); }                \
            case Q_FP16X3: { constexpr int P = Q_FP16X3; OCCK_TR_NP(np, call); }                \
            default: return cudaErrorInvalidValue;                                              \
        }                                                                                       \
    } while (0)
#define OCCK_TR_NP(np, call)                                     \
    switch (np) {                                                \
        case 16: { constexpr int NP = 16; return call; }         \
        case 32: { constexpr int NP = 32; return call; }         \
        case 64: { constexpr int NP = 64; return call; }         \
        case 128: { constexpr int NP = 128; return call; }       \
        default: return cudaErrorInvalidValue;                   \
    }

cudaError_t tr_build_panels(int prec, const double* ops, int nops, int nc, const int* opinfo, const double* scd,
                            int nlev, uint8_t* pan, float* ops_scaled, cudaStream_t s) {
    const int np = tr_np(nc);
    if (nops > 0) {
        k_tr_ops_scaled<<<nops, 256, 0, s>>>(ops, nops, nc, opinfo, scd, nlev, ops_scaled);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    OCCK_TR_DISPATCH(prec, np, (op_panels_typed<P, NP>(ops, nops, nc, opinfo, scd, nlev, pan, s)));
    return cudaErrorInvalidValue;
}

cudaError_t tr_translate(int prec, const TrArgs& h, int mode, int tgt0, int ntgt, const int* ptr, const int* list,
                         const int* opidx, const float* in, float* out, int accumulate, cudaStream_t s) {
    const int np = tr_np(h.nc);
    OCCK_TR_DISPATCH(prec, np, (tr_typed<P, NP>(h, mode, tgt0, ntgt, ptr, list, opidx, in, out, accumulate, s)));
    return cudaErrorInvalidValue;
}

size_t tr_slot_box_bytes(int prec, int nc, int ntile) {
    const int np = tr_np(nc);
    const int m = tc_mode(prec);
    if (!np || m < 0) return 0;
    const int esz = m == Q_TF32 ? 4 : 2;
    const int parts = (m == Q_BF16X3 || m == Q_FP16X3) ? 2 : 1;
    return (size_t)ntile * 128 * np * esz * parts;
}

cudaError_t tr_slot_translate(int prec, const SlotArgs& h, int mode, int tgt0, int ntgt, const int* ptr,
                              const int* list, const int* opidx, const uint8_t* in, uint8_t* out, int accumulate,
                              cudaStream_t s) {
    const int np = tr_np(h.nc);
    OCCK_TR_DISPATCH(prec, np,
                     (slot_translate_typed<P, NP>(h, mode, tgt0, ntgt, ptr, list, opidx, in, out, accumulate, s)));
    return cudaErrorInvalidValue;
}

template <int P, int NP>
static cudaError_t pack_typed(bool pack, const float* X, float* Xo, int nc, int Ppairs, int ntile, int box0,
                              int nbox, const uint8_t* sin, uint8_t* sout, cudaStream_t s) {
    if (nbox <= 0) return cudaSuccess;
    dim3 g(ntile, nbox);
    if (pack)
        k_slots_pack<P, NP><<<g, 128, 0, s>>>(X, nc, Ppairs, ntile, box0, sout);
    else
        k_slots_unpack<P, NP><<<g, 128, 0, s>>>(sin, nc, Ppairs, ntile, box0, Xo);
    return cudaGetLastError();
}

cudaError_t tr_slots_pack(int prec, int nc, const float* X, int Ppairs, int ntile, int box0, int nbox,
                          uint8_t* slots, cudaStream_t s) {
    const int np = tr_np(nc);
    OCCK_TR_DISPATCH(prec, np,
                     (pack_typed<P, NP>(true, X, nullptr, nc, Ppairs, ntile, box0, nbox, nullptr, slots, s)));
    return cudaErrorInvalidValue;
}

cudaError_t tr_slots_unpack(int prec, int nc, const uint8_t* slots, int Ppairs, int ntile, int box0, int nbox,
                            float* X, cudaStream_t s) {
    const int np = tr_np(nc);
    OCCK_TR_DISPATCH(prec, np,
                     (pack_typed<P, NP>(false, nullptr, X, nc, Ppairs, ntile, box0, nbox, slots, nullptr, s)));
    return cudaErrorInvalidValue;
}

}  // namespace occk
