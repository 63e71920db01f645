// Steps (a), (c), (e) on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators), for the mixed-precision forms of the far-field exchange.
//
// Data stay FP32 in HBM.  Each CTA (128 threads) stages operand tiles into
// shared memory in the K-major canonical layout, converting on the fly to
// BF16, FP16 or TF32 -- and, for the split forms, into hi + lo parts whose
// three products hi*hi + hi*lo + lo*hi recover most of the FP32 digits.  One
// thread issues tcgen05.mma (M = 128) into a TMEM accumulator and commits to
// an mbarrier per stage; two stages double-buffer the loads against the MMAs.
// Every wait is bounded and records an error word instead of hanging.
//
// Per-level scaling: component l of a multipole is divided by s^l and of a
// local expansion multiplied by s^(l+1) (s = box side of the level) before it
// enters a low-precision format, so every operand is O(1) and the FP16 range
// is never left; the scale is undone in FP32 in the epilogue.
//
//   (a) O[B][lm][i][j] = sum_r C_ri W[lm][r][j]            A = C_S^T, B = W^T
//   (e) KB[r][i] = sum_lm w_lm sum_j W[lm][r][j] M[B][lm][i][j]
//   (c) M[t][lm][p] = sum_src sum_c T_src[lm][c] O[src][c][p]   A = O^T, B = T
#include <cstdio>

#include "occk_internal.h"
#include "tc.cuh"

namespace occk {

int tc_mode(int prec);

namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kRowBytes = 128;                 // bytes of one operand row per stage
constexpr uint32_t kLBO = 128;                 // K-adjacent core matrices
constexpr uint32_t kSBO = 8 * 128;             // 8-row groups
constexpr uint32_t kWaitLimit = 1u << 24;      // bounded mbarrier polls

enum PM { PM_BF16 = 0, PM_FP16 = 1, PM_TF32 = 2, PM_BF16X3 = 3, PM_FP16X3 = 4 };

template <int P>
struct PrecT {
    static constexpr bool split = (P == PM_BF16X3 || P == PM_FP16X3);
    static constexpr int esz = (P == PM_TF32) ? 4 : 2;
    static constexpr int BK = kRowBytes / esz;       // elements per row per stage
    static constexpr int KSTEP = (P == PM_TF32) ? 8 : 16;
    static constexpr int EPC = 16 / esz;             // elements per 16-byte chunk
    static constexpr uint32_t fmt = (P == PM_BF16 || P == PM_BF16X3) ? 1u : (P == PM_TF32 ? 2u : 0u);
    // FP16 lo parts are stored scaled by 2^11 (they would otherwise fall into
    // FP16 subnormals) and accumulate in a second TMEM accumulator that the
    // epilogue adds back with weight 2^-11
    static constexpr bool dual = (P == PM_FP16X3);
};
constexpr float kLoScale = 2048.f;

// rank l of real-form component index c = l*l + ...
__device__ __forceinline__ int lrank(int c) {
    int l = (int)sqrtf((float)c);
    while (l * l > c) --l;
    while ((l + 1) * (l + 1) <= c) ++l;
    return l;
}

__device__ __forceinline__ uint32_t tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Store one 16-byte chunk of a row (EPC values) into the hi (and lo) tile.
template <int P>
__device__ __forceinline__ void put_chunk(uint8_t* hi, uint8_t* lo, int row, int chunk, const float* v) {
    const uint32_t off = (uint32_t)(row >> 3) * kSBO + (uint32_t)chunk * kLBO + (uint32_t)(row & 7) * 16u;
    if constexpr (P == PM_TF32) {
        uint4 h;
        h.x = tf32_round(v[0]);
        h.y = tf32_round(v[1]);
        h.z = tf32_round(v[2]);
        h.w = tf32_round(v[3]);
        *reinterpret_cast<uint4*>(hi + off) = h;
    } else {
        using S = typename std::conditional<(P == PM_BF16 || P == PM_BF16X3), SplitBF16, SplitFP16>::type;
        typename S::T h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if constexpr (PrecT<P>::dual) {
                h[q] = __float2half_rn(v[q]);
                l[q] = __float2half_rn((v[q] - __half2float(h[q])) * kLoScale);
            } else {
                S::split(v[q], h[q], l[q]);
            }
        }
        *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<uint4*>(h);
        if constexpr (PrecT<P>::split) *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<uint4*>(l);
    }
}

// Shared-memory plan: per stage A_hi, A_lo, B_hi, B_lo tiles of 128 rows.
template <int P>
struct Smem {
    static constexpr int tile = 128 * kRowBytes;                     // 16 KB
    static constexpr int per_stage = tile * (PrecT<P>::split ? 4 : 2);
    static constexpr int stages = 2;
    static constexpr int bytes = per_stage * stages;
};

struct EngineState {
    uint64_t bar[2];
    uint32_t tmem;
    int err;
};

// Issue the MMAs of one stage (called by one thread).
template <int P>
__device__ __forceinline__ void issue_stage(uint8_t* stage, uint32_t tmem, uint32_t idesc, bool first, int N) {
    constexpr int T = Smem<P>::tile;
    const uint32_t a_hi = smem_u32(stage), b_hi = smem_u32(stage + T);
    const uint32_t a_lo = smem_u32(stage + 2 * T), b_lo = smem_u32(stage + 3 * T);
    constexpr int nks = PrecT<P>::BK / PrecT<P>::KSTEP;
#pragma unroll
    for (int ks = 0; ks < nks; ++ks) {
        const uint32_t adv = (uint32_t)ks * 2u * kLBO;   // two core matrices per K step
        const uint64_t dah = smem_desc(a_hi + adv, kLBO, kSBO), dbh = smem_desc(b_hi + adv, kLBO, kSBO);
        const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
        if constexpr (P == PM_TF32) {
            mma_tf32(tmem, dah, dbh, idesc, acc0);
        } else {
            mma_f16(tmem, dah, dbh, idesc, acc0);
            if constexpr (PrecT<P>::split) {
                const uint64_t dal = smem_desc(a_lo + adv, kLBO, kSBO), dbl = smem_desc(b_lo + adv, kLBO, kSBO);
                const uint32_t t2 = PrecT<P>::dual ? tmem + (uint32_t)N : tmem;
                mma_f16(t2, dah, dbl, idesc, PrecT<P>::dual ? acc0 : 1u);
                mma_f16(t2, dal, dbh, idesc, 1u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The engine: K loop over stages with a Mode policy providing the row values.
//   Mode::nchunks(ctx)                         number of K stages
//   Mode::fill(ctx, kc, t, k0, a[8], b[8], &hasb)  elements k0..k0+7 of row t
//                                              of A and B in stage kc
//   Mode::epilogue(ctx, warp, lane, tmem, valid)
// ---------------------------------------------------------------------------
// Add the accumulator buffer at `base` (this warp's 32 lanes, N columns) to
// the thread's FP32 registers; the dual form adds its scaled second half.
template <int P, int N>
__device__ __forceinline__ void flush_acc(uint32_t base, int warp, float* acc) {
#pragma unroll
    for (int cc = 0; cc < N / 16; ++cc) {
        float v[16];
        tmem_ld16(base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 16), v);
        if constexpr (PrecT<P>::dual) {
            float w[16];
            tmem_ld16(base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(N + cc * 16), w);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] += w[q] * (1.f / kLoScale);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[cc * 16 + q] += v[q];
    }
}

// The tensor core accumulates in FP32 with a bias toward zero that grows with
// the number of products in one accumulation chain (about -2e-5 relative at
// K = 4096).  So every stage (64 K elements of 16-bit, 32 of TF32) starts a
// fresh accumulator in one of two TMEM buffers, and while the next stage's MMAs
// run, the threads add the finished buffer into FP32 registers (round to
// nearest): the chain never exceeds one stage.
template <int P, int N, class Mode>
__device__ __forceinline__ void engine(typename Mode::Ctx& c, int* err_word) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ EngineState st;
    constexpr int BK = PrecT<P>::BK, EPC = PrecT<P>::EPC;
    static_assert(8 % EPC == 0, "chunk");
    static_assert(N % 16 == 0 && N <= 128, "N");
    constexpr uint32_t kBuf = (uint32_t)N * (PrecT<P>::dual ? 2u : 1u);   // columns per buffer
    constexpr uint32_t kCols = (2 * kBuf <= 32) ? 32u : (2 * kBuf <= 64 ? 64u : (2 * kBuf <= 128 ? 128u : (2 * kBuf <= 256 ? 256u : 512u)));
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 0) {
        tmem_alloc(&st.tmem, kCols);
        tmem_relinquish();
    }
    if (t == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        mbar_fence_init();
        st.err = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = st.tmem;
    const uint32_t idesc = instr_desc(128, N, PrecT<P>::fmt);
    const int nk = Mode::nchunks(c);
    float acc[N];
#pragma unroll
    for (int q = 0; q < N; ++q) acc[q] = 0.f;
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc & 1;
        uint8_t* stage = smem + s * Smem<P>::per_stage;
        if (kc >= 2) {
            if (!mbar_wait_bounded(&st.bar[s], ((kc - 2) >> 1) & 1, kWaitLimit)) ok = false;
        }
        uint8_t* a_hi = stage;
        uint8_t* b_hi = stage + Smem<P>::tile;
        uint8_t* a_lo = stage + 2 * Smem<P>::tile;
        uint8_t* b_lo = stage + 3 * Smem<P>::tile;
        for (int k8 = 0; k8 < BK / 8; ++k8) {
            float a[8], b[8];
            bool hasb = false;
            Mode::fill(c, kc, t, k8 * 8, a, b, hasb);
#pragma unroll
            for (int h = 0; h < 8 / EPC; ++h) {
                put_chunk<P>(a_hi, a_lo, t, k8 * (8 / EPC) + h, a + h * EPC);
                if (hasb) put_chunk<P>(b_hi, b_lo, t, k8 * (8 / EPC) + h, b + h * EPC);
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (t == 0) {
            fence_after_sync();
            issue_stage<P>(stage, tmem + (uint32_t)(kc & 1) * kBuf, idesc, true, N);
            mma_commit(&st.bar[s]);
        }
        if (kc >= 1) {   // flush the previous stage's buffer while this stage's MMAs run
            const int pk = kc - 1;
            if (!mbar_wait_bounded(&st.bar[pk & 1], (pk >> 1) & 1, kWaitLimit)) ok = false;
            fence_after_sync();
            if (ok) flush_acc<P, N>(tmem + (uint32_t)(pk & 1) * kBuf, warp, acc);
            fence_before_sync();
        }
    }
    if (nk > 0) {
        const int pk = nk - 1;
        if (!mbar_wait_bounded(&st.bar[pk & 1], (pk >> 1) & 1, kWaitLimit)) ok = false;
        fence_after_sync();
        if (ok) flush_acc<P, N>(tmem + (uint32_t)(pk & 1) * kBuf, warp, acc);
    }
    if (!ok) atomicExch(&st.err, 1);
    fence_before_sync();
    __syncthreads();
    if (st.err) {
        if (t == 0) atomicExch(err_word, 1);
    } else {
        Mode::template epilogue<N>(c, warp, lane, acc, nk > 0);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ===========================================================================
// Step (a): O[B][lm][i][j] = sum_r C_ri W[lm][r][j]
// ===========================================================================
struct A2Args {
    const int* leaf_rowoff; const int* leaf_aos; const float* Ct; const float* W;
    int nocc, nrow, nc, ntile, leaf_store0;
    const float* lscale;     // [nc] 1/s^l for the leaf level
    float* Obox;
};

template <int P>
struct ModeA2 {
    struct Ctx {
        const A2Args* a;
        int B, lm, ti, tj, rb0, nr;
    };
    __device__ static int nchunks(const Ctx& c) { return (c.nr + PrecT<P>::BK - 1) / PrecT<P>::BK; }
    __device__ static void fill(const Ctx& c, int kc, int t, int k0, float* a, float* b, bool& hasb) {
        constexpr int BK = PrecT<P>::BK;
        const A2Args& A = *c.a;
        const int i = c.ti * 128 + t, j = c.tj * 128 + t;
        const float sc = A.lscale[c.lm];
        const float* Wl = A.W + ((size_t)c.lm * A.nrow + c.rb0) * A.nocc;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = kc * BK + k0 + k;
            const bool rv = r < c.nr;
            a[k] = (rv && i < A.nocc) ? A.Ct[(size_t)A.leaf_aos[c.rb0 + r] * A.nocc + i] : 0.f;
            b[k] = (rv && j < A.nocc) ? Wl[(size_t)r * A.nocc + j] * sc : 0.f;
        }
        hasb = true;
    }
    template <int N>
    __device__ static void epilogue(const Ctx& c, int warp, int lane, const float* acc, bool valid) {
        const A2Args& A = *c.a;
        const size_t P2 = (size_t)A.nocc * (A.nocc + 1) / 2;   // stored pairs i <= j
        float* O = A.Obox + ((size_t)(A.leaf_store0 + c.B) * A.nc + c.lm) * P2;
        const float inv = 1.0f / A.lscale[c.lm];
        const int i = c.ti * 128 + warp * 32 + lane;
#pragma unroll
        for (int cc = 0; cc < N / 16; ++cc) {
            const float* v = acc + cc * 16;
            if (i < A.nocc) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = c.tj * 128 + cc * 16 + q;
                    if (j < A.nocc && j >= i)
                        O[(size_t)i * (2 * A.nocc - i + 1) / 2 + (j - i)] = valid ? v[q] * inv : 0.f;
                }
            }
        }
    }
};

template <int P>
__global__ void __launch_bounds__(kThreads) k_tc_a2(A2Args args, int* err) {
    typename ModeA2<P>::Ctx c;
    c.a = &args;
    c.B = blockIdx.y / args.nc;
    c.lm = blockIdx.y - c.B * args.nc;
    int tt = blockIdx.x, ti = 0;
    while (tt >= args.ntile - ti) {
        tt -= args.ntile - ti;
        ++ti;
    }
    c.ti = ti;
    c.tj = ti + tt;
    c.rb0 = args.leaf_rowoff[c.B];
    c.nr = args.leaf_rowoff[c.B + 1] - c.rb0;
    engine<P, 128, ModeA2<P>>(c, err);
}

// ===========================================================================
// Step (e): KB[rowoff + r][i] = 2 sum_lm w_lm sum_j W[lm][r][j] M[leaf][lm][i][j]
// ===========================================================================
struct L2PArgs {
    const int* leaf_rowoff; const float* W; const float* Mbox;
    int nocc, nrow, nc, leaf_store0;
    const float* lscale;     // [nc] 1/s^l for the leaf level
    double* KB;
};

template <int P>
struct ModeL2P {
    struct Ctx {
        const L2PArgs* a;
        int B, r0, i0, rb0, nr, kpl;   // kpl: K stages per lm
    };
    __device__ static int nchunks(const Ctx& c) { return c.kpl * c.a->nc; }
    __device__ static void fill(const Ctx& c, int kc, int t, int k0, float* a, float* b, bool& hasb) {
        constexpr int BK = PrecT<P>::BK;
        const L2PArgs& A = *c.a;
        const int lm = kc / c.kpl, j0 = (kc - lm * c.kpl) * BK + k0;
        int l = 0;
        while ((l + 1) * (l + 1) <= lm) ++l;
        const float w = (lm == l * l) ? 2.f : (((lm - l * l) & 1) ? 4.f : -4.f);
        const float sa = A.lscale[lm], sb = w / A.lscale[lm];
        const int r = c.r0 + t, i = c.i0 + t;
        const float* Wr = A.W + ((size_t)lm * A.nrow + c.rb0 + r) * A.nocc;
        const size_t P2 = (size_t)A.nocc * (A.nocc + 1) / 2;
        const float* Ml = A.Mbox + ((size_t)(A.leaf_store0 + c.B) * A.nc + lm) * P2;
        const bool rv = r < c.nr, iv = i < A.nocc;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = j0 + k;
            const bool jv = j < A.nocc;
            a[k] = (rv && jv) ? Wr[j] * sa : 0.f;
            // Mcal^{ij} from the packed upper triangle
            const int lo = i < j ? i : j, hi = i < j ? j : i;
            b[k] = (iv && jv) ? Ml[(size_t)lo * (2 * A.nocc - lo + 1) / 2 + (hi - lo)] * sb : 0.f;
        }
        hasb = true;
    }
    template <int N>
    __device__ static void epilogue(const Ctx& c, int warp, int lane, const float* acc, bool valid) {
        const L2PArgs& A = *c.a;
        const int r = c.r0 + warp * 32 + lane;
#pragma unroll
        for (int cc = 0; cc < N / 16; ++cc) {
            const float* v = acc + cc * 16;
            if (r < c.nr) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int i = c.i0 + cc * 16 + q;
                    if (i < A.nocc) A.KB[(size_t)(c.rb0 + r) * A.nocc + i] = valid ? (double)v[q] : 0.0;
                }
            }
        }
    }
};

template <int P>
__global__ void __launch_bounds__(kThreads) k_tc_l2p(L2PArgs args, int* err) {
    typename ModeL2P<P>::Ctx c;
    c.a = &args;
    c.B = blockIdx.z;
    c.rb0 = args.leaf_rowoff[c.B];
    c.nr = args.leaf_rowoff[c.B + 1] - c.rb0;
    c.r0 = blockIdx.x * 128;
    c.i0 = blockIdx.y * 128;
    c.kpl = (args.nocc + PrecT<P>::BK - 1) / PrecT<P>::BK;
    if (c.r0 >= c.nr) return;   // uniform per block
    engine<P, 128, ModeL2P<P>>(c, err);
}

// ===========================================================================
// Step (c): M[t][lm][p] = sum_src sum_c T_src[lm][c] O[src][c][p]
// ===========================================================================
struct M2LArgs {
    int P, nc, L, first_box, tgt0;
    const int* ptr; const int* src; const int* op; const int* lmax_e;
    const float* ops;        // [nops][nc][nc] FP32 operators
    const float* O;          // [box][nc][P]
    float* M;
    const float* box_scale;  // [nbox] side of the box's level
};

template <int P>
struct ModeM2L {
    struct Ctx {
        const M2LArgs* a;
        int tgt, p0, e0, e1, nchunk_src, N;
        float spow[16];      // s^k, s = side of the target level
        float inv_spow[16];
    };
    __device__ static int nchunks(const Ctx& c) { return (c.e1 - c.e0) * c.nchunk_src; }
    __device__ static void fill(const Ctx& c, int kc, int t, int k0, float* a, float* b, bool& hasb) {
        constexpr int BK = PrecT<P>::BK;
        const M2LArgs& A = *c.a;
        const int e = c.e0 + kc / c.nchunk_src, kb = (kc % c.nchunk_src) * BK + k0;
        const int src = A.src[e];
        const int Le = A.lmax_e ? A.lmax_e[e] : A.L;
        const int ncr = (Le + 1) * (Le + 1);
        const float* Os = A.O + (size_t)(src - A.first_box) * A.nc * A.P;
        const int p = c.p0 + t;
        const bool pv = p < A.P;
        // A(p, col) = O[src][col][p] / s^l'
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int col = kb + k;
            a[k] = (pv && col < ncr) ? Os[(size_t)col * A.P + p] * c.inv_spow[lrank(col)] : 0.f;
        }
        // B(n, col) = T[n][col] s^l' s^(l_n + 1), rows n = output components
        hasb = t < c.N;
        if (hasb) {
            const int n = t;
            const float* Tm = A.ops + (size_t)A.op[e] * A.nc * A.nc + (size_t)n * A.nc;
            const float sn = c.spow[lrank(n) + 1];
            const bool nv = n < ncr;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int col = kb + k;
                b[k] = (nv && col < ncr) ? Tm[col] * c.spow[lrank(col)] * sn : 0.f;
            }
        }
    }
    template <int N>
    __device__ static void epilogue(const Ctx& c, int warp, int lane, const float* acc, bool valid) {
        const M2LArgs& A = *c.a;
        const int p = c.p0 + warp * 32 + lane;
        float* Mt = A.M + (size_t)(c.tgt - A.first_box) * A.nc * A.P;
#pragma unroll
        for (int cc = 0; cc < N / 16; ++cc) {
            const float* v = acc + cc * 16;
            if (p < A.P) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = cc * 16 + q;
                    if (n < A.nc) Mt[(size_t)n * A.P + p] = valid ? v[q] * c.inv_spow[lrank(n) + 1] : 0.f;
                }
            }
        }
    }
};

template <int P, int N>
__global__ void __launch_bounds__(kThreads) k_tc_m2l(M2LArgs args, int* err) {
    typename ModeM2L<P>::Ctx c;
    c.a = &args;
    c.tgt = args.tgt0 + blockIdx.y;
    c.p0 = blockIdx.x * 128;
    c.e0 = args.ptr[c.tgt];
    c.e1 = args.ptr[c.tgt + 1];
    c.nchunk_src = (args.nc + PrecT<P>::BK - 1) / PrecT<P>::BK;
    c.N = N;
    const float sd = args.box_scale[c.tgt];
    c.spow[0] = 1.f;
    for (int k = 1; k < 16; ++k) c.spow[k] = c.spow[k - 1] * sd;
    for (int k = 0; k < 16; ++k) c.inv_spow[k] = 1.f / c.spow[k];
    engine<P, N, ModeM2L<P>>(c, err);
}

// ===========================================================================
// Plain GEMM D[M][N] = A[M][K] B[N][K]^T (FP32 in HBM), for checking the engine
// ===========================================================================
struct GemmArgs {
    int M, N, K;
    const float* A; const float* B; float* D;
};

template <int P>
struct ModeGemm {
    struct Ctx {
        const GemmArgs* a;
        int m0, n0;
    };
    __device__ static int nchunks(const Ctx& c) { return (c.a->K + PrecT<P>::BK - 1) / PrecT<P>::BK; }
    __device__ static void fill(const Ctx& c, int kc, int t, int k0, float* a, float* b, bool& hasb) {
        constexpr int BK = PrecT<P>::BK;
        const GemmArgs& G = *c.a;
        const int m = c.m0 + t, n = c.n0 + t;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int kk = kc * BK + k0 + k;
            a[k] = (m < G.M && kk < G.K) ? G.A[(size_t)m * G.K + kk] : 0.f;
            b[k] = (n < G.N && kk < G.K) ? G.B[(size_t)n * G.K + kk] : 0.f;
        }
        hasb = true;
    }
    template <int N>
    __device__ static void epilogue(const Ctx& c, int warp, int lane, const float* acc, bool valid) {
        const GemmArgs& G = *c.a;
        const int m = c.m0 + warp * 32 + lane;
#pragma unroll
        for (int cc = 0; cc < N / 16; ++cc) {
            const float* v = acc + cc * 16;
            if (m < G.M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c.n0 + cc * 16 + q;
                    if (n < G.N) G.D[(size_t)m * G.N + n] = valid ? v[q] : 0.f;
                }
            }
        }
    }
};

template <int P>
__global__ void __launch_bounds__(kThreads) k_tc_gemm(GemmArgs args, int* err) {
    typename ModeGemm<P>::Ctx c;
    c.a = &args;
    c.m0 = blockIdx.x * 128;
    c.n0 = blockIdx.y * 128;
    engine<P, 128, ModeGemm<P>>(c, err);
}

template <int P>
cudaError_t set_smem_attr() {
    cudaError_t e = cudaSuccess;
    const int bytes = Smem<P>::bytes;
    e = cudaFuncSetAttribute(k_tc_a2<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_l2p<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_gemm<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_m2l<P, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_m2l<P, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_m2l<P, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_m2l<P, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <int P>
cudaError_t gemm_typed(const GemmArgs& g, int* err, cudaStream_t s) {
    static bool init = false;
    if (!init) {
        cudaError_t e = set_smem_attr<P>();
        if (e != cudaSuccess) return e;
        init = true;
    }
    dim3 grid((g.M + 127) / 128, (g.N + 127) / 128);
    k_tc_gemm<P><<<grid, kThreads, Smem<P>::bytes, s>>>(g, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t ensure_attr() {
    static bool init = false;
    if (!init) {
        cudaError_t e = set_smem_attr<P>();
        if (e != cudaSuccess) return e;
        init = true;
    }
    return cudaSuccess;
}

template <int P>
cudaError_t a2_typed(const A2Args& a, int nleaf, int* err, cudaStream_t s) {
    cudaError_t e = ensure_attr<P>();
    if (e != cudaSuccess) return e;
    dim3 grid(a.ntile * (a.ntile + 1) / 2, nleaf * a.nc);
    k_tc_a2<P><<<grid, kThreads, Smem<P>::bytes, s>>>(a, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t l2p_typed(const L2PArgs& a, int nleaf, int max_rows, int* err, cudaStream_t s) {
    cudaError_t e = ensure_attr<P>();
    if (e != cudaSuccess) return e;
    dim3 grid((max_rows + 127) / 128, (a.nocc + 127) / 128, nleaf);
    k_tc_l2p<P><<<grid, kThreads, Smem<P>::bytes, s>>>(a, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t m2l_typed(const M2LArgs& a, int ntgt, int* err, cudaStream_t s) {
    cudaError_t e = ensure_attr<P>();
    if (e != cudaSuccess) return e;
    dim3 grid((a.P + 127) / 128, ntgt);
    if (a.nc <= 16)
        k_tc_m2l<P, 16><<<grid, kThreads, Smem<P>::bytes, s>>>(a, err);
    else if (a.nc <= 32)
        k_tc_m2l<P, 32><<<grid, kThreads, Smem<P>::bytes, s>>>(a, err);
    else if (a.nc <= 64)
        k_tc_m2l<P, 64><<<grid, kThreads, Smem<P>::bytes, s>>>(a, err);
    else if (a.nc <= 128)
        k_tc_m2l<P, 128><<<grid, kThreads, Smem<P>::bytes, s>>>(a, err);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

#define OCCK_TC_DISPATCH(prec, call)                      \
    switch (tc_mode(prec)) {                              \
        case PM_BF16: { constexpr int P = PM_BF16; return call; }       \
        case PM_FP16: { constexpr int P = PM_FP16; return call; }       \
        case PM_TF32: { constexpr int P = PM_TF32; return call; }       \
        case PM_BF16X3: { constexpr int P = PM_BF16X3; return call; }   \
        case PM_FP16X3: { constexpr int P = PM_FP16X3; return call; }   \
        default: return cudaErrorInvalidValue;            \
    }

}  // namespace

int tc_mode(int prec) {
    switch (prec) {
        case OCCK_BF16: return PM_BF16;
        case OCCK_FP16: return PM_FP16;
        case OCCK_TF32: return PM_TF32;
        case OCCK_BF16X3: return PM_BF16X3;
        case OCCK_FP16X3: return PM_FP16X3;
        default: return -1;
    }
}

cudaError_t tc_gemm(int prec, int M, int N, int K, const float* A, const float* B, float* D, int* err,
                    cudaStream_t s) {
    GemmArgs g{M, N, K, A, B, D};
    switch (tc_mode(prec)) {
        case PM_BF16: return gemm_typed<PM_BF16>(g, err, s);
        case PM_FP16: return gemm_typed<PM_FP16>(g, err, s);
        case PM_TF32: return gemm_typed<PM_TF32>(g, err, s);
        case PM_BF16X3: return gemm_typed<PM_BF16X3>(g, err, s);
        case PM_FP16X3: return gemm_typed<PM_FP16X3>(g, err, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace occk

namespace occk {

cudaError_t tc_run_a2(int prec, const int* leaf_rowoff, const int* leaf_aos, const float* Ct, const float* W,
                      int nocc, int nrow, int nc, int nleaf, int leaf_store0, const float* lscale, float* Obox,
                      int* err, cudaStream_t s) {
    A2Args a{leaf_rowoff, leaf_aos, Ct, W, nocc, nrow, nc, (nocc + 127) / 128, leaf_store0, lscale, Obox};
    OCCK_TC_DISPATCH(prec, a2_typed<P>(a, nleaf, err, s));
}

cudaError_t tc_run_l2p(int prec, const int* leaf_rowoff, const float* W, const float* Mbox, int nocc, int nrow,
                       int nc, int nleaf, int leaf_store0, int max_rows, const float* lscale, double* KB,
                       int* err, cudaStream_t s) {
    L2PArgs a{leaf_rowoff, W, Mbox, nocc, nrow, nc, leaf_store0, lscale, KB};
    OCCK_TC_DISPATCH(prec, l2p_typed<P>(a, nleaf, max_rows, err, s));
}

cudaError_t tc_run_m2l(int prec, int P2, int nc, int L, int first_box, int tgt0, int ntgt, const int* ptr,
                       const int* src, const int* op, const int* lmax_e, const float* ops, const float* O,
                       float* M, const float* box_scale, int* err, cudaStream_t s) {
    M2LArgs a{P2, nc, L, first_box, tgt0, ptr, src, op, lmax_e, ops, O, M, box_scale};
    OCCK_TC_DISPATCH(prec, m2l_typed<P>(a, ntgt, err, s));
}

}  // namespace occk
