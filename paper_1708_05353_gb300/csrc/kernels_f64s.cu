// The FP64-accurate form off the FP64 pipe.  Steps (a) (full transform) and (e)
// in FP64 from integer slices on tcgen05: the error-free splitting of a matrix
// product into products of small-integer matrices (Ozaki, Ogita, Oishi and
// Rump, Numer. Algorithms 59 (2012) 95-118), with the slice products on the
// tensor core and every sum of them exact.  The half transform and the tree
// passes in double-FP32 arithmetic further down.  Step (e) reads
//
//   KB[row][i] = sum_{lm, j} A[row][(lm, j)] B[i][(lm, j)]              (Eq. kri)
//   A = W[lm][row][j] s_lm,   B = w_lm Mcal[lm](i, j) / s_lm            (FP64)
//
// (s_lm ~ the leaf-level component scale that brings every component to O(1);
// w_lm the real-form weight times the factor 2 of K.)  Each row of A is scaled
// by 2^-e_row and each column i of B by 2^-f_i so that the entries lie in
// (-1, 1); an entry x is then cut into S slices
//   x = sum_{s=1..S} q_s 2^-c_s + r,   c_s = 6 + 7 (s - 1),   |q_s| <= 64,
// q_s = rint(x_{s-1} 2^c_s), x_s = x_{s-1} - q_s 2^-c_s (all exact in FP64),
// |r| <= 2^-(c_S + 1).  The slices are integers, exact in FP16, and the
// product of two is an integer of magnitude <= 2^12.  A product of slices s
// and t carries the scale 2^-(c_s + c_t) = 2^-(12 + 7 (d - 2)), d = s + t, so
// all pairs with the same d add into one TMEM accumulator G_d; the pairs with
// d <= S + 1 are formed: slice s of A meets slices 1 .. S + 1 - s of B in one
// MMA of N = 32 (S + 1 - s), the B slices lying one after another along N and
// the groups one after another in TMEM (S MMAs per K step of 16).  Over a
// chunk of 512 K values |G_d| <= (d - 1) 2^12 512 < 2^24, so the tensor core's
// FP32 accumulation is exact (pinned by tests/test_gpu_mixed.py on integer data);
// after each chunk the epilogue converts G_d to int32 (exact) and adds it to an
// int32 sum per group and column (exact below 2^31, i.e. up to 127 chunks;
// longer K ranges are split).  At the end of a tile
//   KB = 2^(e_row + f_i) sum_d 2^-(12 + 7 (d - 2)) G_d                 (FP64)
// Scaling is by powers of two throughout (the component scales s_lm are
// rounded down to powers of two), and the slices are cut from the bits of the
// FP64 values with integer operations: FP64 arithmetic, two operations per
// clock and SM on this GPU, is left to the final sums.
// The only roundings are the slices' truncation (relative 2^-(c_S + 1) of the
// row's and the column's largest entry per product, 2^-49 for S = 7), the
// dropped pairs d > S + 1 (smaller still) and the final FP64 sum.
//
// GEMM: M = 128 rows, N = 32 orbitals, K = 32 values per stage; A panels hold
// the S slices of a 128 x 32 block (S x 8 KB), B panels of a 32 x 32 block
// (S x 2 KB), each in the K-major no-swizzle canonical layout (8-row x 16-byte
// core matrices, LBO 128 bytes along K, SBO 512 bytes between row groups).
// One CTA per SM walks the tiles (leaf, row tile, orbital tile, K split):
// warp 0 copies panels into a ring of stages (cp.async.bulk, mbarrier
// transaction counts), warp 1 issues the MMAs, warps 2-17 drain the group
// accumulators after every chunk (two TMEM buffers of S x 32 columns
// alternate, so the drain of one chunk overlaps the MMAs of the next) and
// write the tile.  Every wait is bounded; on a timeout the CTA raises the
// error word, waits (bounded) for its copies in flight, frees TMEM and returns.
//
// From 25 components on, M2L runs on the same engine with its K gathered stage
// by stage from the interaction list (rows = occupied pairs, columns = output
// components, K = (edge, input component)); the scalings there are per level
// (see the M2L section below), and the parent's L2L is added in double-FP32.
#include <algorithm>
#include <cstdio>

#include "occk_internal.h"
#include "tc.cuh"

namespace occk {

namespace {

using namespace tc;

constexpr uint32_t kWaitS = 1u << 22;
constexpr int kSK = 32;              // K values of one stage
constexpr int kSN = 32;              // orbitals of one tile
constexpr int kChunk = 16;           // stages of one exact chunk (512 K values)
constexpr int kMaxChunks = 127;      // chunks of one tile (int32 group sums)
constexpr uint32_t kSLBO = 128, kSSBO = 512;
constexpr int kAPart = 128 * kSK * 2;   // bytes of one A slice (8 KB)
constexpr int kBPart = kSN * kSK * 2;   // bytes of one B slice (2 KB)

template <int S>
struct SL {
    static constexpr int a_bytes = S * kAPart, b_bytes = S * kBPart;
    static constexpr int stage = a_bytes + b_bytes;
    static constexpr int ring = S <= 4 ? 4 : 3;
    static constexpr int smem = ring * stage;
    static constexpr uint32_t buf = (uint32_t)S * kSN;   // TMEM columns of one accumulator set
};

__device__ __forceinline__ void s_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void s_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void s_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}
// Polls allowed to the MMA thread's wait for a stage's operands: kWaitS in
// normal use; occk_debug_set_wait_limit lowers it so that a test can make that
// wait give up and exercise the abort path (every other wait keeps kWaitS).
__device__ uint32_t g_s_full_wait = kWaitS;

__device__ __forceinline__ bool s_wait(uint64_t* bar, uint32_t parity, const int* flag, uint32_t limit = kWaitS) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(const volatile int*)flag) return false;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

// byte offset of element (row, k) of one slice in the canonical layout
__device__ __forceinline__ uint32_t s_off(int row, int k) {
    return (uint32_t)(row >> 3) * kSSBO + (uint32_t)(k >> 3) * kSLBO + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Component scales as powers of two: k_lm = floor(log2 s_lm), so that scaling
// is exact and done on exponents; the real-form weight times the factor 2 of
// K (Eq. kri) is +-2^a_lm (2 for m = 0, 4 for cos, -4 for sin).
__device__ __forceinline__ int s_klm(const float* lscale, int lm) { return ilogbf(lscale[lm]); }
__device__ __forceinline__ void s_weight(int lm, int& a, bool& neg) {
    int l = 0;
    while ((l + 1) * (l + 1) <= lm) ++l;
    a = lm == l * l ? 1 : 2;
    neg = lm != l * l && !((lm - l * l) & 1);
}

__device__ __forceinline__ size_t s_tri(int i, int j, int n) {
    return (size_t)i * (size_t)(2 * n - i + 1) / 2 + (size_t)(j - i);
}

// Smallest E with |v| < 2^E (from the exponent field; -2000 for zero and
// subnormal values, which then never set a maximum).
__device__ __forceinline__ int s_expo(double v) {
    const int ef = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    return ef == 0 ? -2000 : ef - 1022;
}

// round(v 2^t) as a 64-bit integer, from the bits of v (integer operations
// only; the caller guarantees |v 2^t| < 2^55)
__device__ __forceinline__ long long s_fixed(double v, int t) {
    const long long bits = __double_as_longlong(v);
    const int ef = (int)((bits >> 52) & 0x7FF);
    long long mant = bits & ((1LL << 52) - 1);
    int E = -1074;
    if (ef != 0) {
        mant |= 1LL << 52;
        E = ef - 1075;
    }
    const int sh = E + t;
    long long r;
    if (sh >= 0) r = mant << min(sh, 10);
    else if (sh > -60) r = (mant + (1LL << (-sh - 1))) >> (-sh);
    else r = 0;
    return bits < 0 ? -r : r;
}

// The same for FP32 operands (the FP32 form): |v| < 2^E, and round(v 2^t).
__device__ __forceinline__ int s_expo(float v) {
    const int ef = (int)((__float_as_uint(v) >> 23) & 0xFF);
    return ef == 0 ? -2000 : ef - 126;
}
__device__ __forceinline__ long long s_fixed(float v, int t) {
    const unsigned bits = __float_as_uint(v);
    const int ef = (int)((bits >> 23) & 0xFF);
    long long mant = bits & 0x7FFFFF;
    int E = -149;
    if (ef != 0) {
        mant |= 1LL << 23;
        E = ef - 150;
    }
    const int sh = E + t;
    long long r;
    if (sh >= 0) r = mant << min(sh, 40);
    else if (sh > -40) r = (mant + (1LL << (-sh - 1))) >> (-sh);
    else r = 0;
    return (bits >> 31) ? -r : r;
}

// 2^k for -1022 <= k <= 1023 (clamped), built from its bits
__device__ __forceinline__ double s_pow2(int k) {
    k = max(-1022, min(1023, k));
    return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ __forceinline__ int s_warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// e_row: one warp per stored row, the exponent bound of max |W 2^k_lm| over (lm, j)
template <typename T>
__global__ void k_s_rowexp(const T* __restrict__ W, const float* __restrict__ lscale, int nrow, int nocc,
                           int nc, int* __restrict__ erow) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= nrow) return;
    int m = -2000;
    for (int lm = 0; lm < nc; ++lm) {
        const int k = s_klm(lscale, lm);
        const T* w = W + ((size_t)lm * nrow + row) * nocc;
        for (int j = lane; j < nocc; j += 32) m = max(m, s_expo(w[j]) + k);
    }
    m = s_warp_max(m);
    if (lane == 0) erow[row] = m <= -1000 ? 0 : m;
}

// f_i: one warp per (leaf, orbital i), the exponent bound of
// max |w_lm Mcal(i, j) 2^-k_lm| over (lm, j)
template <typename T>
__global__ void k_s_colexp(const T* __restrict__ Mbox, const float* __restrict__ lscale, int nleaf, int nocc,
                           int nc, int leaf_store0, int* __restrict__ fcol) {
    const long long x = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (x >= (long long)nleaf * nocc) return;
    const int B = (int)(x / nocc), i = (int)(x % nocc);
    const size_t P = (size_t)nocc * (nocc + 1) / 2;
    int m = -2000;
    for (int lm = 0; lm < nc; ++lm) {
        int a;
        bool neg;
        s_weight(lm, a, neg);
        const int k = a - s_klm(lscale, lm);
        const T* M = Mbox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
        for (int j = lane; j < nocc; j += 32) m = max(m, s_expo(M[i <= j ? s_tri(i, j, nocc) : s_tri(j, i, nocc)]) + k);
    }
    m = s_warp_max(m);
    if (lane == 0) fcol[x] = m <= -1000 ? 0 : m;
}

// Slices of 8 consecutive K values of one row, given as integers round(x 2^55)
// (|x| < 1): slice s is round(r_s 2^-(49 - 7 s)) of the remainder r_s, so
// |q| <= 64 and x = sum_s q_s 2^-(6 + 7 s) + O(2^-49); stored as FP16 in
// 16-byte rows of core matrices, part s at dst + s * part_bytes.
template <int S>
__device__ __forceinline__ void s_put8(uint8_t* dst, uint32_t part_bytes, long long* r) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int sh = 49 - 7 * s;
        __half h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long qs = (r[q] + (1LL << (sh - 1))) >> sh;
            r[q] -= qs << sh;
            h[q] = __int2half_rn((int)qs);
        }
        *reinterpret_cast<uint4*>(dst + (size_t)s * part_bytes) = *reinterpret_cast<uint4*>(h);
    }
}

// A panels: block (stage kc, row tile rt, leaf B), thread = panel row
template <int S, typename T>
__global__ void __launch_bounds__(128)
k_s_panel_A(const int* __restrict__ leaf_rowoff, const T* __restrict__ W, const float* __restrict__ lscale,
            const int* __restrict__ erow, int nocc, int nrow, int jc, int KC, const int* __restrict__ rtA,
            const long long* __restrict__ offA, int B0, long long pan0, uint8_t* __restrict__ pan) {
    const int kc = blockIdx.x, rt = blockIdx.y, B = B0 + blockIdx.z;
    if (rt >= rtA[B]) return;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r = rt * 128 + threadIdx.x;
    const int lm = kc / jc, j0 = (kc % jc) * kSK;
    const bool live = r < nr;
    const T* w = W + ((size_t)lm * nrow + rb0 + (live ? r : 0)) * nocc;
    const int t = s_klm(lscale, lm) - (live ? erow[rb0 + r] : 0) + 55;
    uint8_t* panel = pan + (size_t)(offA[B] - pan0 + (long long)rt * KC + kc) * SL<S>::a_bytes;
#pragma unroll
    for (int k8 = 0; k8 < kSK; k8 += 8) {
        long long v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + k8 + q;
            v[q] = (live && j < nocc) ? s_fixed(w[j], t) : 0;
        }
        s_put8<S>(panel + s_off(threadIdx.x, k8), kAPart, v);
    }
}

// B panels: block (4 stages, orbital tile ct, leaf B), thread = (orbital, stage)
template <int S, typename T>
__global__ void __launch_bounds__(128)
k_s_panel_B(const T* __restrict__ Mbox, const float* __restrict__ lscale, const int* __restrict__ fcol,
            int nocc, int nc, int leaf_store0, int jc, int KC, int nct, int B0, uint8_t* __restrict__ pan) {
    const int kc = blockIdx.x * 4 + (threadIdx.x >> 5), ct = blockIdx.y, B = B0 + blockIdx.z;
    if (kc >= KC) return;
    const int il = threadIdx.x & 31, i = ct * kSN + il;
    const int lm = kc / jc, j0 = (kc % jc) * kSK;
    int a;
    bool neg;
    s_weight(lm, a, neg);
    const size_t P = (size_t)nocc * (nocc + 1) / 2;
    const T* M = Mbox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
    const bool live = i < nocc;
    const int t = a - s_klm(lscale, lm) - (live ? fcol[(size_t)B * nocc + i] : 0) + 55;
    uint8_t* panel = pan + (size_t)(((long long)(B - B0) * nct + ct) * KC + kc) * SL<S>::b_bytes;
#pragma unroll
    for (int k8 = 0; k8 < kSK; k8 += 8) {
        long long v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + k8 + q;
            const long long x = (live && j < nocc) ? s_fixed(M[i <= j ? s_tri(i, j, nocc) : s_tri(j, i, nocc)], t) : 0;
            v[q] = neg ? -x : x;
        }
        s_put8<S>(panel + s_off(il, k8), kBPart, v);
    }
}

// Step (a) operands: A[i][r] = C_ri (rows i, K = the leaf's AO rows r), one
// exponent per (leaf, i); B[j][r] = W[lm][r][j], one exponent per (leaf, lm, j).
template <typename T>
__global__ void k_s_a2_expC(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos,
                            const T* __restrict__ Ct, int nocc, int* __restrict__ eC) {
    const int B = blockIdx.x, i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= nocc) return;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    int m = -2000;
    for (int r = 0; r < nr; ++r) m = max(m, s_expo(Ct[(size_t)leaf_aos[rb0 + r] * nocc + i]));
    eC[(size_t)B * nocc + i] = m <= -1000 ? 0 : m;
}

template <typename T>
__global__ void k_s_a2_expW(const int* __restrict__ leaf_rowoff, const T* __restrict__ W, int nocc, int nrow,
                            int nc, int* __restrict__ eW) {
    const int B = blockIdx.x / nc, lm = blockIdx.x % nc, j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= nocc) return;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const T* w = W + ((size_t)lm * nrow + rb0) * nocc + j;
    int m = -2000;
    for (int r = 0; r < nr; ++r) m = max(m, s_expo(w[(size_t)r * nocc]));
    eW[((size_t)B * nc + lm) * nocc + j] = m <= -1000 ? 0 : m;
}

// A panels of step (a): block (stage kc, row tile ti, leaf B), thread = orbital i
template <int S, typename T>
__global__ void __launch_bounds__(128)
k_s_a2_panel_A(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos, const T* __restrict__ Ct,
               const int* __restrict__ eC, int nocc, int nti, const int* __restrict__ kca,
               const long long* __restrict__ offAa, int B0, long long pan0, uint8_t* __restrict__ pan) {
    const int kc = blockIdx.x, ti = blockIdx.y, B = B0 + blockIdx.z;
    if (kc >= kca[B]) return;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int i = ti * 128 + threadIdx.x;
    const bool live = i < nocc;
    const int t = 55 - (live ? eC[(size_t)B * nocc + i] : 0);
    uint8_t* panel = pan + (size_t)(offAa[B] - pan0 + (long long)ti * kca[B] + kc) * SL<S>::a_bytes;
#pragma unroll
    for (int k8 = 0; k8 < kSK; k8 += 8) {
        long long v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = kc * kSK + k8 + q;
            v[q] = (live && r < nr) ? s_fixed(Ct[(size_t)leaf_aos[rb0 + r] * nocc + i], t) : 0;
        }
        s_put8<S>(panel + s_off(threadIdx.x, k8), kAPart, v);
    }
}

// B panels of step (a): block (4 stages, column tile tj, leaf B * nc + lm),
// thread = (orbital j, stage)
template <int S, typename T>
__global__ void __launch_bounds__(128)
k_s_a2_panel_B(const int* __restrict__ leaf_rowoff, const T* __restrict__ W, const int* __restrict__ eW,
               int nocc, int nrow, int nc, int nct, const int* __restrict__ kca, const long long* __restrict__ offBa,
               int B0, long long pan0, uint8_t* __restrict__ pan) {
    const int B = B0 + blockIdx.z / nc, lm = blockIdx.z % nc, tj = blockIdx.y;
    const int kc = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (kc >= kca[B]) return;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int jl = threadIdx.x & 31, j = tj * kSN + jl;
    const bool live = j < nocc;
    const int t = 55 - (live ? eW[((size_t)B * nc + lm) * nocc + j] : 0);
    const T* w = W + ((size_t)lm * nrow + rb0) * nocc + j;
    uint8_t* panel = pan + (size_t)(offBa[B] - pan0 + ((long long)lm * nct + tj) * kca[B] + kc) * SL<S>::b_bytes;
#pragma unroll
    for (int k8 = 0; k8 < kSK; k8 += 8) {
        long long v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = kc * kSK + k8 + q;
            v[q] = (live && r < nr) ? s_fixed(w[(size_t)r * nocc], t) : 0;
        }
        s_put8<S>(panel + s_off(jl, k8), kBPart, v);
    }
}

struct SState {
    uint64_t full[4], empty[4], accf[2], acce[2];
    uint32_t tmem;
    int abort;
    uint32_t gp, gm;   // stages issued by the producer, consumed by the MMA thread
};

// step (e): tiles (leaf, row tile, orbital tile, K split)
struct SGemmE {
    const int* leaf_rowoff; const int* rtA; const long long* offA; const long long* item0;
    const int* erow; const int* fcol;
    const uint8_t* panA; const uint8_t* panB;
    double* KB;
    int nleaf, nocc, nrow, KC, nct, nsplit;
    int B0;                                  // first leaf of the batch (panels hold leaves B0 ..)
    long long it0, nitems, panA0;            // items it0 .. it0 + nitems - 1; offA of leaf B0
    int* err;
};

// step (a): tiles (leaf, lm, triangular pair of a 128-orbital row tile and a
// 32-orbital column tile)
struct SGemmA {
    const int* kca; const long long* offAa; const long long* offBa; const int* tpair;
    const int* eC; const int* eW;
    const uint8_t* panA; const uint8_t* panB;
    void* Obox;                              // double (FP64 form) or float (FP32 form)
    int nleaf, nocc, nc, nct, ntp, leaf_store0;
    int B0;                                  // first leaf of the batch
    long long nitems, panA0, panB0;          // offAa, offBa of leaf B0
    int* err;
};

constexpr int kSEpi = 16;                       // epilogue warps: four per TMEM lane quarter
constexpr int kSThreads = 64 + kSEpi * 32;
constexpr int kSCols = kSN / (kSEpi / 4);        // orbitals per epilogue thread

// TMEM -> registers: 32 lanes x 8 columns of 32 bit (completion by s_tmem_wait)
__device__ __forceinline__ void s_tmem_ld8(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void s_tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Stage kc of an item whose panels lie one after another along K
template <int S>
struct SContig {
    __device__ __forceinline__ bool operator()(long long, int kc, const uint8_t* A, const uint8_t* B,
                                               const uint8_t*& a, const uint8_t*& b) const {
        a = A + (size_t)kc * SL<S>::a_bytes;
        b = B + (size_t)kc * SL<S>::b_bytes;
        return true;
    }
};

// One CTA per SM walks items it = blockIdx.x, + gridDim.x, ...:
// src(it, A, B, nk) gives an item's first A and B panels and its number of
// stages; at(it, kc, A, B, a, b) the panels of stage kc (false: an address
// outside the workspace, which aborts the CTA before any copy is issued);
// out(it, row, part, acc) receives the exact group sums of one output row and
// kSCols columns (part) at the end of the item.
template <int S, typename Src, typename Out, typename At = SContig<S>>
__device__ __forceinline__ void s_gemm_body(long long nitems, Src src, Out out, int* err, At at = At()) {
    using C = SL<S>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ SState st;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 2) {
        tmem_alloc(&st.tmem, 512);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int r = 0; r < C::ring; ++r) {
            mbar_init(&st.full[r], 1);
            mbar_init(&st.empty[r], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&st.accf[b], 1);
            mbar_init(&st.acce[b], kSEpi * 32);
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
    auto stA = [&](int r) { return sbase + (uint32_t)r * C::stage; };
    auto stB = [&](int r) { return sbase + (uint32_t)r * C::stage + C::a_bytes; };
    if (warp == 0) {
        if (lane == 0) {   // producer
            uint32_t gs = 0;
            for (long long it = blockIdx.x; it < nitems && !*(volatile int*)&st.abort; it += gridDim.x) {
                const uint8_t *A, *Bp;
                int nk;
                src(it, A, Bp, nk);
                for (int kc = 0; kc < nk; ++kc, ++gs) {
                    const int r = (int)(gs % C::ring);
                    if (gs >= (uint32_t)C::ring && !s_wait(&st.empty[r], ((gs / C::ring) - 1) & 1, &st.abort)) {
                        st.abort = 1;
                        break;
                    }
                    const uint8_t *a, *b;
                    if (!at(it, kc, A, Bp, a, b)) {
                        st.abort = 1;
                        break;
                    }
                    s_expect_tx(&st.full[r], (uint32_t)C::stage);
                    s_bulk_g2s(stA(r), a, C::a_bytes, &st.full[r]);
                    s_bulk_g2s(stB(r), b, C::b_bytes, &st.full[r]);
                    st.gp = gs + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issue
            uint32_t gs = 0, gc = 0;
            const uint32_t full_wait = g_s_full_wait;
            for (long long it = blockIdx.x; it < nitems && !*(volatile int*)&st.abort; it += gridDim.x) {
                const uint8_t *A, *Bp;
                int nk;
                src(it, A, Bp, nk);
                for (int kc = 0; kc < nk; ++kc, ++gs) {
                    const int r = (int)(gs % C::ring), q = kc % kChunk;
                    const int b = (int)(gc & 1);
                    if (!s_wait(&st.full[r], (gs / C::ring) & 1, &st.abort, full_wait) ||
                        (q == 0 && gc >= 2 && !s_wait(&st.acce[b], ((gc >> 1) - 1) & 1, &st.abort))) {
                        st.abort = 1;
                        break;
                    }
                    fence_after_sync();
                    // A slice s against B slices 0 .. S-1-s in one MMA: the B
                    // slices lie one after another along N (32 rows each), and
                    // the products land in groups s .. S-1, 32 TMEM columns each
                    const uint32_t d0 = tmem + (uint32_t)b * C::buf;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const uint32_t idesc = instr_desc(128, kSN * (S - s), 0u);   // FP16 x FP16 -> FP32
#pragma unroll
                        for (int k16 = 0; k16 < kSK / 16; ++k16) {
                            const uint32_t adv = (uint32_t)k16 * 2u * kSLBO;
                            const uint64_t ad = smem_desc(stA(r) + (uint32_t)s * kAPart + adv, kSLBO, kSSBO);
                            const uint64_t bd = smem_desc(stB(r) + adv, kSLBO, kSSBO);
                            const uint32_t acc = (q == 0 && s == 0 && k16 == 0) ? 0u : 1u;
                            mma_f16(d0 + (uint32_t)s * kSN, ad, bd, idesc, acc);
                        }
                    }
                    mma_commit(&st.empty[r]);
                    st.gm = gs + 1;
                    if (q == kChunk - 1 || kc == nk - 1) {
                        mma_commit(&st.accf[b]);
                        ++gc;
                    }
                }
            }
            // every MMA issued is complete before TMEM is given back: the last
            // commit (to the stage's empty barrier, also after an abort in the
            // middle of a chunk) covers all earlier ones
            const uint32_t gl = st.gm;
            if (gl > 0) mbar_wait_bounded(&st.empty[(gl - 1) % C::ring], ((gl - 1) / C::ring) & 1, kWaitS);
        }
    } else {   // warps 2..17: drain the group accumulators, write the tile
        const int q4 = warp & 3, part = (warp - 2) >> 2;   // TMEM lane quarter, share of the orbitals
        const int row = q4 * 32 + lane;
        uint32_t gc = 0;
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
            const uint8_t *A, *Bp;
            int nk;
            src(it, A, Bp, nk);
            const int nch = (nk + kChunk - 1) / kChunk;
            int acc[S][kSCols];   // exact: every chunk adds less than 2^24, at most 127 chunks
#pragma unroll
            for (int d = 0; d < S; ++d)
#pragma unroll
                for (int c = 0; c < kSCols; ++c) acc[d][c] = 0;
            bool ok = true;
            for (int ch = 0; ch < nch; ++ch, ++gc) {
                const int b = (int)(gc & 1);
                if (*(volatile int*)&st.abort || !s_wait(&st.accf[b], (gc >> 1) & 1, &st.abort)) {
                    st.abort = 1;
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t base =
                    tmem + (uint32_t)b * C::buf + (uint32_t)(part * kSCols) + ((uint32_t)(q4 * 32) << 16);
#pragma unroll
                for (int d = 0; d < S; ++d) {
                    uint32_t v[kSCols];
#pragma unroll
                    for (int c8 = 0; c8 < kSCols; c8 += 8) s_tmem_ld8(base + (uint32_t)(d * kSN + c8), v + c8);
                    s_tmem_wait();
#pragma unroll
                    for (int c = 0; c < kSCols; ++c) acc[d][c] += __float2int_rn(__uint_as_float(v[c]));
                }
                fence_before_sync();
                s_arrive(&st.acce[b]);
            }
            if (!ok) break;
            out(it, row, part, acc);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (t == 0 && st.abort) {
        atomicExch(err, 1);
        // copies issued but never consumed: wait (bounded) until they land
        for (uint32_t gs = st.gm; gs < st.gp; ++gs)
            mbar_wait_bounded(&st.full[gs % C::ring], (gs / C::ring) & 1, kWaitS);
    }
    __syncthreads();
    fence_after_sync();
    if (warp == 2) tmem_dealloc(tmem, 512);
}


// sum_d 2^-(12 + 7 d) G_d for kSCols columns.  The groups are first combined
// exactly in two 64-bit integers, vh = sum_{d<3} G_d 2^(7 (2 - d)) (below
// 2^46) and vl = sum_{d>=3} G_d 2^(7 (S - 1 - d)) (below 2^60), so that only
// two conversions and one FMA run on the FP64 pipe (two operations per clock
// and SM on this GPU): vh converts exactly, vl with a rounding far below the
// result's last bit.
template <int S>
__device__ __forceinline__ void s_combine(const int (&acc)[S][kSCols], double* v) {
#pragma unroll
    for (int c = 0; c < kSCols; ++c) {
        long long vh = 0, vl = 0;
#pragma unroll
        for (int d = 0; d < S; ++d) {
            if (d < 3) vh += (long long)acc[d][c] << (7 * (2 - d));
            else vl += (long long)acc[d][c] << (7 * (S - 1 - d));
        }
        v[c] = fma((double)vl, s_pow2(-(12 + 7 * (S - 1))), (double)vh * s_pow2(-26));
    }
}

// Step (e): KB[ks][row][i] for the leaf's rows and a 32-orbital tile
template <int S>
__global__ void __launch_bounds__(kSThreads, 1)
k_s_gemm_e(SGemmE g) {
    using C = SL<S>;
    auto decode = [&](long long it, int& B, int& rt, int& ct, int& ks, int& kc0, int& kc1) {
        it += g.it0;
        int lo = g.B0, hi = g.nleaf - 1;              // last leaf with item0 <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g.item0[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        B = lo;
        int x = (int)(it - g.item0[B]);   // items of one leaf: below 2^31
        ct = x % g.nct;
        x /= g.nct;
        rt = x % g.rtA[B];
        ks = x / g.rtA[B];
        kc0 = g.KC * ks / g.nsplit;       // KC * nsplit below 2^31
        kc1 = g.KC * (ks + 1) / g.nsplit;
    };
    auto src = [&](long long it, const uint8_t*& A, const uint8_t*& Bp, int& nk) {
        int B, rt, ct, ks, kc0, kc1;
        decode(it, B, rt, ct, ks, kc0, kc1);
        A = g.panA + (size_t)(g.offA[B] - g.panA0 + (long long)rt * g.KC + kc0) * C::a_bytes;
        Bp = g.panB + (size_t)(((long long)(B - g.B0) * g.nct + ct) * g.KC + kc0) * C::b_bytes;
        nk = kc1 - kc0;
    };
    auto out = [&](long long it, int row, int part, const int (&acc)[S][kSCols]) {
        int B, rt, ct, ks, kc0, kc1;
        decode(it, B, rt, ct, ks, kc0, kc1);
        const int rb0 = g.leaf_rowoff[B], nr = g.leaf_rowoff[B + 1] - rb0;
        const int rr = rt * 128 + row;
        if (rr >= nr) return;
        double v[kSCols];
        s_combine<S>(acc, v);
        const int er = g.erow[rb0 + rr];
        double* o = g.KB + ((size_t)ks * g.nrow + rb0 + rr) * g.nocc;
        const int* fc = g.fcol + (size_t)B * g.nocc;
#pragma unroll
        for (int c = 0; c < kSCols; ++c) {
            const int i = ct * kSN + part * kSCols + c;
            if (i < g.nocc) o[i] = v[c] * s_pow2(er + fc[i]);
        }
    };
    s_gemm_body<S>(g.nitems, src, out, g.err);
}

// Step (a): O[B][lm][(i, j)] = sum_r C_ri W[lm][r][j] for i <= j, rows i of a
// 128-orbital tile, columns j of a 32-orbital tile (Eq. motrans)
template <int S, typename T>
__global__ void __launch_bounds__(kSThreads, 1)
k_s_gemm_a(SGemmA g) {
    using C = SL<S>;
    auto decode = [&](long long it, int& B, int& lm, int& ti, int& tj) {
        const int tt = (int)(it % g.ntp);
        const long long x = it / g.ntp;
        lm = (int)(x % g.nc);
        B = g.B0 + (int)(x / g.nc);
        ti = g.tpair[tt] & 0xFFFF;
        tj = g.tpair[tt] >> 16;
    };
    auto src = [&](long long it, const uint8_t*& A, const uint8_t*& Bp, int& nk) {
        int B, lm, ti, tj;
        decode(it, B, lm, ti, tj);
        const int kca = g.kca[B];
        A = g.panA + (size_t)(g.offAa[B] - g.panA0 + (long long)ti * kca) * C::a_bytes;
        Bp = g.panB + (size_t)(g.offBa[B] - g.panB0 + ((long long)lm * g.nct + tj) * kca) * C::b_bytes;
        nk = kca;
    };
    const size_t P = (size_t)g.nocc * (g.nocc + 1) / 2;
    auto out = [&](long long it, int row, int part, const int (&acc)[S][kSCols]) {
        int B, lm, ti, tj;
        decode(it, B, lm, ti, tj);
        const int i = ti * 128 + row;
        if (i >= g.nocc) return;
        const int ec = g.eC[(size_t)B * g.nocc + i];
        const int* ew = g.eW + ((size_t)B * g.nc + lm) * g.nocc;
        T* o = (T*)g.Obox + ((size_t)(g.leaf_store0 + B) * g.nc + lm) * P + s_tri(i, i, g.nocc) - (size_t)i;
        if constexpr (sizeof(T) == 4) {
            // an FP32 result: the group sums combined on the FP32 pipe (a few
            // roundings at 2^-24, below the FP32 store's own), off the FP64 pipe
#pragma unroll
            for (int c = 0; c < kSCols; ++c) {
                const int j = tj * kSN + part * kSCols + c;
                float v = 0.f;
#pragma unroll
                for (int d = S - 1; d >= 0; --d)
                    v = fmaf((float)acc[d][c], __int_as_float((127 - (12 + 7 * d)) << 23), v);
                const int k = max(-126, min(127, ec + (j < g.nocc ? ew[j] : 0)));
                if (j >= i && j < g.nocc) o[j] = v * __int_as_float((k + 127) << 23);
            }
        } else {
            double v[kSCols];
            s_combine<S>(acc, v);
#pragma unroll
            for (int c = 0; c < kSCols; ++c) {
                const int j = tj * kSN + part * kSCols + c;
                if (j >= i && j < g.nocc) o[j] = (T)(v[c] * s_pow2(ec + ew[j]));
            }
        }
    };
    s_gemm_body<S>(g.nitems, src, out, g.err);
}

// ---------------------------------------------------------------------------
// M2L with L2L (Eqs. fmmex, fmm2, fmm3) in double-FP32 arithmetic for the
// sliced FP64 form: every value is an unevaluated sum hi + lo of two FP32
// numbers (about 48 significant bits) and every multiply-add is done with the
// error-free product (FMA) and sum (Knuth's TwoSum) of Dekker's and Knuth's
// double-length arithmetic, about 11 FP32 operations on the FP32 pipe, which
// issues 64 times as many operations per clock as the FP64 pipe here.  The
// multipoles are split into (hi, lo) in place before the level loop and the
// local expansions joined back to FP64 after it; the kernel is the per-level
// fused pass of the FP64 form (each target written once from its interaction
// list and its parent's finished expansion), the same sums in the same order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ff_fma(float& h, float& l, float2 w, float2 v) {
    const float p = __fmul_rn(w.x, v.x);
    float e = fmaf(w.x, v.x, -p);                 // p + e = w.x v.x exactly
    e = fmaf(w.x, v.y, e);
    e = fmaf(w.y, v.x, e);
    const float sum = __fadd_rn(h, p);            // TwoSum(h, p)
    const float bb = __fsub_rn(sum, h);
    const float t = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
    l = __fadd_rn(l, __fadd_rn(t, e));
    h = sum;
}

// x (FP64) -> (hi, lo): hi = x rounded to FP32, lo = (x - hi) rounded to FP32
// (x - hi is exact in FP64), in place in the same 8 bytes
__global__ void k_ff_split(double* x, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    {
        const double v = x[k];
        const float h = __double2float_rn(v);
        reinterpret_cast<float2*>(x)[k] = make_float2(h, __double2float_rn(v - (double)h));
    }
}

__global__ void k_ff_join(double* x, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const float2 f = reinterpret_cast<const float2*>(x)[k];
        x[k] = (double)f.x + (double)f.y;
    }
}

__global__ void k_ff_ops(const double* __restrict__ ops, size_t n, float2* __restrict__ out) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double v = ops[k];
        const float h = __double2float_rn(v);
        out[k] = make_float2(h, __double2float_rn(v - (double)h));
    }
}

constexpr int kFFNcMax = 169;

// one level: block (target, 128 pairs, chunk of LMC output components).
// MODE 0: M2M, the target gathers its children (Eq. fmm1); MODE 3: M2L over
// the interaction list, then the parent's finished local expansion (L2L);
// MODE 4: the L2L alone, added to the expansion already in out.
template <int LMC, int MODE, int PPT>
__global__ void __launch_bounds__(128)
k_translate_ff(int P, int nc, int L, int first_box, int tgt0, const int* __restrict__ ptr, const int* __restrict__ list,
               const int* __restrict__ opidx, const int* __restrict__ lmax_e, const int* __restrict__ parent,
               const int* __restrict__ l2l_opidx, const float2* __restrict__ ops, const float2* in, float2* out) {
    __shared__ float2 sop[kFFNcMax][LMC];   // [input component][output component of the chunk]
    const int tgt = tgt0 + blockIdx.x;
    const int pb = blockIdx.y * blockDim.x * PPT + threadIdx.x;   // pairs pb + k * blockDim.x
    const int c0 = blockIdx.z * LMC;
    const int ncl = min(LMC, nc - c0);
    bool live[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) live[k] = pb + k * (int)blockDim.x < P;
    float ah[PPT][LMC], al[PPT][LMC];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
        for (int q = 0; q < LMC; ++q) {
            ah[k][q] = al[k][q] = 0.f;
            if (MODE == 4 && live[k] && q < ncl) {
                const float2 x = out[((size_t)(tgt - first_box) * nc + c0 + q) * P + pb + k * blockDim.x];
                ah[k][q] = x.x;
                al[k][q] = x.y;
            }
        }
    const int e1 = ptr[tgt + 1], e0 = MODE == 4 ? e1 : ptr[tgt];
    const int eend = e1 + ((MODE >= 3 && parent[tgt] >= first_box) ? 1 : 0);   // then the parent's expansion
    int llo = 0;
    while ((llo + 1) * (llo + 1) <= c0) ++llo;
    int lhi = 0;
    while ((lhi + 1) * (lhi + 1) <= c0 + ncl - 1) ++lhi;
    for (int e = e0; e < eend; ++e) {
        const bool l2l = MODE >= 3 && e == e1;
        int src, op, Le = L;
        if (MODE == 0) {
            src = list[e];
            op = opidx[src];
        } else if (!l2l) {
            src = list[e];
            op = opidx[e];
            if (lmax_e) Le = lmax_e[e];
        } else {
            src = parent[tgt];
            op = l2l_opidx[tgt];
        }
        const int ncr = (Le + 1) * (Le + 1);
        if (c0 >= ncr) continue;   // uniform across the block
        // M2M: output rank l takes input ranks up to l; L2L: from l up
        const int cb0 = l2l ? llo * llo : 0, cb1 = MODE == 0 ? min(ncr, (lhi + 1) * (lhi + 1)) : ncr;
        const float2* Tm = ops + (size_t)op * nc * nc;
        __syncthreads();
        for (int x = threadIdx.x; x < LMC * (cb1 - cb0); x += blockDim.x) {
            const int q = x / (cb1 - cb0), c = cb0 + (x - q * (cb1 - cb0));
            sop[c][q] = (q < ncl && c0 + q < ncr) ? Tm[(size_t)(c0 + q) * nc + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2* xs = (l2l ? out : in) + (size_t)(src - first_box) * nc * P + pb;
        for (int cb = cb0; cb < cb1; cb += 4) {
            float2 v[4][PPT];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    v[u][k] = (cb + u < cb1 && live[k]) ? xs[(size_t)(cb + u) * P + k * blockDim.x]
                                                        : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (cb + u >= cb1) break;      // uniform across the block
#pragma unroll
                for (int q = 0; q < LMC; ++q) {
                    const float2 w = sop[cb + u][q];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) ff_fma(ah[k][q], al[k][q], w, v[u][k]);
                }
            }
        }
    }
    float2* o = out + ((size_t)(tgt - first_box) * nc + c0) * P + pb;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!live[k]) continue;
#pragma unroll
        for (int q = 0; q < LMC; ++q)
            if (q < ncl) {
                const float h = __fadd_rn(ah[k][q], al[k][q]);       // renormalise (Fast2Sum)
                o[(size_t)q * P + k * blockDim.x] = make_float2(h, __fsub_rn(al[k][q], __fsub_rn(h, ah[k][q])));
            }
    }
}

// ---------------------------------------------------------------------------
// M2L of the FP64-accurate form from integer slices on the tensor core
// (Eqs. fmmex, fmm2), per level:  Mcal[t][q][p] = sum over the edges (t, s, op)
// of sum_c T_op[q][c] O[s][c][p].  A GEMM with rows = pairs p (128 per tile),
// columns = output components q (32 per chunk) and K = (edge, input component
// c) gathered stage by stage: A panels hold the sliced expansions of every box
// of the level for a batch of pair tiles, B panels the sliced operators.  All
// scaling is by powers of two, exact: component c of the level's expansions is
// scaled by 2^-ec[c] (their largest exponent), pair p then by 2^-gp[p] (the
// largest over boxes and components), and row q of the operators by
// 2^(ec[c] - fq[q]); the product of the two scalings is undone per (p, q) in
// the epilogue.  The expansions arrive in double-FP32 (hi, lo) and leave in it.
// ---------------------------------------------------------------------------
__global__ void k_m2l_init_exp(int* __restrict__ ec, int* __restrict__ fq, int nc) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) ec[c] = fq[c] = -2000;
}

// ec[c] = largest exponent of component c over the level's boxes and pairs:
// block (box, component), threads over the pairs
__global__ void k_m2l_ecomp(const float2* __restrict__ O, int b0s, int nc, size_t P, int* __restrict__ ec) {
    const int b = blockIdx.x / nc, c = blockIdx.x % nc;
    const float2* x = O + ((size_t)(b0s + b) * nc + c) * P;
    int m = -2000;
    for (size_t p = threadIdx.x; p < P; p += blockDim.x) m = max(m, s_expo(x[p].x));
    m = s_warp_max(m);
    if ((threadIdx.x & 31) == 0 && m > -1000) atomicMax(&ec[c], m);
}

// gp[p] = largest exponent of pair p over the level's boxes and components,
// relative to ec (0 for a pair that is zero everywhere)
__global__ void k_m2l_pexp(const float2* __restrict__ O, int b0s, int nb, int nc, size_t P,
                           const int* __restrict__ ec, int* __restrict__ gp) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int m = -2000;
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < nc; ++c) {
            const int e = s_expo(O[((size_t)(b0s + b) * nc + c) * P + p].x);
            if (e > -1000) m = max(m, e - ec[c]);
        }
    gp[p] = m <= -1000 ? 0 : m;
}

// fq[q] = largest exponent of row q of the level's operators scaled by 2^ec[c]
__global__ void k_m2l_fq(const double* __restrict__ ops, const int* __restrict__ oplist, int nc,
                         const int* __restrict__ ec, int* __restrict__ fq) {
    const double* T = ops + (size_t)oplist[blockIdx.x] * nc * nc;
    for (int x = threadIdx.x; x < nc * nc; x += blockDim.x) {
        const int q = x / nc, c = x - q * nc;
        const int e = s_expo(T[x]);
        if (e > -1000 && ec[c] > -1000) atomicMax(&fq[q], e + ec[c]);
    }
}

// B panels: block (K stage cs, output chunk qc, local operator x rank
// variant), thread = output component of the chunk.  Variant v of a learned
// rank selection is the operator restricted to l, l' <= v.
template <int S>
__global__ void __launch_bounds__(32)
k_m2l_panel_B(const double* __restrict__ ops, const int* __restrict__ oplist, int nvar, int L, int nc, int nq,
              int ncs, const int* __restrict__ ec, const int* __restrict__ fq, uint8_t* __restrict__ pan) {
    const int cs = blockIdx.x, qc = blockIdx.y, lop = blockIdx.z / nvar, v = blockIdx.z % nvar;
    const int n = threadIdx.x, q = qc * kSN + n;
    const int Lv = nvar > 1 ? v : L, ncv = min(nc, (Lv + 1) * (Lv + 1));
    const double* T = ops + (size_t)oplist[lop] * nc * nc;
    const int f = q < nc && fq[q] > -1000 ? fq[q] : 0;
    uint8_t* panel = pan + (size_t)((((long long)blockIdx.z * nq + qc) * ncs) + cs) * SL<S>::b_bytes;
#pragma unroll
    for (int k8 = 0; k8 < kSK; k8 += 8) {
        long long x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = cs * kSK + k8 + u;
            x[u] = (q < ncv && c < ncv && ec[c] > -1000) ? s_fixed(T[(size_t)q * nc + c], 55 + ec[c] - f) : 0;
        }
        s_put8<S>(panel + s_off(n, k8), kBPart, x);
    }
}

// Stage list of every (target, output chunk) of the level: thread per pair
// (local target, chunk); entry k = (A panel of the source and K stage, B panel
// of the operator variant, chunk and K stage).  Chunks beyond an edge's rank
// take nothing from it.  Where the chunk and the stage both lie inside the
// edge's rank the restricted operator equals the full one there, so the full
// operator's panel (variant L) serves: only the boundary stages read panels of
// the rank's own variant, and most stages share the full operators' panels.
__global__ void k_m2l_stages(const int* __restrict__ m2l_ptr, const int* __restrict__ m2l_src,
                             const int* __restrict__ edge_bop, const int* __restrict__ lmax_e, int t0, int nt, int L,
                             int nq, int ncs, int nvar, int sb0, const long long* __restrict__ stoff,
                             int2* __restrict__ stab, int* __restrict__ nk) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nt * nq) return;
    const int tl = x / nq, qc = x - tl * nq, t = t0 + tl;
    int2* o = stab + stoff[x];
    int k = 0;
    for (int e = m2l_ptr[t]; e < m2l_ptr[t + 1]; ++e) {
        const int Le = lmax_e ? lmax_e[e] : L, nce = (Le + 1) * (Le + 1);
        if (qc * kSN >= nce) continue;
        const int ncse = min(ncs, (nce + kSK - 1) / kSK);
        const int a0 = (m2l_src[e] - sb0) * ncs;
        const int bv = ((edge_bop[e] * nvar + (nvar > 1 ? Le : 0)) * nq + qc) * ncs;
        const int bf = ((edge_bop[e] * nvar + (nvar > 1 ? L : 0)) * nq + qc) * ncs;
        const bool qin = (qc + 1) * kSN <= nce;
        for (int cs = 0; cs < ncse; ++cs)
            o[k++] = make_int2(a0 + cs, (qin && (cs + 1) * kSK <= nce ? bf : bv) + cs);
    }
    nk[x] = k;
}

// A panels of a batch of pair tiles: block (K stage cs, tile of the batch, box
// of the level), thread = pair row
template <int S>
__global__ void __launch_bounds__(128)
k_m2l_panel_A(const float2* __restrict__ O, int b0s, int nb, int nc, size_t P, int ncs, int T0,
              const int* __restrict__ ec, const int* __restrict__ gp, uint8_t* __restrict__ pan) {
    const int cs = blockIdx.x, tl = blockIdx.y, b = blockIdx.z;
    const size_t p = (size_t)(T0 + tl) * 128 + threadIdx.x;
    const bool live = p < P;
    const int g = live ? gp[p] : 0;
    const float2* x = O + (size_t)(b0s + b) * nc * P + (live ? p : 0);
    uint8_t* panel = pan + (size_t)(((long long)tl * nb + b) * ncs + cs) * SL<S>::a_bytes;
#pragma unroll
    for (int k8 = 0; k8 < kSK; k8 += 8) {
        long long v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = cs * kSK + k8 + u;
            long long r = 0;
            if (live && c < nc && ec[c] > -1000) {
                const float2 h = x[(size_t)c * P];
                r = s_fixed((double)h.x + (double)h.y, 55 - ec[c] - g);   // hi + lo, rounded once
            }
            v[u] = r;
        }
        s_put8<S>(panel + s_off(threadIdx.x, k8), kAPart, v);
    }
}

// 2^E as an FP32 number (0 below the normal range)
__device__ __forceinline__ float s_pow2f(int E) {
    return E < -126 ? 0.f : __int_as_float((min(E, 127) + 127) << 23);
}

// x += a exactly in double-FP32: TwoSum(h, a), the error into l
__device__ __forceinline__ void s_ff_add(float& h, float& l, float a) {
    const float sum = __fadd_rn(h, a);
    const float bb = __fsub_rn(sum, h);
    l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bb)), __fsub_rn(a, bb)));
    h = sum;
}

// x 2^E for any E down to -252 (two exact steps, one final rounding into the
// subnormal range); 0 below
__device__ __forceinline__ float s_ldexpf(float x, int E) {
    if (E >= -126) return x * s_pow2f(E);
    if (E >= -252) return (x * s_pow2f(E + 126)) * s_pow2f(-126);
    return 0.f;
}

// an unsigned integer below 2^23 as an exact FP32 number (magic-number trick)
__device__ __forceinline__ float s_u2f(long long u) { return __int_as_float(0x4B000000 | (int)u) - 8388608.f; }

// The exact group sums of one column as (hi, lo) FP32 numbers times 2^k,
// without FP64 arithmetic.  X 2^(12+7(S-1)) = vh 2^SH + vl (SH = 7(S-1) - 14,
// vh and vl the 64-bit integers of s_combine) is first formed exactly as
// M 2^SH + R (|M| < 2^47, 0 <= R < 2^SH) and its magnitude cut into
// non-negative chunks of at most 21 bits, which convert exactly; summed
// smallest first with TwoSum (no cancellation, all of one sign) they give
// hi + lo within about 2^-47 of |X|, and the scaling by 2^(k - 12 - 7(S-1))
// comes last.
template <int S>
__device__ __forceinline__ float2 s_combine_ff(const int (&acc)[S][kSCols], int c, int k) {
    constexpr int SH = 7 * (S - 1) - 14;
    long long vh = 0, vl = 0;
#pragma unroll
    for (int d = 0; d < S; ++d) {
        if (d < 3) vh += (long long)acc[d][c] << (7 * (2 - d));
        else vl += (long long)acc[d][c] << (7 * (S - 1 - d));
    }
    long long M = vh + (vl >> SH), R = vl & ((1LL << SH) - 1);
    const bool neg = M < 0;
    if (neg) {
        M = -M;
        if (R) {
            M -= 1;
            R = (1LL << SH) - R;
        }
    }
    float h = s_u2f(R & 0x3FFF), l = 0.f;
    s_ff_add(h, l, s_u2f(R >> 14) * s_pow2f(14));
    s_ff_add(h, l, s_u2f(M & 0x1FFFFF) * s_pow2f(SH));
    s_ff_add(h, l, s_u2f((M >> 21) & 0x1FFFFF) * s_pow2f(SH + 21));
    s_ff_add(h, l, s_u2f(M >> 42) * s_pow2f(SH + 42));
    const float hh = __fadd_rn(h, l);                    // renormalise (Fast2Sum)
    const float ll = __fsub_rn(l, __fsub_rn(hh, h));
    const int E = k - (12 + 7 * (S - 1));
    const float x = s_ldexpf(hh, E), y = s_ldexpf(ll, E);
    return neg ? make_float2(-x, -y) : make_float2(x, y);
}

struct SGemmM {
    const int2* stab; const long long* stoff; const int* nk;
    const uint8_t* panA; const uint8_t* panB;
    long long capA, capB;                  // panels in the workspace (bounds of the stage entries)
    const int* gp; const int* fq;
    float2* Mb;                            // local expansions, (hi, lo)
    size_t P;
    int nc, nq, ncs, nb, nt, t0, first_box, T0, tb, qc_outer;
    long long nitems;
    int* err;
};

// items: tile of the batch outermost, so that the CTAs in flight share the
// tile's A panels in L2; then (target, output chunk) with the chunk
// innermost, or with per-edge ranks (ten times the operator panels) the chunk
// outermost, so that one chunk's B panels stay in L2 too (measured best
// each way); x = target * nq + chunk indexes the stage lists
template <int S>
__global__ void __launch_bounds__(kSThreads, 1)
k_s_gemm_m2l(SGemmM g) {
    using C = SL<S>;
    const long long per_tile = (long long)g.nt * g.nq;
    auto sub = [&](long long it, long long& tl) {
        tl = it / per_tile;
        const int r = (int)(it - tl * per_tile);
        if (!g.qc_outer) return r;
        const int qc = r / g.nt;
        return (r - qc * g.nt) * g.nq + qc;
    };
    auto src = [&](long long it, const uint8_t*& A, const uint8_t*& Bp, int& nk) {
        long long tl;
        const int x = sub(it, tl);
        A = g.panA;
        Bp = g.panB;
        nk = g.nk[x];
    };
    auto at = [&](long long it, int kc, const uint8_t*, const uint8_t*, const uint8_t*& a, const uint8_t*& b) {
        long long tl;
        const int x = sub(it, tl);
        const int2 en = g.stab[g.stoff[x] + kc];
        const long long ai = tl * g.nb * g.ncs + en.x, bi = en.y;
        if (en.x < 0 || en.y < 0 || ai >= g.capA || bi >= g.capB) return false;
        a = g.panA + (size_t)ai * C::a_bytes;
        b = g.panB + (size_t)bi * C::b_bytes;
        return true;
    };
    auto out = [&](long long it, int row, int part, const int (&acc)[S][kSCols]) {
        long long tl;
        const int x = sub(it, tl);
        const int t = g.t0 + x / g.nq, qc = x % g.nq;
        const size_t p = (size_t)(g.T0 + tl) * 128 + row;
        if (p >= g.P) return;
        const int e = g.gp[p];
        float2* o = g.Mb + (size_t)(t - g.first_box) * g.nc * g.P + p;
#pragma unroll
        for (int c = 0; c < kSCols; ++c) {
            const int q = qc * kSN + part * kSCols + c;
            if (q < g.nc) o[(size_t)q * g.P] = s_combine_ff<S>(acc, c, e + (g.fq[q] > -1000 ? g.fq[q] : 0));
        }
    };
    s_gemm_body<S>(g.nitems, src, out, g.err, at);
}

// pairs per thread: two for the narrow chunks (each operator element read
// from shared memory feeds two multiply-adds), one for the wide ones
constexpr int ff_ppt(int lmc) { return lmc <= 9 ? 2 : 1; }

template <int MODE, typename... Args>
void launch_translate_ff(int lmc, dim3 g, cudaStream_t s, Args... args) {
    switch (lmc) {
        case 4: k_translate_ff<4, MODE, ff_ppt(4)><<<g, 128, 0, s>>>(args...); break;
        case 9: k_translate_ff<9, MODE, ff_ppt(9)><<<g, 128, 0, s>>>(args...); break;
        case 16: k_translate_ff<16, MODE, ff_ppt(16)><<<g, 128, 0, s>>>(args...); break;
        default: k_translate_ff<25, MODE, ff_ppt(25)><<<g, 128, 0, s>>>(args...); break;
    }
}

// Step (a), first half (Eq. motrans, first line), in double-FP32 arithmetic:
// W[lm][row][j] = sum over the row's ordered entries (r, s) of O^{rs}_lm C_sj,
// one block per (stored AO row, chunk of LMC components), one orbital j per
// thread, entries staged in shared memory CH at a time; C and the pair
// values arrive split into (hi, lo), W leaves in FP64.
template <int LMC>
__global__ void k_half_ff(const int* __restrict__ row_ptr, const int* __restrict__ ent_col,
                          const int* __restrict__ ent_val, const float2* __restrict__ vals, int nc,
                          const float2* __restrict__ Cff, int nocc, int nrow, double* __restrict__ W) {
    constexpr int CH = 64;
    __shared__ float2 sv[CH][LMC];
    __shared__ int scol[CH];
    const int row = blockIdx.x, c0 = blockIdx.y * LMC;
    const int e0 = row_ptr[row], e1 = row_ptr[row + 1];
    const int ncl = min(LMC, nc - c0);
    for (int jb = 0; jb < nocc; jb += blockDim.x) {
        const int j = jb + threadIdx.x;
        float ah[LMC], al[LMC];
#pragma unroll
        for (int q = 0; q < LMC; ++q) ah[q] = al[q] = 0.f;
        for (int ec = e0; ec < e1; ec += CH) {
            const int n = min(CH, e1 - ec);
            __syncthreads();
            for (int x = threadIdx.x; x < n * LMC; x += blockDim.x) {
                const int k = x / LMC, q = x - k * LMC;
                sv[k][q] = q < ncl ? vals[(size_t)ent_val[ec + k] * nc + c0 + q] : make_float2(0.f, 0.f);
            }
            for (int x = threadIdx.x; x < n; x += blockDim.x) scol[x] = ent_col[ec + x];
            __syncthreads();
            for (int k = 0; k < n; ++k) {
                const float2 c = j < nocc ? Cff[(size_t)scol[k] * nocc + j] : make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < LMC; ++q) ff_fma(ah[q], al[q], sv[k][q], c);
            }
        }
        if (j < nocc) {
#pragma unroll
            for (int q = 0; q < LMC; ++q)
                if (q < ncl) W[((size_t)(c0 + q) * nrow + row) * nocc + j] = (double)ah[q] + (double)al[q];
        }
    }
}

template <int S>
cudaError_t l2p_attrs() {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_s_gemm_e<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, SL<S>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_s_gemm_a<S, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, SL<S>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_s_gemm_a<S, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SL<S>::smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return cudaSuccess;
}

template <int S, typename T>
cudaError_t l2p_slices_typed(const SliceArgs& a, cudaStream_t s) {
    const T* W = (const T*)a.W;
    const T* Mbox = (const T*)a.Mbox;
    cudaError_t e0 = l2p_attrs<S>();
    if (e0 != cudaSuccess) return e0;
    const int jc = (a.nocc + kSK - 1) / kSK, KC = a.nc * jc, nct = (a.nocc + kSN - 1) / kSN;
    k_s_rowexp<T><<<(a.nrow + 7) / 8, 256, 0, s>>>(W, a.lscale, a.nrow, a.nocc, a.nc, a.erow);
    const long long ncol = (long long)a.nleaf * a.nocc;
    k_s_colexp<T><<<(unsigned)((ncol + 7) / 8), 256, 0, s>>>(Mbox, a.lscale, a.nleaf, a.nocc, a.nc, a.leaf_store0,
                                                          a.fcol);
    // leaf batches whose panels fit the workspace: build, then multiply
    for (int bt = 0; bt < a.nbatch_e; ++bt) {
        const int B0 = a.batch_e[bt], B1 = a.batch_e[bt + 1];
        if (B1 <= B0) continue;
        const long long pA0 = a.offA_h[B0];
        uint8_t* panB = a.panA + (size_t)(a.offA_h[B1] - pA0) * SL<S>::a_bytes;
        k_s_panel_A<S, T><<<dim3(KC, a.max_rt, B1 - B0), 128, 0, s>>>(a.leaf_rowoff, W, a.lscale, a.erow, a.nocc,
                                                                   a.nrow, jc, KC, a.rtA, a.offA, B0, pA0, a.panA);
        k_s_panel_B<S, T><<<dim3((KC + 3) / 4, nct, B1 - B0), 128, 0, s>>>(Mbox, a.lscale, a.fcol, a.nocc, a.nc,
                                                                        a.leaf_store0, jc, KC, nct, B0, panB);
        SGemmE g{};
        g.leaf_rowoff = a.leaf_rowoff; g.rtA = a.rtA; g.offA = a.offA; g.item0 = a.item0;
        g.erow = a.erow; g.fcol = a.fcol; g.panA = a.panA; g.panB = panB; g.KB = a.KB;
        g.nleaf = B1; g.nocc = a.nocc; g.nrow = a.nrow; g.KC = KC; g.nct = nct; g.nsplit = a.nsplit;
        g.B0 = B0; g.it0 = a.item0_h[B0]; g.nitems = a.item0_h[B1] - a.item0_h[B0]; g.panA0 = pA0;
        g.err = a.err;
        const int grid = (int)std::min<long long>(g.nitems, a.sm_count);
        if (grid > 0) k_s_gemm_e<S><<<grid, kSThreads, SL<S>::smem, s>>>(g);
    }
    return cudaGetLastError();
}

template <int S, typename T>
cudaError_t full_slices_typed(const SliceArgs& a, const T* Ct, T* Obox, cudaStream_t s) {
    const T* W = (const T*)a.W;
    cudaError_t e = l2p_attrs<S>();
    if (e != cudaSuccess) return e;
    const int nct = (a.nocc + kSN - 1) / kSN, nti = (a.nocc + 127) / 128;
    k_s_a2_expC<T><<<dim3(a.nleaf, (a.nocc + 127) / 128), 128, 0, s>>>(a.leaf_rowoff, a.leaf_aos, Ct, a.nocc, a.eC);
    k_s_a2_expW<T><<<dim3(a.nleaf * a.nc, (a.nocc + 127) / 128), 128, 0, s>>>(a.leaf_rowoff, W, a.nocc, a.nrow, a.nc,
                                                                            a.eW);
    for (int bt = 0; bt < a.nbatch_a; ++bt) {
        const int B0 = a.batch_a[bt], B1 = a.batch_a[bt + 1];
        if (B1 <= B0) continue;
        const long long pA0 = a.offAa_h[B0], pB0 = a.offBa_h[B0];
        uint8_t* panB = a.panAa + (size_t)(a.offAa_h[B1] - pA0) * SL<S>::a_bytes;
        k_s_a2_panel_A<S, T><<<dim3(a.max_kca, nti, B1 - B0), 128, 0, s>>>(a.leaf_rowoff, a.leaf_aos, Ct, a.eC, a.nocc,
                                                                         nti, a.kca, a.offAa, B0, pA0, a.panAa);
        k_s_a2_panel_B<S, T><<<dim3((a.max_kca + 3) / 4, nct, (B1 - B0) * a.nc), 128, 0, s>>>(
            a.leaf_rowoff, W, a.eW, a.nocc, a.nrow, a.nc, nct, a.kca, a.offBa, B0, pB0, panB);
        SGemmA g{};
        g.kca = a.kca; g.offAa = a.offAa; g.offBa = a.offBa; g.tpair = a.tpair;
        g.eC = a.eC; g.eW = a.eW; g.panA = a.panAa; g.panB = panB; g.Obox = Obox;
        g.nleaf = a.nleaf; g.nocc = a.nocc; g.nc = a.nc; g.nct = nct; g.ntp = a.ntp; g.leaf_store0 = a.leaf_store0;
        g.B0 = B0; g.nitems = (long long)(B1 - B0) * a.nc * a.ntp; g.panA0 = pA0; g.panB0 = pB0;
        g.err = a.err;
        const int grid = (int)std::min<long long>(g.nitems, a.sm_count);
        if (grid > 0) k_s_gemm_a<S, T><<<grid, kSThreads, SL<S>::smem, s>>>(g);
    }
    return cudaGetLastError();
}

}  // namespace

int slice_stage_k() { return kSK; }
cudaError_t set_slice_wait_limit(long long polls) {
    const uint32_t v = polls < 0 ? kWaitS : (uint32_t)std::min<long long>(polls, 0xffffffffLL);
    return cudaMemcpyToSymbol(g_s_full_wait, &v, sizeof(v));
}

int slice_tile_n() { return kSN; }
int slice_max_stages() { return kChunk * kMaxChunks; }
size_t slice_panel_bytes(int S, bool a) { return (size_t)S * (a ? kAPart : kBPart); }

cudaError_t full_slices(const SliceArgs& a, const void* Ct, void* Obox, cudaStream_t s) {
    if (a.f32) {
        if (a.S == 4) return full_slices_typed<4, float>(a, (const float*)Ct, (float*)Obox, s);
        return cudaErrorInvalidValue;
    }
    if (a.S == 7) return full_slices_typed<7, double>(a, (const double*)Ct, (double*)Obox, s);
    if (a.S == 6) return full_slices_typed<6, double>(a, (const double*)Ct, (double*)Obox, s);
    return cudaErrorInvalidValue;
}

cudaError_t half_ff(const HalfFFArgs& h, cudaStream_t s) {
    const size_t nv = (size_t)h.nvals * h.nc, ncf = (size_t)h.nao * h.nocc;
    k_ff_ops<<<std::max(1, (int)std::min<size_t>((nv + 255) / 256, 8192)), 256, 0, s>>>(h.vals, nv, h.vals_ff);
    k_ff_ops<<<std::max(1, (int)std::min<size_t>((ncf + 255) / 256, 8192)), 256, 0, s>>>(h.Ct, ncf, h.C_ff);
    dim3 g(h.nrow, (h.nc + h.lmc - 1) / h.lmc);
    switch (h.lmc) {
        case 4: k_half_ff<4><<<g, h.nth, 0, s>>>(h.row_ptr, h.ent_col, h.ent_val, h.vals_ff, h.nc, h.C_ff, h.nocc,
                                                 h.nrow, h.W); break;
        case 9: k_half_ff<9><<<g, h.nth, 0, s>>>(h.row_ptr, h.ent_col, h.ent_val, h.vals_ff, h.nc, h.C_ff, h.nocc,
                                                 h.nrow, h.W); break;
        case 25: k_half_ff<25><<<g, h.nth, 0, s>>>(h.row_ptr, h.ent_col, h.ent_val, h.vals_ff, h.nc, h.C_ff, h.nocc,
                                                   h.nrow, h.W); break;
        default: k_half_ff<16><<<g, h.nth, 0, s>>>(h.row_ptr, h.ent_col, h.ent_val, h.vals_ff, h.nc, h.C_ff, h.nocc,
                                                   h.nrow, h.W); break;
    }
    return cudaGetLastError();
}

static int ff_lmc(int nc) { return nc <= 4 ? 4 : nc <= 9 ? 9 : nc <= 16 ? 16 : 25; }

// One level of the sliced M2L: exponents, operator panels and stage lists,
// then per batch of pair tiles the expansions' panels and the GEMM
template <int S>
cudaError_t m2l_slices_level_t(const FFArgs& f, int lev, cudaStream_t s) {
    const SM2LArgs& m = *f.sm;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_s_gemm_m2l<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SL<S>::smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int t0 = m.lt0[lev], nt = m.lnt[lev], nb = nt;   // sources and targets: the level's boxes
    const int b0s = t0 - f.first_box;
    const size_t P = (size_t)f.P;
    const auto* O = reinterpret_cast<const float2*>(f.Ob);
    k_m2l_init_exp<<<1, 256, 0, s>>>(m.ec, m.fq, f.nc);
    k_m2l_ecomp<<<nb * f.nc, 256, 0, s>>>(O, b0s, f.nc, P, m.ec);
    k_m2l_pexp<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(O, b0s, nb, f.nc, P, m.ec, m.gp);
    const int nopl = m.lnopl[lev];
    const int* oplist = m.oplist + m.lopl0[lev];
    if (nopl > 0) {
        k_m2l_fq<<<nopl, 256, 0, s>>>(f.ops, oplist, f.nc, m.ec, m.fq);
        k_m2l_panel_B<S><<<dim3(m.ncs, m.nq, nopl * m.nvar), 32, 0, s>>>(f.ops, oplist, m.nvar, f.L, f.nc, m.nq,
                                                                        m.ncs, m.ec, m.fq, m.panB);
    }
    const long long* stoff = m.stoff + m.lst0[lev];
    k_m2l_stages<<<(nt * m.nq + 127) / 128, 128, 0, s>>>(f.m2l_ptr, f.m2l_src, m.edge_bop, f.lmax_e, t0, nt, f.L,
                                                         m.nq, m.ncs, m.nvar, t0, stoff, m.stab, m.nk);
    const int tb = std::max(1, m.ltb[lev]);
    for (int T0 = 0; T0 < m.ntile; T0 += tb) {
        const int nbt = std::min(tb, m.ntile - T0);
        k_m2l_panel_A<S><<<dim3(m.ncs, nbt, nb), 128, 0, s>>>(O, b0s, nb, f.nc, P, m.ncs, T0, m.ec, m.gp, m.panA);
        SGemmM g{};
        g.stab = m.stab; g.stoff = stoff; g.nk = m.nk;
        g.panA = m.panA; g.panB = m.panB; g.capA = m.capA; g.capB = m.capB;
        g.gp = m.gp; g.fq = m.fq; g.Mb = reinterpret_cast<float2*>(f.Mb); g.P = P;
        g.nc = f.nc; g.nq = m.nq; g.ncs = m.ncs; g.nb = nb; g.nt = nt; g.t0 = t0; g.first_box = f.first_box;
        g.T0 = T0; g.tb = nbt; g.qc_outer = m.nvar > 1 ? 1 : 0;
        g.nitems = (long long)nbt * nt * m.nq;
        g.err = f.err;
        const int grid = (int)std::min<long long>(g.nitems, std::max(f.sm_count, 1));
        k_s_gemm_m2l<S><<<grid, kSThreads, SL<S>::smem, s>>>(g);
    }
    return cudaGetLastError();
}

cudaError_t m2l_slices_level(const FFArgs& f, int lev, cudaStream_t s) {
    switch (f.sm->S) {
        case 7: return m2l_slices_level_t<7>(f, lev, s);
        case 6: return m2l_slices_level_t<6>(f, lev, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t m2m_ff(const FFArgs& f, cudaStream_t s) {
    // the leaves' multipoles (FP64 from step (a)) to (hi, lo); M2M writes
    // the parents' in (hi, lo)
    const size_t nleafv = (size_t)(f.nstore - f.leaf_store0) * f.nc * f.P;
    const int blocks = 4 * std::max(f.sm_count, 1);
    k_ff_split<<<blocks, 256, 0, s>>>(f.Ob + (size_t)f.leaf_store0 * f.nc * f.P, nleafv);
    const size_t nops = (size_t)f.nops * f.nc * f.nc;
    k_ff_ops<<<std::max(1, (int)std::min<size_t>((nops + 255) / 256, 4096)), 256, 0, s>>>(f.ops, nops, f.ops_ff);
    const int lmc = ff_lmc(f.nc), nchunk = (f.nc + lmc - 1) / lmc;
    auto* ob = reinterpret_cast<float2*>(f.Ob);
    for (int lev = f.D; lev >= 3; --lev) {
        const int t0 = f.level_off[lev - 1], nt = f.level_off[lev] - t0;
        if (nt <= 0) continue;
        dim3 g(nt, (unsigned)((f.P + 128 * ff_ppt(lmc) - 1) / (128 * ff_ppt(lmc))), nchunk);
        launch_translate_ff<0>(lmc, g, s, f.P, f.nc, f.L, f.first_box, t0, f.child_ptr, f.child_list, f.m2m_op,
                               (const int*)nullptr, f.parent, (const int*)nullptr, (const float2*)f.ops_ff,
                               (const float2*)ob, ob);
    }
    return cudaGetLastError();
}

cudaError_t ff_join(const FFArgs& f, cudaStream_t s) {
    k_ff_join<<<4 * std::max(f.sm_count, 1), 256, 0, s>>>(f.Ob, (size_t)f.nstore * f.nc * f.P);
    return cudaGetLastError();
}

cudaError_t m2l_ff(const FFArgs& f, cudaStream_t s) {
    const size_t n = (size_t)f.nstore * f.nc * f.P;
    const int blocks = 4 * std::max(f.sm_count, 1);
    if (!f.m2m_done) {   // multipoles still FP64 (the FP64 M2M ran)
        const size_t nops = (size_t)f.nops * f.nc * f.nc;
        k_ff_ops<<<std::max(1, (int)std::min<size_t>((nops + 255) / 256, 4096)), 256, 0, s>>>(f.ops, nops,
                                                                                              f.ops_ff);
        k_ff_split<<<blocks, 256, 0, s>>>(f.Ob, n);
    }
    const int lmc = ff_lmc(f.nc), nchunk = (f.nc + lmc - 1) / lmc;
    for (int lev = 2; lev <= f.D; ++lev) {
        const int t0 = f.level_off[lev], nt = f.level_off[lev + 1] - t0;
        if (nt <= 0) continue;
        dim3 g(nt, (unsigned)((f.P + 128 * ff_ppt(lmc) - 1) / (128 * ff_ppt(lmc))), nchunk);
        if (f.sm) {
            // M2L from slices on the tensor core, then the parent's L2L added
            // in double-FP32
            cudaError_t e = m2l_slices_level(f, lev, s);
            if (e != cudaSuccess) return e;
            if (lev >= 3)
                launch_translate_ff<4>(lmc, g, s, f.P, f.nc, f.L, f.first_box, t0, f.m2l_ptr, f.m2l_src, f.m2l_op,
                                       f.lmax_e, f.parent, f.l2l_op, (const float2*)f.ops_ff,
                                       reinterpret_cast<const float2*>(f.Ob), reinterpret_cast<float2*>(f.Mb));
            continue;
        }
        launch_translate_ff<3>(lmc, g, s, f.P, f.nc, f.L, f.first_box, t0, f.m2l_ptr, f.m2l_src, f.m2l_op, f.lmax_e,
                               f.parent, f.l2l_op, (const float2*)f.ops_ff, reinterpret_cast<const float2*>(f.Ob),
                               reinterpret_cast<float2*>(f.Mb));
    }
    k_ff_join<<<blocks, 256, 0, s>>>(f.Ob, n);
    k_ff_join<<<blocks, 256, 0, s>>>(f.Mb, n);
    return cudaGetLastError();
}

cudaError_t l2p_slices(const SliceArgs& a, cudaStream_t s) {
    if (a.f32) {
        if (a.S == 4) return l2p_slices_typed<4, float>(a, s);
        return cudaErrorInvalidValue;
    }
    if (a.S == 7) return l2p_slices_typed<7, double>(a, s);
    if (a.S == 6) return l2p_slices_typed<6, double>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace occk
