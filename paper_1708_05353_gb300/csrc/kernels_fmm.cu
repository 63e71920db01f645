// Steps (a)-(e) of the far-field occupied exchange on SIMT cores, in FP64
// (DFMA) or FP32 (FFMA); K and the energy are always reduced in FP64.
//
// Layouts in HBM (P = nocc(nocc+1)/2 stored occupied pairs i <= j, packed
// row-major upper triangle; W and KB keep every orbital):
//   Ct   [nao][nocc]            row-major copy of C
//   W    [nc][nrow][nocc]       O^{rj,X}_lm for the AO set S_B of every leaf,
//                               leaves stacked (row = leaf_rowoff[B] + local)
//   Obox [box][nc][P]           O^{ij,X}_lm (i <= j) for boxes of levels 2..D
//   Mbox [box][nc][P]           Mcal^{ij}_lm(X), same boxes
//   KB   [nrow][nocc]           per-leaf partial K rows (FP64)
// Every pair-indexed access is coalesced along p (or along j).
#include <algorithm>
#include <type_traits>
#include <cstdio>

#include "fmm_bodies.cuh"
#include "occk_internal.h"

namespace occk {

namespace {

using body::k_final_energy;
using body::k_zero_K;

template <typename T>
__global__ void k_transpose_C(const double* __restrict__ C, int ldc, int nao, int nocc, T* __restrict__ Ct) {
    body::transpose_body<T>(blockIdx.x, blockIdx.y, 0, C, ldc, nao, nocc, Ct);
}

template <typename T, int LMC>
__global__ void k_half(const int* __restrict__ row_ptr, const int* __restrict__ ent_col,
                       const int* __restrict__ ent_val, const T* __restrict__ vals, int nc,
                       const T* __restrict__ Ct, int nocc, int nrow, T* __restrict__ W) {
    body::half_body<T, LMC>(blockIdx.x, blockIdx.y, 0, row_ptr, ent_col, ent_val, vals, nc, Ct, nocc, nrow, W);
}

template <typename T, int BM, int BK, int TM>
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
k_full(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos, const T* __restrict__ Ct,
       const T* __restrict__ W, int nocc, int nrow, int nc, int ntile, T* __restrict__ Obox, int leaf_store0,
       const unsigned char* __restrict__ tskip) {
    // screened: tiles whose every pair is dropped by the bound are not formed
    if (tskip && tskip[blockIdx.x]) return;
    body::full_body<T, BM, BK, TM>(blockIdx.x, blockIdx.y, 0, leaf_rowoff, leaf_aos, Ct, W, nocc, nrow, nc, ntile,
                                   Obox, leaf_store0);
}

template <typename T, int LMC>
__global__ void __launch_bounds__(128)
k_translate(int mode, int P, int nc, int L, int first_box, int tgt0, const int* __restrict__ ptr,
            const int* __restrict__ list, const int* __restrict__ opidx, const int* __restrict__ lmax_e,
            const int* __restrict__ parent, const T* __restrict__ ops, const T* __restrict__ in,
            T* __restrict__ out, int accumulate, const int* __restrict__ l2l_opidx, const T* parent_in,
            const int* __restrict__ pcount) {
    // blockIdx.x = target, blockIdx.y = pair block: consecutive blocks work on
    // the same pairs of different targets, so the source slices they share
    // stay in L2 (a pair block of every box of a level is well under 1 MB)
    body::translate_body<T, LMC>(blockIdx.y, blockIdx.x, blockIdx.z, mode, P, nc, L, first_box, tgt0, ptr, list,
                                 opidx, lmax_e, parent, ops, in, out, accumulate, l2l_opidx, parent_in, pcount);
}

// grid.y runs over the 128-orbital tiles tile0, tile0 + 1, ... (all of them
// unless a column block restricts the output columns)
template <int TI>
__global__ void __launch_bounds__(256)
k_l2p_r32(int nsplit, const int* __restrict__ leaf_rowoff, const double* __restrict__ W,
          const double* __restrict__ Mbox, int nocc, int nrow, int nc, int leaf_store0, double* __restrict__ KB,
          const unsigned char* __restrict__ tflag, int tile0) {
    body::l2p_rect_body<TI>(blockIdx.x, blockIdx.y + tile0, blockIdx.z, nsplit, leaf_rowoff, W, Mbox, nocc, nrow,
                            nc, leaf_store0, KB, tflag);
}

template <int TI>
__global__ void __launch_bounds__(256)
k_l2p_r96f(int nsplit, const int* __restrict__ leaf_rowoff, const float* __restrict__ W,
           const float* __restrict__ Mbox, int nocc, int nrow, int nc, int leaf_store0, double* __restrict__ KB,
           const unsigned char* __restrict__ tflag, int tile0) {
    body::l2p_rect_body_f<TI>(blockIdx.x, blockIdx.y + tile0, blockIdx.z, nsplit, leaf_rowoff, W, Mbox, nocc, nrow,
                              nc, leaf_store0, KB, tflag);
}

__global__ void k_reduce_K(const int* __restrict__ ao_row_ptr, const int* __restrict__ ao_rows,
                           const double* __restrict__ KB, int nao, int nocc, const double* __restrict__ C, int ldc,
                           double* __restrict__ K, int ldk, double* __restrict__ part, int nsplit,
                           size_t split_stride, int col0, int col1) {
    body::reduce_body(blockIdx.x, 0, gridDim.x, ao_row_ptr, ao_rows, KB, nao, nocc, C, ldc, K, ldk, part, nsplit,
                      split_stride, col0, col1);
}

// ---------------------------------------------------------------------------
// FMA throughput probe: NACC independent accumulators per thread, four FMAs
// on each per loop trip, so neither latency nor loop overhead limits the
// issue rate; the result is consumed so that nothing is removed.  Form 0
// updates a = a m + c (one shared multiplier and addend), form 1 a = b m + a
// with a different multiplicand b per accumulator (the operand pattern of a
// GEMM's inner loop).
// The multiplier and addend come from device memory (mc[0], mc[1]) so that
// they sit in registers like a GEMM's operands, not in the constant bank.
template <typename T, int NACC, int FORM>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T seed, const T* __restrict__ mc) {
    T a[NACC], b[NACC];
    const T m = mc[0], c = mc[1];
#pragma unroll
    for (int q = 0; q < NACC; ++q) {
        a[q] = seed + T(threadIdx.x + q) * c;
        b[q] = c * T(q + 1);
    }
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int q = 0; q < NACC; ++q) {
                if constexpr (FORM == 0)
                    a[q] = fma(a[q], m, c);
                else
                    a[q] = fma(b[q], m, a[q]);
            }
        }
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < NACC; ++q) s += a[q];
    if (s == T(-1.2345)) out[threadIdx.x] = s;
}

template <typename T, int NACC>
void launch_probe(int form, int blocks, T* buf, int iters, cudaStream_t s) {
    const T* mc = buf + 512;
    if (form == 0)
        k_fma_probe<T, NACC, 0><<<blocks, 256, 0, s>>>(buf, iters, T(1), mc);
    else
        k_fma_probe<T, NACC, 1><<<blocks, 256, 0, s>>>(buf, iters, T(1), mc);
}

// ---------------------------------------------------------------------------
// Occupied-pair screening (the paper's proposed extension to localised
// orbitals, Sec. IV): a pair p = (i <= j) is kept when
//   n_p^2 = sum_leaves sum_lm w_lm O[leaf][lm][p]^2 >= tau^2,
// w = 1 for m = 0 and 2 for the Re and Im components of m > 0 (the real form
// of sum over m = -l..l of |O_lm|^2).  The tree passes then run on the kept
// pairs, compacted to the front of every [box][lm] row.
// ---------------------------------------------------------------------------
// Step (a) tiles that screening drops whole (Cauchy-Schwarz over the leaf's
// AO rows):  sum_lm w_lm |O^{ij,X}_lm|^2 <= a2[X][i] b2[X][j] with
// a2[X][i] = sum_{r in S_X} C_ri^2 and b2[X][j] = sum_lm w_lm sum_{r in S_X}
// W_lm[r][j]^2, so n_ij^2 <= sum_X a2[X][i] b2[X][j].  A tile whose largest
// bound is below tau^2 / 2 (the half covers the rounding of the bound) holds
// only pairs that the exact criterion drops; it is not formed.
// grid (leaf X, 128-orbital chunk, 1 + nc): z = 0 writes a2[X][i], z = 1 +
// lm writes the component's part of b2, bp[lm][X][j] = w_lm sum_{r in S_X}
// W_lm[r][j]^2 (summed over lm, in order, by k_bound_tiles).
template <typename T>
__global__ void __launch_bounds__(128)
k_bound_ab(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos, const T* __restrict__ Ct,
           const T* __restrict__ W, int nocc, int nrow, int nleaf, float* __restrict__ a2, float* __restrict__ bp) {
    const int X = blockIdx.x, i = blockIdx.y * blockDim.x + threadIdx.x, z = blockIdx.z;
    if (i >= nocc) return;
    const int r0 = leaf_rowoff[X], r1 = leaf_rowoff[X + 1];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (z == 0) {
        int r = r0;
        for (; r + 4 <= r1; r += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float c = (float)Ct[(size_t)leaf_aos[r + u] * nocc + i];
                acc[u] += c * c;
            }
        }
        for (; r < r1; ++r) {
            const float c = (float)Ct[(size_t)leaf_aos[r] * nocc + i];
            acc[0] += c * c;
        }
        a2[(size_t)X * nocc + i] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        return;
    }
    const int lm = z - 1;
    int l = 0;
    while ((l + 1) * (l + 1) <= lm) ++l;
    const float w = lm == l * l ? 1.f : 2.f;
    const T* Wl = W + (size_t)lm * nrow * nocc + i;
    int r = r0;
    for (; r + 4 <= r1; r += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float x = (float)Wl[(size_t)(r + u) * nocc];
            acc[u] += x * x;
        }
    }
    for (; r < r1; ++r) {
        const float x = (float)Wl[(size_t)r * nocc];
        acc[0] += x * x;
    }
    bp[((size_t)lm * nleaf + X) * nocc + i] = w * ((acc[0] + acc[1]) + (acc[2] + acc[3]));
}

// grid (triangular tile ti <= tj of BM x BM pairs in the order of k_full's
// grid, slab of 8 rows of the tile): a slab holding a pair i <= j with
// sum_X a2[X][i] b2[X][j] >= half_tau2 clears tskip[tile] (set to 1 before).
__global__ void __launch_bounds__(256)
k_bound_tiles(const float* __restrict__ a2, const float* __restrict__ bp, int nleaf, int nc, int nocc, int BM,
              int ntile, float half_tau2, unsigned char* __restrict__ tskip) {
    constexpr int RS = 8;
    __shared__ float sa[32][RS];
    __shared__ float sb[32][128];
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int i0 = ti * BM + blockIdx.y * RS, j0 = tj * BM;
    // each thread owns (RS * BM) / 256 pairs of the slab (4 or 2)
    const int per = (RS * BM) / 256;
    float u[4] = {0.f, 0.f, 0.f, 0.f};
    for (int x0 = 0; x0 < nleaf; x0 += 32) {
        const int nx = min(32, nleaf - x0);
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * RS; e += blockDim.x) {
            const int x = e / RS, c = e % RS;
            sa[x][c] = (x < nx && i0 + c < nocc) ? a2[(size_t)(x0 + x) * nocc + i0 + c] : 0.f;
        }
        for (int e = threadIdx.x; e < 32 * BM; e += blockDim.x) {
            const int x = e / BM, c = e % BM;
            float b = 0.f;
            if (x < nx && j0 + c < nocc)
                for (int lm = 0; lm < nc; ++lm) b += bp[((size_t)lm * nleaf + x0 + x) * nocc + j0 + c];
            sb[x][c] = b;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= per) break;
            const int e = threadIdx.x + 256 * k, ii = e / BM, jj = e % BM;
            float acc = 0.f;
            for (int x = 0; x < nx; ++x) acc += sa[x][ii] * sb[x][jj];
            u[k] += acc;
        }
    }
    bool hit = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= per) break;
        const int e = threadIdx.x + 256 * k, ii = e / BM, jj = e % BM;
        const int i = i0 + ii, j = j0 + jj;
        hit |= i < nocc && j < nocc && i <= j && u[k] >= half_tau2;
    }
    if (__syncthreads_or(hit) && threadIdx.x == 0) tskip[blockIdx.x] = 0;   // every writer stores 0
}

// Column block [col0, col1): sets tskip[t] (tile not formed) for every step
// (a) tile (ti <= tj, k_full's triangular order) none of whose rows or
// columns lies in the block (its pairs touch no column of the block and are
// dropped anyway).
__global__ void k_col_tiles(int ntile, int BM, int col0, int col1, unsigned char* __restrict__ tskip) {
    const int n = ntile * (ntile + 1) / 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int r = t, ti = 0;
        while (r >= ntile - ti) {
            r -= ntile - ti;
            ++ti;
        }
        const int tj = ti + r;
        auto hits = [&](int tt) { return tt * BM < col1 && (tt + 1) * BM > col0; };
        if (!hits(ti) && !hits(tj)) tskip[t] = 1;
    }
}

// Pass 1a: partial norms over groups of kPairLG leaves, part[g][p], in the
// storage type.  A block takes 8 x 256 consecutive pairs of one group and
// walks its leaf-component rows, reading 8 KB contiguous from each.
constexpr int kPairBlk = 256, kPairLG = 8, kPairPPT = 8;

template <typename T>
__global__ void __launch_bounds__(kPairBlk)
k_pair_part(const T* __restrict__ Oleaf, int nleaf, int nc, long long P, T* __restrict__ part) {
    __shared__ T wsh[body::kNcMax];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int l = 0;
        while ((l + 1) * (l + 1) <= c) ++l;
        wsh[c] = c == l * l ? T(1) : T(2);
    }
    __syncthreads();
    const long long base = (long long)blockIdx.x * (kPairBlk * kPairPPT) + threadIdx.x;
    const int B0 = blockIdx.y * kPairLG, B1 = min(nleaf, B0 + kPairLG);
    T acc[kPairPPT];
#pragma unroll
    for (int k = 0; k < kPairPPT; ++k) acc[k] = T(0);
    for (int r = B0 * nc; r < B1 * nc; ++r) {
        const T w = wsh[r % nc];
        const T* row = Oleaf + (size_t)r * P;
        T x[kPairPPT];
#pragma unroll
        for (int k = 0; k < kPairPPT; ++k) {
            const long long p = base + (long long)k * kPairBlk;
            x[k] = p < P ? row[p] : T(0);
        }
#pragma unroll
        for (int k = 0; k < kPairPPT; ++k) acc[k] += w * x[k] * x[k];
    }
#pragma unroll
    for (int k = 0; k < kPairPPT; ++k) {
        const long long p = base + (long long)k * kPairBlk;
        if (p < P) part[(size_t)blockIdx.y * P + p] = acc[k];
    }
}

// Pass 1b (kPairBlk pairs per block): each pair's norm (the groups summed in
// order, in FP64) and keep flag (stored in inv as 1 / 0), and the block's
// count of kept pairs.
// With a column block [col0, col1) (col1 > col0) a pair is kept only if it
// touches the block (i or j in it); with ngrp = 0 no norm is read and the
// threshold tau2 must be 0.
template <typename T>
__global__ void __launch_bounds__(kPairBlk)
k_pair_flag(const T* __restrict__ part, int ngrp, long long P, double tau2, double* __restrict__ n2,
            int* __restrict__ inv, int* __restrict__ bcount, const unsigned char* __restrict__ tskip, int nocc,
            int BM, int col0, int col1) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    if (p < P) {
        bool formed = true;
        const bool colblk = col1 > col0;
        if (tskip || colblk) {
            // pair (i, j) from its packed index; its step (a) tile (ti, tj)
            const double b = 2.0 * nocc + 1.0;
            long long i = (long long)((b - sqrt(b * b - 8.0 * (double)p)) * 0.5);
            auto off = [&](long long r) { return r * (2LL * nocc - r + 1) / 2; };
            if (i < 0) i = 0;
            if (i > nocc - 1) i = nocc - 1;
            while (i > 0 && off(i) > p) --i;
            while (i + 1 < nocc && off(i + 1) <= p) ++i;
            const long long j = i + (p - off(i));
            if (tskip) {
                const int nt = (nocc + BM - 1) / BM, ti = (int)(i / BM), tj = (int)(j / BM);
                const int t = ti * nt - ti * (ti - 1) / 2 + (tj - ti);
                formed = !tskip[t];
            }
            if (colblk) formed = formed && ((i >= col0 && i < col1) || (j >= col0 && j < col1));
        }
        double acc = 0.0;
        if (formed)
            for (int g = 0; g < ngrp; ++g) acc += (double)part[(size_t)g * P + p];
        n2[p] = acc;
        keep = formed && acc >= tau2;
        inv[p] = keep;
    }
    const int n = __syncthreads_count(keep);
    if (threadIdx.x == 0) bcount[blockIdx.x] = n;
}

// Pass 2 (one block): exclusive scan of the block counts in place, total in
// *count.
__global__ void __launch_bounds__(1024) k_pair_scan(int* __restrict__ bcount, int nb, int* __restrict__ count) {
    __shared__ int part[1024];
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int sum = 0;
    for (int b = b0; b < b1; ++b) sum += bcount[b];
    part[threadIdx.x] = sum;
    __syncthreads();
    // inclusive scan of the 1024 partial sums (Hillis-Steele)
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int b = b0; b < b1; ++b) {
        const int t = bcount[b];
        bcount[b] = run;
        run += t;
    }
    if (threadIdx.x == blockDim.x - 1) *count = part[threadIdx.x];
}

// Pass 3 (kPairBlk pairs per block): kept pairs in increasing order (keep[q]
// = p) and the inverse map (inv[p] = q or -1).  Deterministic.
__global__ void __launch_bounds__(kPairBlk)
k_pair_compact(long long P, const int* __restrict__ boff, int* __restrict__ keep, int* __restrict__ inv) {
    __shared__ int wsum[32];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int flag = p < P ? inv[p] : 0;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the warp counts
        const int nw = (int)(blockDim.x >> 5);
        int v = (int)lane < nw ? wsum[lane] : 0;
        const int own = v;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= (unsigned)off) v += u;
        }
        if ((int)lane < nw) wsum[lane] = v - own;
    }
    __syncthreads();
    if (p < P) {
        if (flag) {
            const int q = boff[blockIdx.x] + wsum[warp] + __popc(m & ((1u << lane) - 1u));
            keep[q] = (int)p;
            inv[p] = q;
        } else {
            inv[p] = -1;
        }
    }
}

// Flags of the step (e) tiles that hold a kept pair: tf[i / 128][j / 8] for
// both orderings of every kept pair (i <= j), so that L2P can skip K steps
// whose Mcal tile is all dropped pairs.  tf is zeroed before.
__global__ void k_pair_tiles(const int* __restrict__ keep, const int* __restrict__ count, int nocc,
                             unsigned char* __restrict__ tf) {
    const long long n = *count;
    const int nj8 = (nocc + 7) / 8;
    const double b = 2.0 * nocc + 1.0;
    auto off = [&](long long r) { return r * (2LL * nocc - r + 1) / 2; };
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const long long p = keep[q];
        // row i of the packed triangle: the largest i with off(i) <= p,
        // off(i) = i (2 nocc - i + 1) / 2
        long long i = (long long)((b - sqrt(b * b - 8.0 * (double)p)) * 0.5);
        if (i < 0) i = 0;
        if (i > nocc - 1) i = nocc - 1;
        while (i > 0 && off(i) > p) --i;
        while (i + 1 < nocc && off(i + 1) <= p) ++i;
        const long long j = i + (p - off(i));
        tf[(size_t)(i / 128) * nj8 + j / 8] = 1;
        tf[(size_t)(j / 128) * nj8 + i / 8] = 1;
    }
}

// dst[row][q] = src[row][keep[q]] for q < *count (rows of length P); a fixed
// grid (the kept count is known on the device only) strides over q
template <typename T>
__global__ void k_pair_gather(const T* __restrict__ src, T* __restrict__ dst, long long P,
                              const int* __restrict__ keep, const int* __restrict__ count) {
    const long long n = *count;
    const size_t row = (size_t)blockIdx.y * P;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x)
        dst[row + q] = src[row + keep[q]];
}

// dst[row][p] = src[row][inv[p]], zero for dropped pairs
template <typename T>
__global__ void k_pair_scatter(const T* __restrict__ src, T* __restrict__ dst, long long P,
                               const int* __restrict__ inv) {
    const size_t row = (size_t)blockIdx.y * P;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const int q = inv[p];
        dst[row + p] = q >= 0 ? src[row + q] : T(0);
    }
}

// ---------------------------------------------------------------------------
// Sibling-grouped M2L fused with L2L (FP32), one level: the same sums as
// k_translate's mode 3, in the same order.  A block takes one sibling group
// (the <= 8 children of one parent, one warp each) and 32 * PPW consecutive
// pairs.  It walks the ascending union of the children's interaction lists:
// every source's multipoles for the block's pairs are loaded once into
// shared memory (the next source's prefetched into registers meanwhile) and
// applied by each warp whose child has that source in its list,
//   Mcal^{ij}(child) += T(child, src) O^{ij}(src)    (Eqs. fmmex, fmm2),
// the operator entries read through the read-only cache (the same address
// for all lanes).  Then, at levels >= 3, the parent's finished local
// expansion is translated down (Eq. fmm3) and each child is written once.
// A source shared by several siblings is read once instead of once per
// edge, which is what limits the per-target pass in 3-D clusters.
// ---------------------------------------------------------------------------
template <int NC, int PPW>
__global__ void __launch_bounds__(256)
k_m2l_group(int P, const int* __restrict__ pcount, int first_box, int g0, const int* __restrict__ grp_child,
            const int* __restrict__ grp_parent, const int* __restrict__ grp_ptr, const int* __restrict__ grp_src,
            const int* __restrict__ grp_op, const int* __restrict__ l2l_op, int do_l2l, const float* __restrict__ ops,
            const float* __restrict__ in, const float* parent_in, float* out) {
    constexpr int TP = 32 * PPW;                      // pairs of the block
    constexpr int PER = (NC * TP + 255) / 256;        // tile elements each thread moves
    __shared__ float tile[2][NC][TP];
    const int g = g0 + blockIdx.y;
    const int pb = blockIdx.x * TP;
    const int Pl = pcount ? min(P, *pcount) : P;
    if (pb >= Pl) return;                              // uniform across the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int child = grp_child[g * 8 + warp];
    float acc[NC][PPW];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int p = 0; p < PPW; ++p) acc[c][p] = 0.f;
    float pre[PER];
    auto gload = [&](const float* base, int box) {
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int e = threadIdx.x + 256 * m;
            const int c = e / TP, p = e - c * TP;
            pre[m] = (e < NC * TP && pb + p < Pl) ? base[((size_t)(box - first_box) * NC + c) * P + pb + p] : 0.f;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int e = threadIdx.x + 256 * m;
            const int c = e / TP, p = e - c * TP;
            if (e < NC * TP) tile[buf][c][p] = pre[m];
        }
    };
    auto apply = [&](int buf, int op) {                // warp-uniform op >= 0
        const float* T = ops + (size_t)op * NC * NC;
#pragma unroll
        for (int ci = 0; ci < NC; ++ci) {
            float v[PPW];
#pragma unroll
            for (int p = 0; p < PPW; ++p) v[p] = tile[buf][ci][lane + 32 * p];
#pragma unroll
            for (int co = 0; co < NC; ++co) {
                const float w = __ldg(T + co * NC + ci);
#pragma unroll
                for (int p = 0; p < PPW; ++p) acc[co][p] += w * v[p];
            }
        }
    };
    const int s0 = grp_ptr[g], s1 = grp_ptr[g + 1];
    if (s0 < s1) {
        gload(in, grp_src[s0]);
        sstore(0);
    }
    __syncthreads();
    for (int x = s0; x < s1; ++x) {
        const int buf = (x - s0) & 1;
        if (x + 1 < s1) gload(in, grp_src[x + 1]);
        const int op = child >= 0 ? grp_op[(size_t)x * 8 + warp] : -1;
        if (op >= 0) apply(buf, op);
        if (x + 1 < s1) sstore(buf ^ 1);
        __syncthreads();
    }
    if (do_l2l) {
        const int buf = (s1 - s0) & 1;
        gload(parent_in, grp_parent[g]);
        sstore(buf);
        __syncthreads();
        if (child >= 0) apply(buf, l2l_op[child]);
    }
    if (child < 0) return;
#pragma unroll
    for (int co = 0; co < NC; ++co)
#pragma unroll
        for (int p = 0; p < PPW; ++p) {
            const int q = pb + lane + 32 * p;
            if (q < Pl) out[((size_t)(child - first_box) * NC + co) * P + q] = acc[co][p];
        }
}

template <int NC, int PPW>
void launch_m2l_group(const FmmArgs& a, int lev, int P, const int* pcount, const float* ops, const float* in,
                      float* out, cudaStream_t s) {
    constexpr int TP = 32 * PPW;
    const int g0 = a.grp_level_off[lev], ng = a.grp_level_off[lev + 1] - g0;
    if (ng <= 0) return;
    dim3 g((P + TP - 1) / TP, ng);
    k_m2l_group<NC, PPW><<<g, 256, 0, s>>>(P, pcount, a.first_box, g0, a.grp_child, a.grp_parent, a.grp_ptr,
                                          a.grp_src, a.grp_op, a.l2l_op, lev >= 3 ? 1 : 0, ops, in, out, out);
}

// Components per block of k_half: the instantiated width that leaves the
// fewest padded components (ties: the wider one, fewer blocks).
int half_chunk(int nc) {
    const int cand[] = {25, 16, 9, 4};
    int best = 16, waste = 1 << 30;
    for (int c : cand) {
        const int w = ((nc + c - 1) / c) * c - nc;
        if (w < waste) {
            waste = w;
            best = c;
        }
    }
    return best;
}

// Threads per block of k_half (a multiple of 32, 64..256): each pass covers
// threads x jpt orbitals, so the width with the fewest orbitals past nocc in
// the last pass is chosen (ties: the widest, fewest passes).
int half_threads(int nocc, int jpt) {
    int best = 128, waste = 1 << 30;
    for (int t = 256; t >= 64; t -= 32) {
        const int per = t * jpt, w = ((nocc + per - 1) / per) * per - nocc;
        if (w < waste) {
            waste = w;
            best = t;
        }
    }
    return best;
}

// Output components per block of k_translate: the instantiated width that
// wastes the fewest lanes of the last chunk (rows past nc still cost FMAs).
int translate_chunk(int nc) {
    const int cand[] = {25, 21, 16, 9, 4};
    int best = 25, waste = 1 << 30;
    for (int c : cand) {
        int w = ((nc + c - 1) / c) * c - nc;
        if (w < waste) {
            waste = w;
            best = c;
        }
    }
    return best;
}

template <typename T, typename... Args>
void launch_translate(int lmc, dim3 g, cudaStream_t s, Args... args) {
    switch (lmc) {
        case 4: k_translate<T, 4><<<g, 128, 0, s>>>(args...); break;
        case 9: k_translate<T, 9><<<g, 128, 0, s>>>(args...); break;
        case 16: k_translate<T, 16><<<g, 128, 0, s>>>(args...); break;
        case 21: k_translate<T, 21><<<g, 128, 0, s>>>(args...); break;
        default: k_translate<T, 25><<<g, 128, 0, s>>>(args...); break;
    }
}

// ---------------------------------------------------------------------------
// The step (a) tile bound is accumulated in FP32; below about 1e-30 the
// squares it sums reach FP32's subnormal range, where the 2x margin of the
// comparison no longer covers the rounding.  Such thresholds form every tile
// (the exact FP64 criterion then decides every pair alone).
inline bool bound_usable(double tau2) { return 0.5 * tau2 >= 1e-30; }

template <typename T>
cudaError_t run_typed(const FmmArgs& a, cudaStream_t s) {
    const int nocc = a.nocc, nc = a.nc, D = a.depth;
    const long long P = (long long)body::npairs(nocc);   // stored pairs i <= j
    auto mark = [&](int k) {
        if (a.ev) cudaEventRecord(a.ev[k], s);
    };
    if (D < 2) {
        for (int k = 0; k < OCCK_NSTAGE; ++k) mark(k);
        k_zero_K<<<256, 256, 0, s>>>(a.K, a.ldk, a.nao, nocc, a.Ex_dev);
        mark(OCCK_NSTAGE);
        return cudaGetLastError();
    }
    T* Ct = (T*)a.ct;
    T* W = (T*)a.w;
    T* Ob = (T*)a.obox;
    T* Mb = (T*)a.mbox;
    const T* vals = (const T*)a.pair_vals;
    const T* ops = (const T*)a.ops;
    mark(0);
    {
        dim3 g((a.nao + 31) / 32, (nocc + 31) / 32), b(32, 8);
        k_transpose_C<T><<<g, b, 0, s>>>(a.C, a.ldc, a.nao, nocc, Ct);
    }
    {
        // components per block and threads per block chosen to waste the
        // fewest FMAs (padded components and orbitals past nocc cost as much
        // as real ones)
        const int LMC = half_chunk(nc);
        const int nth = half_threads(nocc, sizeof(T) == 4 ? 4 : 1);
        dim3 g(a.nrow, (nc + LMC - 1) / LMC);
        if (sizeof(T) == 8 && a.slices && a.slices->ff) {
            // the sliced FP64 form: double-FP32 arithmetic (kernels_f64s.cu)
            HalfFFArgs h{};
            h.nao = a.nao; h.nocc = nocc; h.nrow = a.nrow; h.nc = nc; h.nvals = a.slices->nvals;
            h.lmc = LMC; h.nth = nth;
            h.row_ptr = a.row_ptr; h.ent_col = a.ent_col; h.ent_val = a.ent_val;
            h.vals = (const double*)vals; h.Ct = (const double*)Ct;
            h.vals_ff = a.slices->vals_ff; h.C_ff = a.slices->C_ff;
            h.W = (double*)W;
            cudaError_t e2 = half_ff(h, s);
            if (e2 != cudaSuccess) return e2;
        } else switch (LMC) {
            case 4: k_half<T, 4><<<g, nth, 0, s>>>(a.row_ptr, a.ent_col, a.ent_val, vals, nc, Ct, nocc, a.nrow, W); break;
            case 9: k_half<T, 9><<<g, nth, 0, s>>>(a.row_ptr, a.ent_col, a.ent_val, vals, nc, Ct, nocc, a.nrow, W); break;
            case 25: k_half<T, 25><<<g, nth, 0, s>>>(a.row_ptr, a.ent_col, a.ent_val, vals, nc, Ct, nocc, a.nrow, W); break;
            default: k_half<T, 16><<<g, nth, 0, s>>>(a.row_ptr, a.ent_col, a.ent_val, vals, nc, Ct, nocc, a.nrow, W); break;
        }
    }
    const int leaf_store0 = a.leaf0 - a.first_box;
    const bool tcm = sizeof(T) == 4 && tc_mode(a.prec) >= 0;
    mark(1);
    PanelArgs pa{};
    if (tcm) {
        pa.rtA = a.pp_rtA; pa.offA = a.pp_offA; pa.KC = a.pp_KC; pa.jc = a.pp_jc; pa.it = a.pp_it;
        pa.kca = a.pp_kca; pa.offAa = a.pp_offAa; pa.offBa = a.pp_offBa;
        pa.max_rt = a.pp_max_rt; pa.max_kca = a.pp_max_kca; pa.nleaf = a.nleaf;
        pa.leaf_rowoff = a.leaf_rowoff; pa.leaf_aos = a.leaf_aos; pa.leaf_rowoff_host = a.leaf_rowoff_host;
        pa.Ct = (const float*)Ct; pa.W = (const float*)W; pa.Mbox = (const float*)Mb; pa.Obox = (float*)Ob;
        pa.KB = a.kb; pa.lscale = a.lscale;
        pa.nocc = nocc; pa.nrow = a.nrow; pa.nc = nc; pa.leaf_store0 = leaf_store0;
        pa.scaled = a.tr_on; pa.inv_h_leaf = a.inv_h_leaf;
        pa.nsplit = a.l2p_nsplit;
        pa.sm_count = a.sm_count;
        pa.err = a.err_word;
        pa.panA = a.pan_a2A;
        pa.panB = a.pan_a2B;
        cudaError_t e2 = panel_a2(a.prec, pa, s);
        if (e2 != cudaSuccess) return e2;
    } else if (a.slices && a.slices->full) {
        // from integer slices on the tensor core, exact sums (kernels_f64s.cu)
        cudaError_t e2 = full_slices(*a.slices, Ct, Ob, s);
        if (e2 != cudaSuccess) return e2;
    } else if constexpr (sizeof(T) == 8) {
        constexpr int BM = kFullTileFP64, BK = 8, TM = 4;
        int nt = (nocc + BM - 1) / BM;
        if (a.screen) {
            // tskip[t] = 1: tile t is not formed.  With a usable bound every
            // tile starts skipped and the bound clears the ones that may hold
            // a kept pair; otherwise every tile starts formed.
            const bool bound = a.screen_tau2 > 0 && bound_usable(a.screen_tau2);
            cudaMemsetAsync(a.scr_tskip, bound ? 1 : 0, (size_t)nt * (nt + 1) / 2, s);
            if (bound) {
                k_bound_ab<T><<<dim3(a.nleaf, (nocc + 127) / 128, nc + 1), 128, 0, s>>>(
                    a.leaf_rowoff, a.leaf_aos, Ct, W, nocc, a.nrow, a.nleaf, a.scr_a2, a.scr_b2);
                k_bound_tiles<<<dim3(nt * (nt + 1) / 2, BM / 8), 256, 0, s>>>(
                    a.scr_a2, a.scr_b2, a.nleaf, nc, nocc, BM, nt, (float)(0.5 * a.screen_tau2), a.scr_tskip);
            }
            if (a.col1 > a.col0)
                k_col_tiles<<<std::max(1, (nt * (nt + 1) / 2 + 255) / 256), 256, 0, s>>>(nt, BM, a.col0, a.col1,
                                                                                         a.scr_tskip);
        }
        dim3 g(nt * (nt + 1) / 2, a.nleaf * nc);
        k_full<T, BM, BK, TM><<<g, (BM / TM) * (BM / TM), 0, s>>>(a.leaf_rowoff, a.leaf_aos, Ct, W, nocc,
                                                                 a.nrow, nc, nt, Ob, leaf_store0,
                                                                 a.screen ? a.scr_tskip : nullptr);
    } else {
        // 128 x 128 tiles (8 x 8 per thread) or 96 x 96 (6 x 6), whichever
        // wastes fewer FMAs on padding and on the lower halves of diagonal
        // tiles (full_tile_fp32)
        auto launch = [&](auto tile) {
            constexpr int BM = decltype(tile)::value, BK = 16, TM = BM == 96 ? 6 : 8;
            const int nt = (nocc + BM - 1) / BM;
            if (a.screen) {
                const bool bound = a.screen_tau2 > 0 && bound_usable(a.screen_tau2);
                cudaMemsetAsync(a.scr_tskip, bound ? 1 : 0, (size_t)nt * (nt + 1) / 2, s);
                if (bound) {
                    k_bound_ab<T><<<dim3(a.nleaf, (nocc + 127) / 128, nc + 1), 128, 0, s>>>(
                        a.leaf_rowoff, a.leaf_aos, Ct, W, nocc, a.nrow, a.nleaf, a.scr_a2, a.scr_b2);
                    k_bound_tiles<<<dim3(nt * (nt + 1) / 2, BM / 8), 256, 0, s>>>(
                        a.scr_a2, a.scr_b2, a.nleaf, nc, nocc, BM, nt, (float)(0.5 * a.screen_tau2), a.scr_tskip);
                }
                if (a.col1 > a.col0)
                    k_col_tiles<<<std::max(1, (nt * (nt + 1) / 2 + 255) / 256), 256, 0, s>>>(nt, BM, a.col0,
                                                                                             a.col1, a.scr_tskip);
            }
            dim3 g(nt * (nt + 1) / 2, a.nleaf * nc);
            k_full<T, BM, BK, TM><<<g, (BM / TM) * (BM / TM), 0, s>>>(a.leaf_rowoff, a.leaf_aos, Ct, W, nocc,
                                                                     a.nrow, nc, nt, Ob, leaf_store0,
                                                                     a.screen ? a.scr_tskip : nullptr);
        };
        if (full_tile_fp32(nocc) == 96)
            launch(std::integral_constant<int, 96>{});
        else
            launch(std::integral_constant<int, 128>{});
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // occupied-pair screening: the tree passes run on the kept pairs, whose
    // leaf multipoles are gathered to the front of each row of scr_o
    T* Ot = Ob;
    T* Mt = Mb;
    const int* pcnt = nullptr;
    // gather / scatter grid: one row of blocks per leaf component, at most 16
    // blocks along the pairs
    const dim3 gpair((unsigned)std::min<long long>((P + 255) / 256, 16), (unsigned)(a.nleaf * nc));
    if (a.screen) {
        const int nb = (int)((P + kPairBlk - 1) / kPairBlk);
        const int ngrp = (a.nleaf + kPairLG - 1) / kPairLG;
        // the partial norms live in scr_m (idle until the tree passes; it
        // holds at least nleaf x nc rows of P)
        T* part = (T*)a.scr_m;
        const dim3 gpart((unsigned)((P + kPairBlk * kPairPPT - 1) / (kPairBlk * kPairPPT)), (unsigned)ngrp);
        // a column block alone (no threshold) reads no norm
        const bool norms = a.screen_tau2 > 0;
        if (norms)
            k_pair_part<T><<<gpart, kPairBlk, 0, s>>>(Ob + (size_t)leaf_store0 * nc * P, a.nleaf, nc, P, part);
        k_pair_flag<T><<<nb, kPairBlk, 0, s>>>(part, norms ? ngrp : 0, P, a.screen_tau2, a.scr_norm, a.scr_inv,
                                                a.scr_bcount, tcm ? nullptr : a.scr_tskip, nocc,
                                                sizeof(T) == 8 ? kFullTileFP64 : full_tile_fp32(nocc), a.col0,
                                                a.col1);
        k_pair_scan<<<1, 1024, 0, s>>>(a.scr_bcount, nb, a.scr_count);
        k_pair_compact<<<nb, kPairBlk, 0, s>>>(P, a.scr_bcount, a.scr_keep, a.scr_inv);
        cudaMemsetAsync(a.scr_tiles, 0, (size_t)((nocc + 127) / 128) * ((nocc + 7) / 8), s);
        k_pair_tiles<<<std::max(1, a.sm_count) * 4, 256, 0, s>>>(a.scr_keep, a.scr_count, nocc, a.scr_tiles);
        Ot = (T*)a.scr_o;
        Mt = (T*)a.scr_m;
        pcnt = a.scr_count;
        k_pair_gather<T><<<gpair, 256, 0, s>>>(Ob + (size_t)leaf_store0 * nc * P, Ot + (size_t)leaf_store0 * nc * P,
                                               P, a.scr_keep, a.scr_count);
    }
    const int LMC = translate_chunk(nc);
    const int nchunk = (nc + LMC - 1) / LMC;
    const unsigned pblocks = (unsigned)((P + 128 * body::translate_ppt<T>() - 1) / (128 * body::translate_ppt<T>()));
    // (b) M2M: parents at level lev-1 gather their children at level lev
    // tensor-core translations for the mixed forms (multipoles kept in FP32
    // between steps, operands scaled per component, see kernels_tc_translate.cu)
    const bool trc = tcm && a.tr_on;
    const T* tops = trc ? (const T*)a.ops_scaled : ops;   // SIMT operators matching the storage
    TrArgs th{};
    if (trc) {
        th.P = (int)P; th.nc = nc; th.first_box = a.first_box; th.nlev = a.tr_nlev; th.sm_count = a.sm_count;
        th.parent = a.parent; th.box_level = a.box_level;
        th.pan = a.tr_pan; th.err = a.err_word;
    }
    // slot pipeline: the leaf multipoles of step (a) go into slots once, all
    // three translations read and write slots, the leaf local expansions come
    // back as FP32 for step (e)
    const bool slots = trc && a.slot_o != nullptr;
    // M2L and L2L both on the SIMT kernel: one fused pass per level
    const bool fused = !slots && !(trc && (a.tr_mask & 2)) && !(trc && (a.tr_mask & 4));
    SlotArgs sh{};
    const int ntile = (int)((P + 127) / 128);
    if (slots) {
        sh.P = (int)P; sh.nc = nc; sh.ntile = ntile; sh.first_box = a.first_box; sh.sm_count = a.sm_count;
        sh.parent = a.parent; sh.pan = a.tr_pan; sh.err = a.err_word;
    }
    mark(2);
    if (slots) {
        cudaError_t e2 = tr_slots_pack(a.prec, nc, (const float*)Ob, (int)P, ntile, leaf_store0, a.nbox - a.leaf0,
                                       a.slot_o, s);
        for (int lev = D; lev >= 3 && e2 == cudaSuccess; --lev) {
            int t0 = a.level_off[lev - 1], nt = a.level_off[lev] - t0;
            e2 = tr_slot_translate(a.prec, sh, 0, t0, nt, a.child_ptr, a.child_list, a.m2m_op, a.slot_o, a.slot_o,
                                   0, s);
        }
        if (e2 != cudaSuccess) return e2;
    }
    // the sliced FP64 form: M2M in double-FP32 arithmetic; for the learned
    // selector, whose features read the FP64 multipoles of every box, they
    // are joined back to FP64 after it (and split again for M2L)
    FFArgs ffa{};
    bool m2m_ff_done = false;
    if constexpr (sizeof(T) == 8) {
        if (a.slices && a.slices->ff && !a.screen) {
            ffa.P = (int)P; ffa.nc = nc; ffa.L = a.L; ffa.D = D; ffa.first_box = a.first_box;
            ffa.nstore = a.nbox - a.first_box; ffa.leaf_store0 = leaf_store0; ffa.nops = a.slices->nops;
            ffa.sm_count = a.sm_count; ffa.level_off = a.level_off;
            ffa.m2l_ptr = a.m2l_ptr; ffa.m2l_src = a.m2l_src; ffa.m2l_op = a.m2l_op;
            ffa.parent = a.parent; ffa.l2l_op = a.l2l_op;
            ffa.child_ptr = a.child_ptr; ffa.child_list = a.child_list; ffa.m2m_op = a.m2m_op;
            ffa.ops = (const double*)tops; ffa.ops_ff = a.slices->ops_ff;
            ffa.Ob = (double*)Ob; ffa.Mb = (double*)Mb;
            ffa.sm = a.slices->m2l;
            ffa.err = a.slices->err;
            cudaError_t e2 = m2m_ff(ffa, s);
            if (e2 == cudaSuccess && a.learned) e2 = ff_join(ffa, s);
            if (e2 != cudaSuccess) return e2;
            m2m_ff_done = true;
            ffa.m2m_done = a.learned ? 0 : 1;
        }
    }
    for (int lev = D; lev >= 3 && !slots && !m2m_ff_done; --lev) {
        int t0 = a.level_off[lev - 1], nt = a.level_off[lev] - t0;
        if (trc && (a.tr_mask & 1)) {
            cudaError_t e2 = tr_translate(a.prec, th, 0, t0, nt, a.child_ptr, a.child_list, a.m2m_op,
                                          (const float*)Ob, (float*)Ob, 0, s);
            if (e2 != cudaSuccess) return e2;
            continue;
        }
        dim3 g(nt, pblocks, nchunk);
        launch_translate<T>(LMC, g, s, 0, (int)P, nc, a.L, a.first_box, t0, a.child_ptr,
                                             a.child_list, a.m2m_op, nullptr, a.parent, tops, Ot, Ot, 0,
                                             (const int*)nullptr, (const T*)nullptr, pcnt);
    }
    // learned ranks: features from the multipoles of every box, FP16 MLP,
    // budgeted choice; M2L then reads the per-edge ranks
    const int* lmax_e = a.m2l_lmax;
    if (a.learned) {
        cudaError_t e2 = edge_features(sizeof(T) == 8, Ob, a.first_box, a.nbox, nc, a.L, P, nocc, a.nm2l, a.m2l_tgt,
                                       a.m2l_src, a.box_key, a.box_level, a.hlev, D, a.nrm, a.feat, s);
        if (e2 == cudaSuccess)
            e2 = mlp_predict_fp16(a.mlp_prm, (__half*)a.mlp_h, a.mlp_norm, a.feat, a.nm2l, a.pred, s);
        if (e2 == cudaSuccess) e2 = select_ranks(a.pred, a.nm2l, a.L, a.tau, a.ranks, a.rank_err, s);
        if (e2 != cudaSuccess) return e2;
        lmax_e = a.ranks;
    }
    // (c) M2L: every box of levels 2..D, all levels in one launch
    mark(3);
    if (slots) {
        int t0 = a.level_off[2], nt = a.nbox - t0;
        cudaError_t e2 = tr_slot_translate(a.prec, sh, 1, t0, nt, a.m2l_ptr, a.m2l_src, a.m2l_op, a.slot_o, a.slot_m,
                                           0, s);
        if (e2 != cudaSuccess) return e2;
    } else if (trc && (a.tr_mask & 2)) {
        int t0 = a.level_off[2], nt = a.nbox - t0;
        cudaError_t e2 = tr_translate(a.prec, th, 1, t0, nt, a.m2l_ptr, a.m2l_src, a.m2l_op, (const float*)Ob,
                                      (float*)Mb, 0, s);
        if (e2 != cudaSuccess) return e2;
    } else if (fused) {
        // (c) and (d) together, level by level: each target is written once
        // from its interaction list and its parent's finished expansion
        bool done = false;
        if constexpr (sizeof(T) == 8) {
            if (a.slices && a.slices->ff && !a.screen) {
                // the sliced FP64 form: the same pass in double-FP32 arithmetic
                ffa.lmax_e = lmax_e;
                cudaError_t e2 = m2l_ff(ffa, s);
                if (e2 != cudaSuccess) return e2;
                done = true;
            }
        }
        for (int lev = 2; lev <= D && !done; ++lev) {
            int t0 = a.level_off[lev], nt = a.level_off[lev + 1] - t0;
            if (nt <= 0) continue;
            if constexpr (sizeof(T) == 4) {
                if (((a.grp_use >> lev) & 1u) && lmax_e == nullptr) {
                    const float* fo = (const float*)tops;
                    if (nc == 9)
                        launch_m2l_group<9, 4>(a, lev, (int)P, pcnt, fo, (const float*)Ot, (float*)Mt, s);
                    else if (nc == 16)
                        launch_m2l_group<16, 2>(a, lev, (int)P, pcnt, fo, (const float*)Ot, (float*)Mt, s);
                    else
                        launch_m2l_group<4, 4>(a, lev, (int)P, pcnt, fo, (const float*)Ot, (float*)Mt, s);
                    continue;
                }
            }
            dim3 g(nt, pblocks, nchunk);
            launch_translate<T>(LMC, g, s, 3, (int)P, nc, a.L, a.first_box, t0, a.m2l_ptr, a.m2l_src,
                                a.m2l_op, lmax_e, a.parent, tops, Ot, Mt, 0, a.l2l_op, (const T*)Mt, pcnt);
        }
    } else {
        int t0 = a.level_off[2], nt = a.nbox - t0;
        dim3 g(nt, pblocks, nchunk);
        launch_translate<T>(LMC, g, s, 1, (int)P, nc, a.L, a.first_box, t0, a.m2l_ptr, a.m2l_src,
                                             a.m2l_op, lmax_e, a.parent, tops, Ob, Mb, 0,
                                             (const int*)nullptr, (const T*)nullptr, (const int*)nullptr);
    }
    // (d) L2L: children at level lev accumulate their parent's expansion
    mark(4);
    if (slots) {
        cudaError_t e2 = cudaSuccess;
        for (int lev = 3; lev <= D && e2 == cudaSuccess; ++lev) {
            int t0 = a.level_off[lev], nt = a.level_off[lev + 1] - t0;
            e2 = tr_slot_translate(a.prec, sh, 2, t0, nt, nullptr, nullptr, a.l2l_op, a.slot_m, a.slot_m, 1, s);
        }
        if (e2 != cudaSuccess) return e2;
    }
    for (int lev = 3; lev <= D && !slots && !fused; ++lev) {
        int t0 = a.level_off[lev], nt = a.level_off[lev + 1] - t0;
        if (trc && (a.tr_mask & 4)) {
            cudaError_t e2 = tr_translate(a.prec, th, 2, t0, nt, nullptr, nullptr, a.l2l_op, (const float*)Mb,
                                          (float*)Mb, 1, s);
            if (e2 != cudaSuccess) return e2;
            continue;
        }
        dim3 g(nt, pblocks, nchunk);
        launch_translate<T>(LMC, g, s, 2, (int)P, nc, a.L, a.first_box, t0, nullptr, nullptr,
                                             a.l2l_op, nullptr, a.parent, tops, Mb, Mb, 1,
                                             (const int*)nullptr, (const T*)nullptr, (const int*)nullptr);
    }
    // screened: the kept pairs' leaf local expansions back to their places,
    // zero for the dropped pairs
    if (a.screen)
        k_pair_scatter<T><<<gpair, 256, 0, s>>>(Mt + (size_t)leaf_store0 * nc * P, Mb + (size_t)leaf_store0 * nc * P,
                                                P, a.scr_inv);
    // (e) L2P: with a column block only the 128-orbital tiles of its columns
    const bool colblk = a.col1 > a.col0;
    const int itile0 = colblk ? a.col0 / 128 : 0;
    const int itile1 = colblk ? (a.col1 + 127) / 128 : (nocc + 127) / 128;
    mark(5);
    if (slots) {
        cudaError_t e2 = tr_slots_unpack(a.prec, nc, a.slot_m, (int)P, ntile, leaf_store0, a.nbox - a.leaf0,
                                         (float*)Mb, s);
        if (e2 != cudaSuccess) return e2;
    }
    if (tcm) {
        pa.panA = a.pan_l2pA;
        pa.panB = a.pan_l2pB;
        cudaError_t e2 = panel_l2p(a.prec, pa, s);
        if (e2 != cudaSuccess) return e2;
    } else if (a.slices) {
        // from integer slices on the tensor core, exact sums (kernels_f64s.cu)
        cudaError_t e2 = l2p_slices(*a.slices, s);
        if (e2 != cudaSuccess) return e2;
    } else if constexpr (sizeof(T) == 8) {
        // 32 AO rows x 128 orbitals per block: leaves hold ~70-600 AOs, and a
        // 64-row tile would spend a third of the DFMA on padding
        // the last 128-orbital tile, when it holds 32 orbitals or fewer, runs
        // as a 32-column launch of its own (no DFMAs on padded columns)
        const bool tail = nocc - (itile1 - 1) * 128 <= 32;
        dim3 g((a.max_rows + 31) / 32, itile1 - itile0 - (tail ? 1 : 0), a.nleaf * a.l2p_nsplit);
        if (g.y > 0)
            k_l2p_r32<8><<<g, 256, 0, s>>>(a.l2p_nsplit, a.leaf_rowoff, (const double*)W, (const double*)Mb, nocc,
                                           a.nrow, nc, leaf_store0, a.kb, a.screen ? a.scr_tiles : nullptr, itile0);
        if (tail) {
            g.y = 1;
            k_l2p_r32<2><<<g, 256, 0, s>>>(a.l2p_nsplit, a.leaf_rowoff, (const double*)W, (const double*)Mb, nocc,
                                           a.nrow, nc, leaf_store0, a.kb, a.screen ? a.scr_tiles : nullptr,
                                           itile1 - 1);
        }
    } else {
        const int nsplit = a.l2p_nsplit;
        // the last orbital tile with 32 orbitals or fewer as a 32-column launch
        const bool tail = nocc - (itile1 - 1) * 128 <= 32;
        dim3 g((a.max_rows + 95) / 96, itile1 - itile0 - (tail ? 1 : 0), a.nleaf * nsplit);
        if (g.y > 0)
            k_l2p_r96f<8><<<g, 256, 0, s>>>(nsplit, a.leaf_rowoff, (const float*)W, (const float*)Mb, nocc, a.nrow,
                                            nc, leaf_store0, a.kb, a.screen ? a.scr_tiles : nullptr, itile0);
        if (tail) {
            g.y = 1;
            k_l2p_r96f<2><<<g, 256, 0, s>>>(nsplit, a.leaf_rowoff, (const float*)W, (const float*)Mb, nocc, a.nrow,
                                            nc, leaf_store0, a.kb, a.screen ? a.scr_tiles : nullptr, itile1 - 1);
        }
    }
    mark(6);
    constexpr int kRedBlocks = kFarfieldPartials;
    const int nsplit = a.l2p_nsplit;
    k_reduce_K<<<kRedBlocks, 256, 0, s>>>(a.ao_row_ptr, a.ao_rows, a.kb, a.nao, nocc, a.C, a.ldc, a.K,
                                          a.ldk, a.part, nsplit, (size_t)a.nrow * nocc, colblk ? a.col0 : 0,
                                          colblk ? a.col1 : -1);
    k_final_energy<<<1, 256, 0, s>>>(a.part, kRedBlocks, a.Ex_dev);
    mark(OCCK_NSTAGE);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Far-field Coulomb matrix (Sec. II, Eq. fmmc and the J^ff formula), FP64:
// density multipoles of the leaves, the tree passes on one density channel
// (k_translate with one "pair"), then J^ff on every kept AO pair.
// ---------------------------------------------------------------------------

// q[leaf][lm] = sum over the leaf's ordered entries (r, s) of D_rs O^{rs}_lm
// (both orderings of a pair are entries, as in the half transform).
__global__ void __launch_bounds__(256)
k_j_density(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos, const int* __restrict__ row_ptr,
            const int* __restrict__ ent_col, const int* __restrict__ ent_val, const double* __restrict__ vals, int nc,
            const double* __restrict__ D, int ldd, double* __restrict__ q) {
    const int B = blockIdx.x, lm = blockIdx.y;
    const int r0 = leaf_rowoff[B], r1 = leaf_rowoff[B + 1];
    double acc = 0.0;
    for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
        const int r = leaf_aos[row];
        for (int e = row_ptr[row]; e < row_ptr[row + 1]; ++e)
            acc += D[(size_t)ent_col[e] * ldd + r] * vals[(size_t)ent_val[e] * nc + lm];
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) q[(size_t)B * nc + lm] = red[0];
}

// J^ff_rs = sum_lm w_lm O^{rs}_lm Mcal_lm(X) on the leaf's entries (real form:
// w = 1 for m = 0, 2 for Re m > 0, -2 for Im m > 0), and the leaf's part of
// E_J = 1/2 sum_rs D_rs J_rs.
__global__ void __launch_bounds__(256)
k_j_l2p(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos, const int* __restrict__ row_ptr,
        const int* __restrict__ ent_col, const int* __restrict__ ent_val, const double* __restrict__ vals, int nc,
        const double* __restrict__ Mleaf, const double* __restrict__ D, int ldd, double* __restrict__ J, int ldj,
        double* __restrict__ part) {
    const int B = blockIdx.x;
    __shared__ double wm[body::kNcMax];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int l = 0;
        while ((l + 1) * (l + 1) <= c) ++l;
        const double w = c == l * l ? 1.0 : (((c - l * l) & 1) ? 2.0 : -2.0);
        wm[c] = w * Mleaf[(size_t)B * nc + c];
    }
    __syncthreads();
    const int r0 = leaf_rowoff[B], r1 = leaf_rowoff[B + 1];
    double e_acc = 0.0;
    for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
        const int r = leaf_aos[row];
        for (int e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
            const int sidx = ent_col[e];
            const double* v = vals + (size_t)ent_val[e] * nc;
            double j = 0.0;
            for (int c = 0; c < nc; ++c) j += v[c] * wm[c];
            J[(size_t)sidx * ldj + r] = j;
            e_acc += D[(size_t)sidx * ldd + r] * j;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = e_acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[B] = red[0];
}

__global__ void k_zero_square(double* M, int ld, int n) {
    const long long tot = (long long)n * n;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(x / n), r = (int)(x - (long long)c * n);
        M[(size_t)c * ld + r] = 0.0;
    }
}

__global__ void k_j_energy(const double* __restrict__ part, int n, double* __restrict__ E) {
    __shared__ double red[256];
    double s = 0.0;
    for (int x = threadIdx.x; x < n; x += blockDim.x) s += part[x];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = 0.5 * red[0];
}

}  // namespace

cudaError_t run_farfield_J(const JArgs& a, cudaStream_t s) {
    k_zero_square<<<256, 256, 0, s>>>(a.J, a.ldj, a.nao);
    if (a.depth < 2 || a.nleaf == 0) {
        cudaMemsetAsync(a.Ej_dev, 0, sizeof(double), s);
        return cudaGetLastError();
    }
    const int nc = a.nc, D = a.depth;
    const int leaf_store0 = a.leaf0 - a.first_box;
    double* Ob = a.ob;
    double* Mb = a.mb;
    k_j_density<<<dim3(a.nleaf, nc), 256, 0, s>>>(a.leaf_rowoff, a.leaf_aos, a.row_ptr, a.ent_col, a.ent_val, a.vals,
                                                  nc, a.D, a.ldd, Ob + (size_t)leaf_store0 * nc);
    const int LMC = translate_chunk(nc);
    const int nchunk = (nc + LMC - 1) / LMC;
    for (int lev = D; lev >= 3; --lev) {
        const int t0 = a.level_off[lev - 1], nt = a.level_off[lev] - t0;
        launch_translate<double>(LMC, dim3(nt, 1, nchunk), s, 0, 1, nc, a.L, a.first_box, t0, a.child_ptr,
                                 a.child_list, a.m2m_op, nullptr, a.parent, a.ops, Ob, Ob, 0,
                                 (const int*)nullptr, (const double*)nullptr, (const int*)nullptr);
    }
    {
        const int t0 = a.level_off[2], nt = a.nbox - t0;
        launch_translate<double>(LMC, dim3(nt, 1, nchunk), s, 1, 1, nc, a.L, a.first_box, t0, a.m2l_ptr, a.m2l_src,
                                 a.m2l_op, nullptr, a.parent, a.ops, Ob, Mb, 0, (const int*)nullptr,
                                 (const double*)nullptr, (const int*)nullptr);
    }
    for (int lev = 3; lev <= D; ++lev) {
        const int t0 = a.level_off[lev], nt = a.level_off[lev + 1] - t0;
        launch_translate<double>(LMC, dim3(nt, 1, nchunk), s, 2, 1, nc, a.L, a.first_box, t0, nullptr, nullptr,
                                 a.l2l_op, nullptr, a.parent, a.ops, Mb, Mb, 1, (const int*)nullptr,
                                 (const double*)nullptr, (const int*)nullptr);
    }
    k_j_l2p<<<a.nleaf, 256, 0, s>>>(a.leaf_rowoff, a.leaf_aos, a.row_ptr, a.ent_col, a.ent_val, a.vals, nc,
                                    Mb + (size_t)leaf_store0 * nc, a.D, a.ldd, a.J, a.ldj, a.part);
    k_j_energy<<<1, 256, 0, s>>>(a.part, a.nleaf, a.Ej_dev);
    return cudaGetLastError();
}

cudaError_t energy_from_K(int nao, int nocc, const double* C, int ldc, const double* K, int ldk, double* part,
                          double* E, cudaStream_t s) {
    body::k_energy_parts<<<kFarfieldPartials, 256, 0, s>>>(nao, nocc, C, ldc, K, ldk, part);
    k_final_energy<<<1, 256, 0, s>>>(part, kFarfieldPartials, E);
    return cudaGetLastError();
}

cudaError_t run_farfield(const FmmArgs& a, cudaStream_t s) {
    if (a.prec == OCCK_FP64) return run_typed<double>(a, s);
    return run_typed<float>(a, s);
}

cudaError_t probe_fma(int prec, int sm_count, double* flops, cudaStream_t s) {
    // best rate over the two operand forms, occupancies of 4 and 8 blocks of
    // 256 threads per SM and 8, 16 or 32 accumulators, each timed three
    // times after one warm-up
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 1024 * 8);
    if (e != cudaSuccess) return e;
    {
        // multiplier 0.999999 and addend 1e-7 at element 512 of the buffer
        const double md[2] = {0.999999, 1e-7};
        const float mf[2] = {0.999999f, 1e-7f};
        e = prec == OCCK_FP64 ? cudaMemcpy((double*)buf + 512, md, sizeof(md), cudaMemcpyHostToDevice)
                              : cudaMemcpy((float*)buf + 512, mf, sizeof(mf), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(buf);
            return e;
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256;
    double best_rate = 0.0;
    for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
        for (int bps : {4, 8}) {
            const int blocks = sm_count * bps;
            for (int nacc : {8, 16, 32}) {
                // about 2^27 FMAs per thread-block wave for FP32, 2^21 for FP64
                const int iters = prec == OCCK_FP64 ? (1 << 12) / (nacc / 8) : (1 << 16) / (nacc / 8);
                for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                    cudaEventRecord(e0, s);
                    if (prec == OCCK_FP64) {
                        double* b = (double*)buf;
                        if (nacc == 8) launch_probe<double, 8>(form, blocks, b, iters, s);
                        if (nacc == 16) launch_probe<double, 16>(form, blocks, b, iters, s);
                        if (nacc == 32) launch_probe<double, 32>(form, blocks, b, iters, s);
                    } else {
                        float* b = (float*)buf;
                        if (nacc == 8) launch_probe<float, 8>(form, blocks, b, iters, s);
                        if (nacc == 16) launch_probe<float, 16>(form, blocks, b, iters, s);
                        if (nacc == 32) launch_probe<float, 32>(form, blocks, b, iters, s);
                    }
                    cudaEventRecord(e1, s);
                    e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) break;
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    const double nfma = (double)blocks * threads * nacc * 4.0 * iters;
                    if (rep > 0 && ms > 0) best_rate = std::max(best_rate, 2.0 * nfma / (ms * 1e-3));
                }
            }
        }
    }
    *flops = best_rate;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace occk
