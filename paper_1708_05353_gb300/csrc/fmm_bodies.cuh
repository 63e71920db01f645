// Device bodies of the SIMT steps, shared by the single-system kernels
// (kernels_fmm.cu) and the persistent batched kernels (kernels_batch.cu).
// Each body takes the block coordinates (bx, by, bz) explicitly so that a
// persistent block can run many work items.
#pragma once

#include "occk_internal.h"

namespace occk {
namespace body {



// Occupied pairs are stored once: p = (i, j) with i <= j, row-major upper
// triangle (O^{ij} = O^{ji} and Mcal^{ij} = Mcal^{ji}).
__host__ __device__ __forceinline__ size_t tri_index(int i, int j, int n) {
    return (size_t)i * (size_t)(2 * n - i + 1) / 2 + (size_t)(j - i);
}
__host__ __device__ __forceinline__ size_t npairs(int n) { return (size_t)n * (size_t)(n + 1) / 2; }

constexpr int kNcMax = 169;   // (12+1)^2

// ---------------------------------------------------------------------------
// C (column-major, ldc) -> Ct (row-major), 32x32 tiles through shared memory
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void transpose_body(int bx, int by, int bz, const double* __restrict__ C, int ldc, int nao, int nocc,
                              T* __restrict__ Ct) {
    __shared__ double tile[32][33];
    int r0 = bx * 32, i0 = by * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int r = r0 + threadIdx.x, i = i0 + k;
        tile[k][threadIdx.x] = (r < nao && i < nocc) ? C[(size_t)i * ldc + r] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int r = r0 + k, i = i0 + threadIdx.x;
        if (r < nao && i < nocc) Ct[(size_t)r * nocc + i] = (T)tile[threadIdx.x][k];
    }
}

// ---------------------------------------------------------------------------
// Step (a), first half (Eq. motrans, first line):
//   W[lm][row][j] = sum_{entries (row, s, v)} O^{rs}_lm C_sj
// grid (nrow, lm chunks); threads stride over j.
// ---------------------------------------------------------------------------
template <typename T, int LMC>
__device__ __forceinline__ void half_body(int bx, int by, int bz, const int* __restrict__ row_ptr, const int* __restrict__ ent_col,
                       const int* __restrict__ ent_val, const T* __restrict__ vals, int nc,
                       const T* __restrict__ Ct, int nocc, int nrow, T* __restrict__ W) {
    // One block per (AO row, chunk of LMC components).  The row's pair values
    // and partner AOs are staged in shared memory (CH entries at a time); in
    // FP32 each thread accumulates JPT = 4 orbitals j, so every shared value
    // feeds 4 FMAs (FP64 is DFMA-bound and keeps one orbital per thread).
    constexpr int JPT = sizeof(T) == 4 ? 4 : 1, CH = 64;
    __shared__ T sv[CH][LMC];
    __shared__ int scol[CH];
    const int row = bx;
    const int c0 = by * LMC;
    const int e0 = row_ptr[row], e1 = row_ptr[row + 1];
    const int ncl = min(LMC, nc - c0);
    const int nth = blockDim.x;
    for (int jb = 0; jb < nocc; jb += nth * JPT) {
        T acc[JPT][LMC];
#pragma unroll
        for (int u = 0; u < JPT; ++u)
#pragma unroll
            for (int q = 0; q < LMC; ++q) acc[u][q] = T(0);
        for (int ec = e0; ec < e1; ec += CH) {
            const int n = min(CH, e1 - ec);
            __syncthreads();
            for (int x = threadIdx.x; x < n * LMC; x += nth) {
                const int k = x / LMC, q = x - k * LMC;
                sv[k][q] = q < ncl ? vals[(size_t)ent_val[ec + k] * nc + c0 + q] : T(0);
            }
            for (int x = threadIdx.x; x < n; x += nth) scol[x] = ent_col[ec + x];
            __syncthreads();
            for (int k = 0; k < n; ++k) {
                const T* crow = Ct + (size_t)scol[k] * nocc + jb + threadIdx.x;
                T cs[JPT];
#pragma unroll
                for (int u = 0; u < JPT; ++u) cs[u] = jb + threadIdx.x + u * nth < nocc ? crow[u * nth] : T(0);
#pragma unroll
                for (int q = 0; q < LMC; ++q) {
                    const T w = sv[k][q];
#pragma unroll
                    for (int u = 0; u < JPT; ++u) acc[u][q] += w * cs[u];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < JPT; ++u) {
            const int jj = jb + threadIdx.x + u * nth;
            if (jj >= nocc) continue;
#pragma unroll
            for (int q = 0; q < LMC; ++q)
                if (q < ncl) W[((size_t)(c0 + q) * nrow + row) * nocc + jj] = acc[u][q];
        }
    }
}

// ---------------------------------------------------------------------------
// Register-tiled GEMM core shared by steps (a) and (e):
//   acc[tm][tn] += sum_k As[k][ty*TM+tm] * Bs[k][tx*TN+tn]
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK, int TM, int TN>
struct Tile {
    static constexpr int NT = (BM / TM) * (BN / TN);
};

// Step (a), second half (Eq. motrans, second line), per leaf B and component lm:
//   O[B][lm][i][j] = sum_{r in S_B} C_ri W[lm][rowoff_B + r][j]
// Only tiles with ti <= tj are computed; O^{ij} = O^{ji} fills the rest.
template <typename T, int BM, int BK, int TM>
__device__ __forceinline__ void full_body(int bx, int by, int bz, const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos,
       const T* __restrict__ Ct, const T* __restrict__ W, int nocc, int nrow, int nc,
       int ntile, T* __restrict__ Obox, int leaf_store0) {
    constexpr int NTH = (BM / TM) * (BM / TM);
    constexpr int NL = (BK * BM) / NTH;          // elements per operand one thread moves per step
    // FP32 with 8 columns per thread: a thread owns columns tx*4..tx*4+3 and
    // BM/2 + tx*4.., so a quarter warp's 16-byte loads cover 128 contiguous bytes
    constexpr bool kSplitCols = sizeof(T) == 4 && TM == 8 && BM / 2 == (BM / TM) * 4;
    __shared__ __align__(16) T As[2][BK][BM];
    __shared__ __align__(16) T Bs[2][BK][BM];
    const int B = by / nc;
    const int lm = by - B * nc;
    // triangular tile index -> (ti, tj), ti <= tj
    int t = bx, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int i0 = ti * BM, j0 = tj * BM;
    // FP64 (DFMA-bound): a warp owns a stripe of 2 * TM columns over all rows,
    // so that in a tile whose columns run past nocc the warps holding only
    // such columns skip their FMAs; FP32 keeps row stripes and 16-byte loads
    constexpr bool kColWarps = sizeof(T) == 8;
    const int tx = kColWarps ? threadIdx.x / (BM / TM) : threadIdx.x % (BM / TM);
    const int ty = kColWarps ? threadIdx.x % (BM / TM) : threadIdx.x / (BM / TM);
    const bool warp_live = !kColWarps || j0 + ((threadIdx.x >> 5) * 32 / (BM / TM)) * TM < nocc;
    const T* Wl = W + ((size_t)lm * nrow + rb0) * nocc;
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    // the next K step is loaded into registers while the current one is
    // multiplied; one barrier per step
    T ra[NL], rb[NL];
    auto gload = [&](int k0) {
#pragma unroll
        for (int m = 0; m < NL; ++m) {
            const int e = threadIdx.x + NTH * m;
            const int kk = e / BM, c = e - kk * BM;
            const int r = k0 + kk;
            const int ao = r < nr ? leaf_aos[rb0 + r] : -1;
            ra[m] = (ao >= 0 && i0 + c < nocc) ? Ct[(size_t)ao * nocc + i0 + c] : T(0);
            rb[m] = (r < nr && j0 + c < nocc) ? Wl[(size_t)r * nocc + j0 + c] : T(0);
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int m = 0; m < NL; ++m) {
            const int e = threadIdx.x + NTH * m;
            const int kk = e / BM, c = e - kk * BM;
            As[buf][kk][c] = ra[m];
            Bs[buf][kk][c] = rb[m];
        }
    };
    const int nk = (nr + BK - 1) / BK;
    if (nk > 0) {
        gload(0);
        sstore(0);
    }
    __syncthreads();
    for (int ks = 0; ks < nk; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < nk) gload((ks + 1) * BK);
        if (warp_live) {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TM];
            if constexpr (kSplitCols) {   // float4 shared loads; B columns tx*4.. and BM/2 + tx*4..
#pragma unroll
                for (int q = 0; q < TM; q += 4) {
                    const float4 av = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM + q]);
                    const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][(q / 4) * (BM / 2) + tx * 4]);
                    a[q] = av.x; a[q + 1] = av.y; a[q + 2] = av.z; a[q + 3] = av.w;
                    b[q] = bv.x; b[q + 1] = bv.y; b[q + 2] = bv.z; b[q + 3] = bv.w;
                }
            } else if constexpr (sizeof(T) == 4 && TM % 2 == 0) {   // float2 shared loads (conflict-free for TM = 6)
#pragma unroll
                for (int q = 0; q < TM; q += 2) {
                    const float2 av = *reinterpret_cast<const float2*>(&As[buf][kk][ty * TM + q]);
                    const float2 bv = *reinterpret_cast<const float2*>(&Bs[buf][kk][tx * TM + q]);
                    a[q] = av.x; a[q + 1] = av.y;
                    b[q] = bv.x; b[q + 1] = bv.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < TM; ++q) {
                    a[q] = As[buf][kk][ty * TM + q];
                    b[q] = Bs[buf][kk][tx * TM + q];
                }
            }
#pragma unroll
            for (int x = 0; x < TM; ++x)
#pragma unroll
                for (int y = 0; y < TM; ++y) acc[x][y] += a[x] * b[y];
        }
        }
        if (ks + 1 < nk) sstore(buf ^ 1);
        __syncthreads();
    }
    const size_t P = npairs(nocc);
    T* O = Obox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
#pragma unroll
    for (int x = 0; x < TM; ++x) {
        int i = i0 + ty * TM + x;
        if (i >= nocc) continue;
#pragma unroll
        for (int y = 0; y < TM; ++y) {
            int j = j0 + (kSplitCols ? (y / 4) * (BM / 2) + tx * 4 + (y % 4) : tx * TM + y);
            if (j >= nocc || j < i) continue;
            O[tri_index(i, j, nocc)] = acc[x][y];
        }
    }
}

// ---------------------------------------------------------------------------
// Steps (b), (c), (d): out[tgt][lm][p] (+)= sum_src sum_l'm' T_src[lm][l'm'] in[src][l'm'][p]
// mode 0: M2M, sources = children of tgt, operator m2m_op[child], lower in l
// mode 1: M2L, sources = interaction list of tgt, operator m2l_op[e], rank lmax_e
// mode 2: L2L, source = parent of tgt, operator l2l_op[tgt], upper in l
// mode 3: M2L and L2L of one level in one pass: the interaction list as in
//         mode 1, then the parent's finished local expansion (read from
//         `parent_in`, operator l2l_opidx[tgt]) when the parent is stored
//         (level >= 3); the target is written once, with no read-modify-write
// grid (pair blocks, targets, lm chunks).
// ---------------------------------------------------------------------------
// Pairs per thread of the translations: FP32 reuses each operator entry read
// from shared memory for 4 pairs (one broadcast load per 4 FMAs); FP64 is
// bound by the DFMA rate and keeps one.
template <typename T>
__host__ __device__ constexpr int translate_ppt() { return sizeof(T) == 4 ? 4 : 1; }

template <typename T, int LMC>
__device__ __forceinline__ void translate_body(int bx, int by, int bz, int mode, int P, int nc, int L, int first_box, int tgt0, const int* __restrict__ ptr,
            const int* __restrict__ list, const int* __restrict__ opidx, const int* __restrict__ lmax_e,
            const int* __restrict__ parent, const T* __restrict__ ops, const T* __restrict__ in,
            T* __restrict__ out, int accumulate, const int* __restrict__ l2l_opidx = nullptr,
            const T* parent_in = nullptr, const int* __restrict__ pcount = nullptr) {
    constexpr int PPT = translate_ppt<T>();
    // pcount (device, nullable): only the first *pcount pairs of each row are
    // live (compacted pairs after occupied-pair screening); P stays the row
    // stride
    const int Pl = pcount ? min(P, *pcount) : P;
    if (bx * (int)blockDim.x * PPT >= Pl) return;     // uniform across the block
    __shared__ T sop[kNcMax][LMC];      // [input component][output component of the chunk]
    const int tgt = tgt0 + by;
    const int c0 = bz * LMC;
    const int ncl = min(LMC, nc - c0);
    const int pb = bx * blockDim.x * PPT + threadIdx.x;      // pairs pb + k * blockDim.x
    bool live[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) live[k] = pb + k * (int)blockDim.x < Pl;
    T acc[PPT][LMC];
    T* o = out + ((size_t)(tgt - first_box) * nc + c0) * P + pb;
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
        for (int q = 0; q < LMC; ++q)
            acc[k][q] = (accumulate && live[k] && q < ncl) ? o[(size_t)q * P + k * blockDim.x] : T(0);
    int e0, e1, eend;
    if (mode == 2) {
        e0 = 0;
        e1 = 1;
    } else {
        e0 = ptr[tgt];
        e1 = ptr[tgt + 1];
    }
    // mode 3: one more step for the parent's local expansion
    eend = e1 + ((mode == 3 && parent[tgt] >= first_box) ? 1 : 0);
    // output rank range of this chunk
    int lhi = 0;
    while ((lhi + 1) * (lhi + 1) <= c0 + ncl - 1) ++lhi;
    int llo = 0;
    while ((llo + 1) * (llo + 1) <= c0) ++llo;
    for (int e = e0; e < eend; ++e) {
        int src, op, Le = L;
        // the L2L step of mode 3 behaves as mode 2
        const bool l2l = mode == 2 || e == e1;
        if (mode == 0) {
            src = list[e];
            op = opidx[src];
        } else if (!l2l) {
            src = list[e];
            op = opidx[e];
            if (lmax_e) Le = lmax_e[e];
        } else {
            src = parent[tgt];
            op = mode == 2 ? opidx[tgt] : l2l_opidx[tgt];
        }
        const int ncr = (Le + 1) * (Le + 1);
        if (c0 >= ncr) continue;   // uniform across the block
        int cb0 = 0, cb1 = ncr;
        if (mode == 0) cb1 = min(ncr, (lhi + 1) * (lhi + 1));
        if (l2l) cb0 = llo * llo;
        const T* Tm = ops + (size_t)op * nc * nc;
        __syncthreads();
        for (int x = threadIdx.x; x < LMC * (cb1 - cb0); x += blockDim.x) {
            int q = x / (cb1 - cb0), c = cb0 + (x - q * (cb1 - cb0));
            sop[c][q] = (q < ncl && c0 + q < ncr) ? Tm[(size_t)(c0 + q) * nc + c] : T(0);
        }
        __syncthreads();
        const T* x = (mode == 3 && l2l ? parent_in : in) + (size_t)(src - first_box) * nc * P + pb;
        // CB input components at a time: all their loads are issued before
        // the first FMA that needs them
        constexpr int CB = (sizeof(T) == 4 && LMC <= 9) ? 8 : 4;
        for (int cb = cb0; cb < cb1; cb += CB) {
            T v[CB][PPT];
#pragma unroll
            for (int u = 0; u < CB; ++u)
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    v[u][k] = (cb + u < cb1 && live[k]) ? x[(size_t)(cb + u) * P + k * blockDim.x] : T(0);
#pragma unroll
            for (int u = 0; u < CB; ++u) {
                if (cb + u >= cb1) break;      // uniform across the block
#pragma unroll
                for (int q = 0; q < LMC; ++q) {
                    const T w = sop[cb + u][q];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) acc[k][q] += w * v[u][k];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!live[k]) continue;
#pragma unroll
        for (int q = 0; q < LMC; ++q)
            if (q < ncl) o[(size_t)q * P + k * blockDim.x] = acc[k][q];
    }
}

// ---------------------------------------------------------------------------
// Step (e), Eq. kri, per leaf B:
//   KB[rowoff_B + r][i] = 2 sum_lm w_lm sum_j W[lm][rowoff_B + r][j] Mcal[B][lm][i][j]
// with w = 1 for m = 0, 2 for Re(m>0), -2 for Im(m>0): the real form of
// sum_{m=-l..l} O_lm Mcal_lm for real densities.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BK, int TM>
__device__ __forceinline__ void l2p_body(int bx, int by, int bz, const int* __restrict__ leaf_rowoff, const T* __restrict__ W, const T* __restrict__ Mbox,
      int nocc, int nrow, int nc, int leaf_store0, double* __restrict__ KB) {
    constexpr int NTH = (BM / TM) * (BM / TM);
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BM + 1];
    const int B = bz;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r0 = bx * BM, i0 = by * BM;
    if (r0 >= nr) return;
    const int tx = threadIdx.x % (BM / TM), ty = threadIdx.x / (BM / TM);
    const size_t P = npairs(nocc);
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    for (int lm = 0; lm < nc; ++lm) {
        int l = 0;
        while ((l + 1) * (l + 1) <= lm) ++l;
        const T w = (lm == l * l) ? T(2) : (((lm - l * l) & 1) ? T(4) : T(-4));
        const T* Wl = W + ((size_t)lm * nrow + rb0) * nocc;
        const T* Ml = Mbox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
        for (int k0 = 0; k0 < nocc; k0 += BK) {
            const bool below = k0 + BK <= i0;   // every j < every i: packed rows j, contiguous in i
            for (int e = threadIdx.x; e < BK * BM; e += NTH) {
                int row = e / BK, kk = e - row * BK;
                int r = r0 + row, j = k0 + kk;
                As[kk][row] = (r < nr && j < nocc) ? Wl[(size_t)r * nocc + j] : T(0);
                int rb = below ? e % BM : row, kb = below ? e / BM : kk;
                int i = i0 + rb, jb = k0 + kb;
                Bs[kb][rb] = (i < nocc && jb < nocc)
                                 ? w * Ml[i <= jb ? tri_index(i, jb, nocc) : tri_index(jb, i, nocc)]
                                 : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T a[TM], b[TM];
#pragma unroll
                for (int q = 0; q < TM; ++q) {
                    a[q] = As[kk][ty * TM + q];
                    b[q] = Bs[kk][tx * TM + q];
                }
#pragma unroll
                for (int x = 0; x < TM; ++x)
#pragma unroll
                    for (int y = 0; y < TM; ++y) acc[x][y] += a[x] * b[y];
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int x = 0; x < TM; ++x) {
        int r = r0 + ty * TM + x;
        if (r >= nr) continue;
#pragma unroll
        for (int y = 0; y < TM; ++y) {
            int i = i0 + tx * TM + y;
            if (i < nocc) KB[(size_t)(rb0 + r) * nocc + i] = (double)acc[x][y];
        }
    }
}

// FP64 step (e) with a 32-row x 16 TI-column block tile (thread tile 2 x TI)
// over the orbitals i0 = 128 by .. i0 + 16 TI - 1: TI = 8 covers a whole
// 128-orbital tile; TI = 2 covers only the first 32 columns of one, for the
// last tile when it holds 32 orbitals or fewer (the other 96 columns would
// be padding that costs DFMAs).  Same sum as l2p_body, less padding on
// leaves with a few dozen AOs.  Block z = leaf * nsplit + split: the split
// covers its share of the flattened (lm, j-chunk) range and writes its own
// copy of KB (summed by the K reduction), so that short grids still fill the
// GPU.
template <int TI = 8>
__device__ __forceinline__ void l2p_rect_body(int bx, int by, int bz, int nsplit, const int* __restrict__ leaf_rowoff,
                                              const double* __restrict__ W, const double* __restrict__ Mbox,
                                              int nocc, int nrow, int nc, int leaf_store0, double* __restrict__ KB,
                                              const unsigned char* __restrict__ tflag = nullptr) {
    constexpr int BR = 32, BI = 16 * TI, BK = 8, TR = 2;
    __shared__ double As[BK][BR + 1];
    __shared__ double Bs[BK][BI + 1];
    const int B = bz / nsplit, ks = bz % nsplit;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r0 = bx * BR, i0 = by * 128;
    if (r0 >= nr) return;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const size_t P = npairs(nocc);
    double acc[TR][TI];
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TI; ++b) acc[a][b] = 0.0;
    const int jt = (nocc + BK - 1) / BK, nkt = nc * jt;
    const int kt0 = (int)((long long)nkt * ks / nsplit), kt1 = (int)((long long)nkt * (ks + 1) / nsplit);
    for (int kt = kt0; kt < kt1; ++kt) {
        const int lm = kt / jt, k0 = (kt - lm * jt) * BK;
        // screened pairs: skip K steps whose Mcal tile holds no kept pair
        if (tflag && !tflag[(size_t)by * jt + k0 / 8]) continue;     // uniform across the block
        int l = 0;
        while ((l + 1) * (l + 1) <= lm) ++l;
        const double w = (lm == l * l) ? 2.0 : (((lm - l * l) & 1) ? 4.0 : -4.0);
        const double* Wl = W + ((size_t)lm * nrow + rb0) * nocc;
        const double* Ml = Mbox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
        {   // A: 32 rows x 8 columns, one element per thread, times the
            // real-form weight w (a power of two, so w a b is rounded exactly
            // as a (w b); 256 multiplies per step instead of 1024 on B)
            const int row = threadIdx.x / BK, kk = threadIdx.x % BK;
            const int r = r0 + row, j = k0 + kk;
            As[kk][row] = (r < nr && j < nocc) ? w * Wl[(size_t)r * nocc + j] : 0.0;
        }
        // B: 128 rows (i) x 8 columns (j) of the symmetric Mcal, read from
        // the packed upper triangle; thread order follows the stored rows
        const bool below = k0 + BK <= i0;
        for (int e = threadIdx.x; e < BK * BI; e += 256) {
            const int row = below ? e % BI : e / BK, kk = below ? e / BI : e % BK;
            const int i = i0 + row, j = k0 + kk;
            Bs[kk][row] = (i < nocc && j < nocc) ? Ml[i <= j ? tri_index(i, j, nocc) : tri_index(j, i, nocc)] : 0.0;
        }
        __syncthreads();
        // a warp covers rows r0 + 4w .. r0 + 4w + 3: skip warps past the leaf's rows
        if (r0 + (threadIdx.x >> 5) * 2 * TR < nr) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double a[TR], b[TI];
#pragma unroll
                for (int q = 0; q < TR; ++q) a[q] = As[kk][ty * TR + q];
#pragma unroll
                for (int q = 0; q < TI; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
                for (int x = 0; x < TR; ++x)
#pragma unroll
                    for (int y = 0; y < TI; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < TR; ++x) {
        const int r = r0 + ty * TR + x;
        if (r >= nr) continue;
#pragma unroll
        for (int y = 0; y < TI; ++y) {
            const int i = i0 + tx + 16 * y;
            if (i < nocc) KB[(size_t)ks * nrow * nocc + (size_t)(rb0 + r) * nocc + i] = acc[x][y];
        }
    }
}

// FP32 step (e): 96 AO rows x 128 orbitals per block (256 threads, thread
// tile 6 rows x 8 orbitals, the orbitals in two groups of 4 at tx*4 and
// 64 + tx*4 so that a quarter warp's 16-byte loads are conflict-free; K step
// 32).  The (lm, j) range may be split over `nsplit` blocks, each writing its
// own copy of KB (summed by the K reduction), so that the grid covers the GPU
// in several waves instead of one and a sliver.  A leaf of up to 96 AOs is
// one row tile, so each element of the packed Mcal is read once per leaf;
// shared-memory operands are read as float2/float4 (5 loads per 48 FMAs).
//
// TI = 2 covers only the first 32 orbitals of the 128-orbital tile `by`
// (columns tx + 16 y), for the last tile when it holds 32 or fewer.
template <int TI = 8>
__device__ __forceinline__ void l2p_rect_body_f(int bx, int by, int bz, int nsplit, const int* __restrict__ leaf_rowoff,
                                                const float* __restrict__ W, const float* __restrict__ Mbox,
                                                int nocc, int nrow, int nc, int leaf_store0,
                                                double* __restrict__ KB,
                                                const unsigned char* __restrict__ tflag = nullptr) {
    constexpr int BR = 96, BI = 16 * TI, BK = 32, TR = 6;
    __shared__ __align__(16) float As[BK][BR + 4];
    __shared__ __align__(16) float Bs[BK][BI + 4];
    // block z = leaf * nsplit + split: the split covers its share of the
    // flattened (lm, j-chunk) range and writes its own copy of KB
    const int B = bz / nsplit, ks = bz % nsplit;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r0 = bx * BR, i0 = by * 128;
    if (r0 >= nr) return;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const size_t P = npairs(nocc);
    float acc[TR][TI];
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TI; ++b) acc[a][b] = 0.f;
    // rows of this warp: r0 + 12 w .. r0 + 12 w + 11
    const bool warp_live = r0 + (threadIdx.x >> 5) * 2 * TR < nr;
    const int jt = (nocc + BK - 1) / BK, nkt = nc * jt;
    const int kt0 = (int)((long long)nkt * ks / nsplit), kt1 = (int)((long long)nkt * (ks + 1) / nsplit);
    const int nj8 = (nocc + 7) / 8;
    for (int kt = kt0; kt < kt1; ++kt) {
        const int lm = kt / jt, k0 = (kt - lm * jt) * BK;
        if (tflag) {
            // screened pairs: skip K steps whose Mcal tile holds no kept pair
            // (flags per 128 orbitals x 8 j; this step covers four)
            bool any = false;
#pragma unroll
            for (int u = 0; u < BK / 8; ++u)
                if (k0 / 8 + u < nj8) any |= tflag[(size_t)by * nj8 + k0 / 8 + u] != 0;
            if (!any) continue;     // uniform across the block
        }
        int l = 0;
        while ((l + 1) * (l + 1) <= lm) ++l;
        const float w = (lm == l * l) ? 2.f : (((lm - l * l) & 1) ? 4.f : -4.f);
        const float* Wl = W + ((size_t)lm * nrow + rb0) * nocc;
        const float* Ml = Mbox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
#pragma unroll
        for (int m = 0; m < (BR * BK) / 256; ++m) {
            const int e = threadIdx.x + 256 * m;
            const int row = e / BK, kk = e % BK;
            const int r = r0 + row, j = k0 + kk;
            As[kk][row] = (r < nr && j < nocc) ? Wl[(size_t)r * nocc + j] : 0.f;
        }
        const bool below = k0 + BK <= i0;
#pragma unroll
        for (int m = 0; m < (BI * BK) / 256; ++m) {
            const int e = threadIdx.x + 256 * m;
            const int row = below ? e % BI : e / BK, kk = below ? e / BI : e % BK;
            const int i = i0 + row, j = k0 + kk;
            // packed index of (min, max) in 32-bit arithmetic (P < 2^32)
            const unsigned a = (unsigned)min(i, j), bb = (unsigned)max(i, j);
            const unsigned q = ((a * (2u * (unsigned)nocc + 1u - a)) >> 1) + (bb - a);
            Bs[kk][row] = (i < nocc && j < nocc) ? w * Ml[q] : 0.f;
        }
        __syncthreads();
        if (warp_live) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float2 a0 = *reinterpret_cast<const float2*>(&As[kk][ty * TR]);
                const float2 a1 = *reinterpret_cast<const float2*>(&As[kk][ty * TR + 2]);
                const float2 a2 = *reinterpret_cast<const float2*>(&As[kk][ty * TR + 4]);
                const float av[6] = {a0.x, a0.y, a1.x, a1.y, a2.x, a2.y};
                float bv[TI];
                if constexpr (TI == 8) {
                    // columns tx*4.. and 64 + tx*4..: each quarter warp reads
                    // 128 contiguous bytes (no bank conflict)
                    const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
                    const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
                    bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
                    bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
                } else {
#pragma unroll
                    for (int y = 0; y < TI; ++y) bv[y] = Bs[kk][tx + 16 * y];
                }
#pragma unroll
                for (int x = 0; x < TR; ++x)
#pragma unroll
                    for (int y = 0; y < TI; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < TR; ++x) {
        const int r = r0 + ty * TR + x;
        if (r >= nr) continue;
#pragma unroll
        for (int y = 0; y < TI; ++y) {
            const int i = i0 + (TI == 8 ? (y >> 2) * 64 + tx * 4 + (y & 3) : tx + 16 * y);
            if (i < nocc) KB[(size_t)ks * nrow * nocc + (size_t)(rb0 + r) * nocc + i] = (double)acc[x][y];
        }
    }
}

// ---------------------------------------------------------------------------
// K[r + i*ldk] = sum over the leaf rows of AO r of KB[row][i] (summed over the
// nsplit copies of KB when step (e) split its K range), in FP64, and the
// per-block partial of E = -1/2 sum_ri C_ri K_ri.
// ---------------------------------------------------------------------------
// With a column block [col0, col1) only those columns are reduced and
// written (elements x = i * nao + r from col0 * nao on, in the same order).
static __device__ __forceinline__ void reduce_body(int bx, int by, int bz, const int* __restrict__ ao_row_ptr, const int* __restrict__ ao_rows,
                           const double* __restrict__ KB, int nao, int nocc,
                           const double* __restrict__ C, int ldc, double* __restrict__ K, int ldk,
                           double* __restrict__ part, int nsplit = 1, size_t split_stride = 0, int col0 = 0,
                           int col1 = -1) {
    __shared__ double red[256];
    double e = 0.0;
    const long long x0 = (long long)nao * col0;
    const long long n = (long long)nao * (col1 < 0 ? nocc : col1);
    for (long long x = x0 + (long long)bx * blockDim.x + threadIdx.x; x < n;
         x += (long long)bz * blockDim.x) {
        int i = (int)(x / nao), r = (int)(x - (long long)i * nao);
        double s = 0.0;
        for (int q = ao_row_ptr[r]; q < ao_row_ptr[r + 1]; ++q)
            for (int sp = 0; sp < nsplit; ++sp) s += KB[sp * split_stride + (size_t)ao_rows[q] * nocc + i];
        K[(size_t)i * ldk + r] = s;
        e += C[(size_t)i * ldc + r] * s;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[bx] = red[0];
}

static __global__ void k_final_energy(const double* __restrict__ part, int n, double* __restrict__ E) {
    __shared__ double red[256];
    double s = 0.0;
    for (int x = threadIdx.x; x < n; x += blockDim.x) s += part[x];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = -0.5 * red[0];
}

// Per-block partials of E = -1/2 sum_ri C_ri K_ri from a stored K, with the
// element order, grid and per-thread accumulation of reduce_body (same grid),
// so that k_final_energy then gives the energy of that K bit for bit as the
// far-field call would have.
static __global__ void k_energy_parts(int nao, int nocc, const double* __restrict__ C, int ldc,
                                      const double* __restrict__ K, int ldk, double* __restrict__ part) {
    __shared__ double red[256];
    double e = 0.0;
    const long long n = (long long)nao * nocc;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(x / nao), r = (int)(x - (long long)i * nao);
        e += C[(size_t)i * ldc + r] * K[(size_t)i * ldk + r];
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

static __global__ void k_zero_K(double* K, int ldk, int nao, int nocc, double* E) {
    long long n = (long long)nao * nocc;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (long long)gridDim.x * blockDim.x) {
        int i = (int)(x / nao), r = (int)(x - (long long)i * nao);
        K[(size_t)i * ldk + r] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *E = 0.0;
}


}  // namespace body
}  // namespace occk
