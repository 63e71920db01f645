// Steps (a)-(e) of the far-field occupied exchange on SIMT cores, in FP64
// (DFMA) or FP32 (FFMA); K and the energy are always reduced in FP64.
//
// Layouts in HBM (P = nocc^2 occupied pairs, pair index p = i*nocc + j):
//   Ct   [nao][nocc]            row-major copy of C
//   W    [nc][nrow][nocc]       O^{rj,X}_lm for the AO set S_B of every leaf,
//                               leaves stacked (row = leaf_rowoff[B] + local)
//   Obox [box][nc][P]           O^{ij,X}_lm for boxes of levels 2..D
//   Mbox [box][nc][P]           Mcal^{ij}_lm(X), same boxes
//   KB   [nrow][nocc]           per-leaf partial K rows (FP64)
// Every pair-indexed access is coalesced along p (or along j).
#include <algorithm>
#include <cstdio>

#include "occk_internal.h"

namespace occk {

namespace {

constexpr int kNcMax = 169;   // (12+1)^2

// ---------------------------------------------------------------------------
// C (column-major, ldc) -> Ct (row-major), 32x32 tiles through shared memory
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_transpose_C(const double* __restrict__ C, int ldc, int nao, int nocc,
                              T* __restrict__ Ct) {
    __shared__ double tile[32][33];
    int r0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
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
__global__ void k_half(const int* __restrict__ row_ptr, const int* __restrict__ ent_col,
                       const int* __restrict__ ent_val, const T* __restrict__ vals, int nc,
                       const T* __restrict__ Ct, int nocc, int nrow, T* __restrict__ W) {
    const int row = blockIdx.x;
    const int c0 = blockIdx.y * LMC;
    const int e0 = row_ptr[row], e1 = row_ptr[row + 1];
    const int ncl = min(LMC, nc - c0);
    for (int j = threadIdx.x; j < nocc; j += blockDim.x) {
        T acc[LMC];
#pragma unroll
        for (int q = 0; q < LMC; ++q) acc[q] = T(0);
        for (int e = e0; e < e1; ++e) {
            const T cs = Ct[(size_t)ent_col[e] * nocc + j];
            const T* v = vals + (size_t)ent_val[e] * nc + c0;
#pragma unroll
            for (int q = 0; q < LMC; ++q)
                if (q < ncl) acc[q] += v[q] * cs;
        }
#pragma unroll
        for (int q = 0; q < LMC; ++q)
            if (q < ncl) W[((size_t)(c0 + q) * nrow + row) * nocc + j] = acc[q];
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
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
k_full(const int* __restrict__ leaf_rowoff, const int* __restrict__ leaf_aos,
       const T* __restrict__ Ct, const T* __restrict__ W, int nocc, int nrow, int nc,
       int ntile, T* __restrict__ Obox, int leaf_store0) {
    constexpr int NTH = (BM / TM) * (BM / TM);
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BM];
    __shared__ int aos[BK];
    const int B = blockIdx.y / nc;
    const int lm = blockIdx.y - B * nc;
    // triangular tile index -> (ti, tj), ti <= tj
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int i0 = ti * BM, j0 = tj * BM;
    const int tx = threadIdx.x % (BM / TM), ty = threadIdx.x / (BM / TM);
    const T* Wl = W + ((size_t)lm * nrow + rb0) * nocc;
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < nr; k0 += BK) {
        if (threadIdx.x < BK) aos[threadIdx.x] = (k0 + threadIdx.x < nr) ? leaf_aos[rb0 + k0 + threadIdx.x] : -1;
        __syncthreads();
        for (int e = threadIdx.x; e < BK * BM; e += NTH) {
            int kk = e / BM, c = e - kk * BM;
            int ao = aos[kk];
            int ii = i0 + c, jj = j0 + c;
            As[kk][c] = (ao >= 0 && ii < nocc) ? Ct[(size_t)ao * nocc + ii] : T(0);
            Bs[kk][c] = (ao >= 0 && jj < nocc) ? Wl[(size_t)(k0 + kk) * nocc + jj] : T(0);
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
    const size_t P = (size_t)nocc * nocc;
    T* O = Obox + ((size_t)(leaf_store0 + B) * nc + lm) * P;
#pragma unroll
    for (int x = 0; x < TM; ++x) {
        int i = i0 + ty * TM + x;
        if (i >= nocc) continue;
#pragma unroll
        for (int y = 0; y < TM; ++y) {
            int j = j0 + tx * TM + y;
            if (j >= nocc) continue;
            O[(size_t)i * nocc + j] = acc[x][y];
            if (ti != tj) O[(size_t)j * nocc + i] = acc[x][y];
        }
    }
}

// ---------------------------------------------------------------------------
// Steps (b), (c), (d): out[tgt][lm][p] (+)= sum_src sum_l'm' T_src[lm][l'm'] in[src][l'm'][p]
// mode 0: M2M, sources = children of tgt, operator m2m_op[child], lower in l
// mode 1: M2L, sources = interaction list of tgt, operator m2l_op[e], rank lmax_e
// mode 2: L2L, source = parent of tgt, operator l2l_op[tgt], upper in l
// grid (pair blocks, targets, lm chunks).
// ---------------------------------------------------------------------------
template <typename T, int LMC>
__global__ void __launch_bounds__(128)
k_translate(int mode, int P, int nc, int L, int first_box, int tgt0, const int* __restrict__ ptr,
            const int* __restrict__ list, const int* __restrict__ opidx, const int* __restrict__ lmax_e,
            const int* __restrict__ parent, const T* __restrict__ ops, const T* __restrict__ in,
            T* __restrict__ out, int accumulate) {
    __shared__ T sop[LMC][kNcMax];
    const int tgt = tgt0 + blockIdx.y;
    const int c0 = blockIdx.z * LMC;
    const int ncl = min(LMC, nc - c0);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = p < P;
    T acc[LMC];
    T* o = out + ((size_t)(tgt - first_box) * nc + c0) * P + p;
#pragma unroll
    for (int q = 0; q < LMC; ++q) acc[q] = (accumulate && live && q < ncl) ? o[(size_t)q * P] : T(0);
    int e0, e1;
    if (mode == 2) {
        e0 = 0;
        e1 = 1;
    } else {
        e0 = ptr[tgt];
        e1 = ptr[tgt + 1];
    }
    // output rank range of this chunk
    int lhi = 0;
    while ((lhi + 1) * (lhi + 1) <= c0 + ncl - 1) ++lhi;
    int llo = 0;
    while ((llo + 1) * (llo + 1) <= c0) ++llo;
    for (int e = e0; e < e1; ++e) {
        int src, op, Le = L;
        if (mode == 0) {
            src = list[e];
            op = opidx[src];
        } else if (mode == 1) {
            src = list[e];
            op = opidx[e];
            if (lmax_e) Le = lmax_e[e];
        } else {
            src = parent[tgt];
            op = opidx[tgt];
        }
        const int ncr = (Le + 1) * (Le + 1);
        if (c0 >= ncr) continue;   // uniform across the block
        int cb0 = 0, cb1 = ncr;
        if (mode == 0) cb1 = min(ncr, (lhi + 1) * (lhi + 1));
        if (mode == 2) cb0 = llo * llo;
        const T* Tm = ops + (size_t)op * nc * nc;
        __syncthreads();
        for (int x = threadIdx.x; x < LMC * (cb1 - cb0); x += blockDim.x) {
            int q = x / (cb1 - cb0), c = cb0 + (x - q * (cb1 - cb0));
            sop[q][c] = (q < ncl && c0 + q < ncr) ? Tm[(size_t)(c0 + q) * nc + c] : T(0);
        }
        __syncthreads();
        if (live) {
            const T* x = in + (size_t)(src - first_box) * nc * P + p;
            for (int c = cb0; c < cb1; ++c) {
                const T v = x[(size_t)c * P];
#pragma unroll
                for (int q = 0; q < LMC; ++q) acc[q] += sop[q][c] * v;
            }
        }
    }
    if (live) {
#pragma unroll
        for (int q = 0; q < LMC; ++q)
            if (q < ncl) o[(size_t)q * P] = acc[q];
    }
}

// ---------------------------------------------------------------------------
// Step (e), Eq. kri, per leaf B:
//   KB[rowoff_B + r][i] = 2 sum_lm w_lm sum_j W[lm][rowoff_B + r][j] Mcal[B][lm][i][j]
// with w = 1 for m = 0, 2 for Re(m>0), -2 for Im(m>0): the real form of
// sum_{m=-l..l} O_lm Mcal_lm for real densities.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BK, int TM>
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
k_l2p(const int* __restrict__ leaf_rowoff, const T* __restrict__ W, const T* __restrict__ Mbox,
      int nocc, int nrow, int nc, int leaf_store0, double* __restrict__ KB) {
    constexpr int NTH = (BM / TM) * (BM / TM);
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BM + 1];
    const int B = blockIdx.z;
    const int rb0 = leaf_rowoff[B], nr = leaf_rowoff[B + 1] - rb0;
    const int r0 = blockIdx.x * BM, i0 = blockIdx.y * BM;
    if (r0 >= nr) return;
    const int tx = threadIdx.x % (BM / TM), ty = threadIdx.x / (BM / TM);
    const size_t P = (size_t)nocc * nocc;
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
            for (int e = threadIdx.x; e < BK * BM; e += NTH) {
                int row = e / BK, kk = e - row * BK;
                int r = r0 + row, i = i0 + row, j = k0 + kk;
                As[kk][row] = (r < nr && j < nocc) ? Wl[(size_t)r * nocc + j] : T(0);
                Bs[kk][row] = (i < nocc && j < nocc) ? w * Ml[(size_t)i * nocc + j] : T(0);
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

// ---------------------------------------------------------------------------
// K[r + i*ldk] = sum over the leaf rows of AO r of KB[row][i], in FP64, and the
// per-block partial of E = -1/2 sum_ri C_ri K_ri.
// ---------------------------------------------------------------------------
__global__ void k_reduce_K(const int* __restrict__ ao_row_ptr, const int* __restrict__ ao_rows,
                           const double* __restrict__ KB, int nao, int nocc,
                           const double* __restrict__ C, int ldc, double* __restrict__ K, int ldk,
                           double* __restrict__ part) {
    __shared__ double red[256];
    double e = 0.0;
    const long long n = (long long)nao * nocc;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (long long)gridDim.x * blockDim.x) {
        int i = (int)(x / nao), r = (int)(x - (long long)i * nao);
        double s = 0.0;
        for (int q = ao_row_ptr[r]; q < ao_row_ptr[r + 1]; ++q) s += KB[(size_t)ao_rows[q] * nocc + i];
        K[(size_t)i * ldk + r] = s;
        e += C[(size_t)i * ldc + r] * s;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_final_energy(const double* __restrict__ part, int n, double* __restrict__ E) {
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

__global__ void k_zero_K(double* K, int ldk, int nao, int nocc, double* E) {
    long long n = (long long)nao * nocc;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (long long)gridDim.x * blockDim.x) {
        int i = (int)(x / nao), r = (int)(x - (long long)i * nao);
        K[(size_t)i * ldk + r] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *E = 0.0;
}

// ---------------------------------------------------------------------------
// FMA throughput probe: 8 independent dependent chains per thread.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fma_probe(T* out, int iters, T seed) {
    T a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5,
      a6 = a0 + 6, a7 = a0 + 7;
    const T m = T(0.999999), c = T(1e-7);
    for (int k = 0; k < iters; ++k) {
        a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
        a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
    }
    T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == T(-1.2345)) out[threadIdx.x] = s;
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
template <typename T>
cudaError_t run_typed(const FmmArgs& a, cudaStream_t s) {
    const int nocc = a.nocc, nc = a.nc, D = a.depth;
    const long long P = (long long)nocc * nocc;
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
        constexpr int LMC = 16;
        dim3 g(a.nrow, (nc + LMC - 1) / LMC);
        k_half<T, LMC><<<g, 128, 0, s>>>(a.row_ptr, a.ent_col, a.ent_val, vals, nc, Ct, nocc, a.nrow, W);
    }
    const int leaf_store0 = a.leaf0 - a.first_box;
    const bool tcm = sizeof(T) == 4 && tc_mode(a.prec) >= 0;
    mark(1);
    if (tcm) {
        cudaError_t e2 = tc_run_a2(a.prec, a.leaf_rowoff, a.leaf_aos, (const float*)Ct, (const float*)W, nocc,
                                   a.nrow, nc, a.nleaf, leaf_store0, a.lscale, (float*)Ob, a.err_word, s);
        if (e2 != cudaSuccess) return e2;
    } else if constexpr (sizeof(T) == 8) {
        constexpr int BM = 64, BK = 8, TM = 4;
        int nt = (nocc + BM - 1) / BM;
        dim3 g(nt * (nt + 1) / 2, a.nleaf * nc);
        k_full<T, BM, BK, TM><<<g, (BM / TM) * (BM / TM), 0, s>>>(a.leaf_rowoff, a.leaf_aos, Ct, W, nocc,
                                                                 a.nrow, nc, nt, Ob, leaf_store0);
    } else {
        constexpr int BM = 128, BK = 8, TM = 8;
        int nt = (nocc + BM - 1) / BM;
        dim3 g(nt * (nt + 1) / 2, a.nleaf * nc);
        k_full<T, BM, BK, TM><<<g, (BM / TM) * (BM / TM), 0, s>>>(a.leaf_rowoff, a.leaf_aos, Ct, W, nocc,
                                                                 a.nrow, nc, nt, Ob, leaf_store0);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int LMC = translate_chunk(nc);
    const int nchunk = (nc + LMC - 1) / LMC;
    const unsigned pblocks = (unsigned)((P + 127) / 128);
    // (b) M2M: parents at level lev-1 gather their children at level lev
    mark(2);
    for (int lev = D; lev >= 3; --lev) {
        int t0 = a.level_off[lev - 1], nt = a.level_off[lev] - t0;
        dim3 g(pblocks, nt, nchunk);
        launch_translate<T>(LMC, g, s, 0, (int)P, nc, a.L, a.first_box, t0, a.child_ptr,
                                             a.child_list, a.m2m_op, nullptr, a.parent, ops, Ob, Ob, 0);
    }
    // learned ranks: features from the multipoles of every box, FP16 MLP,
    // budgeted choice; M2L then reads the per-edge ranks
    const int* lmax_e = a.m2l_lmax;
    if (a.learned) {
        cudaError_t e2 = edge_features(sizeof(T) == 8, Ob, a.first_box, a.nbox, nc, a.L, P, a.nm2l, a.m2l_tgt,
                                       a.m2l_src, a.box_key, a.box_level, a.hlev, D, a.nrm, a.feat, s);
        if (e2 == cudaSuccess)
            e2 = mlp_predict_fp16(a.mlp_prm, (__half*)a.mlp_h, a.mlp_norm, a.feat, a.nm2l, a.pred, s);
        if (e2 == cudaSuccess) e2 = select_ranks(a.pred, a.nm2l, a.L, a.tau, a.ranks, s);
        if (e2 != cudaSuccess) return e2;
        lmax_e = a.ranks;
    }
    // (c) M2L: every box of levels 2..D, all levels in one launch
    mark(3);
    if (tcm && nc <= 128) {
        int t0 = a.level_off[2], nt = a.nbox - t0;
        cudaError_t e2 = tc_run_m2l(a.prec, (int)P, nc, a.L, a.first_box, t0, nt, a.m2l_ptr, a.m2l_src, a.m2l_op,
                                    lmax_e, (const float*)ops, (const float*)Ob, (float*)Mb, a.box_scale,
                                    a.err_word, s);
        if (e2 != cudaSuccess) return e2;
    } else {
        int t0 = a.level_off[2], nt = a.nbox - t0;
        dim3 g(pblocks, nt, nchunk);
        launch_translate<T>(LMC, g, s, 1, (int)P, nc, a.L, a.first_box, t0, a.m2l_ptr, a.m2l_src,
                                             a.m2l_op, lmax_e, a.parent, ops, Ob, Mb, 0);
    }
    // (d) L2L: children at level lev accumulate their parent's expansion
    mark(4);
    for (int lev = 3; lev <= D; ++lev) {
        int t0 = a.level_off[lev], nt = a.level_off[lev + 1] - t0;
        dim3 g(pblocks, nt, nchunk);
        launch_translate<T>(LMC, g, s, 2, (int)P, nc, a.L, a.first_box, t0, nullptr, nullptr,
                                             a.l2l_op, nullptr, a.parent, ops, Mb, Mb, 1);
    }
    // (e) L2P
    mark(5);
    if (tcm) {
        cudaError_t e2 = tc_run_l2p(a.prec, a.leaf_rowoff, (const float*)W, (const float*)Mb, nocc, a.nrow, nc,
                                    a.nleaf, leaf_store0, a.max_rows, a.lscale, a.kb, a.err_word, s);
        if (e2 != cudaSuccess) return e2;
    } else if constexpr (sizeof(T) == 8) {
        constexpr int BM = 64, BK = 8, TM = 4;
        dim3 g((a.max_rows + BM - 1) / BM, (nocc + BM - 1) / BM, a.nleaf);
        k_l2p<T, BM, BK, TM><<<g, (BM / TM) * (BM / TM), 0, s>>>(a.leaf_rowoff, W, Mb, nocc, a.nrow, nc,
                                                                 leaf_store0, a.kb);
    } else {
        constexpr int BM = 128, BK = 8, TM = 8;
        dim3 g((a.max_rows + BM - 1) / BM, (nocc + BM - 1) / BM, a.nleaf);
        k_l2p<T, BM, BK, TM><<<g, (BM / TM) * (BM / TM), 0, s>>>(a.leaf_rowoff, W, Mb, nocc, a.nrow, nc,
                                                                 leaf_store0, a.kb);
    }
    mark(6);
    constexpr int kRedBlocks = 1024;
    k_reduce_K<<<kRedBlocks, 256, 0, s>>>(a.ao_row_ptr, a.ao_rows, a.kb, a.nao, nocc, a.C, a.ldc, a.K,
                                          a.ldk, a.part);
    k_final_energy<<<1, 256, 0, s>>>(a.part, kRedBlocks, a.Ex_dev);
    mark(OCCK_NSTAGE);
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_farfield(const FmmArgs& a, cudaStream_t s) {
    if (a.prec == OCCK_FP64) return run_typed<double>(a, s);
    return run_typed<float>(a, s);
}

cudaError_t probe_fma(int prec, int sm_count, double* flops, cudaStream_t s) {
    const int iters = 1 << 14;
    const int blocks = sm_count * 8, threads = 256;
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 1024 * 8);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        if (prec == OCCK_FP64)
            k_fma_probe<double><<<blocks, threads, 0, s>>>((double*)buf, iters, 1.0);
        else
            k_fma_probe<float><<<blocks, threads, 0, s>>>((float*)buf, iters * 8, 1.0f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    const double nfma = (double)blocks * threads * 8.0 * (prec == OCCK_FP64 ? iters : iters * 8.0);
    *flops = 2.0 * nfma / (best * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace occk
