// Learned multipole-rank selector for M2L (an addition to the paper's method).
//
// A 3-layer MLP (16 -> 64 -> 64 -> 8, ReLU) maps features of an M2L edge (box
// geometry, separation ratio, per-box multipole norms) to the predicted
// log10 truncation error of that edge's energy at ranks 2..9 relative to rank
// 10.  Training (full-batch Adam, MSE) and inference run in these kernels:
// FP32 training, FP16 inference (FP16 weights and activations, FP32 sums).
//
// Labels come from the method itself: the far-field energy splits exactly
// over M2L edges because M2M and L2L are exact re-expansions, so
//   e_edge(L') = -sum_p sum_{c,c' <= L'} w_c T_e[c][c'] O_t[c][p] O_s[c'][p]
// with w the real-form weights (1, 2, -2) and p all occupied pairs; it is
// evaluated through the pair-summed Gram matrix G_e = O_t O_s^T over the
// stored pairs i <= j, off-diagonal pairs counted twice.
//
// Rank choice: minimise sum_e (L_e+1)^4 (the M2L cost) subject to
// sum_e err_e(L_e) <= tau, by bisection on the Lagrange multiplier; edges
// whose prediction is not finite keep the full rank.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdio>

#include "occk_internal.h"

namespace occk {

namespace {

constexpr int NIN = OCCK_MLP_NIN, H = OCCK_MLP_HIDDEN, NOUT = OCCK_MLP_NOUT;
constexpr int NP = NIN * H + H + H * H + H + H * NOUT + NOUT;
constexpr int OFF_W1 = 0, OFF_B1 = NIN * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * NOUT;

// ---------------------------------------------------------------------------
// Forward: one thread per sample, weights in shared memory.  norm = [mean_x
// (NIN), std_x (NIN), mean_y (NOUT), std_y (NOUT)].  Writes the normalised
// input, the pre-activations (for backward) and the normalised output.
// ---------------------------------------------------------------------------
__global__ void k_mlp_fwd(const float* __restrict__ prm, const float* __restrict__ norm,
                          const float* __restrict__ X, int n, float* __restrict__ Xn, float* __restrict__ Z1,
                          float* __restrict__ Z2, float* __restrict__ Y) {
    __shared__ float w[NP];
    for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = prm[k];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[NIN], h1[H];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        x[i] = (X[(size_t)s * NIN + i] - norm[i]) / norm[NIN + i];
        if (Xn) Xn[(size_t)s * NIN + i] = x[i];
    }
    for (int j = 0; j < H; ++j) {
        float z = w[OFF_B1 + j];
#pragma unroll
        for (int i = 0; i < NIN; ++i) z += x[i] * w[OFF_W1 + i * H + j];
        if (Z1) Z1[(size_t)s * H + j] = z;
        h1[j] = z > 0.f ? z : 0.f;
    }
    float y[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) y[k] = w[OFF_B3 + k];
    for (int j = 0; j < H; ++j) {
        float z = w[OFF_B2 + j];
        for (int i = 0; i < H; ++i) z += h1[i] * w[OFF_W2 + i * H + j];
        if (Z2) Z2[(size_t)s * H + j] = z;
        const float h2 = z > 0.f ? z : 0.f;
#pragma unroll
        for (int k = 0; k < NOUT; ++k) y[k] += h2 * w[OFF_W3 + j * NOUT + k];
    }
#pragma unroll
    for (int k = 0; k < NOUT; ++k) Y[(size_t)s * NOUT + k] = y[k];
}

// FP16 inference: weights and activations in half precision, FP32 sums;
// output de-normalised to log10 errors.
__global__ void k_mlp_fwd_h(const __half* __restrict__ prm, const float* __restrict__ norm,
                            const float* __restrict__ X, int n, float* __restrict__ Y) {
    __shared__ __half w[NP];
    for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = prm[k];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    __half x[NIN], h1[H];
#pragma unroll
    for (int i = 0; i < NIN; ++i) x[i] = __float2half((X[(size_t)s * NIN + i] - norm[i]) / norm[NIN + i]);
    for (int j = 0; j < H; ++j) {
        float z = __half2float(w[OFF_B1 + j]);
#pragma unroll
        for (int i = 0; i < NIN; ++i) z += __half2float(__hmul(x[i], w[OFF_W1 + i * H + j]));
        h1[j] = __float2half(z > 0.f ? z : 0.f);
    }
    float y[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) y[k] = __half2float(w[OFF_B3 + k]);
    for (int j = 0; j < H; ++j) {
        float z = __half2float(w[OFF_B2 + j]);
        for (int i = 0; i < H; ++i) z += __half2float(__hmul(h1[i], w[OFF_W2 + i * H + j]));
        const __half h2 = __float2half(z > 0.f ? z : 0.f);
#pragma unroll
        for (int k = 0; k < NOUT; ++k) y[k] += __half2float(__hmul(h2, w[OFF_W3 + j * NOUT + k]));
    }
    const float* my = norm + 2 * NIN;
    const float* sy = norm + 2 * NIN + NOUT;
#pragma unroll
    for (int k = 0; k < NOUT; ++k) Y[(size_t)s * NOUT + k] = y[k] * sy[k] + my[k];
}

// dY = 2 (Y - T) / (n NOUT) and the per-block partial of sum (Y - T)^2.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int n, float* __restrict__ dY,
                      double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    const long long tot = (long long)n * NOUT;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < tot;
         x += (long long)gridDim.x * blockDim.x) {
        const float d = Y[x] - T[x];
        dY[x] = 2.f * d / (float)tot;
        acc += (double)d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dZ2 = (dY W3^T) * [Z2 > 0], dZ1 = (dZ2 W2^T) * [Z1 > 0], one thread per sample.
__global__ void k_mlp_dz(const float* __restrict__ prm, const float* __restrict__ Z1,
                         const float* __restrict__ Z2, const float* __restrict__ dY, int n,
                         float* __restrict__ dZ1, float* __restrict__ dZ2) {
    __shared__ float w[NP];
    for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = prm[k];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float dy[NOUT], dz2[H];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) dy[k] = dY[(size_t)s * NOUT + k];
    for (int j = 0; j < H; ++j) {
        float g = 0.f;
#pragma unroll
        for (int k = 0; k < NOUT; ++k) g += dy[k] * w[OFF_W3 + j * NOUT + k];
        dz2[j] = Z2[(size_t)s * H + j] > 0.f ? g : 0.f;
        dZ2[(size_t)s * H + j] = dz2[j];
    }
    for (int i = 0; i < H; ++i) {
        float g = 0.f;
        for (int j = 0; j < H; ++j) g += dz2[j] * w[OFF_W2 + i * H + j];
        dZ1[(size_t)s * H + i] = Z1[(size_t)s * H + i] > 0.f ? g : 0.f;
    }
}

// Parameter gradients, one thread per parameter, fixed-order sums over samples:
//   gW1 = Xn^T dZ1, gb1 = sum dZ1, gW2 = relu(Z1)^T dZ2, gb2 = sum dZ2,
//   gW3 = relu(Z2)^T dY, gb3 = sum dY.
__global__ void k_mlp_wgrad(const float* __restrict__ Xn, const float* __restrict__ Z1,
                            const float* __restrict__ Z2, const float* __restrict__ dZ1,
                            const float* __restrict__ dZ2, const float* __restrict__ dY, int n,
                            float* __restrict__ grad) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NP) return;
    double acc = 0.0;
    if (q < OFF_B1) {
        const int i = q / H, j = q % H;
        for (int s = 0; s < n; ++s) acc += (double)Xn[(size_t)s * NIN + i] * dZ1[(size_t)s * H + j];
    } else if (q < OFF_W2) {
        const int j = q - OFF_B1;
        for (int s = 0; s < n; ++s) acc += dZ1[(size_t)s * H + j];
    } else if (q < OFF_B2) {
        const int i = (q - OFF_W2) / H, j = (q - OFF_W2) % H;
        for (int s = 0; s < n; ++s) {
            const float h = Z1[(size_t)s * H + i];
            if (h > 0.f) acc += (double)h * dZ2[(size_t)s * H + j];
        }
    } else if (q < OFF_W3) {
        const int j = q - OFF_B2;
        for (int s = 0; s < n; ++s) acc += dZ2[(size_t)s * H + j];
    } else if (q < OFF_B3) {
        const int i = (q - OFF_W3) / NOUT, k = (q - OFF_W3) % NOUT;
        for (int s = 0; s < n; ++s) {
            const float h = Z2[(size_t)s * H + i];
            if (h > 0.f) acc += (double)h * dY[(size_t)s * NOUT + k];
        }
    } else {
        const int k = q - OFF_B3;
        for (int s = 0; s < n; ++s) acc += dY[(size_t)s * NOUT + k];
    }
    grad[q] = (float)acc;
}

__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int np, float lr, float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float mm = b1 * m[q] + (1.f - b1) * g[q];
    const float vv = b2 * v[q] + (1.f - b2) * g[q] * g[q];
    m[q] = mm;
    v[q] = vv;
    prm[q] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
}

__global__ void k_to_half(const float* __restrict__ a, __half* __restrict__ b, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) b[q] = __float2half(a[q]);
}

// ---------------------------------------------------------------------------
// Per-box multipole norms: nrm[box][l] = sqrt(sum_{c in rank l} sum_p O[box][c][p]^2)
// ---------------------------------------------------------------------------
// Pairs are stored once (i <= j); a stored off-diagonal pair stands for two
// entries of the full i,j square, so sums over pairs weigh it by 2.
__device__ __forceinline__ double pair_weight(long long p, int n) {
    // p is diagonal iff p == i(2n - i + 1)/2 for some i; solve for i
    const double b = 2.0 * n + 1.0;
    int i = (int)floor((b - sqrt(b * b - 8.0 * (double)p)) * 0.5);
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    while (i > 0 && (long long)i * (2 * n - i + 1) / 2 > p) --i;
    while (i < n - 1 && (long long)(i + 1) * (2 * n - i) / 2 <= p) ++i;
    return ((long long)i * (2 * n - i + 1) / 2 == p) ? 1.0 : 2.0;
}

template <typename T>
__global__ void k_box_norms(const T* __restrict__ O, int first_box, int nc, int L, long long P, int nocc,
                            double* __restrict__ nrm) {
    __shared__ double red[256];
    const int box = first_box + blockIdx.x;
    const int l = blockIdx.y;
    double acc = 0.0;
    const T* base = O + (size_t)blockIdx.x * nc * P;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) {
        const double w = pair_weight(p, nocc);
        for (int c = l * l; c < (l + 1) * (l + 1); ++c) {
            const double v = (double)base[(size_t)c * P + p];
            acc += w * v * v;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) nrm[(size_t)box * (L + 1) + l] = sqrt(red[0]);
}

// Edge features (NIN = 16): level/depth, |R|/h, sorted |R_k|/|R| (3), log10 h,
// log10(n_l / h^l) of target (5) and source (5) for l = 0, 2, 4, 6, 8 (clamped
// to the rank of the run).
__global__ void k_edge_features(int nedge, const int* __restrict__ tgt, const int* __restrict__ src,
                                const int* __restrict__ box_key, const int* __restrict__ box_level,
                                const double* __restrict__ hlev, int depth, int L,
                                const double* __restrict__ nrm, float* __restrict__ F) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nedge) return;
    const int t = tgt[e], s = src[e];
    const int lev = box_level[t];
    const double h = hlev[lev];
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = fabs((double)(box_key[3 * t + k] - box_key[3 * s + k]));
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    // sort descending
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2 - a; ++b)
            if (d[b] < d[b + 1]) {
                double x = d[b];
                d[b] = d[b + 1];
                d[b + 1] = x;
            }
    float* f = F + (size_t)e * NIN;
    f[0] = (float)lev / (float)max(depth, 1);
    f[1] = (float)r;
    f[2] = (float)(d[0] / r);
    f[3] = (float)(d[1] / r);
    f[4] = (float)(d[2] / r);
    f[5] = (float)log10(h);
    for (int l = 0; l <= 4; ++l) {
        const int ll = min(2 * l, L);
        const double sc = pow(h, (double)ll);
        f[6 + l] = (float)log10(nrm[(size_t)t * (L + 1) + ll] / sc + 1e-300);
        f[11 + l] = (float)log10(nrm[(size_t)s * (L + 1) + ll] / sc + 1e-300);
    }
}

// ---------------------------------------------------------------------------
// Gram matrices G_e[c][c'] = sum_p O_t[c][p] O_s[c'][p] (FP64 accumulation),
// one block per (edge, 16x16 tile, pair slice).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_edge_gram(const int* __restrict__ tgt, const int* __restrict__ src, const T* __restrict__ O,
                            int first_box, int nc, long long P, int nocc, int ntile, int nslice,
                            double* __restrict__ G) {
    __shared__ double At[16][65], Bs[16][65];
    const int e = blockIdx.x;
    const int tile = blockIdx.y;
    const int ti = tile / ntile, tj = tile % ntile;
    const int slice = blockIdx.z;
    const int c0 = ti * 16, d0 = tj * 16;
    const T* Ot = O + (size_t)(tgt[e] - first_box) * nc * P;
    const T* Os = O + (size_t)(src[e] - first_box) * nc * P;
    const long long per = (P + nslice - 1) / nslice;
    const long long p0 = (long long)slice * per, p1 = min(P, p0 + per);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc = 0.0;
    for (long long pb = p0; pb < p1; pb += 64) {
        for (int x = threadIdx.x; x < 16 * 64; x += blockDim.x) {
            const int r = x / 64, q = x % 64;
            const long long p = pb + q;
            const bool pv = p < p1;
            At[r][q] = (pv && c0 + r < nc) ? pair_weight(p, nocc) * (double)Ot[(size_t)(c0 + r) * P + p] : 0.0;
            Bs[r][q] = (pv && d0 + r < nc) ? (double)Os[(size_t)(d0 + r) * P + p] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 64; ++q) acc += At[ty][q] * Bs[tx][q];
        __syncthreads();
    }
    if (c0 + ty < nc && d0 + tx < nc) atomicAdd(&G[((size_t)e * nc + c0 + ty) * nc + d0 + tx], acc);
}

// e(L') for L' = 0..L from G and the FP64 operator of each edge.
__global__ void k_edge_energy(const double* __restrict__ G, const double* __restrict__ ops,
                              const int* __restrict__ opidx, int nc, int L, double* __restrict__ out) {
    __shared__ double bucket[32];
    const int e = blockIdx.x;
    if (threadIdx.x < 32) bucket[threadIdx.x] = 0.0;
    __syncthreads();
    const double* T = ops + (size_t)opidx[e] * nc * nc;
    const double* g = G + (size_t)e * nc * nc;
    for (int x = threadIdx.x; x < nc * nc; x += blockDim.x) {
        const int c = x / nc, d = x % nc;
        int l = 0;
        while ((l + 1) * (l + 1) <= c) ++l;
        int lp = 0;
        while ((lp + 1) * (lp + 1) <= d) ++lp;
        const double w = (c == l * l) ? 1.0 : (((c - l * l) & 1) ? 2.0 : -2.0);
        atomicAdd(&bucket[max(l, lp)], -w * T[x] * g[x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int k = 0; k <= L; ++k) {
            run += bucket[k];
            out[(size_t)e * (L + 1) + k] = run;
        }
    }
}

// ---------------------------------------------------------------------------
// Rank selection by bisection on the Lagrange multiplier (one block): each
// edge takes the rank L in 2..Lmax that minimises (L+1)^4 + 10^loglam err_L.
// pred[e][k] = log10 err at rank 2+k (k < NOUT); rank Lmax has error 0 when
// Lmax == 2 + NOUT, else its predicted value.
// ---------------------------------------------------------------------------
// The choice for one edge from tabulated values: er[L] = 10^(predicted log10
// error) of rank L (-1 for a prediction that is not finite, which keeps rank
// Lmax), cost[L] = (L+1)^4 and lam = 10^loglam, each computed once.
__device__ __forceinline__ int choose_rank_tab(const double* er, const double* cost, int Lmax, double lam,
                                               double* err_out) {
    int best = Lmax;
    double bestv = 1e300, besterr = 0.0;
    for (int L = 2; L <= Lmax; ++L) {
        const double err = er[L];
        if (err < 0.0) {
            if (err_out) *err_out = 0.0;
            return Lmax;
        }
        const double v = cost[L] + lam * err;
        if (v < bestv) {
            bestv = v;
            best = L;
            besterr = err;
        }
    }
    if (err_out) *err_out = besterr;
    return best;
}

// er[e][L] for every edge, once, on the whole GPU (the bisection below reads
// them 61 times)
__global__ void k_rank_err(const float* __restrict__ pred, int nedge, int Lmax, double* __restrict__ er) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nedge) return;
    double* o = er + (size_t)e * (Lmax + 1);
    for (int L = 2; L <= Lmax; ++L) {
        double v = 0.0;
        if (L - 2 < NOUT) {
            const float y = pred[(size_t)e * NOUT + L - 2];
            v = isfinite(y) ? pow(10.0, (double)y) : -1.0;
        }
        o[L] = v;
    }
}

__global__ void k_select(const double* __restrict__ er, int nedge, int Lmax, double tau, int* __restrict__ ranks) {
    __shared__ double red[1024];
    __shared__ double lo, hi, lam;
    __shared__ double cost[64];
    if (threadIdx.x <= Lmax && threadIdx.x < 64) cost[threadIdx.x] = pow((double)(threadIdx.x + 1), 4.0);
    if (threadIdx.x == 0) {
        lo = -10.0;
        hi = 60.0;
    }
    __syncthreads();
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (threadIdx.x == 0) lam = pow(10.0, mid);
        __syncthreads();
        double s = 0.0;
        for (int e = threadIdx.x; e < nedge; e += blockDim.x) {
            double err;
            choose_rank_tab(er + (size_t)e * (Lmax + 1), cost, Lmax, lam, &err);
            s += err;
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (red[0] <= tau)
                hi = mid;     // feasible: try a smaller multiplier (cheaper)
            else
                lo = mid;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) lam = pow(10.0, hi);
    __syncthreads();
    for (int e = threadIdx.x; e < nedge; e += blockDim.x)
        ranks[e] = choose_rank_tab(er + (size_t)e * (Lmax + 1), cost, Lmax, lam, nullptr);
}

}  // namespace

int mlp_nparams() { return NP; }

cudaError_t mlp_forward_train(const float* prm, const float* norm, const float* X, int n, float* Xn, float* Z1,
                              float* Z2, float* Y, cudaStream_t s) {
    k_mlp_fwd<<<(n + 127) / 128, 128, 0, s>>>(prm, norm, X, n, Xn, Z1, Z2, Y);
    return cudaGetLastError();
}

cudaError_t mlp_backward(const float* prm, const float* Xn, const float* Z1, const float* Z2, const float* Y,
                         const float* T, int n, float* dY, float* dZ1, float* dZ2, float* grad, double* part,
                         int npart, cudaStream_t s) {
    k_mse<<<npart, 256, 0, s>>>(Y, T, n, dY, part);
    k_mlp_dz<<<(n + 127) / 128, 128, 0, s>>>(prm, Z1, Z2, dY, n, dZ1, dZ2);
    k_mlp_wgrad<<<(NP + 127) / 128, 128, 0, s>>>(Xn, Z1, Z2, dZ1, dZ2, dY, n, grad);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* prm, const float* g, float* m, float* v, int t, float lr, cudaStream_t s) {
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    k_adam<<<(NP + 255) / 256, 256, 0, s>>>(prm, g, m, v, NP, lr, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_predict_fp16(const float* prm, __half* prm_h, const float* norm, const float* X, int n,
                             float* Y, cudaStream_t s) {
    k_to_half<<<(NP + 255) / 256, 256, 0, s>>>(prm, prm_h, NP);
    if (n > 0) k_mlp_fwd_h<<<(n + 127) / 128, 128, 0, s>>>(prm_h, norm, X, n, Y);
    return cudaGetLastError();
}

cudaError_t edge_features(bool fp64, const void* O, int first_box, int nbox, int nc, int L, long long P,
                          int nocc, int nedge, const int* tgt, const int* src, const int* box_key, const int* box_level,
                          const double* hlev, int depth, double* nrm, float* F, cudaStream_t s) {
    const int nst = nbox - first_box;
    if (nst <= 0 || nedge == 0) return cudaSuccess;
    dim3 g(nst, L + 1);
    if (fp64)
        k_box_norms<double><<<g, 256, 0, s>>>((const double*)O, first_box, nc, L, P, nocc, nrm);
    else
        k_box_norms<float><<<g, 256, 0, s>>>((const float*)O, first_box, nc, L, P, nocc, nrm);
    k_edge_features<<<(nedge + 127) / 128, 128, 0, s>>>(nedge, tgt, src, box_key, box_level, hlev, depth, L, nrm, F);
    return cudaGetLastError();
}

cudaError_t edge_energies(bool fp64, const void* O, int first_box, int nc, int L, long long P, int nocc,
                          int nedge,
                          const int* tgt, const int* src, const double* ops, const int* opidx, double* G,
                          double* out, cudaStream_t s) {
    if (nedge == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)nedge * nc * nc, s);
    if (e != cudaSuccess) return e;
    const int ntile = (nc + 15) / 16;
    const int nslice = (int)std::min<long long>(64, std::max<long long>(1, P / 4096));
    dim3 g(nedge, ntile * ntile, nslice);
    if (fp64)
        k_edge_gram<double><<<g, 256, 0, s>>>(tgt, src, (const double*)O, first_box, nc, P, nocc, ntile, nslice, G);
    else
        k_edge_gram<float><<<g, 256, 0, s>>>(tgt, src, (const float*)O, first_box, nc, P, nocc, ntile, nslice, G);
    k_edge_energy<<<nedge, 256, 0, s>>>(G, ops, opidx, nc, L, out);
    return cudaGetLastError();
}

cudaError_t select_ranks(const float* pred, int nedge, int Lmax, double tau, int* ranks, double* er,
                         cudaStream_t s) {
    if (nedge == 0) return cudaSuccess;
    if (Lmax >= 64) return cudaErrorInvalidValue;
    k_rank_err<<<(nedge + 255) / 256, 256, 0, s>>>(pred, nedge, Lmax, er);
    k_select<<<1, 1024, 0, s>>>(er, nedge, Lmax, tau, ranks);
    return cudaGetLastError();
}

}  // namespace occk
