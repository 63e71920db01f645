// Step a0 on the device, FP64: scaled solid harmonics, the real-form
// translation operators, and the AO-pair multipole integrals.
//
// Scaled solid harmonics (Sec. I, the definitions after Eq. mmexp), with the
// associated Legendre functions taken WITHOUT the Condon-Shortley phase:
//   O_lm(r) = eps_m r^l/(l+|m|)! P_l|m|(cos t) e^{-i m phi}
//   M_lm(r) = eps_m (l-|m|)!/r^(l+1) P_l|m|(cos t) e^{+i m phi}
// evaluated by recurrences in Cartesian form (m >= 0):
//   O_00 = 1,  O_mm = O_{m-1,m-1} (x - i y)/(2m),
//   (l^2 - m^2) O_lm = (2l-1) z O_{l-1,m} - r^2 O_{l-2,m}
//   M_00 = 1/r, M_mm = (2m-1) (x + i y)/r^2 M_{m-1,m-1},
//   M_lm = [(2l-1) z M_{l-1,m} - ((l-1)^2 - m^2) M_{l-2,m}] / r^2
// and X_{l,-m} = (-1)^m conj(X_lm).
//
// Translation operators (Sec. II, Eqs. fmm1, fmm2, fmm3) act on the real form
// of an expansion (for each l: Re m=0, then Re/Im for m = 1..l); the entries
// for m' < 0 inputs are folded in through the conjugate symmetry of a real
// charge distribution.
//
// AO-pair multipoles (Sec. II, definition after Eq. eri) use the fact that a
// Gaussian exp(-p|r-P|^2) is radially symmetric about P: by the addition
// theorem only the l'=0 term survives, so
//   int exp(-p|r-P|^2) O_lm(r-X) dr = (pi/p)^(3/2) O_lm(P-X).
// Cartesian p factors are written about P, (x_k - A_k) = (x_k - P_k) + PA_k, and
// (x_k - P_k) G = (1/2p) dG/dP_k, so p functions need the gradient of O_lm,
//   d_z O_lm = O_{l-1,m}, d_x O_lm = (O_{l-1,m-1} - O_{l-1,m+1})/2,
//   d_y O_lm = -i (O_{l-1,m-1} + O_{l-1,m+1})/2
// (the linear term of the addition theorem, Eq. fmm1).
#include "occk_internal.h"

namespace occk {

namespace {

struct cplx {
    double r, i;
};

__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return {a.r * s, a.i * s}; }
// -i/2 * a
__device__ __forceinline__ cplx cmi_half(cplx a) { return {0.5 * a.i, -0.5 * a.r}; }

__host__ __device__ __forceinline__ int tri(int l, int m) { return l * (l + 1) / 2 + m; }

__device__ void regular_table(double x, double y, double z, int L, cplx* O) {
    const double r2 = x * x + y * y + z * z;
    O[0] = {1.0, 0.0};
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            cplx p = O[tri(m - 1, m - 1)];
            double inv = 1.0 / (2.0 * m);
            O[tri(m, m)] = {(p.r * x + p.i * y) * inv, (p.i * x - p.r * y) * inv};
        }
        if (m + 1 <= L) {
            cplx p = O[tri(m, m)];
            O[tri(m + 1, m)] = {z * p.r, z * p.i};
        }
        for (int l = m + 2; l <= L; ++l) {
            double inv = 1.0 / (double)(l * l - m * m);
            cplx a = O[tri(l - 1, m)], b = O[tri(l - 2, m)];
            O[tri(l, m)] = {((2 * l - 1) * z * a.r - r2 * b.r) * inv,
                            ((2 * l - 1) * z * a.i - r2 * b.i) * inv};
        }
    }
}

__device__ void irregular_table(double x, double y, double z, int L, cplx* M) {
    const double r2 = x * x + y * y + z * z;
    const double ir2 = 1.0 / r2;
    M[0] = {1.0 / sqrt(r2), 0.0};
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            cplx p = M[tri(m - 1, m - 1)];
            double f = (2.0 * m - 1.0) * ir2;
            M[tri(m, m)] = {(p.r * x - p.i * y) * f, (p.r * y + p.i * x) * f};
        }
        if (m + 1 <= L) {
            cplx p = M[tri(m, m)];
            double f = (2.0 * m + 1.0) * z * ir2;
            M[tri(m + 1, m)] = {p.r * f, p.i * f};
        }
        for (int l = m + 2; l <= L; ++l) {
            cplx a = M[tri(l - 1, m)], b = M[tri(l - 2, m)];
            double ca = (2 * l - 1) * z, cb = (double)((l - 1) * (l - 1) - m * m);
            M[tri(l, m)] = {(ca * a.r - cb * b.r) * ir2, (ca * a.i - cb * b.i) * ir2};
        }
    }
}

// X_{l,m} for any m from the m >= 0 table; zero outside 0 <= |m| <= l <= Lt.
__device__ __forceinline__ cplx fetch(const cplx* H, int l, int m, int Lt) {
    if (l < 0 || l > Lt) return {0.0, 0.0};
    int am = m < 0 ? -m : m;
    if (am > l) return {0.0, 0.0};
    cplx v = H[tri(l, am)];
    if (m < 0) {
        double s = (am & 1) ? -1.0 : 1.0;
        return {s * v.r, -s * v.i};
    }
    return v;
}

// real-form index -> (l, m, part) with part 0 = Re, 1 = Im
__device__ __forceinline__ void decode(int idx, int& l, int& m, int& part) {
    int ll = (int)floor(sqrt((double)idx) + 1e-9);
    while (ll * ll > idx) --ll;
    while ((ll + 1) * (ll + 1) <= idx) ++ll;
    int r = idx - ll * ll;
    l = ll;
    if (r == 0) {
        m = 0;
        part = 0;
    } else {
        m = (r + 1) / 2;
        part = (r & 1) ? 0 : 1;
    }
}

// Complex coefficient of input (lp, mp) in output (l, m) for each operator.
__device__ __forceinline__ cplx op_coef(int kind, const cplx* H, int Lt, int l, int m, int lp, int mp) {
    if (kind == 0) {          // M2M, Eq. fmm1: O_{l-l', m-m'}(Xc - Xp)
        if (lp > l) return {0.0, 0.0};
        return fetch(H, l - lp, m - mp, Lt);
    } else if (kind == 1) {   // L2L, Eq. fmm3: O_{l'-l, m'-m}(Xc - Xp)
        if (lp < l) return {0.0, 0.0};
        return fetch(H, lp - l, mp - m, Lt);
    } else {                  // M2L, Eq. fmm2: (-1)^l M_{l+l', m+m'}(X - X')
        cplx v = fetch(H, l + lp, m + mp, Lt);
        return (l & 1) ? cplx{-v.r, -v.i} : v;
    }
}

__global__ void k_gen_ops(const OpDesc* desc, int L, double* out, float* out_f) {
    extern __shared__ cplx H[];
    const OpDesc d = desc[blockIdx.x];
    const int Lt = d.kind == 2 ? 2 * L : L;
    if (threadIdx.x == 0) {
        if (d.kind == 2)
            irregular_table(d.d[0], d.d[1], d.d[2], Lt, H);
        else
            regular_table(d.d[0], d.d[1], d.d[2], Lt, H);
    }
    __syncthreads();
    const int nc = (L + 1) * (L + 1);
    const size_t base = (size_t)blockIdx.x * nc * nc;
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
        int a = e / nc, b = e - a * nc;
        int l, m, pa, lp, k, pb;
        decode(a, l, m, pa);
        decode(b, lp, k, pb);
        cplx gp = op_coef(d.kind, H, Lt, l, m, lp, k);
        double v;
        if (k == 0) {
            v = pa == 0 ? gp.r : gp.i;
        } else {
            cplx gm = op_coef(d.kind, H, Lt, l, m, lp, -k);
            double s = (k & 1) ? -1.0 : 1.0;
            if (pa == 0 && pb == 0) v = gp.r + s * gm.r;
            else if (pa == 0) v = -gp.i + s * gm.i;
            else if (pb == 0) v = gp.i + s * gm.i;
            else v = gp.r - s * gm.r;
        }
        out[base + e] = v;
        out_f[base + e] = (float)v;
    }
}

// Gradient of O_lm: D_k[O](l, m), k = 0 (x), 1 (y), 2 (z).
__device__ __forceinline__ cplx dO(const cplx* O, int L, int k, int l, int m) {
    if (k == 2) return fetch(O, l - 1, m, L);
    cplx a = fetch(O, l - 1, m - 1, L), b = fetch(O, l - 1, m + 1, L);
    if (k == 0) return cscale(csub(a, b), 0.5);
    return cmi_half(cadd(a, b));
}

// Second derivative d_k d_q O_lm = D_k[D_q[O]](l, m).
__device__ __forceinline__ cplx d2O(const cplx* O, int L, int k, int q, int l, int m) {
    if (k == 2) return dO(O, L, q, l - 1, m);
    cplx a = dO(O, L, q, l - 1, m - 1), b = dO(O, L, q, l - 1, m + 1);
    if (k == 0) return cscale(csub(a, b), 0.5);
    return cmi_half(cadd(a, b));
}

constexpr int kMaxL = 12;
constexpr int kMaxTab = (kMaxL + 1) * (kMaxL + 2) / 2;
constexpr int kMaxNc = (kMaxL + 1) * (kMaxL + 1);

// One thread per (shell pair, AO component pair).
__global__ void k_pair_multipoles(const PairDesc* pairs, int npair, const double* pexp,
                                  const double* pcoef, int L, double* vals, float* vals_f) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ip = (int)(tid / 9);
    const int comp = (int)(tid - (long long)ip * 9);
    if (ip >= npair) return;
    const PairDesc pd = pairs[ip];
    const int na = pd.la ? 3 : 1, nb = pd.lb ? 3 : 1;
    if (comp >= na * nb) return;
    const int ia = comp / nb, ib = comp - ia * nb;
    const int nc = (L + 1) * (L + 1);
    cplx O[kMaxTab];
    double acc[kMaxNc];
    for (int c = 0; c < nc; ++c) acc[c] = 0.0;
    const double ABx = pd.A[0] - pd.B[0], ABy = pd.A[1] - pd.B[1], ABz = pd.A[2] - pd.B[2];
    const double AB2 = ABx * ABx + ABy * ABy + ABz * ABz;
    for (int p = 0; p < pd.nprim_a; ++p) {
        const double ea = pexp[pd.prim_a + p], da = pcoef[pd.prim_a + p];
        for (int q = 0; q < pd.nprim_b; ++q) {
            const double eb = pexp[pd.prim_b + q], db = pcoef[pd.prim_b + q];
            const double pp = ea + eb;
            const double ipp = 1.0 / pp;
            double P[3], PA[3], PB[3];
            for (int k = 0; k < 3; ++k) {
                P[k] = (ea * pd.A[k] + eb * pd.B[k]) * ipp;
                PA[k] = P[k] - pd.A[k];
                PB[k] = P[k] - pd.B[k];
            }
            const double pref = da * db * exp(-ea * eb * ipp * AB2) * pow(M_PI * ipp, 1.5);
            regular_table(P[0] - pd.X[0], P[1] - pd.X[1], P[2] - pd.X[2], L, O);
            const double h1 = 0.5 * ipp, h2 = 0.25 * ipp * ipp;
            for (int l = 0; l <= L; ++l) {
                for (int m = 0; m <= l; ++m) {
                    cplx o = O[tri(l, m)];
                    cplx v;
                    if (!pd.la && !pd.lb) {
                        v = o;
                    } else if (pd.la && !pd.lb) {
                        v = cadd(cscale(dO(O, L, ia, l, m), h1), cscale(o, PA[ia]));
                    } else if (!pd.la && pd.lb) {
                        v = cadd(cscale(dO(O, L, ib, l, m), h1), cscale(o, PB[ib]));
                    } else {
                        cplx t2 = d2O(O, L, ia, ib, l, m);
                        if (ia == ib) t2 = cadd(t2, cscale(o, 2.0 * pp));
                        v = cscale(t2, h2);
                        v = cadd(v, cscale(dO(O, L, ia, l, m), PB[ib] * h1));
                        v = cadd(v, cscale(dO(O, L, ib, l, m), PA[ia] * h1));
                        v = cadd(v, cscale(o, PA[ia] * PB[ib]));
                    }
                    if (m == 0) {
                        acc[l * l] += pref * v.r;
                    } else {
                        acc[l * l + 2 * m - 1] += pref * v.r;
                        acc[l * l + 2 * m] += pref * v.i;
                    }
                }
            }
        }
    }
    const size_t row = (size_t)(pd.val_off + comp);
    for (int c = 0; c < nc; ++c) {
        vals[row * nc + c] = acc[c];
        vals_f[row * nc + c] = (float)acc[c];
    }
}

}  // namespace

cudaError_t launch_gen_ops(const OpDesc* d_desc, int nops, int L, double* d_out, float* d_out_f,
                           cudaStream_t s) {
    if (nops <= 0) return cudaSuccess;
    const int Lt = 2 * L;
    size_t shm = sizeof(cplx) * (size_t)(Lt + 1) * (Lt + 2) / 2;
    k_gen_ops<<<nops, 256, shm, s>>>(d_desc, L, d_out, d_out_f);
    return cudaGetLastError();
}

cudaError_t launch_pair_multipoles(const PairDesc* d_pairs, int npair, const double* d_exp,
                                   const double* d_coef, int L, double* d_vals, float* d_vals_f,
                                   int nvals, cudaStream_t s) {
    (void)nvals;
    if (L > kMaxL) return cudaErrorInvalidValue;
    long long nthreads = (long long)npair * 9;
    int bs = 128;
    long long nb = (nthreads + bs - 1) / bs;
    if (nb <= 0) return cudaSuccess;
    k_pair_multipoles<<<(unsigned)nb, bs, 0, s>>>(d_pairs, npair, d_exp, d_coef, L, d_vals, d_vals_f);
    return cudaGetLastError();
}

}  // namespace occk
