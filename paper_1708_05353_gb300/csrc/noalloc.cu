// Exchange energy from caller-owned K and C with no device allocation.
//
// The regular path (occk_farfield_K) reduces E = -1/2 sum_ri C_ri K_ri through
// per-block partial sums held in a context workspace obtained with
// cudaMalloc.  Some callers cannot let a library allocate device memory: an
// application whose own allocator owns all device memory (a framework caching
// allocator or a fixed memory pool), or a latency-sensitive loop in which a
// cudaMalloc would synchronise the device.  This file gives them the same
// reduction with its scratch in a statically sized __device__ array, which
// every GPU that loads the library holds until the process exits.
#include <mutex>

#include "occk_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// One partial sum per occupied column.  Shared by every call on a device and
// never cleared between calls: each call overwrites the first nocc entries
// before reading them, and calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_col_energy[OCCK_NOALLOC_MAX_OCC];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Column sums: col[i] = sum_r C_ri K_ri, one block per column, fixed order.
__global__ void k_col_energy(const double* __restrict__ C, int ldc, const double* __restrict__ K, int ldk,
                             int nao, int nocc, double* __restrict__ col) {
    __shared__ double red[256];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < nao; r += blockDim.x)
        s += C[(size_t)i * ldc + r] * K[(size_t)i * ldk + r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) col[i] = red[0];
}

__global__ void k_sum_cols(const double* __restrict__ col, int nocc, double* __restrict__ E) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nocc; i += blockDim.x) s += col[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = -0.5 * red[0];
}

}  // namespace

extern "C" occk_status occk_exchange_energy_noalloc(occk_ctx* ctx, int nao, int nocc, const double* C_dev,
                                                    int ldc, const double* K_dev, int ldk, double* E_dev,
                                                    void* stream) {
    if (!ctx) return OCCK_ERR_ARG;
    if (ctx->device < 0 || ctx->device >= kMaxDevices) {
        ctx->err = "occk_exchange_energy_noalloc: context has no usable device";
        return OCCK_ERR_UNSUPPORTED;
    }
    if (!C_dev || !K_dev || !E_dev || nao <= 0 || nocc <= 0) {
        ctx->err = "occk_exchange_energy_noalloc: null buffer or non-positive size";
        return OCCK_ERR_ARG;
    }
    if (ldc < nao || ldk < nao) {
        ctx->err = "occk_exchange_energy_noalloc: ldc/ldk < nao";
        return OCCK_ERR_SHAPE;
    }
    if (nocc > OCCK_NOALLOC_MAX_OCC) {
        ctx->err = "occk_exchange_energy_noalloc: nocc exceeds OCCK_NOALLOC_MAX_OCC (" +
                   std::to_string(OCCK_NOALLOC_MAX_OCC) + "); use occk_farfield_K's energy instead";
        return OCCK_ERR_SHAPE;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        ctx->err = std::string("occk_exchange_energy_noalloc: cudaSetDevice: ") + cudaGetErrorString(e);
        return OCCK_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Device address of the static array (the host-side symbol is only a
    // stand-in, not a device address).  Outside stream capture it is looked up
    // on every call, with this device current, so a device reset or a new
    // primary context never leaves a stale address behind; during capture the
    // address of the last uncaptured call on this device is used, so the first
    // call on a device must come before any capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) {
        ctx->err = std::string("occk_exchange_energy_noalloc: cudaStreamIsCapturing: ") + cudaGetErrorString(e);
        return OCCK_ERR_CUDA;
    }
    double* col = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_col_energy);
            if (e != cudaSuccess) {
                ctx->err = std::string("occk_exchange_energy_noalloc: cudaGetSymbolAddress: ") +
                           cudaGetErrorString(e);
                return OCCK_ERR_CUDA;
            }
            g_addr[ctx->device] = static_cast<double*>(p);
        } else if (!g_addr[ctx->device]) {
            ctx->err = "occk_exchange_energy_noalloc: first call on this device made during stream capture; "
                       "call it once outside capture first";
            return OCCK_ERR_STATE;
        }
        col = g_addr[ctx->device];
    }
    k_col_energy<<<nocc, 256, 0, s>>>(C_dev, ldc, K_dev, ldk, nao, nocc, col);
    k_sum_cols<<<1, 256, 0, s>>>(col, nocc, E_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("occk_exchange_energy_noalloc: launch: ") + cudaGetErrorString(e);
        return OCCK_ERR_CUDA;
    }
    return OCCK_OK;
}
