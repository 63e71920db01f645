// Batched far-field exchange: many systems of uneven size in one launch
// sequence.
//
// A batch plan turns every step of every system into work items (system,
// block coordinates).  One persistent kernel per step -- per tree level for the
// dependent M2M and L2L passes -- sweeps the items of all systems with a
// static stride (no queue, no spin-wait), so a batch of 20 systems costs the
// launches of one deep tree, and the whole sequence is captured once into a
// CUDA graph and replayed.  The tile shapes (components per translation block,
// SIMT GEMM tile, persistent blocks per SM) come from a small autotuner that
// times the candidates on the batch itself and caches the winner in a text
// file keyed by GPU, rank, precision and batch shape.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "fmm_bodies.cuh"
#include "occk_internal.h"

namespace occk {

struct SysDesc {
    int nao, nocc, ldc, ldk, nc, L, depth, nbox, first_box, nleaf, leaf0, nrow, max_rows;
    long long P;
    const double* C;
    double* K;
    const int *row_ptr, *ent_col, *ent_val, *leaf_rowoff, *leaf_aos, *ao_row_ptr, *ao_rows;
    const int *child_ptr, *child_list, *m2m_op, *l2l_op, *parent, *m2l_ptr, *m2l_src, *m2l_op;
    const void* vals;
    const void* ops;
    void *ct, *w, *obox, *mbox;
    double *kb, *part;
};

struct Item {
    int sys, a, b, c;
};

struct TItem {   // translation item
    int sys, mode, tgt, pblk, chunk, acc;
};

namespace {

constexpr int kRedBlocks = 64;   // reduction blocks per system

// ---- persistent kernels: one block sweeps items blockIdx.x, +gridDim.x, ... ----
template <typename T>
__global__ void kb_transpose(const SysDesc* __restrict__ S, const Item* __restrict__ it, int n) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Item w = it[k];
        const SysDesc& s = S[w.sys];
        body::transpose_body<T>(w.a, w.b, 0, s.C, s.ldc, s.nao, s.nocc, (T*)s.ct);
        __syncthreads();
    }
}

template <typename T, int LMC>
__global__ void kb_half(const SysDesc* __restrict__ S, const Item* __restrict__ it, int n) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Item w = it[k];
        const SysDesc& s = S[w.sys];
        body::half_body<T, LMC>(w.a, w.b, 0, s.row_ptr, s.ent_col, s.ent_val, (const T*)s.vals, s.nc,
                                (const T*)s.ct, s.nocc, s.nrow, (T*)s.w);
    }
}

template <typename T, int BM, int BK, int TM>
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
kb_full(const SysDesc* __restrict__ S, const Item* __restrict__ it, int n) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Item w = it[k];
        const SysDesc& s = S[w.sys];
        const int ntile = (s.nocc + BM - 1) / BM;
        body::full_body<T, BM, BK, TM>(w.a, w.b, 0, s.leaf_rowoff, s.leaf_aos, (const T*)s.ct, (const T*)s.w,
                                       s.nocc, s.nrow, s.nc, ntile, (T*)s.obox, s.leaf0 - s.first_box);
    }
}

template <typename T, int LMC>
__global__ void __launch_bounds__(128) kb_translate(const SysDesc* __restrict__ S, const TItem* __restrict__ it, int n) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const TItem w = it[k];
        const SysDesc& s = S[w.sys];
        const bool m2m = w.mode == 0, m2l = w.mode == 1;
        const int* ptr = m2m ? s.child_ptr : (m2l ? s.m2l_ptr : nullptr);
        const int* list = m2m ? s.child_list : (m2l ? s.m2l_src : nullptr);
        const int* opidx = m2m ? s.m2m_op : (m2l ? s.m2l_op : s.l2l_op);
        const T* in = (const T*)(w.mode == 2 ? s.mbox : s.obox);
        T* out = (T*)(w.mode == 0 ? s.obox : s.mbox);
        body::translate_body<T, LMC>(w.pblk, 0, w.chunk, w.mode, (int)s.P, s.nc, s.L, s.first_box, w.tgt, ptr, list,
                                     opidx, nullptr, s.parent, (const T*)s.ops, in, out, w.acc);
    }
}

template <typename T, int BM, int BK, int TM>
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
kb_l2p(const SysDesc* __restrict__ S, const Item* __restrict__ it, int n) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Item w = it[k];
        const SysDesc& s = S[w.sys];
        body::l2p_body<T, BM, BK, TM>(w.a, w.b, w.c, s.leaf_rowoff, (const T*)s.w, (const T*)s.mbox, s.nocc, s.nrow,
                                      s.nc, s.leaf0 - s.first_box, s.kb);
        __syncthreads();
    }
}

__global__ void kb_reduce(const SysDesc* __restrict__ S, const Item* __restrict__ it, int n) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Item w = it[k];
        const SysDesc& s = S[w.sys];
        body::reduce_body(w.a, 0, kRedBlocks, s.ao_row_ptr, s.ao_rows, s.kb, s.nao, s.nocc, s.C, s.ldc, s.K, s.ldk,
                          s.part);
        __syncthreads();
    }
}

__global__ void kb_energy(const SysDesc* __restrict__ S, const int* __restrict__ sys, int n, double* __restrict__ E) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const SysDesc& s = S[sys[k]];
        __shared__ double red[256];
        double acc = 0.0;
        for (int x = threadIdx.x; x < kRedBlocks; x += blockDim.x) acc += s.part[x];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) E[sys[k]] = -0.5 * red[0];
        __syncthreads();
    }
}

template <typename V>
cudaError_t up(V** dst, const std::vector<V>& v) {
    *dst = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dst, sizeof(V) * v.size());
    if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

int translate_chunk_batch(int nc);

}  // namespace occk

using occk::Item;
using occk::SysDesc;
using occk::TItem;

extern "C" void occk_batch_destroy(occk_batch* b);

// mode 0: level-synchronous persistent kernels over all systems' work items;
// mode 1: each system's own pipeline (the single-system kernels) on one of
// several forked streams, joined at the end (a fork-join graph when captured)
struct BatchCfg {
    int lmc = 9, bps = 8, tile = 128, mode = 0;
};

struct occk_batch {
    occk_ctx* ctx = nullptr;
    int nsys = 0, prec = 0, L = 0, maxD = 0;
    std::vector<const occk_tree*> trees;
    std::vector<int> nocc;
    std::vector<SysDesc> h_sys;
    SysDesc* d_sys = nullptr;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    double* E = nullptr;
    // items per stage
    Item *it_tr = nullptr, *it_half = nullptr, *it_full64 = nullptr, *it_full128 = nullptr, *it_l2p64 = nullptr,
         *it_l2p128 = nullptr, *it_red = nullptr;
    int n_tr = 0, n_half = 0, n_full64 = 0, n_full128 = 0, n_l2p64 = 0, n_l2p128 = 0, n_red = 0;
    std::vector<int> lmc_of_items;  // lmc used to build translate items
    std::vector<TItem*> it_m2m, it_l2l;
    std::vector<int> n_m2m, n_l2l;
    TItem* it_m2l = nullptr;
    int n_m2l = 0;
    int* en_sys = nullptr;
    int n_en = 0;
    std::vector<int> zero_sys;   // systems without a far field
    int half_lmc = 16;
    BatchCfg cfg;
    int built_lmc = -1;
    // graph
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_valid = false;
    int sm_count = 0;
    // mode 1: per-system pipelines on forked streams, largest system first
    std::vector<occk::FmmArgs> fargs;
    std::vector<int> order;
    std::vector<cudaStream_t> fs;
    std::vector<cudaEvent_t> fev;
    cudaEvent_t ev_fork = nullptr;
    int* err = nullptr;
};

namespace {

occk_status bfail(occk_ctx* ctx, occk_status code, const std::string& m) {
    if (ctx) ctx->err = m;
    return code;
}

void free_items(occk_batch* b) {
    for (auto p : b->it_m2m) cudaFree(p);
    for (auto p : b->it_l2l) cudaFree(p);
    b->it_m2m.clear();
    b->it_l2l.clear();
    b->n_m2m.clear();
    b->n_l2l.clear();
    if (b->it_m2l) cudaFree(b->it_m2l);
    b->it_m2l = nullptr;
}

// Translation items for chunk width lmc.
cudaError_t build_translate_items(occk_batch* b, int lmc) {
    free_items(b);
    const int ppt = b->prec == OCCK_FP64 ? occk::body::translate_ppt<double>() : occk::body::translate_ppt<float>();
    cudaError_t e = cudaSuccess;
    const int steps = std::max(b->maxD - 2, 0);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        std::vector<TItem> m2m, l2l;
        for (int s = 0; s < b->nsys; ++s) {
            const occk_tree* t = b->trees[s];
            const SysDesc& sd = b->h_sys[s];
            if (sd.depth < 3) continue;
            const int nch = (sd.nc + lmc - 1) / lmc;
            const int pb = (int)((sd.P + 128 * ppt - 1) / (128 * ppt));
            // pair block outermost: consecutive items share source pairs (L2 reuse)
            const int child = sd.depth - k;          // M2M: children at this level
            if (child >= 3) {
                for (int p = 0; p < pb; ++p)
                    for (int tg = t->level_off[child - 1]; tg < t->level_off[child]; ++tg)
                        for (int c = 0; c < nch; ++c) m2m.push_back(TItem{s, 0, tg, p, c, 0});
            }
            const int lev = 3 + k;                   // L2L: children at this level
            if (lev <= sd.depth) {
                for (int p = 0; p < pb; ++p)
                    for (int tg = t->level_off[lev]; tg < t->level_off[lev + 1]; ++tg)
                        for (int c = 0; c < nch; ++c) l2l.push_back(TItem{s, 2, tg, p, c, 1});
            }
        }
        TItem *dm = nullptr, *dl = nullptr;
        e = occk::up(&dm, m2m);
        if (e == cudaSuccess) e = occk::up(&dl, l2l);
        b->it_m2m.push_back(dm);
        b->it_l2l.push_back(dl);
        b->n_m2m.push_back((int)m2m.size());
        b->n_l2l.push_back((int)l2l.size());
    }
    std::vector<TItem> m2l;
    for (int s = 0; s < b->nsys; ++s) {
        const occk_tree* t = b->trees[s];
        const SysDesc& sd = b->h_sys[s];
        if (sd.depth < 2) continue;
        const int nch = (sd.nc + lmc - 1) / lmc;
        const int pb = (int)((sd.P + 128 * ppt - 1) / (128 * ppt));
        for (int p = 0; p < pb; ++p)
            for (int tg = t->level_off[2]; tg < sd.nbox; ++tg)
                for (int c = 0; c < nch; ++c) m2l.push_back(TItem{s, 1, tg, p, c, 0});
    }
    if (e == cudaSuccess) e = occk::up(&b->it_m2l, m2l);
    b->n_m2l = (int)m2l.size();
    b->built_lmc = lmc;
    return e;
}

template <typename T, typename... A>
void launch_kb_translate(int lmc, int grid, cudaStream_t s, A... args) {
    switch (lmc) {
        case 4: occk::kb_translate<T, 4><<<grid, 128, 0, s>>>(args...); break;
        case 9: occk::kb_translate<T, 9><<<grid, 128, 0, s>>>(args...); break;
        case 16: occk::kb_translate<T, 16><<<grid, 128, 0, s>>>(args...); break;
        case 21: occk::kb_translate<T, 21><<<grid, 128, 0, s>>>(args...); break;
        default: occk::kb_translate<T, 25><<<grid, 128, 0, s>>>(args...); break;
    }
}

template <typename T>
cudaError_t enqueue_typed(occk_batch* b, cudaStream_t s) {
    const BatchCfg& c = b->cfg;
    const int cap = std::max(1, b->sm_count * c.bps);
    auto grid = [&](int n) { return std::max(1, std::min(n, cap)); };
    for (int sys : b->zero_sys) {
        const SysDesc& sd = b->h_sys[sys];
        cudaMemsetAsync(sd.K, 0, sizeof(double) * (size_t)sd.ldk * sd.nocc, s);
        cudaMemsetAsync(b->E + sys, 0, sizeof(double), s);
    }
    if (b->n_tr) occk::kb_transpose<T><<<grid(b->n_tr), dim3(32, 8), 0, s>>>(b->d_sys, b->it_tr, b->n_tr);
    if (b->n_half) {
        switch (b->half_lmc) {
            case 4: occk::kb_half<T, 4><<<grid(b->n_half), 128, 0, s>>>(b->d_sys, b->it_half, b->n_half); break;
            case 9: occk::kb_half<T, 9><<<grid(b->n_half), 128, 0, s>>>(b->d_sys, b->it_half, b->n_half); break;
            default: occk::kb_half<T, 16><<<grid(b->n_half), 128, 0, s>>>(b->d_sys, b->it_half, b->n_half); break;
        }
    }
    if constexpr (sizeof(T) == 8) {
        if (b->n_full64) occk::kb_full<T, 64, 8, 4><<<grid(b->n_full64), 256, 0, s>>>(b->d_sys, b->it_full64, b->n_full64);
    } else {
        if (c.tile == 128) {
            if (b->n_full128)
                occk::kb_full<T, 128, 8, 8><<<grid(b->n_full128), 256, 0, s>>>(b->d_sys, b->it_full128, b->n_full128);
        } else if (b->n_full64) {
            occk::kb_full<T, 64, 8, 4><<<grid(b->n_full64), 256, 0, s>>>(b->d_sys, b->it_full64, b->n_full64);
        }
    }
    for (size_t k = 0; k < b->it_m2m.size(); ++k)
        if (b->n_m2m[k]) launch_kb_translate<T>(c.lmc, grid(b->n_m2m[k]), s, b->d_sys, b->it_m2m[k], b->n_m2m[k]);
    if (b->n_m2l) launch_kb_translate<T>(c.lmc, grid(b->n_m2l), s, b->d_sys, b->it_m2l, b->n_m2l);
    for (size_t k = 0; k < b->it_l2l.size(); ++k)
        if (b->n_l2l[k]) launch_kb_translate<T>(c.lmc, grid(b->n_l2l[k]), s, b->d_sys, b->it_l2l[k], b->n_l2l[k]);
    if constexpr (sizeof(T) == 8) {
        if (b->n_l2p64) occk::kb_l2p<T, 64, 8, 4><<<grid(b->n_l2p64), 256, 0, s>>>(b->d_sys, b->it_l2p64, b->n_l2p64);
    } else {
        if (c.tile == 128) {
            if (b->n_l2p128)
                occk::kb_l2p<T, 128, 8, 8><<<grid(b->n_l2p128), 256, 0, s>>>(b->d_sys, b->it_l2p128, b->n_l2p128);
        } else if (b->n_l2p64) {
            occk::kb_l2p<T, 64, 8, 4><<<grid(b->n_l2p64), 256, 0, s>>>(b->d_sys, b->it_l2p64, b->n_l2p64);
        }
    }
    if (b->n_red) occk::kb_reduce<<<grid(b->n_red), 256, 0, s>>>(b->d_sys, b->it_red, b->n_red);
    if (b->n_en) occk::kb_energy<<<grid(b->n_en), 256, 0, s>>>(b->d_sys, b->en_sys, b->n_en, b->E);
    return cudaGetLastError();
}

cudaError_t enqueue_streams(occk_batch* b, cudaStream_t s) {
    const int ns = (int)b->fs.size();
    cudaError_t e = cudaEventRecord(b->ev_fork, s);
    for (int j = 0; j < ns && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(b->fs[j], b->ev_fork, 0);
    for (size_t k = 0; k < b->order.size() && e == cudaSuccess; ++k) {
        const int sys = b->order[k];
        e = occk::run_farfield(b->fargs[sys], b->fs[k % ns]);
    }
    for (int j = 0; j < ns && e == cudaSuccess; ++j) {
        e = cudaEventRecord(b->fev[j], b->fs[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->fev[j], 0);
    }
    return e;
}

cudaError_t enqueue(occk_batch* b, cudaStream_t s) {
    if (b->cfg.mode == 1) return enqueue_streams(b, s);
    if (b->built_lmc != b->cfg.lmc) {
        cudaError_t e = build_translate_items(b, b->cfg.lmc);
        if (e != cudaSuccess) return e;
    }
    return b->prec == OCCK_FP64 ? enqueue_typed<double>(b, s) : enqueue_typed<float>(b, s);
}

std::string cfg_key(occk_batch* b) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, b->ctx->device);
    long long sumP = 0;
    for (auto& s : b->h_sys) sumP += s.P;
    int bucket = 0;
    while ((1LL << bucket) < sumP) ++bucket;
    std::ostringstream k;
    std::string name(prop.name);
    for (auto& ch : name)
        if (ch == ' ') ch = '_';
    k << name << "|L" << b->L << "|prec" << b->prec << "|nsys" << b->nsys << "|P2^" << bucket << "|D" << b->maxD;
    return k.str();
}

}  // namespace

// ===========================================================================
// ABI
// ===========================================================================

extern "C" occk_status occk_batch_create(occk_ctx* ctx, int nsys, occk_tree* const* trees, const int* nocc,
                                         int prec, occk_batch** out) {
    if (!ctx || !trees || !nocc || !out || nsys <= 0) return bfail(ctx, OCCK_ERR_ARG, "bad argument");
    *out = nullptr;
    if (ctx->device < 0) return bfail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    if (prec != OCCK_FP64 && prec != OCCK_FP32)
        return bfail(ctx, OCCK_ERR_UNSUPPORTED, "batches run in OCCK_FP64 or OCCK_FP32");
    const int L = trees[0] ? trees[0]->lmax : -1;
    for (int s = 0; s < nsys; ++s) {
        if (!trees[s] || trees[s]->device != ctx->device) return bfail(ctx, OCCK_ERR_ARG, "tree on another device");
        if (trees[s]->lmax < 0) return bfail(ctx, OCCK_ERR_STATE, "call occk_pair_multipoles on every tree");
        if (trees[s]->lmax != L) return bfail(ctx, OCCK_ERR_SHAPE, "all trees of a batch need the same lmax");
        if (nocc[s] <= 0) return bfail(ctx, OCCK_ERR_ARG, "nocc must be positive");
    }
    cudaSetDevice(ctx->device);
    occk_batch* b = new occk_batch();
    b->ctx = ctx;
    b->nsys = nsys;
    b->prec = prec;
    b->L = L;
    b->sm_count = ctx->sm_count;
    b->trees.assign(trees, trees + nsys);
    b->nocc.assign(nocc, nocc + nsys);
    const size_t es = prec == OCCK_FP64 ? 8 : 4;
    const int nc = occk::ncomp(L);
    // ---- arena layout
    std::vector<size_t> off;
    size_t tot = 0;
    auto take = [&](size_t bytes) {
        size_t o = (tot + 255) & ~(size_t)255;
        tot = o + bytes;
        return o;
    };
    struct Offs {
        size_t C, K, ct, w, obox, mbox, kb, part;
    };
    std::vector<Offs> o(nsys);
    for (int s = 0; s < nsys; ++s) {
        const occk_tree* t = trees[s];
        const int nbox = (int)t->parent.size();
        const int first = t->depth >= 2 ? t->level_off[2] : nbox;
        const size_t P = (size_t)nocc[s] * (nocc[s] + 1) / 2;   // stored pairs i <= j
        const size_t nrow = t->leaf_aos.size();
        o[s].C = take(8 * (size_t)t->nao * nocc[s]);
        o[s].K = take(8 * (size_t)t->nao * nocc[s]);
        o[s].ct = take(es * (size_t)t->nao * nocc[s]);
        o[s].w = take(es * (size_t)nc * nrow * nocc[s]);
        o[s].obox = take(es * (size_t)(nbox - first) * nc * P + 8);
        o[s].mbox = take(es * (size_t)(nbox - first) * nc * P + 8);
        o[s].kb = take(8 * nrow * nocc[s]);
        // room for the persistent reduction's partials and for those of the
        // single-system pipeline (mode 1)
        o[s].part = take(8 * (size_t)std::max(occk::kRedBlocks, occk::kFarfieldPartials));
    }
    size_t eoff = take(8 * (size_t)nsys);
    cudaError_t e = cudaMalloc(&b->arena, tot);
    if (e != cudaSuccess) {
        delete b;
        return bfail(ctx, OCCK_ERR_OOM, "batch arena");
    }
    b->arena_bytes = tot;
    char* base = (char*)b->arena;
    b->E = (double*)(base + eoff);
    for (int s = 0; s < nsys; ++s) {
        const occk_tree* t = trees[s];
        SysDesc d{};
        d.nao = t->nao;
        d.nocc = nocc[s];
        d.ldc = t->nao;
        d.ldk = t->nao;
        d.nc = nc;
        d.L = L;
        d.depth = t->depth;
        d.nbox = (int)t->parent.size();
        d.first_box = t->depth >= 2 ? t->level_off[2] : d.nbox;
        d.nleaf = (int)t->leaf_rowoff.size() - 1;
        d.leaf0 = t->level_off[t->depth];
        d.nrow = (int)t->leaf_aos.size();
        int mr = 0;
        for (int B = 0; B < d.nleaf; ++B) mr = std::max(mr, t->leaf_rowoff[B + 1] - t->leaf_rowoff[B]);
        d.max_rows = mr;
        d.P = (long long)nocc[s] * (nocc[s] + 1) / 2;
        d.C = (const double*)(base + o[s].C);
        d.K = (double*)(base + o[s].K);
        auto& td = t->dev;
        d.row_ptr = td.row_ptr; d.ent_col = td.ent_col; d.ent_val = td.ent_val;
        d.leaf_rowoff = td.leaf_rowoff; d.leaf_aos = td.leaf_aos;
        d.ao_row_ptr = td.ao_row_ptr; d.ao_rows = td.ao_rows;
        d.child_ptr = td.child_ptr; d.child_list = td.child_list; d.m2m_op = td.m2m_op; d.l2l_op = td.l2l_op;
        d.parent = td.parent; d.m2l_ptr = td.m2l_ptr; d.m2l_src = td.m2l_src; d.m2l_op = td.m2l_op;
        d.vals = prec == OCCK_FP64 ? (const void*)td.pair_vals : (const void*)td.pair_vals_f;
        d.ops = prec == OCCK_FP64 ? (const void*)td.ops : (const void*)td.ops_f;
        d.ct = base + o[s].ct;
        d.w = base + o[s].w;
        d.obox = base + o[s].obox;
        d.mbox = base + o[s].mbox;
        d.kb = (double*)(base + o[s].kb);
        d.part = (double*)(base + o[s].part);
        b->h_sys.push_back(d);
        b->maxD = std::max(b->maxD, t->depth);
    }
    // ---- items of the untuned stages
    std::vector<Item> tr, half, f64, f128, l64, l128, red;
    std::vector<int> en;
    b->half_lmc = nc <= 4 ? 4 : (nc <= 9 ? 9 : 16);
    for (int s = 0; s < nsys; ++s) {
        const SysDesc& d = b->h_sys[s];
        if (d.depth < 2) {
            b->zero_sys.push_back(s);
            continue;
        }
        for (int x = 0; x < (d.nao + 31) / 32; ++x)
            for (int y = 0; y < (d.nocc + 31) / 32; ++y) tr.push_back(Item{s, x, y, 0});
        const int nchh = (nc + b->half_lmc - 1) / b->half_lmc;
        for (int r = 0; r < d.nrow; ++r)
            for (int c = 0; c < nchh; ++c) half.push_back(Item{s, r, c, 0});
        for (int bm : {64, 128}) {
            const int nt = (d.nocc + bm - 1) / bm;
            auto& v = bm == 64 ? f64 : f128;
            for (int tt = 0; tt < nt * (nt + 1) / 2; ++tt)
                for (int y = 0; y < d.nleaf * nc; ++y) v.push_back(Item{s, tt, y, 0});
            auto& w = bm == 64 ? l64 : l128;
            for (int B = 0; B < d.nleaf; ++B) {
                const int nr = b->trees[s]->leaf_rowoff[B + 1] - b->trees[s]->leaf_rowoff[B];
                for (int x = 0; x < (nr + bm - 1) / bm; ++x)
                    for (int y = 0; y < (d.nocc + bm - 1) / bm; ++y) w.push_back(Item{s, x, y, B});
            }
        }
        for (int k = 0; k < occk::kRedBlocks; ++k) red.push_back(Item{s, k, 0, 0});
        en.push_back(s);
    }
    e = cudaSuccess;
    if (e == cudaSuccess) e = occk::up(&b->d_sys, b->h_sys);
    if (e == cudaSuccess) e = occk::up(&b->it_tr, tr);
    if (e == cudaSuccess) e = occk::up(&b->it_half, half);
    if (e == cudaSuccess) e = occk::up(&b->it_full64, f64);
    if (e == cudaSuccess) e = occk::up(&b->it_full128, f128);
    if (e == cudaSuccess) e = occk::up(&b->it_l2p64, l64);
    if (e == cudaSuccess) e = occk::up(&b->it_l2p128, l128);
    if (e == cudaSuccess) e = occk::up(&b->it_red, red);
    if (e == cudaSuccess) e = occk::up(&b->en_sys, en);
    b->n_tr = (int)tr.size();
    b->n_half = (int)half.size();
    b->n_full64 = (int)f64.size();
    b->n_full128 = (int)f128.size();
    b->n_l2p64 = (int)l64.size();
    b->n_l2p128 = (int)l128.size();
    b->n_red = (int)red.size();
    b->n_en = (int)en.size();
    b->cfg.lmc = occk::translate_chunk_batch(nc);
    b->cfg.tile = prec == OCCK_FP64 ? 64 : 128;
    if (e == cudaSuccess) e = build_translate_items(b, b->cfg.lmc);
    // per-system pipelines (mode 1): arguments over the same arena buffers,
    // systems ordered by decreasing work and dealt round-robin to the streams
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e == cudaSuccess) {
        std::vector<std::pair<double, int>> work;
        for (int s = 0; s < nsys; ++s) {
            const SysDesc& d = b->h_sys[s];
            b->fargs.push_back(occk::simt_args(ctx, trees[s], nocc[s], prec, d.C, d.ldc, d.K, d.ldk, b->E + s, d.ct,
                                               d.w, d.obox, d.mbox, d.kb, d.part, b->err));
            work.push_back({-(double)d.P * (double)(d.nbox + d.nrow), s});
        }
        std::sort(work.begin(), work.end());
        for (auto& w : work) b->order.push_back(w.second);
        const int ns = std::min(nsys, 8);
        b->fs.resize(ns, nullptr);
        b->fev.resize(ns, nullptr);
        for (int j = 0; j < ns && e == cudaSuccess; ++j) {
            e = cudaStreamCreateWithFlags(&b->fs[j], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fev[j], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        occk_status st = bfail(ctx, OCCK_ERR_CUDA, std::string("occk_batch_create: ") + cudaGetErrorString(e));
        occk_batch_destroy(b);
        return st;
    }
    *out = b;
    return OCCK_OK;
}

extern "C" void occk_batch_destroy(occk_batch* b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cs) cudaStreamDestroy(b->cs);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    for (auto st : b->fs)
        if (st) cudaStreamDestroy(st);
    for (auto ev : b->fev)
        if (ev) cudaEventDestroy(ev);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->err) cudaFree(b->err);
    free_items(b);
    for (void* p : {(void*)b->d_sys, (void*)b->it_tr, (void*)b->it_half, (void*)b->it_full64, (void*)b->it_full128,
                    (void*)b->it_l2p64, (void*)b->it_l2p128, (void*)b->it_red, (void*)b->en_sys, b->arena})
        if (p) cudaFree(p);
    delete b;
}

extern "C" occk_status occk_batch_buffers(occk_batch* b, int sys, double** C_dev, double** K_dev, int* ld,
                                          double** E_dev) {
    if (!b || sys < 0 || sys >= b->nsys) return OCCK_ERR_ARG;
    const SysDesc& d = b->h_sys[sys];
    if (C_dev) *C_dev = const_cast<double*>(d.C);
    if (K_dev) *K_dev = d.K;
    if (ld) *ld = d.nao;
    if (E_dev) *E_dev = b->E;
    return OCCK_OK;
}

extern "C" occk_status occk_batch_run(occk_batch* b, int use_graph, void* stream) {
    if (!b) return OCCK_ERR_ARG;
    occk_ctx* ctx = b->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(b->ev_in, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cs, b->ev_in, 0);
    if (e != cudaSuccess) return bfail(ctx, OCCK_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
    if (use_graph) {
        if (!b->graph_valid) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            b->exec = nullptr;
            b->graph = nullptr;
            if (b->built_lmc != b->cfg.lmc) e = build_translate_items(b, b->cfg.lmc);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue(b, b->cs);
                e = cudaStreamEndCapture(b->cs, &b->graph);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e != cudaSuccess) return bfail(ctx, OCCK_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            b->graph_valid = true;
        }
        e = cudaGraphLaunch(b->exec, b->cs);
    } else {
        e = enqueue(b, b->cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_out, 0);
    if (e != cudaSuccess) return bfail(ctx, OCCK_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    return OCCK_OK;
}

extern "C" occk_status occk_batch_set_config(occk_batch* b, const int* cfg) {
    if (!b || !cfg) return OCCK_ERR_ARG;
    const int lmc = cfg[0], bps = cfg[1], tile = cfg[2], mode = cfg[3];
    if ((lmc != 4 && lmc != 9 && lmc != 16 && lmc != 21 && lmc != 25) || bps < 1 || bps > 64 ||
        (tile != 64 && tile != 128) || (mode != 0 && mode != 1))
        return bfail(b->ctx, OCCK_ERR_ARG, "batch config out of range");
    b->cfg.lmc = lmc;
    b->cfg.bps = bps;
    b->cfg.tile = tile;
    b->cfg.mode = mode;
    b->graph_valid = false;
    return OCCK_OK;
}

extern "C" occk_status occk_batch_tune(occk_batch* b, const char* cache_path, int* cfg_out, void* stream) {
    if (!b) return OCCK_ERR_ARG;
    occk_ctx* ctx = b->ctx;
    cudaSetDevice(ctx->device);
    const std::string key = cfg_key(b);
    // cache lookup: lines "key lmc bps tile mode"
    std::map<std::string, BatchCfg> cache;
    if (cache_path) {
        std::ifstream f(cache_path);
        std::string k;
        BatchCfg c;
        while (f >> k >> c.lmc >> c.bps >> c.tile >> c.mode) cache[k] = c;
    }
    auto it = cache.find(key);
    if (it != cache.end()) {
        b->cfg = it->second;
    } else {
        cudaStream_t s = (cudaStream_t)stream;
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        auto time_cfg = [&](const BatchCfg& c) {
            b->cfg = c;
            float best = 1e30f;
            for (int r = 0; r < 3; ++r) {
                cudaEventRecord(t0, s);
                occk_batch_run(b, 0, stream);
                cudaEventRecord(t1, s);
                cudaEventSynchronize(t1);
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                if (r > 0) best = std::min(best, ms);
            }
            return best;
        };
        BatchCfg best = b->cfg;
        best.mode = 0;
        float tb = time_cfg(best);
        for (int lmc : {4, 9, 16, 21, 25}) {
            BatchCfg c = best;
            c.lmc = lmc;
            float t = time_cfg(c);
            if (t < tb) { tb = t; best = c; }
        }
        for (int bps : {2, 4, 8, 16, 32}) {
            BatchCfg c = best;
            c.bps = bps;
            float t = time_cfg(c);
            if (t < tb) { tb = t; best = c; }
        }
        if (b->prec == OCCK_FP32) {
            for (int tile : {64, 128}) {
                BatchCfg c = best;
                c.tile = tile;
                float t = time_cfg(c);
                if (t < tb) { tb = t; best = c; }
            }
        }
        {
            BatchCfg c = best;
            c.mode = 1;
            float t = time_cfg(c);
            if (t < tb) { tb = t; best = c; }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        b->cfg = best;
        cache[key] = best;
        if (cache_path) {
            std::ofstream f(cache_path);
            for (auto& kv : cache)
                f << kv.first << " " << kv.second.lmc << " " << kv.second.bps << " " << kv.second.tile << " "
                  << kv.second.mode << "\n";
        }
    }
    b->graph_valid = false;
    if (b->built_lmc != b->cfg.lmc) {
        cudaError_t e = build_translate_items(b, b->cfg.lmc);
        if (e != cudaSuccess) return bfail(ctx, OCCK_ERR_CUDA, "translate items");
    }
    if (cfg_out) {
        cfg_out[0] = b->cfg.lmc;
        cfg_out[1] = b->cfg.bps;
        cfg_out[2] = b->cfg.tile;
        cfg_out[3] = b->cfg.mode;
    }
    return OCCK_OK;
}

namespace occk {
int translate_chunk_batch(int nc) {
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
}  // namespace occk
