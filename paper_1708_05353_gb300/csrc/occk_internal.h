// Internal declarations shared by the host ABI layer and the CUDA kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/occk.h"

namespace occk {

// Real form of a rank-L expansion: nc = (L+1)^2 reals, for each l: Re m=0,
// then (Re, Im) for m = 1..l.
inline int ncomp(int L) { return (L + 1) * (L + 1); }

// One translation operator to generate: kind 0 = M2M (d = Xc - Xp),
// 1 = L2L (d = Xc - Xp), 2 = M2L (d = X - X').
struct OpDesc {
    double d[3];
    int kind;
    int pad;
};

// Device-side shell data for pair multipoles (one record per kept shell pair).
struct PairDesc {
    double A[3], B[3], X[3];   // shell centres and the leaf centre
    int prim_a, nprim_a;       // offsets into prim arrays
    int prim_b, nprim_b;
    int la, lb;
    int val_off;               // first value row (na*nb rows of nc reals)
    int pad;
};

// Workspace buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace occk

struct occk_tree {
    int device = -1;
    // ---- host copy -------------------------------------------------------
    int natom = 0, nshell = 0, nao = 0, depth = 0;
    double x0[3] = {0, 0, 0};
    double side = 0;
    std::vector<double> h;                  // [depth+1]
    std::vector<int> level_off;             // [depth+2]
    std::vector<int> box_key;               // [nbox*3]
    std::vector<int> parent;                // [nbox]
    std::vector<double> centre;             // [nbox*3]
    std::vector<int> m2l_tgt, m2l_src;      // sorted by (tgt, src)
    std::vector<int> pair_a, pair_b, pair_leaf;
    std::vector<double> pair_centre;        // [npair*3]
    std::vector<int> leaf_rowoff;           // [nleaf+1]
    std::vector<int> leaf_aos;              // [nrow]
    // shells
    std::vector<double> shell_xyz;          // [nshell*3]
    std::vector<int> shell_l, shell_prim_off, shell_nprim, shell_ao_off;
    std::vector<double> prim_exp, prim_coef;  // coef includes primitive and contracted norm
    // ordered AO-pair entries grouped by (leaf, local row)
    std::vector<int> row_ptr;               // [nrow+1]
    std::vector<int> ent_col;               // AO index s
    std::vector<int> ent_val;               // value row in the pair-multipole array
    int nvals = 0;                          // rows of pair multipole values
    // AO -> rows (for the K reduction)
    std::vector<int> ao_row_ptr;            // [nao+1]
    std::vector<int> ao_rows;               // row ids
    // translation schedule
    std::vector<occk::OpDesc> ops;          // distinct operators
    std::vector<int> m2l_op;                // per M2L edge
    std::vector<int> m2m_op;                // per box (child), -1 if none
    std::vector<int> l2l_op;                // per box (child), -1 if none
    // per-level CSR for M2M (parents gather children)
    std::vector<int> child_ptr;             // [nbox+1]
    std::vector<int> child_list;            // children box ids
    // M2L CSR by target box, restricted to levels 2..D
    std::vector<int> m2l_ptr;               // [nbox+1]
    std::vector<int> edge_lmax;             // per M2L edge (policy 1), empty if unset
    int lmax = -1;
    // sibling groups of the M2L pass: the boxes of each level 2..D grouped by
    // parent (groups in parent order, children in box order, at most 8); per
    // group the ascending union of its children's interaction lists with the
    // operator of each (child slot, source) edge, -1 where the source is not
    // in that child's list
    std::vector<int> grp_level_off;         // [depth+2]: first group of level l (l = 2..D+1)
    std::vector<int> grp_child;             // [ngroup*8], -1 for unused slots
    std::vector<int> grp_parent;            // [ngroup]
    std::vector<int> grp_ptr;               // [ngroup+1] into grp_src
    std::vector<int> grp_src;               // union sources
    std::vector<int> grp_op;                // [nsrc*8]
    std::vector<double> grp_gain;           // [depth+1]: M2L edges / union sources of the level

    // ---- device copy -----------------------------------------------------
    struct {
        int* row_ptr = nullptr; int* ent_col = nullptr; int* ent_val = nullptr;
        int* leaf_rowoff = nullptr; int* leaf_aos = nullptr;
        int* ao_row_ptr = nullptr; int* ao_rows = nullptr;
        int* child_ptr = nullptr; int* child_list = nullptr; int* m2m_op = nullptr;
        int* l2l_op = nullptr;
        int* m2l_ptr = nullptr; int* m2l_src = nullptr; int* m2l_op = nullptr;
        int* m2l_lmax_full = nullptr;  // all = lmax
        int* m2l_lmax_edge = nullptr;  // policy 1
        int* parent = nullptr;
        occk::PairDesc* pairs = nullptr;
        double* prim_exp = nullptr; double* prim_coef = nullptr;
        double* pair_vals = nullptr;   // [nvals][nc]
        float* pair_vals_f = nullptr;
        double* ops = nullptr;         // [nops][nc][nc]
        float* ops_f = nullptr;
        occk::OpDesc* opdesc = nullptr;
        float* lscale = nullptr;       // [nc] sqrt((l+m)!(l-m)!) / h_leaf^l
        float* box_scale = nullptr;    // [nbox]
        int* box_key = nullptr;        // [nbox*3]
        int* box_level = nullptr;      // [nbox]
        double* hlev = nullptr;        // [depth+1]
        int* m2l_tgt = nullptr;        // [nm2l]
        int* grp_child = nullptr; int* grp_parent = nullptr; int* grp_ptr = nullptr;
        int* grp_src = nullptr; int* grp_op = nullptr;
    } dev;
    int nops_alloc_lmax = -1;
    long long gen = 0;                      // changes whenever the operators are regenerated
};

struct occk_ctx {
    int device = -1;
    std::string err;
    int sm_count = 0;
    // workspaces
    occk::DevBuf ct, w, obox, mbox, kb, part, edev, scratch;
    // last run (for debug fetch)
    int last_prec = -1, last_nocc = 0, last_lmax = -1, last_first_box = 0;
    const occk_tree* last_tree = nullptr;
    // learned rank selector
    int mlp_ready = 0, mlp_t = 0;
    double tau = 1e-6;
    occk::DevBuf mlp_prm, mlp_norm, mlp_m, mlp_v, mlp_h, mlp_grad, mlp_ws, feat, pred, ranks, nrm, gram, rank_err;
    int ranks_valid = 0;
    // panel plan cache (tensor-core steps a and e)
    occk::DevBuf pplan, panels;
    const occk_tree* pp_tree = nullptr;
    int pp_nocc = -1, pp_nc = -1, pp_esz = -1, pp_pbytes = -1;
    int pp_KC = 0, pp_jc = 0, pp_it = 0, pp_max_rt = 0, pp_max_kca = 0;
    size_t pp_l2pA = 0, pp_l2pB = 0, pp_a2A = 0, pp_a2B = 0;   // panel counts
    // operator panels of the tensor-core translations
    occk::DevBuf tpan, tscale, tops;
    long long tp_gen = -1;
    int tp_prec = -1, tp_ok = 0;
    std::vector<double> tp_scd;             // [2][nlev][nc] scales of the last panel build (host)
    int last_scaled = 0;                    // last run kept O and Mcal in scaled form
    int tr_engine = -1;                     // occk_set_translate_engine mask
    int m2l_group = -1;                     // occk_set_m2l_group: -1 auto, 0 off, 1 on
    occk::DevBuf sob, smb;                  // slot storage of O~ and Mcal~ (slot pipeline)
    occk::DevBuf jbox;                      // far-field J: density multipoles, local expansions, partials
    double screen_tau = 0.0;                // occupied-pair screening threshold (0: off)
    int col_i0 = 0, col_i1 = 0;             // occk_set_column_block (col_i1 == 0: off)
    int last_screen = 0;                    // the last occk_farfield_K screened
    size_t last_screen_P = 0;               // its stored pair count (offset of the kept count)
    size_t last_tskip_n = 0;                // its step (a) bound tiles (SIMT forms; 0 otherwise)
    const unsigned char* last_tskip = nullptr;   // their flags (0 = tile skipped)
    occk::DevBuf scr_o, scr_m, scr_aux;     // compacted pair expansions; norms, keep/inverse maps, count
    int last_slot = 0;                      // last run used the slot pipeline
    int l2p_split = 0;                      // FP32 step (e) K-range splits (0: automatic)
    int f64_slices = 0;                     // FP64 steps (a), (e) from integer slices on the tensor core (0: DFMA)
    int f32_slices = 0;                     // FP32 steps (a), (e) from 4 integer slices (0: SIMT FFMA)
    int last_sliced = 0;                    // the last occk_farfield_K ran steps (a), (e) from slices
    size_t slice_budget = 0;                // largest slice-panel workspace (0: 32 GB)
    int slice_m2l = 1;                      // FP64-accurate form: M2L from slices too (from 25 components)
    occk::DevBuf splan, spanels;            // its plan (row tiles, panel and item offsets, exponents), panels
    // stage timers
    int timing = 0;
    cudaEvent_t ev[OCCK_NSTAGE + 1] = {};
    int ev_recorded = 0;
};

namespace occk {

// ----- kernel launchers (kernels_*.cu) ------------------------------------
cudaError_t launch_gen_ops(const OpDesc* d_desc, int nops, int L, double* d_out, float* d_out_f,
                           cudaStream_t s);
cudaError_t launch_pair_multipoles(const PairDesc* d_pairs, int npair, const double* d_exp,
                                   const double* d_coef, int L, double* d_vals, float* d_vals_f,
                                   int nvals, cudaStream_t s);

struct SliceArgs;
struct FmmArgs {
    int nao, nocc, ldc, ldk, nc, L, depth;
    int nbox, first_box;             // boxes [first_box, nbox) are stored
    int nleaf, leaf0, nrow;
    const int* level_off;            // host
    int prec;                        // OCCK_FP64 / OCCK_FP32
    const double* C;                 // column-major
    double* K;                       // column-major
    double* Ex_dev;
    // tree (device)
    const int* row_ptr; const int* ent_col; const int* ent_val;
    const int* leaf_rowoff; const int* leaf_aos;
    const int* ao_row_ptr; const int* ao_rows;
    const int* child_ptr; const int* child_list; const int* m2m_op; const int* l2l_op;
    const int* parent;
    const int* m2l_ptr; const int* m2l_src; const int* m2l_op; const int* m2l_lmax;
    const void* pair_vals;           // double or float
    const void* ops;                 // double or float
    // workspaces
    void* ct; void* w; void* obox; void* mbox; double* kb; double* part;
    const int* leaf_rowoff_host;     // host copy (max rows)
    int max_rows;
    int l2p_nsplit;                  // step (e) K-range splits, FP32 and mixed forms (KB holds that many copies)
    const SliceArgs* slices;         // FP64 steps (a), (e) from integer slices (nullptr: DFMA kernels)
    cudaEvent_t* ev;                 // OCCK_NSTAGE+1 events or nullptr
    // tensor-core forms
    const float* lscale;             // [nc] sqrt((l+m)!(l-m)!) / h_leaf^l
    const float* box_scale;          // [nbox] side of each box's level
    int* err_word;                   // device error word (bounded waits)
    // panel plan of the tensor-core steps (a) and (e)
    const int* pp_rtA; const long long* pp_offA; const int* pp_kca; const long long* pp_offAa;
    const long long* pp_offBa; int pp_KC, pp_jc, pp_it, pp_max_rt, pp_max_kca;
    uint8_t* pan_l2pA; uint8_t* pan_l2pB; uint8_t* pan_a2A; uint8_t* pan_a2B;
    // tensor-core translations (tr_on: steps b-d on tcgen05, multipoles and
    // local expansions stored in scaled form; otherwise SIMT, unscaled)
    // tr_mask: bit 0 M2M, bit 1 M2L, bit 2 L2L on the tensor core (the others
    // run on SIMT with the scaled FP32 operators ops_scaled)
    const uint8_t* tr_pan; const float* ops_scaled; int tr_nlev, tr_on, tr_mask, sm_count;
    float inv_h_leaf;
    // slot pipeline (tr_mask == 15): O~ and Mcal~ of every stored box in slots
    uint8_t* slot_o; uint8_t* slot_m;
    // learned selector (lmax_policy 2); learned == 0 when unused
    int learned;
    const float* mlp_prm; void* mlp_h; const float* mlp_norm;
    float* feat; float* pred; int* ranks; double* nrm; double* rank_err; double tau; int nm2l;
    const int* m2l_tgt; const int* box_key; const int* box_level; const double* hlev;
    // occupied-pair screening (screen != 0, FP64 and FP32): pairs with
    // n^2 < screen_tau2 are dropped before M2M; the tree passes run on the
    // kept pairs, compacted in scr_o / scr_m (same shape as obox / mbox)
    int screen; double screen_tau2;
    void* scr_o; void* scr_m; double* scr_norm; int* scr_keep; int* scr_inv; int* scr_count; int* scr_bcount;
    unsigned char* scr_tiles;        // [nocc/128][nocc/8] step (e) tiles holding a kept pair
    float* scr_a2; float* scr_b2;    // bound factors of the SIMT step (a): a2 [nleaf][nocc], b2 parts [nc][nleaf][nocc]
    unsigned char* scr_tskip;        // step (a) tiles (k_full's triangular order) dropped whole by the bound
    // sibling-grouped FP32 M2L (fused with L2L) per level: grp_use[lev] != 0
    // runs level lev with k_m2l_group instead of the per-target pass
    const int* grp_level_off;        // host [depth+2]
    const int* grp_child; const int* grp_parent; const int* grp_ptr; const int* grp_src; const int* grp_op;
    unsigned grp_use;                // bit lev set: level lev grouped
    // occupied column block [col0, col1) (col1 > col0; both 0 when unused):
    // only pairs touching the block are kept (screen != 0), step (e) and the
    // K reduction cover only the block's columns, Ex_dev gets their part of E
    int col0, col1;
};
cudaError_t run_farfield(const FmmArgs& a, cudaStream_t s);
// E = -1/2 sum C K from a stored K with the far-field reduction's order
// (kFarfieldPartials partials in `part`, then one final block).
cudaError_t energy_from_K(int nao, int nocc, const double* C, int ldc, const double* K, int ldk, double* part,
                          double* E, cudaStream_t s);
// Far-field Coulomb matrix (FP64; kernels_fmm.cu).
struct JArgs {
    int nao, nc, L, depth, nbox, first_box, nleaf, leaf0;
    const int* level_off;            // host
    const int* leaf_rowoff; const int* leaf_aos; const int* row_ptr; const int* ent_col; const int* ent_val;
    const int* child_ptr; const int* child_list; const int* m2m_op; const int* l2l_op; const int* parent;
    const int* m2l_ptr; const int* m2l_src; const int* m2l_op;
    const double* vals; const double* ops;
    const double* D; int ldd;        // column-major density matrix
    double* J; int ldj;              // column-major output
    double* Ej_dev;
    double* ob; double* mb;          // [stored boxes][nc] density multipoles, local expansions
    double* part;                    // [nleaf]
};
cudaError_t run_farfield_J(const JArgs& a, cudaStream_t s);
// partial energies run_farfield writes to FmmArgs::part (its K reduction blocks)
constexpr int kFarfieldPartials = 1024;
// orbital tile of the SIMT step (a) O^{ij} kernel (k_full): 64 x 64 in FP64;
// in FP32 128 x 128 (8 x 8 per thread) unless 96 x 96 (6 x 6 per thread)
// covers a third more useful pairs i <= j with its triangle of tiles
// (measured on GB300: 660 orbitals 18.1 -> 15.3 ms with 96; 601 orbitals
// 0.75 -> 0.95 ms, so 128 there).  The screening's step (a) tile flags use
// the same tiles.
constexpr int kFullTileFP64 = 64;
inline int full_tile_fp32(int nocc) {
    auto useful = [nocc](int bm) {
        const double nt = (nocc + bm - 1) / bm;
        return (double)nocc * (nocc + 1) / 2 / (nt * (nt + 1) / 2 * (double)bm * bm);
    };
    return useful(96) > 1.15 * useful(128) ? 96 : 128;
}
// Arguments of the SIMT FP64/FP32 path for one tree with caller-provided
// workspaces (the batch's per-system pipelines; host.cpp).
FmmArgs simt_args(const occk_ctx* ctx, const occk_tree* t, int nocc, int prec, const double* C, int ldc, double* K,
                  int ldk, double* Ex, void* ct, void* w, void* obox, void* mbox, double* kb, double* part,
                  int* err_word);
size_t workspace_elems_w(const FmmArgs& a);

cudaError_t probe_fma(int prec, int sm_count, double* flops, cudaStream_t s);

// ----- learned selector (kernels_mlp.cu) ------------------------------------
int mlp_nparams();
cudaError_t mlp_forward_train(const float* prm, const float* norm, const float* X, int n, float* Xn, float* Z1,
                              float* Z2, float* Y, cudaStream_t s);
cudaError_t mlp_backward(const float* prm, const float* Xn, const float* Z1, const float* Z2, const float* Y,
                         const float* T, int n, float* dY, float* dZ1, float* dZ2, float* grad, double* part,
                         int npart, cudaStream_t s);
cudaError_t mlp_adam(float* prm, const float* g, float* m, float* v, int t, float lr, cudaStream_t s);
cudaError_t mlp_predict_fp16(const float* prm, __half* prm_h, const float* norm, const float* X, int n,
                             float* Y, cudaStream_t s);
cudaError_t edge_features(bool fp64, const void* O, int first_box, int nbox, int nc, int L, long long P,
                          int nocc, int nedge, const int* tgt, const int* src, const int* box_key, const int* box_level,
                          const double* hlev, int depth, double* nrm, float* F, cudaStream_t s);
cudaError_t edge_energies(bool fp64, const void* O, int first_box, int nc, int L, long long P, int nocc,
                          int nedge,
                          const int* tgt, const int* src, const double* ops, const int* opidx, double* G,
                          double* out, cudaStream_t s);
cudaError_t select_ranks(const float* pred, int nedge, int Lmax, double tau, int* ranks, double* er,
                         cudaStream_t s);   // er: [nedge][Lmax+1] workspace

// ----- panel tensor-core GEMMs (kernels_tc2.cu) -----------------------------
struct PanelArgs {
    const int* rtA; const long long* offA; int KC, jc, it;       // step (e) plan
    const int* kca; const long long* offAa; const long long* offBa;  // step (a) plan
    int max_rt, max_kca, nleaf;
    const int* leaf_rowoff; const int* leaf_aos;
    const int* leaf_rowoff_host;           // host copy (row tiles of step (e))
    const float* Ct; const float* W; const float* Mbox; float* Obox; double* KB;
    const float* lscale;
    int nocc, nrow, nc, leaf_store0;
    int scaled; float inv_h_leaf;          // scaled storage of O and Mcal (see kernels_tc_translate.cu)
    int nsplit;                            // step (e): K-range splits (KB copies)
    int sm_count;                          // persistent grids
    uint8_t* panA; uint8_t* panB;
    int* err;
};
int panel_elem_bytes(int prec);
int panel_bytes(int prec);
cudaError_t panel_l2p(int prec, const PanelArgs& a, cudaStream_t s);
cudaError_t panel_a2(int prec, const PanelArgs& a, cudaStream_t s);
// ----- FP64 steps (a) and (e) from integer slices on the tensor core (kernels_f64s.cu) -----
struct SM2LArgs;
struct SliceArgs {
    int S;                                  // slices per operand (6 or 7)
    int nocc, nc, nrow, nleaf, leaf_store0, max_rt, nsplit, sm_count;
    long long nitems;                       // GEMM tiles (leaf, row tile, orbital tile, K split)
    const int* leaf_rowoff;
    int f32;                                // operands FP32 (the FP32 form) instead of FP64
    const SM2LArgs* m2l;                    // M2L from slices too (nullptr: double-FP32)
    const void* W; const void* Mbox; const float* lscale;
    int* erow; int* fcol;                   // row and column exponents (written)
    const int* rtA; const long long* offA; const long long* item0;   // plan
    uint8_t* panA;                          // panels of a leaf batch: A, then B
    double* KB;
    int* err;
    // step (a) (the full transform) from slices
    int full;                               // step (a) too
    int max_kca, ntp;                       // K stages of the largest leaf, triangular tile pairs
    const int* leaf_aos;
    const int* kca; const long long* offAa; const long long* offBa; const int* tpair;
    int* eC; int* eW;                       // exponents of C (leaf, i) and W (leaf, lm, j)
    uint8_t* panAa;                         // (the same workspace)
    // leaf batches whose panels fit the workspace (host): leaves
    // batch_e[b] .. batch_e[b+1]-1 for step (e), batch_a[] for step (a);
    // host copies of the panel and item offsets
    int nbatch_e, nbatch_a;
    const int* batch_e; const int* batch_a;
    const long long* offA_h; const long long* item0_h; const long long* offAa_h; const long long* offBa_h;
    // steps (c), (d) in double-FP32 arithmetic
    int ff, nops, nvals;
    float2* ops_ff;                         // [nops][nc][nc] (hi, lo) operators (workspace)
    float2* vals_ff; float2* C_ff;          // (hi, lo) pair values and transposed C (workspace)
};
int slice_stage_k();                        // K values of one panel stage
int slice_tile_n();                         // orbitals of one GEMM tile
int slice_max_stages();                     // stages of one tile (exact int32 group sums)
size_t slice_panel_bytes(int S, bool a);    // bytes of one A (a) or B panel
cudaError_t l2p_slices(const SliceArgs& a, cudaStream_t s);
cudaError_t full_slices(const SliceArgs& a, const void* Ct, void* Obox, cudaStream_t s);
// M2L with L2L, fused per level, in double-FP32 arithmetic on the FP32 pipe
// (the sliced FP64 form); O and Mcal are FP64 before and after the call
// M2L of the FP64-accurate form from integer slices (kernels_f64s.cu): the
// host plan per level and the device workspace (inside the slice panels)
struct SM2LArgs {
    int S, nq, ncs, nvar, ntile;
    const int* lt0; const int* lnt;         // host, per level: first target (box id), targets
    const int* lopl0; const int* lnopl;     // host, per level: first entry in oplist, distinct operators
    const long long* lst0;                  // host, per level: first entry in stoff
    const int* ltb;                         // host, per level: pair tiles per batch
    const int* edge_bop;                    // device [nm2l]: the edge's operator within its level
    const int* oplist;                      // device: distinct operators of each level
    const long long* stoff;                 // device: first stage entry of each (target, chunk)
    int2* stab; int* nk; int* ec; int* fq; int* gp;   // device workspace
    uint8_t* panB; uint8_t* panA;
    long long capA, capB;                   // panels that fit
};

struct FFArgs {
    int P, nc, L, D, first_box, nstore, leaf_store0, nops, sm_count;
    int m2m_done;                           // m2m_ff ran: the multipoles are (hi, lo) already
    const int* level_off;                   // host
    const int* m2l_ptr; const int* m2l_src; const int* m2l_op; const int* lmax_e;
    const int* parent; const int* l2l_op;
    const int* child_ptr; const int* child_list; const int* m2m_op;
    const double* ops; float2* ops_ff;      // FP64 operators; their (hi, lo) copy (written)
    double* Ob; double* Mb;
    const SM2LArgs* sm;                     // M2L from slices (nullptr: double-FP32)
    int* err;                               // device error word of the slice GEMM
};
cudaError_t m2m_ff(const FFArgs& f, cudaStream_t s);   // (b) in double-FP32; splits the leaves first
cudaError_t m2l_ff(const FFArgs& f, cudaStream_t s);
cudaError_t ff_join(const FFArgs& f, cudaStream_t s);  // every stored box's multipoles back to FP64
// step (a), first half, in double-FP32 arithmetic (the sliced FP64 form)
struct HalfFFArgs {
    int nao, nocc, nrow, nc, nvals, lmc, nth;
    const int* row_ptr; const int* ent_col; const int* ent_val;
    const double* vals; const double* Ct;   // FP64 inputs
    float2* vals_ff; float2* C_ff;          // their (hi, lo) copies (workspace, written)
    double* W;
};
cudaError_t half_ff(const HalfFFArgs& h, cudaStream_t s);

// Polls allowed to the MMA thread's operand wait in the panel GEMMs of steps
// (a) and (e) on the current device (< 0 restores the default 2^22).
cudaError_t set_mma_wait_limit(long long polls);
cudaError_t set_slice_wait_limit(long long polls);   // the sliced GEMMs (kernels_f64s.cu)

// ----- tensor-core translations, steps (b)-(d) (kernels_tc_translate.cu) --------
struct TrArgs {
    int P, nc, first_box, nlev, sm_count;
    const int* parent; const int* box_level;
    const uint8_t* pan;                    // operator panels
    int* err;
};
int tr_np(int nc);                          // N of the GEMM (0: no tensor-core form for this nc)
size_t tr_panel_bytes(int prec, int nc);    // bytes of one operator's panels
cudaError_t tr_build_panels(int prec, const double* ops, int nops, int nc, const int* opinfo, const double* scd,
                            int nlev, uint8_t* pan, float* ops_scaled, cudaStream_t s);
cudaError_t tr_translate(int prec, const TrArgs& h, int mode, int tgt0, int ntgt, const int* ptr, const int* list,
                         const int* opidx, const float* in, float* out, int accumulate, cudaStream_t s);

// Slot pipeline (all three translations on the tensor core, operands kept in
// the tensor core's layout between the steps; kernels_tc_translate.cu).
struct SlotArgs {
    int P, nc, ntile, first_box, sm_count;
    const int* parent;
    const uint8_t* pan;                    // operator panels
    int* err;
};
size_t tr_slot_box_bytes(int prec, int nc, int ntile);   // slot bytes of one box
cudaError_t tr_slot_translate(int prec, const SlotArgs& h, int mode, int tgt0, int ntgt, const int* ptr,
                              const int* list, const int* opidx, const uint8_t* in, uint8_t* out, int accumulate,
                              cudaStream_t s);
// FP32 [box][nc][P] (boxes box0 .. box0+nbox-1, counted from the first stored
// box) <-> slots
cudaError_t tr_slots_pack(int prec, int nc, const float* X, int Ppairs, int ntile, int box0, int nbox,
                          uint8_t* slots, cudaStream_t s);
cudaError_t tr_slots_unpack(int prec, int nc, const uint8_t* slots, int Ppairs, int ntile, int box0, int nbox,
                            float* X, cudaStream_t s);

// ----- plain tensor-core GEMM for checking the engine (kernels_tc2.cu) --------
int tc_mode(int prec);
size_t tc_gemm_panel_bytes(int prec, int M, int N, int K);
cudaError_t tc_gemm(int prec, int M, int N, int K, const float* A, const float* B, float* D, uint8_t* panels,
                    int* err, cudaStream_t s);

}  // namespace occk
