/*
 * occk.h -- C ABI of the far-field occupied-orbital FMM exchange (occ-FMM-K)
 * on one NVIDIA GB300 (sm_103a).
 *
 * The library computes the far-field part of the occupied exchange block
 *     K_ri = 2 sum_j (rj|ji)                          (paper, Eq. occex)
 * for AO index r and occupied orbitals i, j, with the multipole machinery of
 * Le & Shiozaki, "Occupied-orbital fast multipole method for efficient exact
 * exchange evaluation" (arXiv:1708.05353), Sec. II:
 *   (a) AO-pair multipoles transformed to occupied pairs   (Eq. motrans)
 *   (b) occupied M2M up the box hierarchy                  (Eq. fmm1, per ij)
 *   (c) occupied M2L over interaction lists                (Eq. fmmex / fmm2)
 *   (d) occupied L2L down the hierarchy                    (Eq. fmm3, per ij)
 *   (e) K^ff_ri = 2 sum_j sum_lm O^{rj,X}_lm Mcal^{ij}_lm(X) (Eq. kri; the factor
 *       2 of Eq. occex is applied) and E^ff_x = -1/2 sum_ri C_ri K^ff_ri.
 *
 * Conventions shared by every entry point
 *   - Every function returns occk_status: 0 on success, a negative code on
 *     failure.  No C++ exception crosses the ABI.  The message of the last
 *     failure on a context is available from occk_last_error().
 *   - Units: bohr and hartree.  AO order is shell order; a p shell contributes
 *     Cartesian (x, y, z) in that order.  Only s (l = 0) and p (l = 1) shells.
 *   - The caller owns every buffer it passes; the library never frees caller
 *     memory.  The library owns what it allocates (context workspaces, tree
 *     data) and releases it in occk_destroy / occk_tree_destroy.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued asynchronously on it.
 *   - One context per host thread; a context and its trees belong to one
 *     device.
 */
#ifndef OCCK_H
#define OCCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int occk_status;
#define OCCK_OK               0
#define OCCK_ERR_ARG         -1   /* null pointer, bad size, bad enum */
#define OCCK_ERR_SHAPE       -2   /* inconsistent dimensions (nocc, ld, lmax) */
#define OCCK_ERR_CUDA        -3   /* a CUDA runtime call failed */
#define OCCK_ERR_OOM         -4   /* device or host allocation failed */
#define OCCK_ERR_TIMEOUT     -5   /* a bounded device wait gave up */
#define OCCK_ERR_UNSUPPORTED -6   /* l > 1 shells, lmax out of range, no device */
#define OCCK_ERR_STATE       -7   /* call order violated (e.g. no multipoles) */

typedef struct occk_ctx  occk_ctx;    /* opaque: device, workspaces, MLP, tuning */
typedef struct occk_tree occk_tree;   /* opaque: boxes, lists, pair multipoles, operators */

/* Contracted s/p Gaussian basis (paper, Sec. II: AO basis functions phi_r;
 * contracted shells as used in the paper's implementation).  All arrays are
 * host memory, read during occk_build_tree only. */
typedef struct {
    int natom;
    const double* xyz;          /* [natom][3] atom positions, bohr */
    int nshell;
    const int* shell_atom;      /* [nshell] atom of each shell */
    const int* shell_l;         /* [nshell] 0 (s) or 1 (p) */
    const int* shell_nprim;     /* [nshell] primitives per shell, >= 1 */
    const double* exps;         /* [sum nprim] exponents, shell-major */
    const double* coefs;        /* [sum nprim] coefficients of NORMALISED
                                   primitives; each contracted function is
                                   renormalised to unit self-overlap */
} occk_basis;

/* Box-hierarchy parameters (paper, Sec. II: depth N_s, well-separatedness). */
typedef struct {
    int depth;                       /* subdivisions D >= 1; 0 => choose D in
                                        1..12 whose mean atoms per non-empty
                                        leaf is closest to target */
    double target_atoms_per_leaf;    /* used when depth == 0 (e.g. 8) */
    int ws_boxes;                    /* must be 1: nearest-neighbour boxes are
                                        near field */
    double pair_thresh;              /* shell-pair screen (default 1e-14): keep
                                        (a,b) if max_pq |c_p c_q| (2 sqrt(a_p a_q)
                                        /(a_p+a_q))^1.5 exp(-mu_pq R_ab^2) > thresh */
} occk_tree_params;

typedef enum {
    OCCK_FP64 = 0,     /* all steps in FP64 (DFMA) */
    OCCK_FP32 = 1,     /* all contractions in FP32 FMA; K, E reduced in FP64 */
    OCCK_TF32 = 2,     /* (a),(c),(e) on tensor cores, TF32 inputs, FP32 accumulate */
    OCCK_BF16 = 3,     /* (a),(c),(e) on tensor cores, BF16 inputs, FP32 accumulate */
    OCCK_FP16 = 4,     /* (a),(c),(e) on tensor cores, FP16 inputs, FP32 accumulate */
    OCCK_BF16X3 = 5,   /* BF16 hi/lo split, three products (hi*hi + hi*lo + lo*hi) */
    OCCK_FP16X3 = 6    /* FP16 hi/lo split of both operands, three products */
} occk_precision;

typedef struct {
    int nao, natom, nshell, depth;
    int nbox;                  /* non-empty boxes, all levels */
    int nleaf;                 /* non-empty leaf boxes */
    int npair;                 /* kept shell pairs */
    int nentry;                /* ordered AO-pair entries (both orders) */
    int nrow;                  /* sum over leaves of |S_B| (AOs touched per leaf) */
    int nm2l;                  /* M2L edges (target, source), all levels */
    int lmax;                  /* rank of the last occk_pair_multipoles, -1 if none */
    double x0[3];              /* root cube min corner */
    double side;               /* root cube side */
} occk_tree_info;

/* Context.  device >= 0 binds CUDA device `device`; device = -1 makes a
 * host-only context that can build and query trees but runs no kernel
 * (occk_pair_multipoles / occk_farfield_K then fail with UNSUPPORTED). */
occk_status occk_create(occk_ctx** out, int device);
void occk_destroy(occk_ctx* ctx);
const char* occk_last_error(const occk_ctx* ctx);

/* Build the box hierarchy on the host (paper, Sec. II: "hierarchy of boxes",
 * interaction list = non-neighbouring boxes of the same level whose parents
 * are the parent's neighbours).  Steps: screen shell pairs (a <= b); pair
 * centre = sum_pq w_pq P_pq / sum_pq w_pq with w_pq = exp(-mu_pq R_ab^2) (the
 * whole pair goes to one box: "X is unique to each pair r, s"); root cube =
 * bounding box of the centres widened by 1e-6 of its largest extent; leaf
 * index floor((x - x0)/h), clamped; empty boxes dropped; boxes ordered by
 * (level, ix, iy, iz).  Floating-point decisions use IEEE double without
 * contraction, so the integer tree is reproducible.  Host work only; with a
 * device context it also uploads the tree.  *out is owned by the caller and
 * released with occk_tree_destroy. */
occk_status occk_build_tree(occk_ctx* ctx, const occk_basis* basis,
                            const occk_tree_params* params, occk_tree** out);
void occk_tree_destroy(occk_tree* tree);
occk_status occk_query(const occk_tree* tree, occk_tree_info* info);

/* Copy one integer/real array of the tree to host memory (for checking the
 * tree against an independent implementation).  `bytes` must equal the
 * array's size exactly, else OCCK_ERR_SHAPE.
 *   OCCK_TREE_LEVEL_OFF  int32 [depth+2]       first box of each level
 *   OCCK_TREE_BOX_KEY    int32 [nbox][3]       integer box coordinates
 *   OCCK_TREE_PARENT     int32 [nbox]          parent box (-1 for the root)
 *   OCCK_TREE_CENTRE     double [nbox][3]      box centres
 *   OCCK_TREE_M2L        int32 [nm2l][2]       (target, source) sorted
 *   OCCK_TREE_PAIRS      int32 [npair][3]      (shell a, shell b, leaf box)
 *   OCCK_TREE_PAIR_CENTRE double [npair][3]
 *   OCCK_TREE_LEAF_AOS   int32 [nrow]          S_B of each leaf, leaves in order
 *   OCCK_TREE_LEAF_ROWOFF int32 [nleaf+1]      offsets into LEAF_AOS */
enum {
    OCCK_TREE_LEVEL_OFF = 0, OCCK_TREE_BOX_KEY = 1, OCCK_TREE_PARENT = 2,
    OCCK_TREE_CENTRE = 3, OCCK_TREE_M2L = 4, OCCK_TREE_PAIRS = 5,
    OCCK_TREE_PAIR_CENTRE = 6, OCCK_TREE_LEAF_AOS = 7, OCCK_TREE_LEAF_ROWOFF = 8
};
occk_status occk_tree_export(const occk_tree* tree, int what, void* host_out, size_t bytes);

/* Step a0, once per geometry and rank (paper, Sec. II, the AO multipole
 * integrals O^{rs,X}_lm = int phi_r O_lm(r - X) phi_s about the centre X of
 * the leaf box that owns the pair; and the translation operators built from
 * the scaled solid harmonics O_lm, M_lm of Sec. I).  Computes, in FP64 on the
 * device: every kept pair's multipoles up to rank lmax (0 <= lmax <= 12), and
 * the real-form M2M, M2L and L2L matrices for every offset used by the tree.
 * Results stay on the device, owned by the tree.  Asynchronous on `stream`. */
occk_status occk_pair_multipoles(occk_ctx* ctx, occk_tree* tree, int lmax, void* stream);

/* Per-edge multipole ranks for M2L (lmax_policy = 1 of occk_farfield_K):
 * ranks[e] in [0, lmax] for every M2L edge e in OCCK_TREE_M2L order; the
 * edge operator keeps output and input ranks <= ranks[e]; M2M and L2L keep
 * the tree's lmax.  Host array, copied.  n must equal nm2l. */
occk_status occk_set_edge_lmax(occk_ctx* ctx, occk_tree* tree, const int* ranks, int n);

/* The far-field exchange, steps (a)-(e) (paper, Sec. II, from "First, for each
 * box at the lowest level ..." to Eq. kri):
 *   C_dev  [nao x nocc] column-major FP64 device, leading dimension ldc >= nao
 *   K_dev  [nao x nocc] column-major FP64 device output, ldk >= nao; holds
 *          K^ff_ri = 2 sum_j sum_lm O^{rj,X}_lm Mcal^{ij}_lm(X) on return
 *   Ex_dev FP64 device scalar output (nullable): E^ff = -1/2 sum_ri C_ri K_ri
 *   Ex_host FP64 host output (nullable); when non-null the call synchronises
 *          `stream` before returning (do not pass it during graph capture)
 *   prec   arithmetic of the contractions (occk_precision)
 *   lmax_policy 0 = the tree's lmax on every edge; 1 = per-edge ranks from
 *          occk_set_edge_lmax (falls back to 0 when none were set); 2 =
 *          learned: after M2M the edge features feed the MLP (FP16) and the
 *          ranks are chosen on the device for the budget of
 *          occk_set_learned_tau (falls back to 0 without a model or when the
 *          tree's lmax < 2)
 * Requires occk_pair_multipoles on this tree and 1 <= nocc <= 65535 (stored
 * occupied pairs i <= j are indexed in 32 bits; OCCK_ERR_SHAPE above).
 * Workspaces are owned by the context and grow on demand (allocation happens
 * outside any timed loop on the first call with a given shape). */
occk_status occk_farfield_K(occk_ctx* ctx, const occk_tree* tree, int nocc,
                            const double* C_dev, int ldc, int prec, int lmax_policy,
                            double* K_dev, int ldk, double* Ex_dev, double* Ex_host,
                            void* stream);

/* Intermediate results of the last occk_farfield_K on this context, copied to
 * host memory, for step-by-step checking (synchronises `stream`).
 *   OCCK_DBG_PAIR_MULT  double [nvals][nc]      pair multipoles (real form)
 *   OCCK_DBG_OBOX       double [nbox][nc][nocc*nocc]  occupied multipoles
 *   OCCK_DBG_MBOX       double [nbox][nc][nocc*nocc]  local expansions
 * Real form of a rank-L expansion, nc = (L+1)^2 reals: for each l, Re m=0,
 * then (Re, Im) for m = 1..l (components with m < 0 follow from
 * X_{l,-m} = (-1)^m conj X_{lm}).  Levels 0-1 are zero (no M2L there).
 * FP32 runs are widened to double.
 *   OCCK_DBG_SCREEN_TILES int32 [2]  of a screened call (occk_set_pair_screen):
 *       {step (a) tiles skipped by the Cauchy-Schwarz bound, step (a) tiles
 *       the bound examined} (SIMT forms only; {0, 0} for the tensor-core
 *       forms, which form every tile) */
enum { OCCK_DBG_PAIR_MULT = 0, OCCK_DBG_OBOX = 1, OCCK_DBG_MBOX = 2, OCCK_DBG_SCREEN_TILES = 3 };
occk_status occk_debug_fetch(occk_ctx* ctx, const occk_tree* tree, int what,
                             void* host_out, size_t bytes, void* stream);

/* Occupied column block for sharding one far-field build over several GPUs
 * (the data-parallel split of the occupied index that the paper's
 * implementation makes over j batches, Sec. III B, here over blocks of i).
 * With 0 <= i0 < i1 set, later occk_farfield_K calls on this context compute
 * K^ff_{r,i} for i0 <= i < i1 only: steps (a)-(d) run on the occupied pairs
 * (i, j) with i or j in the block (a pair's multipoles do not depend on the
 * other pairs, so those columns come out bit for bit as in an unblocked
 * call), step (e) and the K reduction cover the block's columns, the other
 * columns of K_dev are not written, and Ex_dev / Ex_host receive the block's
 * part -1/2 sum_{r, i in block} C_ri K_ri.  Gathering the blocks of all ranks
 * gives the whole K; occk_exchange_energy on it gives E bit for bit as an
 * unblocked call.  i0 = i1 = 0 turns the block off (default).  i1 > nocc
 * fails in occk_farfield_K with OCCK_ERR_SHAPE; the learned selector
 * (lmax_policy 2) is refused with a block (OCCK_ERR_UNSUPPORTED).  The block
 * uses the workspaces and tree passes of occupied-pair screening (both may be
 * on together: a pair is then kept if it touches the block and passes the
 * threshold).  OCCK_ERR_ARG unless i0 = i1 = 0 or 0 <= i0 < i1. */
occk_status occk_set_column_block(occk_ctx* ctx, int i0, int i1);

/* Exchange energy E = -1/2 sum_ri C_ri K_ri of a stored K (FP64), with the
 * same reduction order as the energy of occk_farfield_K, so that for the K an
 * unblocked occk_farfield_K wrote it returns that call's E bit for bit (e.g.
 * on K gathered from column blocks).  C_dev, K_dev [nao x nocc] column-major
 * FP64 device (ldc, ldk >= nao); E_dev FP64 device scalar output, written on
 * `stream`.  Uses the context's reduction workspace (allocated on first use):
 * order it with the context's other calls (one stream). */
occk_status occk_exchange_energy(occk_ctx* ctx, int nao, int nocc, const double* C_dev, int ldc,
                                 const double* K_dev, int ldk, double* E_dev, void* stream);

/* Exchange energy E = -1/2 sum_ri C_ri K_ri from caller buffers, allocating
 * no device memory.  The paper has no counterpart: this entry exists for
 * callers that cannot let a library call cudaMalloc -- an application whose
 * own allocator owns all device memory (a framework caching allocator or a
 * fixed pool), or a latency-sensitive loop in which an allocation would
 * synchronise the device.  It computes the same reduction as the energy of
 * occk_farfield_K (FP64), with its scratch (one double per occupied column)
 * in a file-scope __device__ array of OCCK_NOALLOC_MAX_OCC doubles (64 KB)
 * that every GPU loading the library holds until the process exits.
 *   C_dev [nao x nocc] column-major FP64 device, ldc >= nao
 *   K_dev [nao x nocc] column-major FP64 device, ldk >= nao (e.g. the K of
 *         occk_farfield_K)
 *   E_dev FP64 device scalar output, written on `stream`
 * nocc > OCCK_NOALLOC_MAX_OCC fails with OCCK_ERR_SHAPE (and a message in
 * occk_last_error(ctx)); no cudaMalloc, cudaFree or allocating library call is
 * made.  The device address of the array is looked up (cudaGetSymbolAddress,
 * with the context's device current) on every call made outside stream
 * capture -- the first such call on a device is its set-up, and a later
 * device reset leaves no stale address behind; a call made during capture
 * reuses the address of the last uncaptured call on that device, so make the
 * first call on a device before any stream capture (OCCK_ERR_STATE
 * otherwise).  All calls on a device share the array and each overwrites it:
 * calls that overlap on the GPU race and must be ordered by the caller (e.g.
 * one stream). */
#define OCCK_NOALLOC_MAX_OCC 8192
occk_status occk_exchange_energy_noalloc(occk_ctx* ctx, int nao, int nocc, const double* C_dev, int ldc,
                                         const double* K_dev, int ldk, double* E_dev, void* stream);

/* Opt-in stage timers (CUDA events recorded on the call's stream between
 * stages).  on != 0 enables them for later occk_farfield_K calls on this
 * context.  occk_get_timings synchronises on the last recorded event and
 * writes the durations (ms) of the last call's stages to ms[0..OCCK_NSTAGE-1]:
 *   0 (a) C transpose + AO->MO half transform   1 (a) full transform O^{ij}
 *   2 (b) M2M   3 (c) M2L   4 (d) L2L   5 (e) L2P   6 K reduction + energy
 * n must be >= OCCK_NSTAGE. */
#define OCCK_NSTAGE 7
occk_status occk_set_timing(occk_ctx* ctx, int on);
occk_status occk_get_timings(occk_ctx* ctx, float* ms, int n);

/* ---- Learned per-edge multipole rank (an addition to the paper's method) --
 * A 3-layer MLP (OCCK_MLP_NIN -> 64 -> 64 -> OCCK_MLP_NOUT, ReLU) maps the
 * features of an M2L edge to the predicted log10 |e_edge(L) - e_edge(10)| (Eh)
 * of that edge's far-field energy for L = 2..9.  The network lives in the
 * context: FP32 parameters (row-major W1 [NIN x 64], b1, W2 [64 x 64], b2,
 * W3 [64 x NOUT], b3) and a normalisation vector [mean_x (NIN), std_x (NIN),
 * mean_y (NOUT), std_y (NOUT)]: inputs are standardised, outputs are
 * predicted standardised and mapped back.  Training is full-batch Adam on the
 * mean squared error of the standardised outputs; inference is FP16. */
#define OCCK_MLP_NIN 16
#define OCCK_MLP_HIDDEN 64
#define OCCK_MLP_NOUT 8
#define OCCK_MLP_NPARAM (OCCK_MLP_NIN * 64 + 64 + 64 * 64 + 64 + 64 * OCCK_MLP_NOUT + OCCK_MLP_NOUT)
#define OCCK_MLP_NNORM (2 * OCCK_MLP_NIN + 2 * OCCK_MLP_NOUT)
/* He-uniform weights from a host generator seeded by `seed`, zero biases,
 * identity normalisation; resets the Adam state. */
occk_status occk_mlp_init(occk_ctx* ctx, uint64_t seed);
/* Copy parameters / normalisation in (set) or out (get); host arrays of
 * OCCK_MLP_NPARAM and OCCK_MLP_NNORM floats.  set marks the model usable. */
occk_status occk_mlp_set(occk_ctx* ctx, const float* params, const float* norm);
occk_status occk_mlp_get(occk_ctx* ctx, float* params, float* norm);
/* `steps` full-batch Adam steps (learning rate lr) on X_dev [n x NIN] raw
 * features and T_dev [n x NOUT] standardised targets (device FP32);
 * *loss_host (nullable) receives the loss before the last step.  Synchronises. */
occk_status occk_mlp_train(occk_ctx* ctx, const float* X_dev, const float* T_dev, int n, int steps,
                           float lr, float* loss_host, void* stream);
/* Loss and its gradient with respect to the parameters (grad_dev: device
 * FP32 [OCCK_MLP_NPARAM]), without updating anything.  Synchronises. */
occk_status occk_mlp_grad(occk_ctx* ctx, const float* X_dev, const float* T_dev, int n, float* grad_dev,
                          float* loss_host, void* stream);
/* FP16 inference: Y_dev [n x NOUT] = predicted log10 errors (de-standardised). */
occk_status occk_mlp_predict(occk_ctx* ctx, const float* X_dev, int n, float* Y_dev, void* stream);
/* Features [nm2l x NIN] of every M2L edge from the occupied multipoles of the
 * last occk_farfield_K on this context and tree: level/depth, |R|/h, sorted
 * |R_k|/|R|, log10 h, log10(norm_l / h^l) of target and source for l = 0, 2,
 * 4, 6, 8, clamped to the rank (norm_l = 2-norm over m and all occupied
 * pairs). */
occk_status occk_edge_features(occk_ctx* ctx, const occk_tree* tree, float* F_dev, void* stream);
/* Training labels: E_dev [nm2l x (lmax+1)] = energy of each M2L edge with its
 * operator truncated to ranks 0..lmax, from the last occk_farfield_K (run with
 * lmax_policy 0); exact splitting because M2M and L2L re-expand exactly. */
occk_status occk_edge_energies(occk_ctx* ctx, const occk_tree* tree, double* E_dev, void* stream);
/* Error budget tau (Eh) of lmax_policy 2: ranks minimise sum_e (L_e+1)^4
 * subject to sum_e predicted err_e(L_e) <= tau.  Default 1e-6. */
occk_status occk_set_learned_tau(occk_ctx* ctx, double tau);
/* Ranks chosen by the last lmax_policy 2 call (host int [nm2l]). */
occk_status occk_get_edge_ranks(occk_ctx* ctx, const occk_tree* tree, int* ranks, int n);

/* ---- Batches of uneven systems (an addition to the paper's method) ---------
 * A batch runs the far-field exchange of many systems (same lmax, each tree
 * with its multipoles) as one sequence of persistent kernels -- one per step,
 * and one per tree level for M2M and L2L -- over static work lists of all
 * systems, captured once into a CUDA graph.  The batch owns one device arena
 * with every system's workspace and its input/output buffers.
 * prec: OCCK_FP64 or OCCK_FP32. */
typedef struct occk_batch occk_batch;
occk_status occk_batch_create(occk_ctx* ctx, int nsys, occk_tree* const* trees, const int* nocc, int prec,
                              occk_batch** out);
void occk_batch_destroy(occk_batch* batch);
/* Device buffers of system `sys`, owned by the batch: C (input) and K
 * (output), column-major [nao x nocc] with leading dimension *ld = nao, and
 * the energies E [nsys] (output, one per system).  Any pointer may be NULL. */
occk_status occk_batch_buffers(occk_batch* batch, int sys, double** C_dev, double** K_dev, int* ld,
                               double** E_dev);
/* Run the batch on `stream` (ordered with it through events).  use_graph != 0
 * captures the launch sequence into a CUDA graph on first use (and after a
 * tuning change) and replays it. */
occk_status occk_batch_run(occk_batch* batch, int use_graph, void* stream);
/* Autotune the batch: for the level-synchronous persistent mode (mode 0) its
 * tile shapes -- components per translation block (4, 9, 16, 21, 25),
 * persistent blocks per SM (2..32) and, in FP32, the SIMT GEMM tile (64 or
 * 128) -- by coordinate search, then the per-system mode (mode 1: every
 * system's own single-system pipeline on one of up to 8 forked streams,
 * largest first, joined at the end), timing whole batch runs with CUDA events;
 * the winner is cached in the text file `cache_path` (nullable, one line
 * "key chunk blocks_per_sm tile mode") under a key of GPU name, lmax,
 * precision, number of systems, total pair count and depth, and reused when
 * the key is present.  cfg_out (nullable, 4 ints) receives {chunk, blocks per
 * SM, tile, mode}.  Synchronises `stream`. */
occk_status occk_batch_tune(occk_batch* batch, const char* cache_path, int* cfg_out, void* stream);
/* Set the batch configuration directly: cfg = {chunk (4, 9, 16, 21 or 25),
 * blocks per SM (1..64), tile (64 or 128), mode (0 or 1)}, as occk_batch_tune
 * reports it.  OCCK_ERR_ARG for a value outside those sets. */
occk_status occk_batch_set_config(occk_batch* batch, const int* cfg);

/* Reads the device error word of the last occk_farfield_K on this context
 * (synchronises `stream`).  Returns OCCK_ERR_TIMEOUT if a bounded wait inside
 * a tensor-core kernel gave up (its results are then invalid), else OK. */
occk_status occk_device_status(occk_ctx* ctx, void* stream);

/* Test aid for the failure path of the bounded device waits (no paper
 * counterpart).  Sets how many times the MMA-issuing thread of the
 * tensor-core panel GEMMs of steps (a) and (e) (the mixed forms and the
 * integer-slice forms of occk_set_fp64_slices / occk_set_fp32_slices) polls
 * for a stage's operands
 * before it gives up (polls < 0 restores the default, 2^22; 0 gives up at the
 * first wait).  A wait that gives up makes the kernel raise its abort flag,
 * wait (with the default limit) for its own bulk copies and MMAs in flight,
 * free its TMEM and return; occk_farfield_K then reports OCCK_ERR_TIMEOUT
 * (when it synchronises) and occk_device_status does too, and the next call
 * with the default limit is unaffected.  The setting belongs to the device,
 * not the context: it applies to every context of the process on that device
 * until changed.  Synchronous. */
occk_status occk_debug_set_wait_limit(occk_ctx* ctx, long long polls);

/* Occupied-pair screening for localised occupied orbitals (the extension the
 * paper proposes in Sec. IV).  With tau > 0, occk_farfield_K drops every
 * occupied pair (i, j) whose pair-density multipoles are negligible on all
 * leaves,  n_ij^2 = sum_X sum_{l, m=-l..l} |O^{ij,X}_lm|^2 < tau^2  (Eq.
 * motrans gives O^{ij,X}), before M2M: M2M, M2L and L2L run on the kept pairs
 * only and the dropped pairs have no local expansion and no part in K.  The
 * norm of pair (i, j) is taken from the stored (min, max) ordering, so both
 * orderings share one decision.
 *   tau  absolute threshold, finite and >= 0; 0 turns screening off (default)
 * Screening runs with every precision and lmax_policy 0 or 1 (the learned
 * policy gives OCCK_ERR_UNSUPPORTED while tau > 0); M2M, M2L and L2L then run
 * on the SIMT translation kernel with unscaled storage, whatever
 * occk_set_translate_engine selects.
 * With screening on, occk_debug_fetch returns current values for the leaf
 * boxes only: the leaf local expansions of every pair (zero for dropped
 * pairs), and the leaf multipoles of every pair except, on the FP64 and FP32
 * paths, those in step (a) tiles skipped because a bound placed every pair
 * of the tile below tau.  OCCK_ERR_ARG for a negative, infinite or NaN tau. */
occk_status occk_set_pair_screen(occk_ctx* ctx, double tau);

/* Number of occupied pairs i <= j kept by the last occk_farfield_K call on
 * this context (synchronises `stream`, the stream of that call), or -1 in
 * *kept when that call did not screen. */
occk_status occk_pair_screen_count(occk_ctx* ctx, long long* kept, void* stream);

/* The far-field Coulomb matrix (paper, Sec. II: the density-contracted box
 * multipoles, Eq. fmmc, and J^ff_rs = sum_lm O^{rs,X}_lm Mcal_lm(X)), in FP64,
 * on the same tree, pair multipoles and operators as the exchange:
 *   D_dev  [nao x nao] column-major FP64 device density matrix (symmetric,
 *          for closed shells 2 C C^T), leading dimension ldd >= nao
 *   J_dev  [nao x nao] column-major FP64 device output, ldj >= nao: J^ff on
 *          every kept AO pair (both orders), zero elsewhere (near-field and
 *          screened pairs are outside this far field)
 *   Ej_dev FP64 device scalar output (nullable): E_J^ff = 1/2 sum_rs D_rs J_rs
 *   Ej_host FP64 host output (nullable); when non-null the call synchronises
 *          `stream`
 * Requires occk_pair_multipoles on this tree (its rank is used).  Workspaces
 * are owned by the context.  OCCK_ERR_SHAPE if ldd or ldj < nao. */
occk_status occk_farfield_J(occk_ctx* ctx, const occk_tree* tree, const double* D_dev, int ldd, double* J_dev,
                            int ldj, double* Ej_dev, double* Ej_host, void* stream);

/* Engine of the translations (b) M2M, (c) M2L and (d) L2L in the mixed forms
 * (OCCK_TF32 .. OCCK_FP16X3).  mask = -1 (default): chosen by expansion rank
 * and form (the slot pipeline, mask 15, from rank 4 for TF32/BF16/FP16 and
 * from rank 6 for the split forms, whose tensor-core M2L is less accurate than
 * the FP32 SIMT one; all SIMT below);
 * otherwise bit 0 / 1 / 2 puts M2M / M2L / L2L on the tensor core (tcgen05,
 * scaled operands, see Eqs. fmm1-3), the others on SIMT FP32; mask = 0 keeps
 * all three on SIMT with unscaled storage; mask = 15 runs all three on the
 * tensor core with the multipoles and local expansions kept in the tensor
 * core's operand layout between the steps (bulk-copy pipeline, extra device
 * memory of about NP/nc times the FP32 boxes, NP = nc rounded up to a power of
 * two).  Ignored when per-edge ranks are in use (lmax_policy 1 or 2): the
 * translations then stay on SIMT.  OCCK_ERR_ARG for a mask outside -1..7 and
 * 15.  No paper counterpart: an implementation choice. */
occk_status occk_set_translate_engine(occk_ctx* ctx, int mask);

/* M2L pass of the FP32 SIMT translations (occk_farfield_K with any precision
 * other than OCCK_FP64 whose translations run on SIMT; ranks 1-3):
 * mode = 1 runs every level with the sibling-grouped kernel (one block per
 * parent's children, the union of their interaction lists walked once, so a
 * source shared by several siblings is read once); 0 runs the per-target
 * kernel; -1 (default) groups a level when its M2L edges number at least
 * twice its union sources (3-D clusters).  Both give the same sums in the
 * same order (bit-identical K).  Ignored with per-edge ranks (lmax_policy 1,
 * 2).  OCCK_ERR_ARG outside -1..1.  No paper counterpart: an implementation
 * choice. */
occk_status occk_set_m2l_group(occk_ctx* ctx, int mode);

/* K-range splits of step (e): each of nsplit blocks of a tile sums a share of
 * the (lm, j) range into its own copy of the per-leaf K rows, which the K
 * reduction adds up (in a fixed order).  nsplit = 0 (default) chooses enough
 * splits for about eight waves of the grid (four FP64 or two FP32 SIMT blocks,
 * or one tensor-core CTA per SM), at most 8; 1..64 forces a count.
 * OCCK_ERR_ARG outside 0..64.  No paper counterpart: an implementation
 * choice. */
occk_status occk_set_l2p_split(occk_ctx* ctx, int nsplit);

/* A faster FP64-accurate form of OCCK_FP64 that keeps its arithmetic off
 * the FP64 pipe.  The full transform O^{ij,X}_lm = sum_r C_ri O^{rj,X}_lm
 * (Sec. II, Eq. motrans, second line) and the K assembly K^ff_ri = 2 sum_X
 * sum_{j,lm} O^{rj,X}_lm Mcal^{ij}_lm(X) (Eq. kri) run on the tensor core from
 * integer slices: every operand row (step (a): C's orbital columns per leaf,
 * W's orbital columns per leaf and component; step (e): W's AO rows, Mcal's
 * orbital columns per leaf) is scaled by a power of two into (-1, 1) and cut
 * into `slices` integer slices of at most 7 bits (the error-free splitting of
 * Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012) 95); the slice
 * products are summed exactly (small integers on FP16 MMAs, exact FP32 sums per
 * 512 K values, exact integer sums across them) and combined in FP64.  The
 * half transform W = O^{rj,X} (Eq. motrans, first line) and the M2M, M2L and
 * L2L passes (Eqs. fmm1, fmmex, fmm2, fmm3) run in double-FP32 arithmetic on
 * the FP32 pipe (each value hi + lo, each multiply-add an error-free FMA
 * product and TwoSum; with the learned selector the multipoles are joined back
 * to FP64 after M2M for its features); from L = 4 M2L itself runs from slices
 * on the tensor core as well (occk_set_fp64_slice_m2l).  The reductions and
 * the energy stay FP64.  The result differs
 * from the DFMA form by the slices' truncation, relative to the largest
 * entries of each row and column about 2^-49 per product for 7 slices and
 * 2^-42 for 6 (measured on K: about 1.6e-12 and 1.3e-10 of max|K|; E within
 * about 1e-14 Eh).  slices = 0 (default) keeps the DFMA kernels; 6 or 7
 * enable the form for calls with prec = OCCK_FP64 and no pair screening or
 * column block (those keep the DFMA kernels).  Workspace: the slice panels of
 * a batch of leaves (about 14 x slices bytes per (stored AO row or leaf
 * orbital) x n_occ x (L+1)^2 in all, 18 GB for 3577 AOs, 660 orbitals, L = 2,
 * 7 slices; batches keep it within occk_set_slice_workspace's budget), and
 * double-FP32 copies of C, the pair values and the operators, allocated on
 * the next call and released (after a device synchronisation) when the form
 * is turned off with slices = 0 (and the FP32 form below is off too).  OCCK_ERR_ARG for other values.  No
 * paper counterpart: an implementation choice of this library. */
occk_status occk_set_fp64_slices(occk_ctx* ctx, int slices);

/* Steps (a) (full transform, Eq. motrans) and (e) (Eq. kri) of the OCCK_FP32
 * form on the tensor core from 4 integer slices per operand, with the same
 * engine as occk_set_fp64_slices: 4 slices of at most 7 bits hold every FP32
 * operand within 2^-28 of its row's largest entry (exactly where the row's
 * entries are within a factor 16 of each other), the slice products are summed
 * exactly and combined in FP64, so these two steps carry no FP32 rounding and
 * no bias of the tensor core's accumulation; the half transform, M2M, M2L and
 * L2L stay FP32 SIMT.  slices = 0 (default) keeps the FP32 SIMT GEMMs; 4
 * enables the form for calls with prec = OCCK_FP32 and no pair screening or
 * column block.  Workspace as for occk_set_fp64_slices (4/7 of it per leaf
 * batch), released when both forms are off.  OCCK_ERR_ARG for other values.
 * No paper counterpart: an implementation choice of this library. */
occk_status occk_set_fp32_slices(occk_ctx* ctx, int slices);

/* M2L (Eqs. fmmex, fmm2) of the occk_set_fp64_slices form from integer
 * slices on the tensor core as well (on = 1, the default), for expansions of
 * at least 25 components (L >= 4; below that the double-FP32 pass is used):
 * per level, the sources' expansions and the operators are split into the
 * same number of 7-bit slices after exact power-of-two scalings (per
 * component and pair for the expansions, per output component for the
 * operators), the slice products are summed exactly and combined in FP64, and
 * the parent's L2L is then added in double-FP32.  Learned or set per-edge
 * ranks use the operators restricted to each edge's rank.  The workspace is
 * the slice panels' (occk_set_slice_workspace bounds it; the pairs are taken
 * in batches of 128-pair tiles).  on = 0 keeps the double-FP32 M2L.
 * OCCK_ERR_ARG for other values.  No paper counterpart. */
occk_status occk_set_fp64_slice_m2l(occk_ctx* ctx, int on);

/* Largest workspace of slice panels of the forms above, in bytes (0, the
 * default: 32 GB).  The leaves are processed in batches whose panels fit
 * (a leaf larger than the budget is a batch of its own); the result does not
 * depend on the batching (each output tile is computed the same way).
 * OCCK_ERR_ARG for bytes < 0.  No paper counterpart. */
occk_status occk_set_slice_workspace(occk_ctx* ctx, long long bytes);

/* D = A B^T on the tensor-core engine used by the mixed forms, for checking
 * it: A [M x K], B [N x K], D [M x N], all FP32 row-major device buffers; prec
 * one of OCCK_TF32, _BF16, _FP16, _BF16X3, _FP16X3.  Synchronises `stream`. */
occk_status occk_debug_tc_gemm(occk_ctx* ctx, int prec, int M, int N, int K, const float* A,
                               const float* B, float* D, void* stream);

/* Sustained FMA throughput of this device for one arithmetic (prec =
 * OCCK_FP64 or OCCK_FP32), measured by a kernel in which every thread updates
 * 8, 16 or 32 independent accumulators (four FMAs on each per loop trip; two
 * operand patterns: a = a m + c and a = b m + a), at 4 and 8 resident
 * 256-thread blocks per SM; *flops receives the best rate seen, in FLOP/s (2
 * per FMA), at whatever SM clock the device runs.
 * Synchronises `stream`.  A measurement aid for roofline reporting, not part
 * of the exchange path. */
occk_status occk_probe_fma_peak(occk_ctx* ctx, int prec, double* flops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OCCK_H */
