"""Thin ctypes binding of ``include/occk.h`` (argument marshalling only).

Every function here forwards to the C ABI of ``libocck.so``; no step of the
far-field exchange runs in Python.  PyTorch supplies device memory and the
current CUDA stream.  If the shared library is missing the import fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libocck.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "occk.h")

OCCK_FP64, OCCK_FP32, OCCK_TF32, OCCK_BF16, OCCK_FP16, OCCK_BF16X3, OCCK_FP16X3 = range(7)
PRECISIONS = {"fp64": OCCK_FP64, "fp32": OCCK_FP32, "tf32": OCCK_TF32, "bf16": OCCK_BF16,
              "fp16": OCCK_FP16, "bf16x3": OCCK_BF16X3, "fp16x3": OCCK_FP16X3}
TREE_ARRAYS = {"level_off": 0, "box_key": 1, "parent": 2, "centre": 3, "m2l": 4, "pairs": 5,
               "pair_centre": 6, "leaf_aos": 7, "leaf_rowoff": 8}
DBG = {"pair_mult": 0, "obox": 1, "mbox": 2, "screen_tiles": 3}
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_SHAPE", -3: "ERR_CUDA", -4: "ERR_OOM",
          -5: "ERR_TIMEOUT", -6: "ERR_UNSUPPORTED", -7: "ERR_STATE"}


class OcckError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Basis(ctypes.Structure):
    _fields_ = [("natom", ctypes.c_int), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("nshell", ctypes.c_int), ("shell_atom", ctypes.POINTER(ctypes.c_int)),
                ("shell_l", ctypes.POINTER(ctypes.c_int)), ("shell_nprim", ctypes.POINTER(ctypes.c_int)),
                ("exps", ctypes.POINTER(ctypes.c_double)), ("coefs", ctypes.POINTER(ctypes.c_double))]


class _TreeParams(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("target_atoms_per_leaf", ctypes.c_double),
                ("ws_boxes", ctypes.c_int), ("pair_thresh", ctypes.c_double)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("nao", ctypes.c_int), ("natom", ctypes.c_int), ("nshell", ctypes.c_int),
                ("depth", ctypes.c_int), ("nbox", ctypes.c_int), ("nleaf", ctypes.c_int),
                ("npair", ctypes.c_int), ("nentry", ctypes.c_int), ("nrow", ctypes.c_int),
                ("nm2l", ctypes.c_int), ("lmax", ctypes.c_int), ("x0", ctypes.c_double * 3),
                ("side", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["x0"] = list(self.x0)
        return d


_lib = None
_vp = ctypes.c_void_p
_SIGS = {
    "occk_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
    "occk_destroy": (None, [_vp]),
    "occk_last_error": (ctypes.c_char_p, [_vp]),
    "occk_build_tree": (ctypes.c_int, [_vp, ctypes.POINTER(_Basis), ctypes.POINTER(_TreeParams),
                                       ctypes.POINTER(_vp)]),
    "occk_tree_destroy": (None, [_vp]),
    "occk_query": (ctypes.c_int, [_vp, ctypes.POINTER(TreeInfo)]),
    "occk_tree_export": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t]),
    "occk_pair_multipoles": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "occk_set_edge_lmax": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "occk_farfield_K": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp]),
    "occk_debug_fetch": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "occk_probe_fma_peak": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]),
    "occk_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_set_translate_engine": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_batch_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "occk_set_l2p_split": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_set_fp64_slices": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_set_slice_workspace": (ctypes.c_int, [_vp, ctypes.c_longlong]),
    "occk_set_fp64_slice_m2l": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_set_fp32_slices": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_set_pair_screen": (ctypes.c_int, [_vp, ctypes.c_double]),
    "occk_pair_screen_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong), _vp]),
    "occk_farfield_J": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                       ctypes.POINTER(ctypes.c_double), _vp]),
    "occk_device_status": (ctypes.c_int, [_vp, _vp]),
    "occk_batch_create": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_int, ctypes.POINTER(_vp)]),
    "occk_batch_destroy": (None, [_vp]),
    "occk_batch_buffers": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp)]),
    "occk_batch_run": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "occk_batch_tune": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), _vp]),
    "occk_mlp_init": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "occk_mlp_set": (ctypes.c_int, [_vp, _vp, _vp]),
    "occk_mlp_get": (ctypes.c_int, [_vp, _vp, _vp]),
    "occk_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.POINTER(ctypes.c_float), _vp]),
    "occk_mlp_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_float), _vp]),
    "occk_mlp_predict": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "occk_edge_features": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "occk_edge_energies": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "occk_set_learned_tau": (ctypes.c_int, [_vp, ctypes.c_double]),
    "occk_get_edge_ranks": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "occk_debug_tc_gemm": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                          _vp, _vp]),
    "occk_exchange_energy_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                                    ctypes.c_int, _vp, _vp]),
    "occk_get_timings": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "occk_debug_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_longlong]),
    "occk_set_column_block": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "occk_set_m2l_group": (ctypes.c_int, [_vp, ctypes.c_int]),
    "occk_exchange_energy": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                            ctypes.c_int, _vp, _vp]),
}
NSTAGE = 7
MLP_NIN, MLP_HIDDEN, MLP_NOUT = 16, 64, 8
MLP_NPARAM = MLP_NIN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_NOUT + MLP_NOUT
MLP_NNORM = 2 * MLP_NIN + 2 * MLP_NOUT
STAGES = ["a_half", "a_full", "b_m2m", "c_m2l", "d_l2l", "e_l2p", "reduce"]


def header_functions():
    """Names of the functions declared in include/occk.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(occk_[A-Za-z0-9_]+)\s*\(", src)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    ct = ctypes.c_double if dtype == np.float64 else ctypes.c_int
    return a, a.ctypes.data_as(ctypes.POINTER(ct))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """occk_ctx: device = -1 gives a host-only context (trees only)."""

    def __init__(self, device: int = 0):
        self._h = _vp()
        rc = lib().occk_create(ctypes.byref(self._h), device)
        if rc != 0:
            raise OcckError(rc, f"occk_create(device={device})")
        self.device = device

    def check(self, rc, what):
        if rc != 0:
            msg = lib().occk_last_error(self._h)
            raise OcckError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if self._h:
            lib().occk_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_translate_engine(self, mask: int = -1):
        """Translations of the mixed forms on the tensor core: bit 0 M2M, bit 1
        M2L, bit 2 L2L; 15: all three with the expansions kept in the tensor
        core's operand layout; -1 chooses by expansion rank."""
        self.check(lib().occk_set_translate_engine(self._h, int(mask)), "occk_set_translate_engine")

    def set_m2l_group(self, mode: int = -1):
        """Sibling-grouped FP32 M2L: 1 always, 0 never, -1 by the level's
        sharing of interaction-list sources."""
        self.check(lib().occk_set_m2l_group(self._h, int(mode)), "occk_set_m2l_group")

    def set_l2p_split(self, nsplit: int = 0):
        """K-range splits of the FP32 SIMT step (e); 0 chooses automatically."""
        self.check(lib().occk_set_l2p_split(self._h, int(nsplit)), "occk_set_l2p_split")

    def set_fp64_slices(self, slices: int = 0):
        """FP64 steps (a) and (e) from integer slices on the tensor core (6
        or 7 slices; 0: the DFMA kernels)."""
        self.check(lib().occk_set_fp64_slices(self._h, int(slices)), "occk_set_fp64_slices")

    def set_fp32_slices(self, slices: int = 0):
        """FP32 steps (a) and (e) from 4 integer slices on the tensor core
        with exact sums (0: the FP32 SIMT GEMMs)."""
        self.check(lib().occk_set_fp32_slices(self._h, int(slices)), "occk_set_fp32_slices")

    def set_fp64_slice_m2l(self, on: bool = True):
        """M2L of the FP64-accurate sliced form from slices too (L >= 4)."""
        self.check(lib().occk_set_fp64_slice_m2l(self._h, int(bool(on))), "occk_set_fp64_slice_m2l")

    def set_slice_workspace(self, nbytes: int = 0):
        """Largest slice-panel workspace of the sliced FP64 form (0: 32 GB)."""
        self.check(lib().occk_set_slice_workspace(self._h, int(nbytes)), "occk_set_slice_workspace")

    def set_pair_screen(self, tau: float = 0.0):
        """Occupied-pair screening threshold for occk_farfield_K (0: off)."""
        self.check(lib().occk_set_pair_screen(self._h, float(tau)), "occk_set_pair_screen")

    def set_column_block(self, i0: int = 0, i1: int = 0):
        """Occupied column block [i0, i1) of later far-field calls (0, 0: off)."""
        self.check(lib().occk_set_column_block(self._h, int(i0), int(i1)), "occk_set_column_block")

    def pair_screen_count(self, stream=None) -> int:
        """Pairs i <= j kept by the last occk_farfield_K (-1 if it did not screen)."""
        n = ctypes.c_longlong()
        self.check(lib().occk_pair_screen_count(self._h, ctypes.byref(n), _stream_ptr(stream)),
                   "occk_pair_screen_count")
        return n.value

    def debug_set_wait_limit(self, polls: int = -1):
        """Polls of the tensor-core GEMMs' operand wait before it gives up
        (test aid; -1 restores the default).  Applies to the whole device."""
        self.check(lib().occk_debug_set_wait_limit(self._h, int(polls)), "occk_debug_set_wait_limit")

    def set_timing(self, on: bool):
        self.check(lib().occk_set_timing(self._h, 1 if on else 0), "occk_set_timing")

    def timings(self) -> dict:
        ms = (ctypes.c_float * NSTAGE)()
        self.check(lib().occk_get_timings(self._h, ms, NSTAGE), "occk_get_timings")
        return dict(zip(STAGES, [float(x) for x in ms]))

    def probe_fma_peak(self, prec="fp64", stream=None) -> float:
        out = ctypes.c_double()
        self.check(lib().occk_probe_fma_peak(self._h, PRECISIONS[prec], ctypes.byref(out),
                                             _stream_ptr(stream)), "occk_probe_fma_peak")
        return out.value


class Tree:
    """occk_tree built from a ``paper_1708_05353_gb300.inputs.Basis``."""

    def __init__(self, ctx: Context, basis, depth: int = 0, target_atoms_per_leaf: float = 8.0,
                 pair_thresh: float = 1e-14):
        self.ctx = ctx
        keep = []
        xyz, pxyz = _arr(basis.xyz, np.float64)
        sa, psa = _arr(basis.shell_atom, np.int32)
        sl, psl = _arr(basis.shell_l, np.int32)
        sn, psn = _arr(basis.shell_nprim, np.int32)
        ex, pex = _arr(basis.exps, np.float64)
        co, pco = _arr(basis.coefs, np.float64)
        keep += [xyz, sa, sl, sn, ex, co]
        b = _Basis(basis.natom, pxyz, basis.nshell, psa, psl, psn, pex, pco)
        p = _TreeParams(depth, target_atoms_per_leaf, 1, pair_thresh)
        self._h = _vp()
        ctx.check(lib().occk_build_tree(ctx._h, ctypes.byref(b), ctypes.byref(p), ctypes.byref(self._h)),
                  "occk_build_tree")
        self.nao = int(basis.nao)

    def close(self):
        if self._h:
            lib().occk_tree_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = TreeInfo()
        self.ctx.check(lib().occk_query(self._h, ctypes.byref(inf)), "occk_query")
        return inf.as_dict()

    def export(self, what: str) -> np.ndarray:
        inf = self.info()
        shapes = {"level_off": ((inf["depth"] + 2,), np.int32), "box_key": ((inf["nbox"], 3), np.int32),
                  "parent": ((inf["nbox"],), np.int32), "centre": ((inf["nbox"], 3), np.float64),
                  "m2l": ((inf["nm2l"], 2), np.int32), "pairs": ((inf["npair"], 3), np.int32),
                  "pair_centre": ((inf["npair"], 3), np.float64), "leaf_aos": ((inf["nrow"],), np.int32),
                  "leaf_rowoff": ((inf["nleaf"] + 1,), np.int32)}
        shape, dt = shapes[what]
        out = np.zeros(shape, dtype=dt)
        self.ctx.check(lib().occk_tree_export(self._h, TREE_ARRAYS[what], out.ctypes.data_as(_vp),
                                              out.nbytes), "occk_tree_export")
        return out

    def pair_multipoles(self, lmax: int, stream=None):
        self.ctx.check(lib().occk_pair_multipoles(self.ctx._h, self._h, lmax, _stream_ptr(stream)),
                       "occk_pair_multipoles")

    def set_edge_lmax(self, ranks):
        r = np.ascontiguousarray(ranks, dtype=np.int32)
        self.ctx.check(lib().occk_set_edge_lmax(self.ctx._h, self._h,
                                                r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(r)),
                       "occk_set_edge_lmax")


def fortran(t):
    """Column-major view of a 2-D tensor (copy only when needed)."""
    if t.dim() == 2 and (t.stride(0) == 1 or t.shape[0] == 1) and ld(t) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def ld(t):
    """Leading dimension of a column-major 2-D tensor (a single column has
    no meaningful column stride; use the row count)."""
    return t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])


def empty_fortran(nrow, ncol, dtype=None, device=None):
    import torch
    return torch.empty((ncol, nrow), dtype=dtype or torch.float64, device=device).t()


def _is_fortran(t):
    return t.dim() == 2 and (t.stride(0) == 1 or t.shape[0] == 1) and ld(t) >= max(1, t.shape[0])


def _on_ctx_device(ctx, t):
    return bool(getattr(t, "is_cuda", False)) and ctx.device >= 0 and t.device.index == ctx.device


def _check_matrix(ctx, name, t, shape=None, nrow=None, device=True):
    """Raise OcckError before any library call unless t is a 2-D float64
    tensor of the expected shape on the context's device (the C ABI receives
    bare pointers and cannot check any of this)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64:
        raise OcckError(-1, f"{name} must be a float64 torch tensor, got {getattr(t, 'dtype', type(t))}")
    if t.dim() != 2 or (shape is not None and tuple(t.shape) != tuple(shape)) or \
            (nrow is not None and t.shape[0] != nrow) or t.shape[0] < 1 or t.shape[1] < 1:
        want = shape if shape is not None else (f"[{nrow}, n]" if nrow is not None else "2-D, non-empty")
        raise OcckError(-2, f"{name} has shape {tuple(t.shape)}, expected {want}")
    if device and not _on_ctx_device(ctx, t):
        raise OcckError(-1, f"{name} is on {t.device}, the context is bound to cuda:{ctx.device}")


def _check_scalar(ctx, name, t, device=True):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.dim() != 0:
        raise OcckError(-1, f"{name} must be a 0-d float64 tensor")
    if device and not _on_ctx_device(ctx, t):
        raise OcckError(-1, f"{name} is on {t.device}, the context is bound to cuda:{ctx.device}")


def farfield_K(ctx: Context, tree: Tree, C, prec="fp64", lmax_policy: int = 0, K=None, Ex=None,
               want_energy_host: bool = False, stream=None):
    """occk_farfield_K on torch CUDA tensors.  C: [nao, nocc] float64 (any
    layout; a column-major copy is made if needed).  Returns (K, Ex) with K
    column-major [nao, nocc] and Ex a 0-d device tensor (or a float when
    want_energy_host)."""
    import torch
    nao = tree.nao
    for dev in (False, True):          # dtypes and shapes first, then devices
        _check_matrix(ctx, "C", C, nrow=nao, device=dev)
        if K is not None:
            _check_matrix(ctx, "K", K, shape=tuple(C.shape), device=dev)
        if Ex is not None:
            _check_scalar(ctx, "Ex", Ex, device=dev)
    C = fortran(C)
    nocc = C.shape[1]
    if K is None:
        K = empty_fortran(nao, nocc, torch.float64, C.device)
    elif not _is_fortran(K):
        raise OcckError(-2, "K must be a column-major [nao, nocc] view (see empty_fortran)")
    if Ex is None:
        Ex = torch.empty((), dtype=torch.float64, device=C.device)
    eh = ctypes.c_double()
    rc = lib().occk_farfield_K(ctx._h, tree._h, nocc, _vp(C.data_ptr()), ld(C),
                               PRECISIONS[prec] if isinstance(prec, str) else int(prec), lmax_policy,
                               _vp(K.data_ptr()), ld(K), _vp(Ex.data_ptr()),
                               ctypes.byref(eh) if want_energy_host else None, _stream_ptr(stream))
    ctx.check(rc, "occk_farfield_K")
    return K, (eh.value if want_energy_host else Ex)


def farfield_J(ctx: Context, tree: Tree, D, J=None, Ej=None, want_energy_host: bool = False, stream=None):
    """occk_farfield_J on torch CUDA tensors.  D: [nao, nao] float64 symmetric
    density (a column-major copy is made if needed).  Returns (J, Ej) with J
    column-major [nao, nao] and Ej a 0-d device tensor (or a float when
    want_energy_host)."""
    import torch
    nao = tree.nao
    for dev in (False, True):
        _check_matrix(ctx, "D", D, shape=(nao, nao), device=dev)
        if J is not None:
            _check_matrix(ctx, "J", J, shape=(nao, nao), device=dev)
        if Ej is not None:
            _check_scalar(ctx, "Ej", Ej, device=dev)
    if J is not None and not _is_fortran(J):
        raise OcckError(-2, "J must be a column-major [nao, nao] view (see empty_fortran)")
    D = fortran(D)
    if J is None:
        J = empty_fortran(nao, nao, torch.float64, D.device)
    if Ej is None:
        Ej = torch.empty((), dtype=torch.float64, device=D.device)
    eh = ctypes.c_double()
    rc = lib().occk_farfield_J(ctx._h, tree._h, _vp(D.data_ptr()), ld(D), _vp(J.data_ptr()), ld(J),
                               _vp(Ej.data_ptr()), ctypes.byref(eh) if want_energy_host else None,
                               _stream_ptr(stream))
    ctx.check(rc, "occk_farfield_J")
    return J, (eh.value if want_energy_host else Ej)


# ---- batches ---------------------------------------------------------------------

class Batch:
    """occk_batch over trees (each with pair multipoles at the same lmax)."""

    def __init__(self, ctx: Context, trees, noccs, prec="fp32"):
        self.ctx = ctx
        self.trees = list(trees)
        arr = (_vp * len(trees))(*[t._h for t in trees])
        no = (ctypes.c_int * len(trees))(*noccs)
        self._h = _vp()
        ctx.check(lib().occk_batch_create(ctx._h, len(trees), arr, no, PRECISIONS[prec], ctypes.byref(self._h)),
                  "occk_batch_create")
        self.noccs = list(noccs)

    def buffers(self, sys):
        """(C, K, E) as torch views of the batch-owned device buffers."""
        import torch
        c, k, e = _vp(), _vp(), _vp()
        ld = ctypes.c_int()
        self.ctx.check(lib().occk_batch_buffers(self._h, sys, ctypes.byref(c), ctypes.byref(k), ctypes.byref(ld),
                                                ctypes.byref(e)), "occk_batch_buffers")
        return c.value, k.value, e.value, ld.value

    def run(self, use_graph=True, stream=None):
        self.ctx.check(lib().occk_batch_run(self._h, 1 if use_graph else 0, _stream_ptr(stream)), "occk_batch_run")

    def tune(self, cache_path=None, stream=None):
        cfg = (ctypes.c_int * 4)()
        self.ctx.check(lib().occk_batch_tune(self._h, cache_path.encode() if cache_path else None, cfg,
                                             _stream_ptr(stream)), "occk_batch_tune")
        return dict(chunk=cfg[0], blocks_per_sm=cfg[1], tile=cfg[2], mode=cfg[3])

    def set_config(self, chunk=9, blocks_per_sm=8, tile=128, mode=0):
        """Configuration without tuning (the values occk_batch_tune reports)."""
        cfg = (ctypes.c_int * 4)(chunk, blocks_per_sm, tile, mode)
        self.ctx.check(lib().occk_batch_set_config(self._h, cfg), "occk_batch_set_config")

    def close(self):
        if self._h:
            lib().occk_batch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_view(ptr, shape, dtype, device, strides=None):
    """A torch tensor aliasing library-owned device memory (no copy)."""
    import torch
    n = int(np.prod(shape))
    itemsize = torch.tensor([], dtype=dtype).element_size()

    class _Holder:
        __cuda_array_interface__ = {"shape": (n,), "typestr": {8: "<f8", 4: "<f4"}[itemsize],
                                    "data": (ptr, False), "version": 2}
    flat = torch.as_tensor(_Holder(), device=device)
    if strides is None:
        return flat.view(shape)
    return flat.as_strided(shape, strides)


# ---- learned rank selector --------------------------------------------------

def mlp_init(ctx: Context, seed: int = 1):
    ctx.check(lib().occk_mlp_init(ctx._h, seed), "occk_mlp_init")


def mlp_set(ctx: Context, params, norm):
    p = np.ascontiguousarray(params, dtype=np.float32)
    n = np.ascontiguousarray(norm, dtype=np.float32)
    assert p.size == MLP_NPARAM and n.size == MLP_NNORM
    ctx.check(lib().occk_mlp_set(ctx._h, p.ctypes.data_as(_vp), n.ctypes.data_as(_vp)), "occk_mlp_set")


def mlp_get(ctx: Context):
    p = np.zeros(MLP_NPARAM, dtype=np.float32)
    n = np.zeros(MLP_NNORM, dtype=np.float32)
    ctx.check(lib().occk_mlp_get(ctx._h, p.ctypes.data_as(_vp), n.ctypes.data_as(_vp)), "occk_mlp_get")
    return p, n


def mlp_train(ctx: Context, X, T, steps: int, lr: float, stream=None) -> float:
    loss = ctypes.c_float()
    ctx.check(lib().occk_mlp_train(ctx._h, _vp(X.data_ptr()), _vp(T.data_ptr()), X.shape[0], steps, lr,
                                   ctypes.byref(loss), _stream_ptr(stream)), "occk_mlp_train")
    return loss.value


def mlp_grad(ctx: Context, X, T, stream=None):
    import torch
    g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
    loss = ctypes.c_float()
    ctx.check(lib().occk_mlp_grad(ctx._h, _vp(X.data_ptr()), _vp(T.data_ptr()), X.shape[0], _vp(g.data_ptr()),
                                  ctypes.byref(loss), _stream_ptr(stream)), "occk_mlp_grad")
    return loss.value, g


def mlp_predict(ctx: Context, X, stream=None):
    import torch
    Y = torch.empty((X.shape[0], MLP_NOUT), dtype=torch.float32, device=X.device)
    ctx.check(lib().occk_mlp_predict(ctx._h, _vp(X.data_ptr()), X.shape[0], _vp(Y.data_ptr()),
                                     _stream_ptr(stream)), "occk_mlp_predict")
    return Y


def edge_features(ctx: Context, tree: Tree, stream=None):
    import torch
    n = tree.info()["nm2l"]
    F = torch.empty((max(n, 1), MLP_NIN), dtype=torch.float32, device=f"cuda:{ctx.device}")
    ctx.check(lib().occk_edge_features(ctx._h, tree._h, _vp(F.data_ptr()), _stream_ptr(stream)),
              "occk_edge_features")
    return F[:n]


def edge_energies(ctx: Context, tree: Tree, stream=None):
    import torch
    inf = tree.info()
    E = torch.empty((max(inf["nm2l"], 1), inf["lmax"] + 1), dtype=torch.float64, device=f"cuda:{ctx.device}")
    ctx.check(lib().occk_edge_energies(ctx._h, tree._h, _vp(E.data_ptr()), _stream_ptr(stream)),
              "occk_edge_energies")
    return E[:inf["nm2l"]]


def set_learned_tau(ctx: Context, tau: float):
    ctx.check(lib().occk_set_learned_tau(ctx._h, tau), "occk_set_learned_tau")


def edge_ranks(ctx: Context, tree: Tree):
    n = tree.info()["nm2l"]
    r = np.zeros(max(n, 1), dtype=np.int32)
    ctx.check(lib().occk_get_edge_ranks(ctx._h, tree._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n),
              "occk_get_edge_ranks")
    return r[:n]


def debug_tc_gemm(ctx: Context, prec: str, A, B, stream=None):
    """D = A B^T on the tensor-core engine (A [M,K], B [N,K] float32 CUDA)."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    D = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float32, device=A.device)
    ctx.check(lib().occk_debug_tc_gemm(ctx._h, PRECISIONS[prec], A.shape[0], B.shape[0], A.shape[1],
                                       _vp(A.data_ptr()), _vp(B.data_ptr()), _vp(D.data_ptr()),
                                       _stream_ptr(stream)), "occk_debug_tc_gemm")
    return D


def device_status(ctx: Context, stream=None):
    ctx.check(lib().occk_device_status(ctx._h, _stream_ptr(stream)), "occk_device_status")


def exchange_energy(ctx: Context, C, K, E=None, stream=None):
    """occk_exchange_energy on column-major torch CUDA tensors: -1/2 sum C*K
    with the reduction order of occk_farfield_K's energy.  Returns E (0-d
    device tensor)."""
    import torch
    for dev in (False, True):
        _check_matrix(ctx, "C", C, device=dev)
        _check_matrix(ctx, "K", K, shape=tuple(C.shape), device=dev)
        if E is not None:
            _check_scalar(ctx, "E", E, device=dev)
    C = fortran(C)
    K = fortran(K)
    nao, nocc = C.shape
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=C.device)
    ctx.check(lib().occk_exchange_energy(ctx._h, nao, nocc, _vp(C.data_ptr()), ld(C), _vp(K.data_ptr()), ld(K),
                                         _vp(E.data_ptr()), _stream_ptr(stream)), "occk_exchange_energy")
    return E


def exchange_energy_noalloc(ctx: Context, C, K, E=None, stream=None):
    """occk_exchange_energy_noalloc on column-major torch CUDA tensors: the
    energy -1/2 sum C*K with its scratch in a static device array (the
    library allocates no device memory in this call).  Returns E (0-d device
    tensor; allocate it yourself and pass it in to avoid torch allocating)."""
    import torch
    for dev in (False, True):
        _check_matrix(ctx, "C", C, device=dev)
        _check_matrix(ctx, "K", K, shape=tuple(C.shape), device=dev)
        if E is not None:
            _check_scalar(ctx, "E", E, device=dev)
    C = fortran(C)
    K = fortran(K)
    nao, nocc = C.shape
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=C.device)
    ctx.check(lib().occk_exchange_energy_noalloc(ctx._h, nao, nocc, _vp(C.data_ptr()), ld(C),
                                                 _vp(K.data_ptr()), ld(K), _vp(E.data_ptr()),
                                                 _stream_ptr(stream)), "occk_exchange_energy_noalloc")
    return E


def debug_fetch(ctx: Context, tree: Tree, what: str, nocc: int = 0, stream=None) -> np.ndarray:
    inf = tree.info()
    nc = (inf["lmax"] + 1) ** 2
    if what == "screen_tiles":
        out = np.zeros(2, dtype=np.int32)
        ctx.check(lib().occk_debug_fetch(ctx._h, tree._h, DBG[what], out.ctypes.data_as(_vp), out.nbytes,
                                         _stream_ptr(stream)), "occk_debug_fetch")
        return out
    if what == "pair_mult":
        n = None
        # number of value rows: sum over kept pairs of na*nb
        pairs = tree.export("pairs")
        l = _shell_l_cache.get(id(tree))
        if l is None:
            raise ValueError("call debug_fetch_pair_mult with shell_l")
        n = int(sum((3 if l[a] else 1) * (3 if l[b] else 1) for a, b, _ in pairs))
        out = np.zeros((n, nc))
    else:
        out = np.zeros((inf["nbox"], nc, nocc * nocc))
    ctx.check(lib().occk_debug_fetch(ctx._h, tree._h, DBG[what], out.ctypes.data_as(_vp), out.nbytes,
                                     _stream_ptr(stream)), "occk_debug_fetch")
    return out


_shell_l_cache = {}


def debug_fetch_pair_mult(ctx: Context, tree: Tree, shell_l, stream=None) -> np.ndarray:
    _shell_l_cache[id(tree)] = np.asarray(shell_l)
    try:
        return debug_fetch(ctx, tree, "pair_mult", stream=stream)
    finally:
        _shell_l_cache.pop(id(tree), None)
