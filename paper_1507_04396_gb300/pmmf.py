"""Thin Python binding of the pMMF C-ABI (``include/pmmf.h``).

Argument marshalling only: every step of the factorization, the matrix-free
apply and the preconditioned CG runs inside ``_lib/libpmmf.so``.  The functions
``pmmf_factor``, ``pmmf_apply``, ``pmmf_solve_precond`` and ``pmmf_free`` keep
the C names; ``Factorization`` wraps a handle for convenience.  Arrays are torch
tensors (device data) or numpy arrays (host data).  Importing this module
fails loudly when the compiled library is missing.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpmmf.so")

OK, ERR_INVALID_ARG, ERR_NOT_SYMMETRIC, ERR_NONFINITE, ERR_OOM, ERR_CUDA = 0, 1, 2, 3, 4, 5
ERR_NOT_SPD, ERR_SINGULAR_CORE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = 6, 7, 8, 9, 10
HOST, DEVICE = 0, 1
CSR, DENSE = 0, 1
OP_A, OP_A_INV, OP_U, OP_UT, OP_H, OP_H_INV = 0, 1, 2, 3, 4, 5
OP_A_INV_SQRT, OP_H_INV_SQRT = 6, 7
PREC_FP64, PREC_TF32, PREC_BF16 = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SYMMETRIC", 3: "NONFINITE", 4: "OOM",
                5: "CUDA", 6: "NOT_SPD", 7: "SINGULAR_CORE", 8: "NOT_CONVERGED", 9: "TIMEOUT",
                10: "UNSUPPORTED"}


class PmmfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"pmmf status {status} ({STATUS_NAMES.get(status, '?')}): {message}")
        self.status = status


class Matrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("format", C.c_int), ("location", C.c_int),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("val", C.c_void_p),
                ("ld", C.c_int64)]


class Params(C.Structure):
    _fields_ = [("k", C.c_int), ("eta", C.c_double), ("cluster_size", C.c_int),
                ("core_size", C.c_int), ("seed", C.c_uint64), ("max_stages", C.c_int),
                ("lloyd_iters", C.c_int), ("coords", C.c_void_p), ("coord_dim", C.c_int),
                ("coords_location", C.c_int), ("record_stages", C.c_int),
                ("precision", C.c_int), ("labels", C.c_void_p), ("labels_location", C.c_int),
                ("num_labels", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("stages", C.c_int32), ("core_size", C.c_int64),
                ("rotations", C.c_int64), ("nnz_input", C.c_int64), ("norm_a", C.c_double),
                ("error", C.c_double)]


class StageInfo(C.Structure):
    _fields_ = [("active", C.c_int64), ("clusters", C.c_int64), ("rotations", C.c_int64),
                ("nnz_after", C.c_int64), ("max_levels", C.c_int32), ("contrib", C.c_double)]


EXPORTS = ["pmmf_factor", "pmmf_apply", "pmmf_solve_precond", "pmmf_free", "pmmf_last_error",
           "pmmf_profile_begin", "pmmf_profile_end", "pmmf_profile_records", "pmmf_apply_noalloc",
           "pmmf_get_info", "pmmf_get_stage_info", "pmmf_get_stage_clusters",
           "pmmf_get_stage_rotations", "pmmf_get_h", "pmmf_get_stage_matrix",
           "pmmf_launch_count", "pmmf_alloc_count", "pmmf_probe_fp64", "pmmf_gram_reduced",
           "pmmf_apply_backward", "pmmf_get_angles", "pmmf_set_angles",
           "pmmf_set_h", "pmmf_factor_blockdiag", "pmmf_factor_batched", "pmmf_get_batch",
           "pmmf_get_precision_stats", "pmmf_set_tuning", "pmmf_clear_tuning",
           "pmmf_solve_precond_sym", "pmmf_block_angle_grad", "pmmf_shard_create",
           "pmmf_shard_clusters", "pmmf_shard_search", "pmmf_shard_transform",
           "pmmf_shard_result", "pmmf_shard_sumsq", "pmmf_shard_free"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"pMMF CUDA library not built: {path} is missing "
                          "(run paper_1507_04396_gb300.build.build())")
    L = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.pmmf_factor.restype = i32
    L.pmmf_factor.argtypes = [C.POINTER(Matrix), C.POINTER(Params), C.POINTER(vp), vp]
    L.pmmf_apply.restype = i32
    L.pmmf_apply.argtypes = [vp, i32, vp, vp, i64, i64, vp]
    L.pmmf_solve_precond.restype = i32
    L.pmmf_solve_precond.argtypes = [vp, C.POINTER(Matrix), vp, vp, i64, f64, i32, vp, vp, vp]
    L.pmmf_solve_precond_sym.restype = i32
    L.pmmf_solve_precond_sym.argtypes = [vp, C.POINTER(Matrix), vp, vp, i64, f64, i32, vp, vp, vp]
    L.pmmf_free.restype = None
    L.pmmf_free.argtypes = [vp]
    L.pmmf_last_error.restype = C.c_char_p
    L.pmmf_last_error.argtypes = []
    L.pmmf_get_info.restype = i32
    L.pmmf_get_info.argtypes = [vp, C.POINTER(Info)]
    L.pmmf_get_stage_info.restype = i32
    L.pmmf_get_stage_info.argtypes = [vp, i32, C.POINTER(StageInfo)]
    L.pmmf_get_stage_clusters.restype = i32
    L.pmmf_get_stage_clusters.argtypes = [vp, i32, vp, vp]
    L.pmmf_get_stage_rotations.restype = i32
    L.pmmf_get_stage_rotations.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.pmmf_get_h.restype = i32
    L.pmmf_get_h.argtypes = [vp, vp, vp, vp]
    L.pmmf_get_stage_matrix.restype = i32
    L.pmmf_get_stage_matrix.argtypes = [vp, i32, vp, vp, vp, vp]
    L.pmmf_launch_count.restype = C.c_uint64
    L.pmmf_launch_count.argtypes = []
    L.pmmf_alloc_count.restype = C.c_uint64
    L.pmmf_alloc_count.argtypes = []
    L.pmmf_probe_fp64.restype = i32
    L.pmmf_probe_fp64.argtypes = [vp, vp]
    L.pmmf_gram_reduced.restype = i32
    L.pmmf_gram_reduced.argtypes = [vp, i64, i64, i32, vp, vp]
    L.pmmf_apply_noalloc.restype = i32
    L.pmmf_apply_noalloc.argtypes = [vp, i32, vp, vp, i64, i64, vp]
    L.pmmf_apply_backward.restype = i32
    L.pmmf_apply_backward.argtypes = [vp, i32, vp, vp, i64, i64, vp, vp, vp, vp, vp]
    L.pmmf_get_angles.restype = i32
    L.pmmf_get_angles.argtypes = [vp, vp, vp]
    L.pmmf_set_angles.restype = i32
    L.pmmf_set_angles.argtypes = [vp, vp, vp]
    L.pmmf_block_angle_grad.restype = i32
    L.pmmf_block_angle_grad.argtypes = [vp, vp, vp, vp]
    L.pmmf_set_h.restype = i32
    L.pmmf_set_h.argtypes = [vp, vp, vp, vp]
    L.pmmf_factor_blockdiag.restype = i32
    L.pmmf_factor_blockdiag.argtypes = [C.POINTER(Matrix), i64, vp, C.POINTER(Params),
                                        C.POINTER(vp), vp]
    L.pmmf_factor_batched.restype = i32
    L.pmmf_factor_batched.argtypes = [i64, vp, C.POINTER(Params), C.POINTER(vp), vp]
    L.pmmf_get_batch.restype = i32
    L.pmmf_get_precision_stats.restype = i32
    L.pmmf_get_precision_stats.argtypes = [vp, vp, vp, vp, vp]
    L.pmmf_get_batch.argtypes = [vp, vp, vp, vp, vp, vp]
    L.pmmf_set_tuning.restype = i32
    L.pmmf_set_tuning.argtypes = [i32, i64, i32]
    L.pmmf_clear_tuning.restype = None
    L.pmmf_clear_tuning.argtypes = []
    L.pmmf_shard_create.restype = i32
    L.pmmf_shard_create.argtypes = [i64, C.POINTER(Params), C.POINTER(vp), vp]
    L.pmmf_shard_clusters.restype = i32
    L.pmmf_shard_clusters.argtypes = [vp, i64, i64, vp, C.POINTER(i64), vp, vp, vp, vp]
    L.pmmf_shard_search.restype = i32
    L.pmmf_shard_search.argtypes = [vp, i64, i64, vp, vp, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp,
                                    vp, vp, vp, vp]
    L.pmmf_shard_transform.restype = i32
    L.pmmf_shard_transform.argtypes = [vp, i64, i32, i64, vp, vp, vp, vp, i64, i64, vp, vp, i64,
                                       vp, vp, vp, vp, vp, vp, vp, C.POINTER(i64), C.POINTER(i64),
                                       vp]
    L.pmmf_shard_result.restype = i32
    L.pmmf_shard_result.argtypes = [vp, vp, vp, vp, vp, vp]
    L.pmmf_shard_sumsq.restype = i32
    L.pmmf_shard_sumsq.argtypes = [vp, i64, vp, vp]
    L.pmmf_shard_free.restype = None
    L.pmmf_shard_free.argtypes = [vp]
    L.pmmf_profile_begin.restype = i32
    L.pmmf_profile_begin.argtypes = [C.c_uint]
    L.pmmf_profile_end.restype = i32
    L.pmmf_profile_end.argtypes = [vp, vp, vp, vp]
    L.pmmf_profile_records.restype = i32
    L.pmmf_profile_records.argtypes = [i64, vp, vp, vp, vp, vp]
    _lib = L
    apply_tuning(os.environ.get("PMMF_TUNING", TUNING_PATH))
    return L


TUNING_PATH = os.path.join(_HERE, "tuning.json")
TUNE_PARAMS = {"rows_warps": 0, "gram_warps": 1, "select_warps": 2, "pass1_estimate": 3,
               "reach_clusters": 4, "rows_kernel": 5, "dense_tiles": 6, "select_dsm": 7,
               "apply_fused": 8, "select_blocks": 9,
               "mixed_active": 10, "tc_gram": 11}


def apply_tuning(path: str) -> bool:
    """Load launch shapes chosen by autotune.py ({"buckets": {param: [[max_size,
    value], ...]}}) into the library; False when the file is absent."""
    import json
    if not path or not os.path.exists(path):
        return False
    with open(path) as fh:
        cfg = json.load(fh)
    _lib.pmmf_clear_tuning()
    for name, table in cfg.get("buckets", {}).items():
        for max_size, value in table:
            _check(_lib.pmmf_set_tuning(TUNE_PARAMS[name], int(max_size), int(value)))
    return True


def set_tuning(name: str, value: int, max_size: int = 1 << 30) -> None:
    """Set one launch-shape or kernel-choice knob (TUNE_PARAMS) for clusters
    of up to max_size coordinates."""
    _check(load().pmmf_set_tuning(TUNE_PARAMS[name], int(max_size), int(value)))


FAMILIES = ["partition", "gram", "select", "rows", "apply", "other"]


def pmmf_profile_begin(families) -> None:
    """Start timing the named kernel families (see FAMILIES)."""
    mask = 0
    for f in families:
        mask |= 1 << FAMILIES.index(f)
    _check(load().pmmf_profile_begin(mask))


def pmmf_profile_records() -> list:
    """Launches recorded since pmmf_profile_begin, in launch order:
    [(family, ms, bytes, flops)]."""
    L = load()
    cnt = C.c_int64()
    _check(L.pmmf_profile_records(0, None, None, None, None, C.byref(cnt)))
    n = cnt.value
    fam = np.zeros(max(n, 1), dtype=np.int32)
    ms, by, fl = (np.zeros(max(n, 1)) for _ in range(3))
    _check(L.pmmf_profile_records(n, fam.ctypes.data, ms.ctypes.data, by.ctypes.data,
                                  fl.ctypes.data, C.byref(cnt)))
    return [(FAMILIES[fam[i]], float(ms[i]), float(by[i]), float(fl[i])) for i in range(n)]


def pmmf_profile_end() -> dict:
    """Stop timing; per family: total ms, launches, algorithmic bytes and flops."""
    ms = np.zeros(6)
    la = np.zeros(6, dtype=np.int64)
    by = np.zeros(6)
    fl = np.zeros(6)
    _check(load().pmmf_profile_end(ms.ctypes.data, la.ctypes.data, by.ctypes.data, fl.ctypes.data))
    return {f: dict(ms=float(ms[i]), launches=int(la[i]), bytes=float(by[i]), flops=float(fl[i]))
            for i, f in enumerate(FAMILIES)}


def _check(st: int):
    if st != OK:
        raise PmmfError(st, load().pmmf_last_error().decode(errors="replace"))


def _ptr(a) -> Optional[int]:
    """Address of a torch tensor's or numpy array's data."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _loc(a) -> int:
    return DEVICE if hasattr(a, "is_cuda") and a.is_cuda else HOST


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def make_matrix(a=None, *, n=None, rowptr=None, col=None, val=None, dense=None) -> tuple:
    """Build a pmmf_matrix.  Returns (Matrix, keepalive)."""
    keep = []
    if a is not None and dense is None and hasattr(a, "rowptr"):
        n, rowptr, col, val = a.n, a.rowptr, a.col, a.val
    elif a is not None and dense is None:
        dense = a
    if dense is not None:
        if not hasattr(dense, "data_ptr"):
            dense = np.ascontiguousarray(dense, dtype=np.float64)
        keep.append(dense)
        m = Matrix(dense.shape[0], DENSE, _loc(dense), None, None, _ptr(dense), dense.shape[1])
        return m, keep
    if not hasattr(rowptr, "data_ptr"):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
    keep += [rowptr, col, val]
    m = Matrix(int(n), CSR, _loc(val), _ptr(rowptr), _ptr(col), _ptr(val), 0)
    return m, keep


# ---------------------------------------------------------------- C names

def pmmf_factor(matrix: Matrix, params: Params, stream=None) -> int:
    h = C.c_void_p()
    _check(load().pmmf_factor(C.byref(matrix), C.byref(params), C.byref(h), _stream(stream)))
    return h.value


def pmmf_apply(handle: int, op: int, x, y, nrhs: int, ld: int, stream=None):
    _check(load().pmmf_apply(handle, op, _ptr(x), _ptr(y), nrhs, ld, _stream(stream)))


def pmmf_apply_noalloc(handle: int, op: int, x, y, nrhs: int, ld: int, stream=None):
    """pmmf_apply without any allocation (for callers that must not allocate)."""
    _check(load().pmmf_apply_noalloc(handle, op, _ptr(x), _ptr(y), nrhs, ld, _stream(stream)))


def pmmf_solve_precond(handle: int, matrix: Matrix, b, x, nrhs: int, rtol: float, maxit: int,
                       stream=None):
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs)
    st = load().pmmf_solve_precond(handle, C.byref(matrix), _ptr(b), _ptr(x), nrhs, rtol, maxit,
                                   iters.ctypes.data, relres.ctypes.data, _stream(stream))
    return st, iters, relres


def pmmf_solve_precond_sym(handle: int, matrix: Matrix, b, x, nrhs: int, rtol: float,
                           maxit: int, stream=None):
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs)
    st = load().pmmf_solve_precond_sym(handle, C.byref(matrix), _ptr(b), _ptr(x), nrhs, rtol,
                                       maxit, iters.ctypes.data, relres.ctypes.data,
                                       _stream(stream))
    return st, iters, relres


def pmmf_apply_backward(handle: int, op: int, x, g, nrhs: int, ld: int, dx, dtheta, dhdiag,
                        dcore, stream=None):
    _check(load().pmmf_apply_backward(handle, op, _ptr(x), _ptr(g), nrhs, ld, _ptr(dx),
                                      _ptr(dtheta), _ptr(dhdiag), _ptr(dcore), _stream(stream)))


def pmmf_get_angles(handle: int, theta, stream=None):
    _check(load().pmmf_get_angles(handle, _ptr(theta), _stream(stream)))


def pmmf_set_angles(handle: int, theta, stream=None):
    _check(load().pmmf_set_angles(handle, _ptr(theta), _stream(stream)))


def pmmf_block_angle_grad(handle: int, dO, dtheta, stream=None):
    _check(load().pmmf_block_angle_grad(handle, _ptr(dO), _ptr(dtheta), _stream(stream)))


def pmmf_set_h(handle: int, hdiag, core, stream=None):
    _check(load().pmmf_set_h(handle, _ptr(hdiag), _ptr(core), _stream(stream)))


def pmmf_free(handle: int):
    if handle:
        load().pmmf_free(handle)


def pmmf_launch_count() -> int:
    return int(load().pmmf_launch_count())


def pmmf_alloc_count() -> int:
    return int(load().pmmf_alloc_count())


def pmmf_probe_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    v = C.c_double()
    _check(load().pmmf_probe_fp64(C.byref(v), _stream(stream)))
    return float(v.value)


def pmmf_gram_reduced(x, precision: int, stream=None) -> np.ndarray:
    """The reduced-precision Gram matrix the shortlist search screens with,
    for the rows of x (rows x s, FP64): TF32 (1) or BF16 (2) split, FP32
    16-term chunks on the tensor cores, compensated sums.  FP32 result."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    rows, s = x.shape
    g = np.empty((rows, rows), dtype=np.float32)
    _check(load().pmmf_gram_reduced(x.ctypes.data, rows, s, int(precision), g.ctypes.data,
                                    _stream(stream)))
    return g


# ---------------------------------------------------------------- convenience

@dataclass
class StageView:
    active: int
    clusters: int
    rotations: int
    nnz_after: int
    max_levels: int
    contrib: float


class Factorization:
    """Owns a pmmf_handle; frees it when garbage collected or on close()."""

    def __init__(self, handle: int, k: int):
        self.handle = handle
        self.k = k

    def close(self):
        if self.handle:
            pmmf_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> Info:
        i = Info()
        _check(load().pmmf_get_info(self.handle, C.byref(i)))
        return i

    @property
    def error(self) -> float:
        return self.info().error

    def stage(self, p: int) -> StageView:
        s = StageInfo()
        _check(load().pmmf_get_stage_info(self.handle, p, C.byref(s)))
        return StageView(s.active, s.clusters, s.rotations, s.nnz_after, s.max_levels, s.contrib)

    def clusters(self, p: int):
        s = self.stage(p)
        off = np.zeros(s.clusters + 1, dtype=np.int64)
        mem = np.zeros(s.active, dtype=np.int32)
        _check(load().pmmf_get_stage_clusters(self.handle, p, off.ctypes.data, mem.ctypes.data))
        return off, mem

    def rotations(self, p: int):
        s = self.stage(p)
        nr, K = s.rotations, self.k
        n1 = max(nr, 1)
        cl = np.zeros(n1, dtype=np.int32)
        kk = np.zeros(n1, dtype=np.int32)
        idx = np.zeros((n1, K), dtype=np.int32)
        O = np.zeros((n1, K * K))
        el = np.zeros(n1, dtype=np.int32)
        _check(load().pmmf_get_stage_rotations(self.handle, p, cl.ctypes.data, kk.ctypes.data,
                                               idx.ctypes.data, O.ctypes.data, el.ctypes.data))
        return cl[:nr], kk[:nr], idx[:nr], O[:nr], el[:nr]

    def h(self):
        if self.batch()["nmat"] > 1:
            raise ValueError("a batch handle's H comes in blocks: use h_blocks()")
        i = self.info()
        hd = np.zeros(i.n)
        ci = np.zeros(i.core_size, dtype=np.int32)
        core = np.zeros((i.core_size, i.core_size))
        _check(load().pmmf_get_h(self.handle, hd.ctypes.data, ci.ctypes.data, core.ctypes.data))
        return hd, ci, core

    def stage_matrix(self, p: int):
        nnz = C.c_int64()
        _check(load().pmmf_get_stage_matrix(self.handle, p, None, None, None, C.byref(nnz)))
        n = self.info().n
        rp = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(max(nnz.value, 1), dtype=np.int32)
        val = np.zeros(max(nnz.value, 1))
        _check(load().pmmf_get_stage_matrix(self.handle, p, rp.ctypes.data, col.ctypes.data,
                                            val.ctypes.data, C.byref(nnz)))
        return rp, col[:nnz.value], val[:nnz.value]

    def apply(self, op: int, x, y=None, stream=None):
        """y = op(x) for a CUDA float64 tensor x of shape (n,) or (n, nrhs)."""
        import torch
        assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
        if y is None:
            y = torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        pmmf_apply(self.handle, op, x, y, nrhs, nrhs, stream)
        return y

    def precision_stats(self) -> dict:
        v = [C.c_int64() for _ in range(4)]
        _check(load().pmmf_get_precision_stats(self.handle, *[C.byref(x) for x in v]))
        return dict(rescored=v[0].value, fallbacks=v[1].value, steps=v[2].value,
                    max_shortlist=v[3].value)

    def batch(self) -> dict:
        """nmat, core_stride, block_off, errors, core_dim of a batch handle."""
        nm, cs = C.c_int64(), C.c_int64()
        _check(load().pmmf_get_batch(self.handle, C.byref(nm), C.byref(cs), None, None, None))
        bo = np.zeros(nm.value + 1, dtype=np.int64)
        err = np.zeros(nm.value)
        cd = np.zeros(nm.value, dtype=np.int32)
        _check(load().pmmf_get_batch(self.handle, None, None, bo.ctypes.data, err.ctypes.data,
                                     cd.ctypes.data))
        return dict(nmat=nm.value, core_stride=cs.value, block_off=bo, errors=err, core_dim=cd)

    def hdiag(self, out=None):
        """The diagonal of H (host float64 array of n)."""
        n = self.info().n
        hd = np.empty(n) if out is None else out
        _check(load().pmmf_get_h(self.handle, hd.ctypes.data, None, None))
        return hd

    def h_blocks(self):
        """(hdiag, core_idx [nmat, stride], core [nmat, stride, stride]) of any handle."""
        b = self.batch()
        i = self.info()
        ns = b["nmat"] * b["core_stride"]
        hd = np.zeros(i.n)
        ci = np.zeros(max(ns, 1), dtype=np.int32)
        core = np.zeros(max(ns * b["core_stride"], 1))
        _check(load().pmmf_get_h(self.handle, hd.ctypes.data, ci.ctypes.data, core.ctypes.data))
        st = b["core_stride"]
        return hd, ci[:ns].reshape(b["nmat"], st), core[:ns * st].reshape(b["nmat"], st, st)

    # ---- differentiation (selections fixed)

    def angles(self):
        """Every rotation's angle as a CUDA float64 tensor (stage, cluster, step
        order): [rotations] for k = 2, [rotations, k(k-1)/2] Givens angles of
        each block for k >= 3."""
        import torch
        nr = self.info().rotations
        per = self.k * (self.k - 1) // 2 if self.k > 2 else 1
        th = torch.empty(max(nr * per, 1), dtype=torch.float64, device="cuda")
        pmmf_get_angles(self.handle, th)
        th = th[:nr * per]
        return th.reshape(nr, per) if self.k > 2 else th

    def h_tensors(self):
        """(hdiag, core) as CUDA float64 tensors."""
        import torch
        hd, _, core = self.h()
        return torch.from_numpy(hd).cuda(), torch.from_numpy(core).cuda()

    def set_parameters(self, theta=None, hdiag=None, core=None):
        """Write angles and/or H (CUDA float64 tensors) into the factorization."""
        if theta is not None:
            pmmf_set_angles(self.handle, theta.contiguous())
        if hdiag is not None or core is not None:
            pmmf_set_h(self.handle, None if hdiag is None else hdiag.contiguous(),
                       None if core is None else core.contiguous())

    def backward(self, op: int, x, g):
        """Gradients of sum(g * op(x)): dict with dx, dtheta, dhdiag, dcore; for
        k >= 3 also dO ([rotations, k * k], block entry (a, b) at a * kk + b),
        and dtheta is then [rotations, k(k-1)/2] for the Givens angles of
        angles()."""
        import torch
        assert x.is_cuda and x.dtype == torch.float64 and x.shape == g.shape
        x, g = x.contiguous(), g.contiguous()
        i = self.info()
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        per = self.k * self.k if self.k > 2 else 1
        out = dict(dx=torch.empty_like(x),
                   dtheta=torch.empty(max(i.rotations * per, 1), dtype=torch.float64,
                                      device="cuda"),
                   dhdiag=torch.empty(i.n, dtype=torch.float64, device="cuda"),
                   dcore=torch.empty((i.core_size, i.core_size), dtype=torch.float64,
                                     device="cuda"))
        pmmf_apply_backward(self.handle, op, x, g, nrhs, nrhs, out["dx"], out["dtheta"],
                            out["dhdiag"], out["dcore"])
        if self.k > 2:
            out["dO"] = out.pop("dtheta")[:i.rotations * per].reshape(i.rotations, per)
            pa = self.k * (self.k - 1) // 2
            dth = torch.empty(max(i.rotations * pa, 1), dtype=torch.float64, device="cuda")
            pmmf_block_angle_grad(self.handle, out["dO"].contiguous(), dth)
            out["dtheta"] = dth[:i.rotations * pa].reshape(i.rotations, pa)
        else:
            out["dtheta"] = out["dtheta"][:i.rotations]
        return out

    def solve(self, a, b, rtol=1e-8, maxit=1000, xi=1.0, stream=None):
        """Preconditioned CG for a x = b (b: CUDA float64 (n,) or (n, nrhs)).
        xi = 1: PCG with M^{-1} = A~^{-1}; xi = 0.5: CG on the split system
        A~^{-1/2} a A~^{-1/2} (Sec. 4)."""
        import torch
        if xi not in (1, 1.0, 0.5):
            raise ValueError("xi must be 1 or 0.5")
        m, keep = make_matrix(a)
        x = torch.empty_like(b)
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        fn = pmmf_solve_precond_sym if xi == 0.5 else pmmf_solve_precond
        st, iters, relres = fn(self.handle, m, b, x, nrhs, rtol, maxit, stream)
        return st, x, iters, relres


def factor(a, *, k=2, eta=0.5, cluster_size=256, core_size=16, seed=0, max_stages=0,
           lloyd_iters=10, coords="auto", record_stages=False, precision=PREC_FP64,
           labels=None, stream=None) -> Factorization:
    """Factor a symmetric matrix (SymCSR-like object with numpy or torch arrays, or a
    dense 2-D array/tensor).  coords='auto' uses ``a.coords`` when present.
    labels: optional stage-1 cluster label per coordinate (int32, numpy or
    torch), e.g. grid bricks; num_labels is taken as labels.max() + 1."""
    m, keep = make_matrix(a)
    if isinstance(coords, str):
        coords = getattr(a, "coords", None)
    cp, cd, cl = None, 0, HOST
    if coords is not None:
        if not hasattr(coords, "data_ptr"):
            coords = np.ascontiguousarray(coords, dtype=np.float64)
        keep.append(coords)
        cp, cd, cl = _ptr(coords), coords.shape[1], _loc(coords)
    lp, ll, nl = None, HOST, 0
    if labels is not None:
        if not hasattr(labels, "data_ptr"):
            labels = np.ascontiguousarray(labels, dtype=np.int32)
            nl = int(labels.max()) + 1 if labels.size else 0
        else:
            import torch
            if labels.dtype != torch.int32 or not labels.is_contiguous():
                raise TypeError("labels must be a contiguous int32 tensor")
            nl = int(labels.max().item()) + 1 if labels.numel() else 0
        keep.append(labels)
        lp, ll = _ptr(labels), _loc(labels)
    prm = Params(k, eta, cluster_size, core_size, seed, max_stages, lloyd_iters, cp, cd, cl,
                 1 if record_stages else 0, precision, lp, ll, nl)
    h = pmmf_factor(m, prm, stream)
    return Factorization(h, k)


def factor_blockdiag(a, block_off, *, k=2, eta=0.5, core_size=16, seed=0, stream=None
                     ) -> Factorization:
    """Batched factorization of a block-diagonal matrix (block b spans
    coordinates block_off[b] .. block_off[b+1]-1), each block on its own."""
    m, keep = make_matrix(a)
    bo = np.ascontiguousarray(block_off, dtype=np.int64)
    prm = Params(k, eta, k, core_size, seed, 0, 10, None, 0, HOST, 0)
    h = C.c_void_p()
    _check(load().pmmf_factor_blockdiag(C.byref(m), len(bo) - 1, bo.ctypes.data, C.byref(prm),
                                        C.byref(h), _stream(stream)))
    return Factorization(h.value, k)


def factor_batched(mats, *, k=2, eta=0.5, core_size=16, seed=0, stream=None) -> Factorization:
    """Batched factorization of separate host CSR matrices (pmmf_factor_batched)."""
    ms, keep = [], []
    for a in mats:
        m, kp = make_matrix(a)
        ms.append(m)
        keep += kp
    arr = (Matrix * len(ms))(*ms)
    prm = Params(k, eta, k, core_size, seed, 0, 10, None, 0, HOST, 0)
    h = C.c_void_p()
    _check(load().pmmf_factor_batched(len(ms), arr, C.byref(prm), C.byref(h), _stream(stream)))
    return Factorization(h.value, k)


# ---------------------------------------------------------------- autograd

def _operator_fn():
    import torch

    class PMMFOperator(torch.autograd.Function):
        """y = U^T H U x (op A) or its inverse (op A_INV) as a function of x, the
        rotation angles theta, the wavelet diagonal hdiag and the core of H, with
        the factorization's greedy selections held fixed.  Forward and backward
        run in the CUDA library (pmmf_set_angles / pmmf_set_h / pmmf_apply /
        pmmf_apply_backward); this class only passes tensors through."""

        @staticmethod
        def forward(ctx, x, theta, hdiag, core, fac, op):
            fac.set_parameters(theta.detach(), hdiag.detach(), core.detach())
            y = fac.apply(op, x.detach().contiguous())
            ctx.save_for_backward(x, theta, hdiag, core)
            ctx.fac, ctx.op = fac, op
            return y

        @staticmethod
        def backward(ctx, gy):
            x, theta, hdiag, core = ctx.saved_tensors
            fac = ctx.fac
            # the handle may have been re-parameterised since the forward
            fac.set_parameters(theta.detach(), hdiag.detach(), core.detach())
            gr = fac.backward(ctx.op, x.detach().contiguous(), gy.contiguous())
            return gr["dx"], gr["dtheta"], gr["dhdiag"], gr["dcore"], None, None

    return PMMFOperator


_PMMF_OPERATOR = None


def pmmf_operator(fac: Factorization, x, theta, hdiag, core, op: int = OP_A):
    """Differentiable y = op(x) with parameters (theta, hdiag, core)."""
    global _PMMF_OPERATOR
    if _PMMF_OPERATOR is None:
        _PMMF_OPERATOR = _operator_fn()
    return _PMMF_OPERATOR.apply(x, theta, hdiag, core, fac, op)
