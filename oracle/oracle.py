"""ctypes front end of the plain FP64 CPU oracle (``pmmf_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product library never imports it.  It imports nothing from the product
package: callers hand it plain numpy arrays.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.environ.get("PMMF_ORACLE_SO") or os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "pmmf_oracle.c")

OK, ERR_INVALID_ARG, ERR_NOT_SYMMETRIC, ERR_NONFINITE, ERR_OOM = 0, 1, 2, 3, 4
ERR_NOT_SPD, ERR_NOT_CONVERGED = 6, 8
OP_A, OP_A_INV, OP_U, OP_UT, OP_H, OP_H_INV = 0, 1, 2, 3, 4, 5
OP_A_INV_SQRT, OP_H_INV_SQRT = 6, 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so every fma is explicit)."""
    if os.environ.get("PMMF_ORACLE_SO"):
        return _SO           # a prebuilt library chosen by the caller (mutation tests)
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pmmf_oracle.h"))):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-Wall", "-Wextra", "-Wno-unused-parameter", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")


def build_openmp(force: bool = False):
    """The same source compiled with OpenMP (clusters and rows spread over the
    host's cores, the paper's m-fold CPU parallelism).  Used only to time a
    multi-core CPU baseline; its results equal the single-thread build's.
    Returns the library path, or None if the compiler has no OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pmmf_oracle.h"))):
        tmp = _SO_OMP + f".{os.getpid()}.tmp"
        try:
            subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                                   "-fopenmp", "-Wall", "-Wextra", "-Wno-unused-parameter", "-fPIC",
                                   "-shared", "-o", tmp, _SRC, "-lm"],
                                  stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            return None
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


_lib = None
_lib_omp = None


def _declare_factor(L):
    vp = C.c_void_p
    L.or_factor.restype = vp
    L.or_factor.argtypes = [C.c_int64, vp, vp, vp, vp, C.c_int, vp, C.c_int]
    L.or_free.argtypes = [vp]
    L.or_status.restype = C.c_int
    L.or_status.argtypes = [vp]
    L.or_error.restype = C.c_double
    L.or_error.argtypes = [vp]
    L.or_threads.restype = C.c_int
    L.or_threads.argtypes = []
    L.or_hdiag.argtypes = [vp, vp]


def time_factor_openmp(n, rowptr, col, val, coords=None, *, runs=1, k=2, eta=0.5,
                       cluster_size=256, core_size=16, seed=0, labels=None, hdiag_out=None):
    """Median wall time of `runs` factorizations with the OpenMP build:
    (seconds, relative error, threads), or None without OpenMP.  hdiag_out
    (float64[n], optional) receives the diagonal of H of the last run."""
    import time
    global _lib_omp
    if _lib_omp is None:
        path = build_openmp()
        if path is None:
            return None
        _lib_omp = C.CDLL(path)
        _declare_factor(_lib_omp)
    L = _lib_omp
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    dim, cp = 0, None
    if coords is not None:
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        dim, cp = coords.shape[1], _p(coords)
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
    prm = _Params(k, eta, cluster_size, core_size, seed, 0, 10,
                  None if lab is None else _p(lab), 0 if lab is None else int(lab.max()) + 1)
    ts, err = [], None
    for _ in range(runs):
        t0 = time.perf_counter()
        h = L.or_factor(n, _p(rowptr), _p(col), _p(val), cp, dim, C.byref(prm), 0)
        ts.append(time.perf_counter() - t0)
        if not h:
            raise MemoryError("oracle allocation failed")
        st = L.or_status(h)
        err = L.or_error(h)
        if hdiag_out is not None and st == 0:
            L.or_hdiag(h, _p(hdiag_out))
        L.or_free(h)
        if st:
            raise RuntimeError(f"oracle failed with status {st}")
    ts.sort()
    return ts[len(ts) // 2], err, int(L.or_threads())


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        i64, i32, f64, u64, vp = C.c_int64, C.c_int, C.c_double, C.c_uint64, C.c_void_p
        L.or_factor.restype = vp
        L.or_factor.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32]
        L.or_free.argtypes = [vp]
        for name, rt in [("or_status", i32), ("or_num_stages", i32), ("or_error", f64),
                         ("or_norm_a", f64), ("or_core_size", i64)]:
            getattr(L, name).restype = rt
            getattr(L, name).argtypes = [vp]
        for name, rt in [("or_stage_active", i64), ("or_stage_clusters", i64),
                         ("or_stage_rotations", i64), ("or_stage_contrib", f64),
                         ("or_stage_nnz", i64)]:
            getattr(L, name).restype = rt
            getattr(L, name).argtypes = [vp, i32]
        L.or_stage_cluster_offsets.argtypes = [vp, i32, vp]
        L.or_stage_members.argtypes = [vp, i32, vp]
        L.or_stage_rotation_data.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.or_stage_matrix.restype = i64
        L.or_stage_matrix.argtypes = [vp, i32, vp, vp, vp]
        L.or_core.argtypes = [vp, vp, vp]
        L.or_hdiag.argtypes = [vp, vp]
        L.or_apply.restype = i32
        L.or_apply.argtypes = [vp, i32, vp, vp, i64]
        L.or_pcg.restype = i32
        L.or_pcg.argtypes = [vp, i64, vp, vp, vp, vp, vp, i64, f64, i32, vp, vp]
        L.or_pcg_sym.restype = i32
        L.or_pcg_sym.argtypes = [vp, i64, vp, vp, vp, vp, vp, i64, f64, i32, vp, vp]
        L.or_splitmix64_next.restype = u64
        L.or_splitmix64_next.argtypes = [vp]
        L.or_draw.restype = u64
        L.or_draw.argtypes = [u64, i64, i64, i64]
        L.or_pick.restype = i64
        L.or_pick.argtypes = [u64, i64]
        L.or_jacobi2.argtypes = [f64, f64, f64, vp, vp]
        L.or_jacobik.restype = i32
        L.or_jacobik.argtypes = [i32, vp, vp]
        L.or_block_angles.restype = i32
        L.or_block_angles.argtypes = [i32, vp, vp, vp]
        L.or_block_from_angles.restype = None
        L.or_block_from_angles.argtypes = [i32, vp, vp, vp]
        L.or_block_angle_grad.restype = None
        L.or_block_angle_grad.argtypes = [i32, vp, vp, vp, vp]
        L.or_sym_rotate.argtypes = [vp, i64, i64, i32, vp, vp]
        L.or_gram.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp]
        L.or_partition.restype = i32
        L.or_partition.argtypes = [i64, vp, i32, i64, vp, i64, i32, vp]
        L.or_quantize.argtypes = [i64, vp, i32, vp]
        L.or_total_rotations.restype = i64
        L.or_total_rotations.argtypes = [vp]
        L.or_apply_grad.restype = i32
        L.or_apply_grad.argtypes = [vp, i32, vp, vp, i64, vp, vp, vp, vp, vp]
        L.or_set_rotation.restype = i32
        L.or_set_rotation.argtypes = [vp, i32, i64, vp]
        L.or_set_h.restype = i32
        L.or_set_h.argtypes = [vp, vp, vp]
        L.or_threads.restype = i32
        L.or_threads.argtypes = []
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Params(C.Structure):
    _fields_ = [("k", C.c_int), ("eta", C.c_double), ("cluster_size", C.c_int),
                ("core_size", C.c_int), ("seed", C.c_uint64), ("max_stages", C.c_int),
                ("lloyd_iters", C.c_int), ("labels", C.c_void_p), ("num_labels", C.c_int64)]


@dataclass
class Stage:
    active: int
    offsets: np.ndarray      # cluster offsets into members
    members: np.ndarray      # global ids, cluster by cluster, ascending inside
    rot_cluster: np.ndarray
    rot_k: np.ndarray
    rot_idx: np.ndarray      # [nrot, K] global ids (-1 unused)
    rot_O: np.ndarray        # [nrot, K*K] k x k blocks, row-major with stride k
    rot_elim: np.ndarray
    contrib: float
    nnz: int
    matrix: tuple = None     # (rowptr[n+1], col, val) of A_p[S_p,S_p], if recorded


@dataclass
class Factorization:
    status: int
    n: int = 0
    K: int = 2
    stages: list = field(default_factory=list)
    error: float = float("nan")
    norm_a: float = float("nan")
    core_idx: np.ndarray = None
    core: np.ndarray = None
    hdiag: np.ndarray = None
    _h: int = None

    def __del__(self):
        if self._h:
            lib().or_free(self._h)
            self._h = None

    def apply(self, op: int, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        nrhs = 1 if x.ndim == 1 else x.shape[1]
        y = np.empty_like(x)
        st = lib().or_apply(self._h, op, _p(x), _p(y), nrhs)
        if st:
            raise RuntimeError(f"oracle apply failed with status {st}")
        return y

    def pcg(self, a, b: np.ndarray, rtol: float, maxit: int):
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        x = np.zeros_like(b)
        iters = np.zeros(nrhs, dtype=np.int32)
        relres = np.zeros(nrhs)
        st = lib().or_pcg(self._h, a.n, _p(a.rowptr), _p(a.col), _p(a.val), _p(b), _p(x), nrhs,
                          rtol, maxit, _p(iters), _p(relres))
        return st, x, iters, relres

    def pcg_sym(self, a, b: np.ndarray, rtol: float, maxit: int):
        """xi = 1/2: CG on the split system W A W y = W b, x = W y."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        x = np.zeros_like(b)
        iters = np.zeros(nrhs, dtype=np.int32)
        relres = np.zeros(nrhs)
        st = lib().or_pcg_sym(self._h, a.n, _p(a.rowptr), _p(a.col), _p(a.val), _p(b), _p(x), nrhs,
                              rtol, maxit, _p(iters), _p(relres))
        return st, x, iters, relres

    def total_rotations(self) -> int:
        return sum(len(s.rot_elim) for s in self.stages)

    def apply_grad(self, op: int, x: np.ndarray, g: np.ndarray) -> dict:
        """Gradient of sum(g * op(x)) for op A or A_INV, selections fixed:
        dx, dO [T, K*K], dtheta [T] (k = 2 angles), dhdiag [n], dcore [m, m]."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        nrhs = 1 if x.ndim == 1 else x.shape[1]
        T = int(lib().or_total_rotations(self._h))
        m = len(self.core_idx)
        out = dict(dx=np.empty_like(x), dhdiag=np.zeros(self.n), dcore=np.zeros((m, m)))
        dO = np.zeros((max(T, 1), self.K * self.K))
        dth = np.zeros(max(T, 1))
        st = lib().or_apply_grad(self._h, op, _p(x), _p(g), nrhs, _p(out["dx"]), _p(dO), _p(dth),
                                 _p(out["dhdiag"]), _p(out["dcore"]))
        if st:
            raise RuntimeError(f"oracle gradient failed with status {st}")
        out["dO"], out["dtheta"] = dO[:T], dth[:T]
        return out

    def set_rotation(self, p: int, t: int, O: np.ndarray) -> None:
        """Replace one rotation block inside the oracle (finite-difference pins);
        the exported copy in self.stages is left as it was."""
        O = np.ascontiguousarray(O, dtype=np.float64).ravel()
        if lib().or_set_rotation(self._h, p, t, _p(O)):
            raise ValueError("bad rotation index")

    def set_h(self, hdiag: np.ndarray = None, core: np.ndarray = None) -> None:
        """Replace H inside the oracle (finite-difference pins)."""
        hd = None if hdiag is None else np.ascontiguousarray(hdiag, dtype=np.float64)
        co = None if core is None else np.ascontiguousarray(core, dtype=np.float64)
        if lib().or_set_h(self._h, None if hd is None else _p(hd), None if co is None else _p(co)):
            raise ValueError("set_h failed")


def factor(n, rowptr, col, val, coords=None, *, k=2, eta=0.5, cluster_size=256, core_size=16,
           seed=0, max_stages=0, lloyd_iters=10, record=False, labels=None,
           rows_all=False) -> Factorization:
    """Run the oracle's pMMF (Algorithm 1) and copy every result out.  labels:
    optional stage-1 cluster label per coordinate (0 .. max), e.g. grid bricks.
    rows_all: the variant whose Grams sum over all n rows of the uncompacted
    matrix (dense, small n; record is ignored)."""
    L = lib()
    if not hasattr(L, "_rows_all_ready"):
        L.or_factor_rows_all.restype = C.c_void_p
        L.or_factor_rows_all.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_int, C.c_void_p]
        L._rows_all_ready = True
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    dim = 0
    cp = None
    if coords is not None:
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        dim = coords.shape[1]
        cp = _p(coords)
    lab = None
    if labels is not None:
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        assert lab.shape == (n,)
    prm = _Params(k, eta, cluster_size, core_size, seed, max_stages, lloyd_iters,
                  None if lab is None else _p(lab), 0 if lab is None else int(lab.max()) + 1)
    if rows_all:
        h = L.or_factor_rows_all(n, _p(rowptr), _p(col), _p(val), cp, dim, C.byref(prm))
    else:
        h = L.or_factor(n, _p(rowptr), _p(col), _p(val), cp, dim, C.byref(prm), 1 if record else 0)
    if not h:
        raise MemoryError("oracle allocation failed")
    f = Factorization(status=L.or_status(h), n=n, K=k, _h=h)
    if f.status:
        return f
    for p in range(L.or_num_stages(h)):
        s = L.or_stage_active(h, p)
        m = L.or_stage_clusters(h, p)
        off = np.zeros(m + 1, dtype=np.int64)
        L.or_stage_cluster_offsets(h, p, _p(off))
        mem = np.zeros(s, dtype=np.int32)
        L.or_stage_members(h, p, _p(mem))
        nr = L.or_stage_rotations(h, p)
        rc = np.zeros(max(nr, 1), dtype=np.int32)
        rk = np.zeros(max(nr, 1), dtype=np.int32)
        ri = np.zeros((max(nr, 1), k), dtype=np.int32)
        ro = np.zeros((max(nr, 1), k * k))
        re = np.zeros(max(nr, 1), dtype=np.int32)
        L.or_stage_rotation_data(h, p, _p(rc), _p(rk), _p(ri), _p(ro), _p(re))
        st = Stage(s, off, mem, rc[:nr], rk[:nr], ri[:nr], ro[:nr], re[:nr],
                   L.or_stage_contrib(h, p), L.or_stage_nnz(h, p))
        if record:
            nnz = st.nnz
            rp = np.zeros(n + 1, dtype=np.int64)
            cc = np.zeros(max(nnz, 1), dtype=np.int32)
            vv = np.zeros(max(nnz, 1))
            L.or_stage_matrix(h, p, _p(rp), _p(cc), _p(vv))
            st.matrix = (rp, cc[:nnz], vv[:nnz])
        f.stages.append(st)
    f.error = L.or_error(h)
    f.norm_a = L.or_norm_a(h)
    nc = L.or_core_size(h)
    f.core_idx = np.zeros(nc, dtype=np.int32)
    f.core = np.zeros((nc, nc))
    L.or_core(h, _p(f.core_idx), _p(f.core))
    f.hdiag = np.zeros(n)
    L.or_hdiag(h, _p(f.hdiag))
    return f


def factor_csr(a, coords="auto", **kw) -> Factorization:
    """Convenience wrapper for an object with n / rowptr / col / val (/ coords)."""
    if isinstance(coords, str):
        coords = getattr(a, "coords", None)
    return factor(a.n, a.rowptr, a.col, a.val, coords, **kw)


# ---- building blocks ------------------------------------------------------

def splitmix64_stream(seed: int, count: int) -> list:
    st = C.c_uint64(seed)
    return [lib().or_splitmix64_next(C.byref(st)) for _ in range(count)]


def draw(seed, p, u, t) -> int:
    return lib().or_draw(seed, p, u, t)


def pick(r, count) -> int:
    return lib().or_pick(r, count)


def jacobi2(a, b, d):
    c, s = C.c_double(), C.c_double()
    lib().or_jacobi2(a, b, d, C.byref(c), C.byref(s))
    return c.value, s.value


def jacobik(g: np.ndarray):
    g = np.ascontiguousarray(g, dtype=np.float64)
    k = g.shape[0]
    o = np.zeros((k, k))
    st = lib().or_jacobik(k, _p(g), _p(o))
    return st, o


def sym_rotate(x: np.ndarray, tup, o: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    t = np.ascontiguousarray(tup, dtype=np.int64)
    o = np.ascontiguousarray(o, dtype=np.float64)
    lib().or_sym_rotate(_p(x), x.shape[1], x.shape[0], len(t), _p(t), _p(o))
    return x


def gram(a, members) -> tuple:
    members = np.ascontiguousarray(members, dtype=np.int32)
    cu = len(members)
    g = np.zeros((cu, cu))
    m = np.zeros((cu, cu))
    lib().or_gram(a.n, _p(np.ascontiguousarray(a.rowptr, dtype=np.int64)),
                  _p(np.ascontiguousarray(a.col, dtype=np.int32)),
                  _p(np.ascontiguousarray(a.val, dtype=np.float64)), cu, _p(members), _p(g), _p(m))
    return g, m


def partition(coords: np.ndarray, active: np.ndarray, m: int, iters: int = 10):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    active = np.ascontiguousarray(active, dtype=np.int32)
    lab = np.zeros(len(active), dtype=np.int32)
    st = lib().or_partition(coords.shape[0], _p(coords), coords.shape[1], len(active), _p(active),
                            m, iters, _p(lab))
    if st:
        raise RuntimeError(f"oracle partition failed with status {st}")
    return lab


def quantize(coords: np.ndarray) -> np.ndarray:
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    q = np.zeros(coords.shape, dtype=np.uint32)
    lib().or_quantize(coords.shape[0], _p(coords), coords.shape[1], _p(q))
    return q


def block_angles(O: np.ndarray):
    """Givens angles theta [kk(kk-1)/2] and signs D [kk] of an orthogonal block."""
    O = np.ascontiguousarray(O, dtype=np.float64)
    kk = O.shape[0]
    th = np.zeros(kk * (kk - 1) // 2)
    D = np.zeros(kk)
    if lib().or_block_angles(kk, _p(O), _p(th), _p(D)):
        raise ValueError("bad block size")
    return th, D


def block_from_angles(theta: np.ndarray, D: np.ndarray) -> np.ndarray:
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    kk = len(D)
    O = np.zeros((kk, kk))
    lib().or_block_from_angles(kk, _p(theta), _p(D), _p(O))
    return O


def block_angle_grad(theta: np.ndarray, D: np.ndarray, dO: np.ndarray) -> np.ndarray:
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    dO = np.ascontiguousarray(dO, dtype=np.float64)
    kk = len(D)
    dth = np.zeros(kk * (kk - 1) // 2)
    lib().or_block_angle_grad(kk, _p(theta), _p(D), _p(dO), _p(dth))
    return dth


# ---- one stage's steps, one at a time (for running a stage split over
# several processes in tests) -----------------------------------------------

def _step_lib():
    L = lib()
    if not hasattr(L, "_step_ready"):
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        L.or_step_clusters.restype = i32
        L.or_step_clusters.argtypes = [i64, vp, i32, i64, vp, i32, vp, vp, vp, vp, vp]
        L.or_step_search.restype = i32
        L.or_step_search.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp,
                                     vp, vp]
        L.or_step_transform.restype = i32
        L.or_step_transform.argtypes = [i64, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, i32, vp,
                                        vp, vp, i64, vp]
        L._step_ready = True
    return L


def _params(k, eta, cluster_size, core_size, seed, lloyd_iters=10, labels=None):
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
    prm = _Params(k, eta, cluster_size, core_size, seed, 0, lloyd_iters,
                  None if lab is None else _p(lab), 0 if lab is None else int(lab.max()) + 1)
    return prm, lab


def step_clusters(n, coords, act, p, *, k, eta, cluster_size, core_size, seed, labels=None):
    """Stage p's clusters of the active set act (ascending global ids) and
    their rotation counts (Alg. 1 "cluster", R10, R11): coff, members, e."""
    L = _step_lib()
    act = np.ascontiguousarray(act, dtype=np.int32)
    s = len(act)
    prm, lab = _params(k, eta, cluster_size, core_size, seed, labels=labels)
    dim, cp = 0, None
    if coords is not None:
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        dim, cp = coords.shape[1], _p(coords)
    m = C.c_int64()
    coff = np.zeros(s + 1, dtype=np.int64)
    members = np.zeros(max(s, 1), dtype=np.int32)
    e = np.zeros(max(s, 1), dtype=np.int64)
    st = L.or_step_clusters(n, cp, dim, s, _p(act), p, C.byref(prm), C.byref(m), _p(coff),
                            _p(members), _p(e))
    if st:
        raise RuntimeError(f"or_step_clusters failed with status {st}")
    mm = m.value
    return coff[:mm + 1].copy(), members[:s].copy(), e[:mm].copy()


def step_search(n, rowptr, col, val, coff, members, e, own, p, *, k, eta, cluster_size, core_size,
                seed):
    """Rotation search (Alg. 2) of the clusters own (ordinals) on a CSR over
    all n rows in which at least their members' rows are present: the owned
    clusters' rotations in order: (cluster, kk, idx [T, k], O [T, k*k], elim)."""
    L = _step_lib()
    own = np.ascontiguousarray(own, dtype=np.int32)
    T = int(sum(int(e[u]) for u in own))
    rc = np.zeros(max(T, 1), dtype=np.int32)
    rk = np.zeros(max(T, 1), dtype=np.int32)
    ri = np.zeros((max(T, 1), k), dtype=np.int32)
    ro = np.zeros((max(T, 1), k * k))
    re = np.zeros(max(T, 1), dtype=np.int32)
    prm, _ = _params(k, eta, cluster_size, core_size, seed)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    coff = np.ascontiguousarray(coff, dtype=np.int64)
    members = np.ascontiguousarray(members, dtype=np.int32)
    e = np.ascontiguousarray(e, dtype=np.int64)
    st = L.or_step_search(n, _p(rowptr), _p(col), _p(val), len(coff) - 1, _p(coff), _p(members),
                          _p(e), len(own), _p(own), p, C.byref(prm), _p(rc), _p(rk), _p(ri),
                          _p(ro), _p(re))
    if st:
        raise RuntimeError(f"or_step_search failed with status {st}")
    return rc[:T], rk[:T], ri[:T], ro[:T], re[:T]


def step_transform(n, rowptr, col, val, coff, members, roff, rk, ridx, rO, k):
    """out = in Q^T for the given rows (CSR over them, global column ids) with
    every cluster's rotations of the stage: (rowptr, col, val) of the output."""
    L = _step_lib()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    args = [np.ascontiguousarray(x, dtype=t) for x, t in
            ((coff, np.int64), (members, np.int32), (roff, np.int64), (rk, np.int32),
             (ridx, np.int32), (rO, np.float64))]
    nr = len(rowptr) - 1
    orp = np.zeros(nr + 1, dtype=np.int64)
    need = C.c_int64()
    st = L.or_step_transform(n, nr, _p(rowptr), _p(col), _p(val), len(args[0]) - 1, *map(_p, args),
                             k, _p(orp), None, None, 0, C.byref(need))
    if st:
        raise RuntimeError(f"or_step_transform failed with status {st}")
    oc = np.zeros(max(need.value, 1), dtype=np.int32)
    ov = np.zeros(max(need.value, 1))
    st = L.or_step_transform(n, nr, _p(rowptr), _p(col), _p(val), len(args[0]) - 1, *map(_p, args),
                             k, _p(orp), _p(oc), _p(ov), need.value, C.byref(need))
    if st:
        raise RuntimeError(f"or_step_transform failed with status {st}")
    return orp, oc[:need.value], ov[:need.value]
