"""Cluster-sharded pMMF: the stages of Algorithm 1 split over ranks (Sec. 2.3).

The paper parallelizes a stage over clusters (each cluster's search of
Algorithm 2 is independent) and over blocks of the matrix (the blocked update
Q_u A_uv Q_v^T), storing the matrix in blocks that are redistributed between
stages ("reblocking").  Here one rank per GPU runs the same stage loop:

  1. the clustering of the active set, computed identically on every rank;
  2. ownership: cluster u belongs to rank u mod W, and a rank holds the rows
     of its clusters' coordinates;
  3. the search of Algorithm 2 for its own clusters;
  4. all-gather of the stage's rotations: a row's entries span clusters, so
     the update needs every cluster's rotations (Q is block diagonal);
  5. pass 1 of the update, V = A Q^T, on its rows, giving parts of the rows
     of W = V^T;
  6. all-to-all: each part of a row y of W goes to the owner of y's cluster;
  7. pass 2, A_p = W Q^T, on its rows of W, with the residual of the
     eliminated coordinates, the diagonal of H and the compaction to the
     survivors;
  8. all-reduce of the residual; the eliminated coordinates leave;
  9. the next stage's clustering, then the reblock: all-to-all of rows to
     their new owners.
After the last stage the surviving rows are gathered into the dense core.

Every floating-point step runs in the backend (the CUDA library on a GPU);
this module only routes rows, rotations and counts between ranks, so the
merged factorization is the single-process one: the same clusters, rotations
and H, and the residual up to the order of its sums.

A backend provides (tensors on backend.device; global ids everywhere):
  clusters(p, act) -> (coff[m + 1], members[s], e[m])     replicated step 1
  search(p, rows, act, coff, members, e, own) -> (cluster, kk, idx, O, elim)
  pass1(p, rows, act, coff, members, roff, rot) -> Rows of W (parts)
  pass2(p, wrows, act, coff, members, roff, rot) -> (Rows, h_ids, h_vals, contrib)
  sumsq(rows) -> float                                      sum of squares
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class Rows:
    """Sparse rows held by one rank: ids (int64, ascending) with their entries
    in CSR form (rowptr int64, col int64 global ids, val float64)."""
    ids: torch.Tensor
    rowptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor

    @property
    def count(self) -> int:
        return int(self.ids.numel())

    def to(self, device) -> "Rows":
        return Rows(self.ids.to(device), self.rowptr.to(device), self.col.to(device),
                    self.val.to(device))


@dataclass
class Rotations:
    """One stage's rotations, clusters in ordinal order, step order inside a
    cluster: cluster ordinal, tuple size, tuple [T, k] (global ids, -1 unused),
    block [T, k*k], eliminated id."""
    cluster: torch.Tensor
    kk: torch.Tensor
    idx: torch.Tensor
    O: torch.Tensor
    elim: torch.Tensor


@dataclass
class StageResult:
    active: int
    coff: np.ndarray
    members: np.ndarray
    rot: Rotations
    contrib: float


@dataclass
class ShardedFactorization:
    n: int
    stages: list = field(default_factory=list)
    hdiag: np.ndarray = None
    core_idx: np.ndarray = None
    core: np.ndarray = None
    norm_a: float = 0.0
    error: float = 0.0


# ---------------------------------------------------------------- exchange

class Exchange:
    """The collectives of the stage loop over a torch.distributed group (any
    backend with all_to_all_single and all_reduce: NCCL on GPUs, gloo on host
    tensors); a single process needs no group."""

    def __init__(self, group=None, comm_device=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.on = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if self.on else 1
        self.rank = dist.get_rank(group) if self.on else 0
        if comm_device is None and self.on:
            comm_device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        self.dev = torch.device(comm_device or "cpu")

    def alltoall(self, parts):
        """parts[q] goes to rank q; returns the parts received from every rank."""
        if self.world == 1:
            return [parts[0]]
        out_dev = parts[0].device
        sc = torch.tensor([int(x.numel()) for x in parts], dtype=torch.int64, device=self.dev)
        rc = torch.empty_like(sc)
        self.dist.all_to_all_single(rc, sc, group=self.group)
        send = torch.cat([x.reshape(-1) for x in parts]).to(self.dev)
        rcl = [int(v) for v in rc.tolist()]
        recv = torch.empty(sum(rcl), dtype=send.dtype, device=self.dev)
        self.dist.all_to_all_single(recv, send, rcl, [int(v) for v in sc.tolist()],
                                    group=self.group)
        return [x.to(out_dev) for x in recv.split(rcl)]

    def allgather(self, x):
        """Every rank's x (1-D), in rank order."""
        return self.alltoall([x] * self.world)

    def allreduce_sum(self, x: torch.Tensor) -> torch.Tensor:
        if self.world == 1:
            return x
        y = x.to(self.dev).clone()
        self.dist.all_reduce(y, group=self.group)
        return y.to(x.device)


def _gather_entries(rowptr: torch.Tensor, perm: torch.Tensor):
    """Row pointers and entry indices of the rows perm (in that order)."""
    lens = (rowptr[1:] - rowptr[:-1])[perm]
    starts = rowptr[:-1][perm]
    rp = torch.zeros(perm.numel() + 1, dtype=torch.int64, device=rowptr.device)
    rp[1:] = torch.cumsum(lens, 0)
    tot = int(rp[-1])
    row_of = torch.repeat_interleave(torch.arange(perm.numel(), device=rowptr.device), lens)
    idx = starts[row_of] + (torch.arange(tot, device=rowptr.device) - rp[:-1][row_of])
    return rp, idx


def route_rows(ex: Exchange, rows: Rows, dest: torch.Tensor) -> Rows:
    """Send every row to rank dest[row]; rows arriving with the same id from
    several ranks are merged (their entries concatenated, lower rank first).
    The result's ids are ascending."""
    dev = rows.ids.device
    W = ex.world
    order = torch.sort(dest * (rows.ids.max() + 1 if rows.count else 1) + rows.ids).indices \
        if rows.count else torch.zeros(0, dtype=torch.int64, device=dev)
    rp, eidx = _gather_entries(rows.rowptr, order)
    ids = rows.ids[order]
    lens = rp[1:] - rp[:-1]
    col, val = rows.col[eidx], rows.val[eidx]
    d = dest[order]
    nrow = torch.bincount(d, minlength=W).tolist() if rows.count else [0] * W
    nent = [0] * W
    if rows.count:
        nent = torch.zeros(W, dtype=torch.int64, device=dev).index_add_(0, d, lens).tolist()
    R = ex.alltoall(list(ids.split(nrow)))
    L = ex.alltoall(list(lens.split(nrow)))
    Cc = ex.alltoall(list(col.split(nent)))
    V = ex.alltoall(list(val.split(nent)))
    ids = torch.cat(R)
    lens = torch.cat(L)
    col = torch.cat(Cc)
    val = torch.cat(V)
    rp = torch.zeros(ids.numel() + 1, dtype=torch.int64, device=dev)
    rp[1:] = torch.cumsum(lens, 0)
    # merge rows with equal ids (stable: lower rank's part first)
    perm = torch.sort(ids, stable=True).indices
    rp2, eidx = _gather_entries(rp, perm)
    ids, col, val = ids[perm], col[eidx], val[eidx]
    lens = rp2[1:] - rp2[:-1]
    uid, inv = torch.unique_consecutive(ids, return_inverse=True)
    ulen = torch.zeros(uid.numel(), dtype=torch.int64, device=dev).index_add_(0, inv, lens)
    urp = torch.zeros(uid.numel() + 1, dtype=torch.int64, device=dev)
    urp[1:] = torch.cumsum(ulen, 0)
    return Rows(uid, urp, col, val)


def gather_rotations(ex: Exchange, rot: Rotations, k: int) -> Rotations:
    """Every rank's rotations, ordered by cluster ordinal (each cluster's steps
    stay in order: a cluster has a single owner)."""
    parts = [ex.allgather(x.reshape(-1)) for x in (rot.cluster, rot.kk, rot.idx, rot.O, rot.elim)]
    cl, kk, idx, O, el = (torch.cat(p) for p in parts)
    idx = idx.reshape(-1, k)
    O = O.reshape(-1, k * k)
    order = torch.sort(cl, stable=True).indices
    return Rotations(cl[order], kk[order], idx[order], O[order], el[order])


# ---------------------------------------------------------------- the stage loop

def factor_sharded(backend, n: int, rowptr, col, val, *, core_size: int, max_stages: int = 0,
                   k: int = 2, exchange: Exchange = None) -> ShardedFactorization:
    """Factor the symmetric CSR matrix (rowptr, col, val), given in full to
    every rank, with the stages split over the ranks of `exchange` (see the
    module docstring).  Every rank returns the same ShardedFactorization."""
    ex = exchange or Exchange()
    W, q = ex.world, ex.rank
    dev = backend.device
    rp = torch.as_tensor(np.asarray(rowptr), dtype=torch.int64)
    ci = torch.as_tensor(np.asarray(col), dtype=torch.int64)
    va = torch.as_tensor(np.asarray(val), dtype=torch.float64)
    full = Rows(torch.arange(n, dtype=torch.int64), rp, ci, va).to(dev)
    act = torch.arange(n, dtype=torch.int64, device=dev)
    out = ShardedFactorization(n=n)
    held = None
    hd = torch.zeros(n, dtype=torch.float64, device=dev)
    total = 0.0
    p = 0
    while act.numel() > core_size and (max_stages <= 0 or p < max_stages):
        p += 1
        coff, members, e = backend.clusters(p, act)
        m = coff.numel() - 1
        cl_of = torch.full((n,), -1, dtype=torch.int64, device=dev)
        cl_of[members.to(torch.int64)] = torch.repeat_interleave(
            torch.arange(m, device=dev), (coff[1:] - coff[:-1]).to(torch.int64))
        owner_of_cluster = torch.arange(m, device=dev) % W
        own = torch.nonzero(owner_of_cluster == q).flatten()
        if held is None:
            # every rank was given the whole matrix: keep the rows of its
            # clusters (stage 1 needs no exchange)
            mine = torch.nonzero(owner_of_cluster[cl_of[full.ids]] == q).flatten()
            rpk, eidx = _gather_entries(full.rowptr, mine)
            held = Rows(full.ids[mine], rpk, full.col[eidx], full.val[eidx])
            part = backend.sumsq(held)
            norm2 = float(ex.allreduce_sum(torch.tensor([part], dtype=torch.float64)).item())
        else:
            # reblock: rows to the owners of their coordinates' new clusters
            held = route_rows(ex, held, owner_of_cluster[cl_of[held.ids]])
        mine_rot = backend.search(p, held, act, coff, members, e, own)
        rot = gather_rotations(ex, Rotations(*mine_rot), k)
        roff = torch.zeros(m + 1, dtype=torch.int64, device=dev)
        roff[1:] = torch.cumsum(e.to(torch.int64), 0)
        # pass 1 on this rank's rows; the parts of W's rows to their owners
        wpart = backend.pass1(p, held, act, coff, members, roff, rot)
        wrows = route_rows(ex, wpart, owner_of_cluster[cl_of[wpart.ids]])
        held, h_ids, h_vals, c = backend.pass2(p, wrows, act, coff, members, roff, rot)
        hd[h_ids] = h_vals
        contrib = float(ex.allreduce_sum(torch.tensor([c], dtype=torch.float64)).item())
        total += contrib
        out.stages.append(StageResult(int(act.numel()), coff.cpu().numpy(), members.cpu().numpy(),
                                      Rotations(*(x.cpu() for x in (rot.cluster, rot.kk, rot.idx,
                                                                    rot.O, rot.elim))),
                                      contrib))
        keep = torch.ones(n, dtype=torch.bool, device=dev)
        keep[rot.elim.to(torch.int64)] = False
        act = act[keep[act]]
    if held is None:   # no stage ran: the whole matrix is the core
        held = full if q == 0 else Rows(full.ids[:0], full.rowptr[:1], full.col[:0], full.val[:0])
        part = backend.sumsq(held)
        norm2 = float(ex.allreduce_sum(torch.tensor([part], dtype=torch.float64)).item())
    # the core A_L[S_L, S_L]: every rank's surviving rows, gathered on every
    # rank and placed densely
    lens = held.rowptr[1:] - held.rowptr[:-1]
    ids, lens, cc, vc = (torch.cat(ex.allgather(x)) for x in (held.ids, lens, held.col, held.val))
    rpc = torch.zeros(ids.numel() + 1, dtype=torch.int64, device=dev)
    rpc[1:] = torch.cumsum(lens, 0)
    s = int(act.numel())
    pos = torch.full((n,), -1, dtype=torch.int64, device=dev)
    pos[act] = torch.arange(s, device=dev)
    core = torch.zeros(s, s, dtype=torch.float64, device=dev)
    row_of = torch.repeat_interleave(torch.arange(ids.numel(), device=dev), rpc[1:] - rpc[:-1])
    core[pos[ids[row_of]], pos[cc]] = vc
    hd = ex.allreduce_sum(hd)
    hd[act] = torch.diagonal(core)
    out.hdiag = hd.cpu().numpy()
    out.core_idx = act.cpu().numpy().astype(np.int32)
    out.core = core.cpu().numpy()
    out.norm_a = float(np.sqrt(norm2))
    out.error = float(np.sqrt(total) / out.norm_a) if out.norm_a > 0 else 0.0
    return out


# ---------------------------------------------------------------- the GPU backend

class GpuStageBackend:
    """Each rank's compute on its GPU through the library's stage calls
    (pmmf_shard_*): the same kernels as pmmf_factor.  This class only
    arranges device arrays (row orders, the transposed parts of W) for them."""

    def __init__(self, n, coords, *, k, eta, cluster_size, core_size, seed, labels=None,
                 lloyd_iters=10, device=None, stream=None):
        import ctypes as C
        from . import pmmf
        self.C, self.pm = C, pmmf
        self.L = pmmf.load()
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.n, self.k = n, k
        self.stream = stream
        self._keep = []
        cp, cd, cl = None, 0, pmmf.HOST
        if coords is not None:
            co = np.ascontiguousarray(coords, dtype=np.float64)
            self._keep.append(co)
            cp, cd = co.ctypes.data, co.shape[1]
        lp, nl = None, 0
        if labels is not None:
            lab = np.ascontiguousarray(labels, dtype=np.int32)
            self._keep.append(lab)
            lp, nl = lab.ctypes.data, int(lab.max()) + 1
        prm = pmmf.Params(k, eta, cluster_size, core_size, seed, 0, lloyd_iters, cp, cd, cl, 0, 0,
                          lp, pmmf.HOST, nl)
        h = C.c_void_p()
        pmmf._check(self.L.pmmf_shard_create(n, C.byref(prm), C.byref(h), self._s()))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            self.L.pmmf_shard_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _s(self):
        return self.pm._stream(self.stream)

    @staticmethod
    def _p(t):
        return t.data_ptr() if t is not None and t.numel() > 0 else None

    def clusters(self, p, act):
        C = self.C
        a32 = act.to(torch.int32).contiguous()
        s = a32.numel()
        coff = torch.empty(s + 1, dtype=torch.int64, device=self.device)
        mem = torch.empty(s, dtype=torch.int32, device=self.device)
        e = torch.empty(s, dtype=torch.int64, device=self.device)
        m = C.c_int64()
        self.pm._check(self.L.pmmf_shard_clusters(self.h, p, s, self._p(a32), C.byref(m),
                                                   self._p(coff), self._p(mem), self._p(e),
                                                   self._s()))
        mm = m.value
        return coff[:mm + 1].clone(), mem.to(torch.int64), e[:mm].clone()

    def search(self, p, rows, act, coff, members, e, own):
        k = self.k
        s = act.numel()
        # the held rows as a CSR over the whole active set (ids ascending, so
        # their entries are already in the active order)
        pos = torch.full((self.n,), -1, dtype=torch.int64, device=self.device)
        pos[act] = torch.arange(s, device=self.device)
        lens = torch.zeros(s, dtype=torch.int64, device=self.device)
        lens[pos[rows.ids]] = rows.rowptr[1:] - rows.rowptr[:-1]
        rp = torch.zeros(s + 1, dtype=torch.int64, device=self.device)
        rp[1:] = torch.cumsum(lens, 0)
        col = rows.col.to(torch.int32).contiguous()
        val = rows.val.contiguous()
        T = int(e[own].sum()) if own.numel() else 0
        rc = torch.empty(max(T, 1), dtype=torch.int32, device=self.device)
        rk = torch.empty(max(T, 1), dtype=torch.int32, device=self.device)
        ri = torch.empty(max(T, 1) * k, dtype=torch.int32, device=self.device)
        ro = torch.empty(max(T, 1) * k * k, dtype=torch.float64, device=self.device)
        re = torch.empty(max(T, 1), dtype=torch.int32, device=self.device)
        a32 = act.to(torch.int32).contiguous()
        m32 = members.to(torch.int32).contiguous()
        o32 = own.to(torch.int32).contiguous()
        self.pm._check(self.L.pmmf_shard_search(
            self.h, p, s, self._p(a32), rp.data_ptr(), self._p(col), self._p(val), coff.numel() - 1,
            coff.data_ptr(), m32.data_ptr(), e.data_ptr(), o32.numel(), self._p(o32), rc.data_ptr(),
            rk.data_ptr(), ri.data_ptr(), ro.data_ptr(), re.data_ptr(), self._s()))
        i64 = lambda x: x[:T].to(torch.int64)
        return (i64(rc), i64(rk), ri[:T * k].to(torch.int64).reshape(T, k),
                ro[:T * k * k].reshape(T, k * k), i64(re))

    def _transform(self, p, account, rows, act, coff, members, rot, hdiag=None, contrib=None):
        C = self.C
        i32 = lambda x: x.to(torch.int32).contiguous()
        ids, col = i32(rows.ids), i32(rows.col)
        rc, rk, ri, el = i32(rot.cluster), i32(rot.kk), i32(rot.idx.reshape(-1)), i32(rot.elim)
        O = rot.O.reshape(-1).contiguous()
        m32 = i32(members)
        nr, nz = C.c_int64(), C.c_int64()
        self.pm._check(self.L.pmmf_shard_transform(
            self.h, p, account, rows.count, self._p(ids), rows.rowptr.contiguous().data_ptr(),
            self._p(col), self._p(rows.val.contiguous()), act.numel(), coff.numel() - 1,
            coff.data_ptr(), m32.data_ptr(), rc.numel(), self._p(rc), self._p(rk), self._p(ri),
            self._p(O), self._p(el), self._p(hdiag), self._p(contrib), C.byref(nr), C.byref(nz),
            self._s()))
        oi = torch.empty(nr.value, dtype=torch.int32, device=self.device)
        orp = torch.empty(nr.value + 1, dtype=torch.int64, device=self.device)
        oc = torch.empty(nz.value, dtype=torch.int32, device=self.device)
        ov = torch.empty(nz.value, dtype=torch.float64, device=self.device)
        self.pm._check(self.L.pmmf_shard_result(self.h, self._p(oi), orp.data_ptr(), self._p(oc),
                                                 self._p(ov), self._s()))
        torch.cuda.current_stream(self.device).synchronize()
        return Rows(oi.to(torch.int64), orp, oc.to(torch.int64), ov)

    def pass1(self, p, rows, act, coff, members, roff, rot):
        V = self._transform(p, 0, rows, act, coff, members, rot)
        # the rows of W = V^T, parts from this rank's rows: entry (x, y) of V
        # becomes entry (y, x) of W; rows by y, entries by x
        x = torch.repeat_interleave(V.ids, V.rowptr[1:] - V.rowptr[:-1])
        order = torch.sort(V.col * (self.n + 1) + x).indices
        y, x, v = V.col[order], x[order], V.val[order]
        uid, cnt = torch.unique_consecutive(y, return_counts=True)
        rp = torch.zeros(uid.numel() + 1, dtype=torch.int64, device=self.device)
        rp[1:] = torch.cumsum(cnt, 0)
        return Rows(uid, rp, x, v)

    def pass2(self, p, wrows, act, coff, members, roff, rot):
        hd = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        contrib = torch.zeros(1, dtype=torch.float64, device=self.device)
        out = self._transform(p, 1, wrows, act, coff, members, rot, hd, contrib)
        el = torch.zeros(self.n, dtype=torch.bool, device=self.device)
        el[rot.elim] = True
        h_ids = wrows.ids[el[wrows.ids]]
        return out, h_ids, hd[h_ids], float(contrib.item())

    def sumsq(self, rows):
        C = self.C
        out = C.c_double()
        v = rows.val.contiguous()
        self.pm._check(self.L.pmmf_shard_sumsq(self._p(v), v.numel(), C.byref(out), self._s()))
        return float(out.value)
