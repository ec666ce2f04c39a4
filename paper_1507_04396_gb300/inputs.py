"""Seeded synthetic inputs shaped like the workloads pMMF is run on.

This module only *generates* matrices (and the point coordinates that the
clustering step reads); it performs none of the factorization's arithmetic.
Both the CPU oracle (under ``oracle/``) and the CUDA library consume its
output, so the two sides always see identical bytes.

Every matrix is returned in one common form, ``SymCSR``: a symmetric n x n
matrix in compressed sparse row form with int64 row pointers, int32 column
indices sorted ascending inside each row, and float64 values; entries whose
value is exactly zero are never stored.  Symmetry is exact (entry (i, j) and
entry (j, i) are the same float64 value).

Workloads (the paper measures on graph Laplacians and kernel matrices, §3,
§4 and Fig. 2; its datasets are not available, so these stand in for them):

* ``psd_dense``          dense PSD  X X^T / r + 0.1 I   (small dense case)
* ``knn_laplacian``      Laplacian + 1e-3 I of a symmetrised k-nearest-
                         neighbour graph on uniform points in the unit square
* ``poisson3d``          7-point finite-volume variable-coefficient Poisson
* ``grid_bricks``        stage-1 cluster labels of a structured grid by bricks
* ``rbf_mixture``        dense Gaussian RBF kernel on a 3-D Gaussian mixture
* ``er_laplacian``       Laplacian + 1e-3 I of an Erdos-Renyi graph
* ``block_pairs``        direct sum of random SPD k x k blocks under a random
                         permutation (an exactly factorizable special case)
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class SymCSR:
    n: int
    rowptr: np.ndarray          # int64 [n + 1]
    col: np.ndarray             # int32 [nnz], ascending within each row
    val: np.ndarray             # float64 [nnz], no exact zeros
    coords: Optional[np.ndarray] = None   # float64 [n, d] point per coordinate
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.col] = self.val
        return a


def from_dense(a: np.ndarray, coords=None, name="") -> SymCSR:
    """Store a dense symmetric array as SymCSR (exact zeros dropped)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    mask = a != 0.0
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    r, c = np.nonzero(mask)            # row-major order, columns ascending
    return SymCSR(n, rowptr, c.astype(np.int32), a[r, c].copy(), coords, name)


def _from_scipy(m, coords=None, name="") -> SymCSR:
    m = m.tocsr()
    m.sum_duplicates()
    m.sort_indices()
    m.eliminate_zeros()
    return SymCSR(m.shape[0], m.indptr.astype(np.int64), m.indices.astype(np.int32),
                  m.data.astype(np.float64), coords, name)


def _mirror_upper(a: np.ndarray) -> np.ndarray:
    """Make a float64 array exactly symmetric by copying its upper triangle."""
    return np.triu(a) + np.triu(a, 1).T


def psd_dense(n: int = 256, r: int = 64, seed: int = 0) -> SymCSR:
    """A = X X^T / r + 0.1 I with X an n x r standard normal matrix."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, r))
    a = _mirror_upper(x @ x.T / r) + 0.1 * np.eye(n)
    return from_dense(a, name=f"psd_dense(n={n},r={r},seed={seed})")


def knn_laplacian(n: int = 65536, k: int = 10, seed: int = 1, shift: float = 1e-3) -> SymCSR:
    """L = D - W + shift I of the symmetrised (union) k-NN graph, unit weights.

    Points are uniform in [0, 1]^2; each point links to its k nearest other
    points (Euclidean); the graph is symmetrised by union.
    """
    import scipy.sparse as sp
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    kk = min(k + 1, n)
    _, idx = cKDTree(pts).query(pts, k=kk)
    idx = np.asarray(idx).reshape(n, kk)
    rows = np.repeat(np.arange(n), kk - 1)
    cols = idx[:, 1:].ravel()
    keep = cols != rows
    w = sp.coo_matrix((np.ones(int(keep.sum())), (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    w = ((w + w.T) > 0).astype(np.float64)
    deg = np.asarray(w.sum(axis=1)).ravel()
    lap = sp.diags(deg + shift) - w
    return _from_scipy(lap, coords=pts, name=f"knn_laplacian(n={n},k={k},seed={seed})")


def poisson3d(nx: int = 128, sigma: float = 1.0, seed: int = 4) -> SymCSR:
    """7-point finite-volume Poisson with log-normal cell coefficients.

    kappa = exp(sigma * N(0, 1)) per cell; interior faces use the harmonic
    mean of the two cell coefficients; Dirichlet boundary faces use the cell's
    own coefficient.  Unit grid spacing.  Coordinates are the cell centres.
    """
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    n = nx ** 3
    kap = np.exp(sigma * rng.standard_normal(n)).reshape(nx, nx, nx)
    diag = np.zeros((nx, nx, nx))
    rows, cols, vals = [], [], []
    ids = np.arange(n).reshape(nx, nx, nx)
    for axis in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, nx - 1)
        hi[axis] = slice(1, nx)
        ka, kb = kap[tuple(lo)], kap[tuple(hi)]
        t = 2.0 * ka * kb / (ka + kb)
        diag[tuple(lo)] += t
        diag[tuple(hi)] += t
        ia, ib = ids[tuple(lo)].ravel(), ids[tuple(hi)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-t.ravel(), -t.ravel()]
        # boundary faces on both ends of this axis
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[axis] = 0
        last[axis] = nx - 1
        diag[tuple(first)] += kap[tuple(first)]
        diag[tuple(last)] += kap[tuple(last)]
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag.ravel())
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    g = (np.stack(np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij"),
                  axis=-1).reshape(n, 3) + 0.5)
    return _from_scipy(m, coords=g.astype(np.float64), name=f"poisson3d(nx={nx},seed={seed})")


def grid_bricks(nx: int, ny: int, nz: int, bx: int, by: int, bz: int) -> np.ndarray:
    """Label of each cell of an nx x ny x nz grid (cell id (x * ny + y) * nz + z,
    the poisson3d order) by its bx x by x bz brick, bricks numbered in
    lexicographic (x, y, z) brick order."""
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    nby, nbz = -(-ny // by), -(-nz // bz)
    lab = ((x // bx) * nby + (y // by)) * nbz + (z // bz)
    return lab.reshape(-1).astype(np.int32)


def rbf_mixture(n: int = 16384, components: int = 20, seed: int = 2) -> SymCSR:
    """Dense Gaussian RBF kernel on points of a 3-D Gaussian mixture.

    Means uniform in [-5, 5]^3, unit covariance, equal weights.  Bandwidth
    sigma = lower median of all pairwise distances (i < j);
    K_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)).
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-5.0, 5.0, (components, 3))
    lab = rng.integers(0, components, n)
    pts = means[lab] + rng.standard_normal((n, 3))
    sq = (pts * pts).sum(1)
    d2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * pts @ pts.T, 0.0)
    iu = np.triu_indices(n, 1)
    dd = np.sqrt(d2[iu])
    sigma = np.partition(dd, (dd.size - 1) // 2)[(dd.size - 1) // 2]
    del dd, iu
    kmat = np.exp(-d2 / (2.0 * sigma * sigma))
    kmat = _mirror_upper(kmat)
    return from_dense(kmat, coords=pts, name=f"rbf_mixture(n={n},seed={seed})")


def er_laplacian(n: int, rng: np.random.Generator, avg_deg: float = 8.0,
                 shift: float = 1e-3) -> SymCSR:
    """Laplacian + shift I of an Erdos-Renyi graph, p = avg_deg / n, weights U(0.5, 1.5)."""
    import scipy.sparse as sp
    p = min(1.0, avg_deg / n)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    iu, ju = iu[keep], ju[keep]
    w = rng.uniform(0.5, 1.5, iu.size)
    wm = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([iu, ju]), np.concatenate([ju, iu]))),
                       shape=(n, n)).tocsr()
    deg = np.asarray(wm.sum(axis=1)).ravel()
    lap = sp.diags(deg + shift) - wm
    return _from_scipy(lap, name=f"er_laplacian(n={n})")


def er_laplacian_batch(count: int = 4096, lo: int = 64, hi: int = 1024, seed: int = 3):
    """A batch of independent ER Laplacians with sizes uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, count)
    return [er_laplacian(int(s), rng) for s in sizes]


def blockdiag(mats):
    """Stack independent matrices into one block-diagonal SymCSR; returns it and
    the block offsets (block b spans coordinates off[b] .. off[b+1]-1)."""
    off = np.zeros(len(mats) + 1, dtype=np.int64)
    for b, m in enumerate(mats):
        off[b + 1] = off[b] + m.n
    nnz = np.array([len(m.val) for m in mats], dtype=np.int64)
    eoff = np.concatenate([[0], np.cumsum(nnz)])
    rowptr = np.zeros(off[-1] + 1, dtype=np.int64)
    col = np.empty(eoff[-1], dtype=np.int32)
    val = np.empty(eoff[-1])
    for b, m in enumerate(mats):
        rowptr[off[b] + 1:off[b + 1] + 1] = m.rowptr[1:] + eoff[b]
        col[eoff[b]:eoff[b + 1]] = m.col + off[b]
        val[eoff[b]:eoff[b + 1]] = m.val
    return SymCSR(int(off[-1]), rowptr, col, val, None, f"blockdiag({len(mats)})"), off


def block_pairs(nblocks: int, k: int = 2, seed: int = 5) -> SymCSR:
    """Direct sum of random SPD k x k blocks, symmetrically permuted.

    Its exact MMF with k-point rotations has zero residual once every block
    has been rotated into its eigenbasis.
    """
    rng = np.random.default_rng(seed)
    n = nblocks * k
    a = np.zeros((n, n))
    for b in range(nblocks):
        y = rng.standard_normal((k, k))
        blk = y @ y.T + 0.5 * np.eye(k)
        a[b * k:(b + 1) * k, b * k:(b + 1) * k] = _mirror_upper(blk)
    perm = rng.permutation(n)
    a = a[np.ix_(perm, perm)]
    return from_dense(a, name=f"block_pairs(nblocks={nblocks},k={k},seed={seed})")


