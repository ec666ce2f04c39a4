"""Batched factorization (many independent matrices in one block-diagonal
handle) against the oracle run on each matrix alone.

Matrix b of a batch must come out exactly as the oracle's factorization of
that matrix by itself with one cluster per stage and seed + b: the same
rotation tuples, rotation blocks bit for bit, eliminations, H (diagonal and
core block), and the relative error within 1e-10.
"""

import numpy as np
import pytest

from helpers import gpu, gpu_lib
from paper_1507_04396_gb300 import inputs as I

OP_A, OP_A_INV = 0, 1


def _oracle(m, seed, core):
    from oracle import oracle as O
    o = O.factor(m.n, m.rowptr, m.col, m.val, None, k=2, eta=0.5, cluster_size=max(m.n, 2),
                 core_size=min(core, m.n), seed=seed)
    assert o.status == 0
    return o


def _check_matrix(g, b, off, o, cache):
    """Compare matrix b of batch handle g with its oracle factorization o."""
    lo, hi = int(off[b]), int(off[b + 1])
    nst = g.info().stages
    op = 0
    for p in range(nst):
        if p not in cache:
            cache[p] = (g.clusters(p), g.rotations(p))
        (coff, mem), (cl, kk, idx, O, el) = cache[p]
        first = mem[coff[:-1]]
        hit = np.nonzero((first >= lo) & (first < hi))[0]
        if len(hit) == 0:
            continue
        u = int(hit[0])
        assert op < len(o.stages), f"matrix {b}: more stages than the oracle"
        so = o.stages[op]
        np.testing.assert_array_equal(mem[coff[u]:coff[u + 1]] - lo, so.members)
        sel = cl == u
        np.testing.assert_array_equal(idx[sel] - lo, so.rot_idx)
        np.testing.assert_array_equal(el[sel] - lo, so.rot_elim)
        assert np.array_equal(O[sel].view(np.uint64), so.rot_O.view(np.uint64)), f"matrix {b} stage {op}"
        op += 1
    assert op == len(o.stages), f"matrix {b}: {op} stages vs oracle {len(o.stages)}"


def _check_h(g, off, oracles, mats):
    hd, ci, core = g.h_blocks()
    bi = g.batch()
    for b, o in oracles.items():
        lo, hi = int(off[b]), int(off[b + 1])
        d = int(bi["core_dim"][b])
        assert d == len(o.core_idx)
        np.testing.assert_array_equal(ci[b, :d] - lo, o.core_idx)
        assert np.array_equal(core[b, :d, :d], o.core)
        assert np.array_equal(hd[lo:hi], o.hdiag)
        assert abs(bi["errors"][b] - o.error) <= 1e-10 * max(o.error, 1e-300) + 1e-15


@gpu
def test_batch_matches_oracle_per_matrix():
    """24 matrices of 10..150 coordinates (some below the core size)."""
    import torch
    pm = gpu_lib()
    mats = I.er_laplacian_batch(24, lo=10, hi=150, seed=11)
    core, seed = 16, 5
    g = pm.factor_batched(mats, k=2, eta=0.5, core_size=core, seed=seed)
    big, off = I.blockdiag(mats)
    assert g.batch()["nmat"] == 24
    np.testing.assert_array_equal(g.batch()["block_off"], off)
    oracles = {b: _oracle(m, seed + b, core) for b, m in enumerate(mats)}
    cache = {}
    for b, o in oracles.items():
        _check_matrix(g, b, off, o, cache)
    _check_h(g, off, oracles, mats)
    # the block-diagonal operator: U x, A~ x bit for bit, A~^-1 x to 1e-10
    rng = np.random.default_rng(3)
    x = rng.standard_normal((big.n, 3))
    xd = torch.from_numpy(x).cuda()
    for op, exact in ((OP_A, True), (2, True), (OP_A_INV, False)):
        y = g.apply(op, xd).cpu().numpy()
        for b, o in oracles.items():
            lo, hi = int(off[b]), int(off[b + 1])
            want = o.apply(op, x[lo:hi])
            if exact:
                assert np.array_equal(y[lo:hi], want), (op, b)
            else:
                np.testing.assert_allclose(y[lo:hi], want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


@gpu
def test_blockdiag_entry_point_and_validation():
    import torch
    pm = gpu_lib()
    mats = I.er_laplacian_batch(6, lo=40, hi=90, seed=2)
    big, off = I.blockdiag(mats)
    g1 = pm.factor_blockdiag(big, off, core_size=8, seed=1)
    g2 = pm.factor_batched(mats, core_size=8, seed=1)
    for p in range(g1.info().stages):
        a, b = g1.rotations(p), g2.rotations(p)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
    # device-resident block-diagonal input gives the same factorization
    dev = I.SymCSR(big.n, torch.from_numpy(big.rowptr).cuda(), torch.from_numpy(big.col).cuda(),
                   torch.from_numpy(big.val).cuda())
    g3 = pm.factor_blockdiag(dev, off, core_size=8, seed=1)
    assert np.array_equal(g3.rotations(0)[3], g1.rotations(0)[3])
    # an entry coupling two blocks is rejected
    bad = np.array(off)
    bad[1] += 1
    with pytest.raises(pm.PmmfError) as ei:
        pm.factor_blockdiag(big, bad, core_size=8, seed=1)
    assert ei.value.status == pm.ERR_INVALID_ARG


@gpu
def test_batch_pcg_converges():
    import torch
    pm = gpu_lib()
    mats = I.er_laplacian_batch(12, lo=50, hi=300, seed=4)
    big, off = I.blockdiag(mats)
    g = pm.factor_blockdiag(big, off, core_size=16, seed=0)
    b = torch.from_numpy(np.random.default_rng(0).standard_normal((big.n, 4))).cuda()
    st, x, iters, relres = g.solve(big, b, rtol=1e-8, maxit=500)
    assert st == 0 and np.all(relres <= 1e-8), (st, iters, relres)


@gpu
def test_batch_full_size_sampled():
    """4,096 matrices of 64..1024 coordinates (the batched workload); 12
    sampled matrices checked against the oracle."""
    pm = gpu_lib()
    mats = I.er_laplacian_batch(4096, lo=64, hi=1024, seed=3)
    core, seed = 16, 0
    g = pm.factor_batched(mats, k=2, eta=0.5, core_size=core, seed=seed)
    off = g.batch()["block_off"]
    sizes = np.diff(off)
    picks = list(np.argsort(sizes)[-4:]) + list(np.argsort(sizes)[:4]) + [7, 1000, 2048, 4095]
    oracles = {int(b): _oracle(mats[int(b)], seed + int(b), core) for b in picks}
    cache = {}
    for b, o in oracles.items():
        _check_matrix(g, b, off, o, cache)
    _check_h(g, off, oracles, mats)
