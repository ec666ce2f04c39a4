"""The symmetric preconditioner of Sec. 4 (xi = 1/2) on the GPU against the
oracle.

The GPU forms the core's inverse square root by the coupled Newton-Schulz
iteration; the oracle by a cyclic Jacobi eigendecomposition.  The two agree to
rounding (1e-9 relative to the largest entry for these well-conditioned
cores), the operator squares to A~^{-1} (formed by Gauss-Jordan, a third
method), and the split-system CG matches the oracle's iteration counts and
solution.
"""

import numpy as np
import pytest

from helpers import factor_both, gpu, gpu_lib
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu

OP_A_INV, OP_H_INV, OP_A_INV_SQRT, OP_H_INV_SQRT = 1, 5, 6, 7


def _close(got, want, tol):
    assert np.abs(got - want).max() <= tol * np.abs(want).max(), np.abs(got - want).max()


@pytest.mark.parametrize("make,kw", [
    (lambda: I.knn_laplacian(3000, seed=5), dict(cluster_size=150, core_size=60, seed=6)),
    (lambda: I.poisson3d(14, seed=4), dict(cluster_size=64, core_size=64, seed=4)),
    (lambda: I.knn_laplacian(1500, seed=2), dict(cluster_size=100, core_size=7, seed=1)),
], ids=["knn3000-core60", "poisson14-core64", "knn1500-core7-ragged-tile"])
def test_inverse_sqrt_ops_match_oracle(make, kw):
    import torch
    a = make()
    g, o = factor_both(a, k=2, eta=0.5, **kw)
    x = np.random.default_rng(0).standard_normal((a.n, 3))
    xd = torch.from_numpy(x).cuda()
    for op in (OP_H_INV_SQRT, OP_A_INV_SQRT):
        _close(g.apply(op, xd).cpu().numpy(), o.apply(op, x), 1e-9)
    # W (W x) = A~^{-1} x with the inverse from Gauss-Jordan; W symmetric
    w = g.apply(OP_A_INV_SQRT, xd)
    _close(g.apply(OP_A_INV_SQRT, w).cpu().numpy(), g.apply(OP_A_INV, xd).cpu().numpy(), 1e-9)
    z = torch.from_numpy(np.random.default_rng(1).standard_normal((a.n, 3))).cuda()
    lhs = float((z * w).sum())
    rhs = float((g.apply(OP_A_INV_SQRT, z) * xd).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_inverse_sqrt_full_size_core():
    """The 32,768-point Poisson workload with its 1,024 x 1,024 core (the
    largest core the solver workloads use): W^2 = A~^{-1} to rounding."""
    import torch
    pm = gpu_lib()
    a = I.poisson3d(32, seed=4)
    g = pm.factor(a, k=2, eta=0.5, cluster_size=256, core_size=1024, seed=0)
    assert g.info().core_size == 1024
    x = torch.from_numpy(np.random.default_rng(2).standard_normal((a.n, 2))).cuda()
    w2 = g.apply(OP_A_INV_SQRT, g.apply(OP_A_INV_SQRT, x))
    _close(w2.cpu().numpy(), g.apply(OP_A_INV, x).cpu().numpy(), 1e-9)


def test_ill_conditioned_core_square():
    """A dense RBF kernel core (condition number near 1e11): W^2 = A~^{-1}
    to the accuracy that conditioning allows."""
    import torch
    pm = gpu_lib()
    a = I.rbf_mixture(2048, seed=2)
    g = pm.factor(a, k=3, eta=0.5, cluster_size=512, core_size=128, seed=0)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal((a.n, 1))).cuda()
    w2 = g.apply(OP_A_INV_SQRT, g.apply(OP_A_INV_SQRT, x)).cpu().numpy()
    _close(w2, g.apply(OP_A_INV, x).cpu().numpy(), 1e-4)


def test_split_cg_matches_oracle():
    import torch
    a = I.poisson3d(14, seed=4)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=64, core_size=64, seed=4)
    b = np.random.default_rng(4).standard_normal((a.n, 4))
    st, x, iters, rel = g.solve(a, torch.from_numpy(b).cuda(), rtol=1e-8, maxit=500, xi=0.5)
    ost, ox, oit, orel = o.pcg_sym(a, b, 1e-8, 500)
    assert st == 0 and ost == 0
    assert (rel <= 1e-7).all(), rel
    assert (np.abs(iters - oit) <= 2).all(), (iters, oit)
    np.testing.assert_allclose(x.cpu().numpy(), ox, rtol=0, atol=1e-6 * np.abs(ox).max())
    # the same iterates as xi = 1 PCG: iteration counts within a step or two
    st1, x1, it1, _ = g.solve(a, torch.from_numpy(b).cuda(), rtol=1e-8, maxit=500)
    assert st1 == 0 and (np.abs(iters - it1) <= 2).all(), (iters, it1)


def test_split_cg_exact_preconditioner_one_step():
    import torch
    pm = gpu_lib()
    a = I.poisson3d(6, seed=2)
    g = pm.factor(a, k=2, eta=0.5, cluster_size=27, core_size=a.n, seed=1)
    b = torch.from_numpy(np.random.default_rng(5).standard_normal((a.n, 2))).cuda()
    st, x, iters, rel = g.solve(a, b, rtol=1e-10, maxit=10, xi=0.5)
    assert st == 0 and (iters == 1).all() and (rel <= 1e-10).all(), (iters, rel)


def test_batch_inverse_sqrt_per_matrix():
    """Block cores of a batch (sizes below and at the core size)."""
    import torch
    from oracle import oracle as O
    pm = gpu_lib()
    mats = I.er_laplacian_batch(10, lo=8, hi=120, seed=6)
    g = pm.factor_batched(mats, k=2, eta=0.5, core_size=16, seed=2)
    big, off = I.blockdiag(mats)
    x = np.random.default_rng(6).standard_normal((big.n, 2))
    y = g.apply(OP_A_INV_SQRT, torch.from_numpy(x).cuda()).cpu().numpy()
    for b, m in enumerate(mats):
        o = O.factor(m.n, m.rowptr, m.col, m.val, None, k=2, eta=0.5, cluster_size=max(m.n, 2),
                     core_size=min(16, m.n), seed=2 + b)
        lo, hi = int(off[b]), int(off[b + 1])
        _close(y[lo:hi], o.apply(OP_A_INV_SQRT, x[lo:hi]), 1e-9)


def test_not_positive_definite_is_reported():
    """A core with a negative eigenvalue, and a negative wavelet entry: the
    oracle and the GPU both refuse the inverse square root."""
    import torch
    from oracle import oracle as O
    pm = gpu_lib()
    a = I.knn_laplacian(2000, seed=7)
    g = pm.factor(a, k=2, eta=0.5, cluster_size=100, core_size=32, seed=3)
    hd, ci, core = g.h()
    x = torch.ones(a.n, 1, dtype=torch.float64, device="cuda")
    bad = core.copy()
    bad[0, 0] = -10.0 * np.abs(core).max()
    g.set_parameters(core=torch.from_numpy(bad).cuda())
    with pytest.raises(pm.PmmfError) as e:
        g.apply(OP_A_INV_SQRT, x)
    assert e.value.status == pm.ERR_NOT_SPD
    # a valid core again clears the state
    g.set_parameters(core=torch.from_numpy(core).cuda())
    g.apply(OP_A_INV_SQRT, x)
    hb = hd.copy()
    w = np.nonzero(~np.isin(np.arange(a.n), ci))[0][0]
    hb[w] = -1.0
    g.set_parameters(hdiag=torch.from_numpy(hb).cuda())
    with pytest.raises(pm.PmmfError) as e:
        g.apply(OP_H_INV_SQRT, x)
    assert e.value.status == pm.ERR_NOT_SPD
    # the oracle agrees on the indefinite core
    o = O.factor(a.n, a.rowptr, a.col, a.val, None, k=2, eta=0.5, cluster_size=100,
                 core_size=32, seed=3)
    o.set_h(None, bad)
    with pytest.raises(RuntimeError):
        o.apply(OP_A_INV_SQRT, np.ones((a.n, 1)))
