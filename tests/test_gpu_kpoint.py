"""k-point rotations (k >= 3) on the GPU against the oracle.

Same bar as the Givens path: clusters, tuples, eliminations, every k x k
block, every stage's A_p and H bit-identical; U x, U^T x, H x, A~ x
bit-identical; A~^{-1} x within 1e-10; the error within 1e-10 relative.
"""

import numpy as np
import pytest

from helpers import assert_same_factorization, factor_both, gpu, gpu_lib
from oracle import oracle as O
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu


def test_dense_k3_one_cluster():
    a = I.psd_dense(80, 20, seed=2)
    g, o = factor_both(a, coords=None, k=3, eta=0.5, cluster_size=80, core_size=10, seed=11)
    assert_same_factorization(g, o)


@pytest.mark.parametrize("k,eta", [(3, 0.5), (4, 0.4), (5, 0.3)])
def test_knn_clustered_kpoint(k, eta):
    a = I.knn_laplacian(1500, seed=6)
    g, o = factor_both(a, k=k, eta=eta, cluster_size=96, core_size=40, seed=4)
    assert_same_factorization(g, o)


def test_exact_block_sum_k3():
    """Direct sum of random SPD 3 x 3 blocks: one cluster, exact factorization."""
    a = I.block_pairs(40, k=3, seed=7)
    g, o = factor_both(a, coords=None, k=3, eta=1.0 / 3 + 1e-9, cluster_size=a.n,
                       core_size=80, seed=2)
    assert_same_factorization(g, o)
    assert g.info().error <= 1e-13


def test_apply_k3_matches_oracle():
    import torch
    a = I.knn_laplacian(2500, seed=9)
    g, o = factor_both(a, k=3, eta=0.5, cluster_size=128, core_size=60, seed=1)
    assert_same_factorization(g, o)
    x = np.random.default_rng(2).standard_normal((a.n, 3))
    xd = torch.from_numpy(x).cuda()
    for op in (O.OP_U, O.OP_UT, O.OP_H, O.OP_A):
        assert np.array_equal(g.apply(op, xd).cpu().numpy(), o.apply(op, x)), op
    y = g.apply(O.OP_A_INV, xd).cpu().numpy()
    want = o.apply(O.OP_A_INV, x)
    assert np.abs(y - want).max() <= 1e-10 * np.abs(want).max()


def test_batch_k3_matches_oracle():
    pm = gpu_lib()
    mats = I.er_laplacian_batch(10, lo=30, hi=160, seed=8)
    g = pm.factor_batched(mats, k=3, eta=0.5, core_size=12, seed=3)
    big, off = I.blockdiag(mats)
    hd, ci, core = g.h_blocks()
    for b, m in enumerate(mats):
        o = O.factor(m.n, m.rowptr, m.col, m.val, None, k=3, eta=0.5, cluster_size=m.n,
                     core_size=12, seed=3 + b)
        assert o.status == 0
        lo, hi = int(off[b]), int(off[b + 1])
        assert np.array_equal(hd[lo:hi], o.hdiag)
        d = len(o.core_idx)
        assert np.array_equal(core[b, :d, :d], o.core)


def test_angle_entry_points_reject_what_they_do_not_cover():
    """The block-angle chain rule is for k >= 3 (k = 2 rotations are angles
    already); a batch handle has no angle parameterisation."""
    import torch
    pm = gpu_lib()
    a = I.knn_laplacian(300, seed=1)
    g2 = pm.factor(a, k=2, eta=0.5, cluster_size=64, core_size=20, seed=0)
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PmmfError) as e:
        pm.pmmf_block_angle_grad(g2.handle, z, z)
    assert e.value.status == pm.ERR_UNSUPPORTED
    mats = I.er_laplacian_batch(3, lo=20, hi=40, seed=1)
    gb = pm.factor_batched(mats, k=3, eta=0.5, core_size=8, seed=0)
    with pytest.raises(pm.PmmfError) as e:
        gb.angles()
    assert e.value.status == pm.ERR_UNSUPPORTED
