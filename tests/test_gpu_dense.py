"""Dense inputs kept dense on the GPU (dense Gram and dense blocked update)
against the oracle: the same bar as the sparse path (bit-identical
selections, rotations, stage matrices, H and products)."""

import numpy as np
import pytest

from helpers import assert_same_factorization, gpu, gpu_lib
from oracle import oracle as O
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu


def _both(a, coords, **kw):
    import torch
    pm = gpu_lib()
    dense = torch.from_numpy(a.to_dense()).cuda()
    g = pm.factor(dense, coords=coords, record_stages=True, **kw)
    o = O.factor(a.n, a.rowptr, a.col, a.val, coords, record=True, **kw)
    assert o.status == 0
    return g, o


def test_dense_psd_one_cluster():
    """X X^T/64 + 0.1 I, n = 256, one cluster, core 16."""
    a = I.psd_dense(256, 64, seed=0)
    g, o = _both(a, None, k=2, eta=0.5, cluster_size=256, core_size=16, seed=0)
    assert_same_factorization(g, o)


@pytest.mark.parametrize("k", [2, 3])
def test_dense_rbf_clustered(k):
    """Gaussian RBF kernel of a 3-D mixture, k-means clusters of 128."""
    a = I.rbf_mixture(1024, components=8, seed=5)
    g, o = _both(a, a.coords, k=k, eta=0.5, cluster_size=128, core_size=64, seed=3)
    assert_same_factorization(g, o)


def test_sparse_matrix_given_dense():
    """A sparse Laplacian passed as a dense array: zeros must not change a bit."""
    a = I.knn_laplacian(1200, seed=4)
    g, o = _both(a, a.coords, k=2, eta=0.5, cluster_size=100, core_size=50, seed=2)
    assert_same_factorization(g, o)


def test_dense_apply_matches_oracle():
    import torch
    a = I.rbf_mixture(768, components=6, seed=1)
    g, o = _both(a, a.coords, k=3, eta=0.5, cluster_size=96, core_size=48, seed=1)
    x = np.random.default_rng(0).standard_normal((a.n, 2))
    xd = torch.from_numpy(x).cuda()
    for op in (O.OP_U, O.OP_UT, O.OP_H, O.OP_A):
        assert np.array_equal(g.apply(op, xd).cpu().numpy(), o.apply(op, x)), op


def test_dense_rbf_c3_shape():
    """The shape of the dense RBF workload (20-component 3-D mixture, k-means
    clusters of 512, 3-point rotations, core 512) at n = 4,096: eight clusters
    of ~512 at the first stage, so the k-point search runs at its largest
    cluster size.  Bit-identical to the oracle."""
    a = I.rbf_mixture(4096, components=20, seed=2)
    g, o = _both(a, a.coords, k=3, eta=0.5, cluster_size=512, core_size=512, seed=0)
    sizes = np.diff(o.stages[0].offsets)
    assert len(sizes) == 8 and sizes.max() > 400, sizes
    assert_same_factorization(g, o)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("k", [2, 3])
def test_dense_update_kernels_agree_with_oracle(kernel, k):
    """The dense update in cluster-ordered TMA tiles (1, the default) and one
    CTA per row (2), each forced: bit-identical to the oracle, with ragged
    k-means clusters (runs padded to 16 columns) and a row count that leaves
    partial tiles."""
    pm = gpu_lib()
    L = pm.load()
    a = I.rbf_mixture(1000, components=7, seed=8)
    try:
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["dense_tiles"], 1 << 30, kernel) == 0
        g, o = _both(a, a.coords, k=k, eta=0.5, cluster_size=90, core_size=37, seed=4)
        assert_same_factorization(g, o)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)
