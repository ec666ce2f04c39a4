"""Reduced-precision (TF32 / BF16 tensor-core) Gram shortlist on dense inputs.

The shortlist only screens partners; the choice is made on FP64 scores, so
the selections (clusters, tuples, eliminated coordinates) must equal the
oracle's, and the relative error must match the oracle's closely (stated per
test below).  The shortlist must stay short (full-row fallbacks rare), which
also shows that the tensor-core Gram is accurate to its bound.
"""

import numpy as np
import pytest

from helpers import gpu, gpu_lib
from oracle import oracle as O
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu


@pytest.fixture(autouse=True)
def _shortlist_on_every_stage():
    """These inputs are small: without a setting their stages would take the
    FP64 Gram (a stage uses the reduced-precision one only while it has at
    least 12 clusters).  Every stage takes the shortlist here (threshold 0)."""
    pm = gpu_lib()
    L = pm.load()
    assert L.pmmf_set_tuning(pm.TUNE_PARAMS["mixed_active"], 1 << 30, 0) == 0
    yield
    L.pmmf_clear_tuning()
    pm.apply_tuning(pm.TUNING_PATH)


def _run(a, precision, **kw):
    import torch
    pm = gpu_lib()
    dense = torch.from_numpy(a.to_dense()).cuda()
    return pm.factor(dense, coords=a.coords, precision=precision, **kw)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("k", [2, 3])
def test_shortlist_selects_like_fp64(precision, k):
    a = I.rbf_mixture(1024, components=8, seed=5)
    kw = dict(k=k, eta=0.5, cluster_size=128, core_size=64, seed=3)
    f64 = _run(a, 0, **kw)
    mp = _run(a, precision, **kw)
    assert mp.info().stages == f64.info().stages
    for p in range(f64.info().stages):
        r64, rmp = f64.rotations(p), mp.rotations(p)
        np.testing.assert_array_equal(rmp[2], r64[2])     # tuples
        np.testing.assert_array_equal(rmp[4], r64[4])     # eliminated coordinates
        # rotation blocks agree to FP64 rounding of differently ordered sums
        np.testing.assert_allclose(rmp[3], r64[3], rtol=0, atol=1e-9)
    e64, emp = f64.info().error, mp.info().error
    assert abs(emp - e64) <= 1e-8 * e64, (emp, e64)
    st = mp.precision_stats()
    assert st["steps"] == f64.info().rotations
    # the certified bound is a worst case (Cauchy-Schwarz on the row norms), so
    # the shortlists of a smooth kernel matrix hold tens of candidates; with
    # TF32 they stay well below the cluster size (BF16, 8 significant bits,
    # separates the leading candidates of this matrix less well)
    if precision == 1:
        assert st["rescored"] <= 0.25 * 128 * st["steps"], st


def test_shortlist_rejects_sparse_input():
    pm = gpu_lib()
    a = I.knn_laplacian(500, seed=1)
    with pytest.raises(pm.PmmfError) as e:
        pm.factor(a, k=2, eta=0.5, cluster_size=64, core_size=20, precision=1)
    assert e.value.status == pm.ERR_UNSUPPORTED


def _against_oracle(a, precision, **kw):
    mp = _run(a, precision, **kw)
    o = O.factor(a.n, a.rowptr, a.col, a.val, a.coords, **kw)
    assert o.status == 0
    assert mp.info().stages == len(o.stages)
    for p, so in enumerate(o.stages):
        off, mem = mp.clusters(p)
        np.testing.assert_array_equal(off, so.offsets)
        np.testing.assert_array_equal(mem, so.members)
        r = mp.rotations(p)
        np.testing.assert_array_equal(r[2], so.rot_idx)      # tuples
        np.testing.assert_array_equal(r[4], so.rot_elim)     # eliminated coordinates
        # the blocks come from FP64 rows rotated and re-dotted rather than an
        # FP64 Gram rotated: equal to rounding
        np.testing.assert_allclose(r[3], so.rot_O, rtol=0, atol=1e-9)
    hd, ci, core = mp.h()
    np.testing.assert_array_equal(ci, o.core_idx)
    # the error against the oracle's: relative gap stated and bounded
    gap = abs(mp.info().error - o.error) / o.error
    assert gap <= 1e-8, gap
    return mp, o


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("k", [2, 3])
def test_shortlist_selects_like_the_oracle(precision, k):
    """TF32 (1) and BF16 (2) shortlists against the FP64 oracle directly."""
    a = I.rbf_mixture(1024, components=8, seed=5)
    _against_oracle(a, precision, k=k, eta=0.5, cluster_size=128, core_size=64, seed=3)


@pytest.mark.parametrize("precision", [1, 2])
def test_shortlist_rbf_workload_shape(precision):
    """The dense RBF workload's shape (20-component mixture, clusters of 512,
    k = 3, core 512) at n = 2,048: four clusters of ~512 per early stage."""
    a = I.rbf_mixture(2048, components=20, seed=2)
    mp, o = _against_oracle(a, precision, k=3, eta=0.5, cluster_size=512, core_size=512, seed=0)
    assert np.diff(o.stages[0].offsets).max() > 400


def test_per_stage_choice_of_the_reduced_precision_gram():
    """With the default rule (reduced precision while a stage has at least 12
    clusters) the first stages of an n = 4,096 RBF matrix with clusters of 128
    (32, then 16 clusters) take the shortlist and the later ones the FP64
    Gram: the selections still equal the oracle's."""
    pm = gpu_lib()
    L = pm.load()
    L.pmmf_clear_tuning()
    pm.apply_tuning(pm.TUNING_PATH)
    a = I.rbf_mixture(4096, components=8, seed=6)
    mp, o = _against_oracle(a, 1, k=2, eta=0.5, cluster_size=128, core_size=64, seed=3)
    st = mp.precision_stats()
    assert st["steps"] > 0                                        # the first stage's shortlist
    assert st["steps"] < sum(len(x.rot_elim) for x in o.stages)   # not every stage's
