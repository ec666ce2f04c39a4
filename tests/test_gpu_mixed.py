"""Reduced-precision (TF32 / BF16 tensor-core) Gram shortlist on dense inputs.

The shortlist only screens partners; the choice is made on FP64 scores, so
the selections must equal those of the FP64 mode (which is bit-identical to
the oracle), and the relative error must match it closely.  The shortlist
must stay short (full-row fallbacks rare), which also shows that the
tensor-core Gram is accurate to its bound.
"""

import numpy as np
import pytest

from helpers import gpu, gpu_lib
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu


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
