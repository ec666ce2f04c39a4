"""The reduced-precision Gram matrix of the shortlist search, kernel by kernel.

`pmmf_gram_reduced` runs the factorization's own split and tensor-core Gram
(the tcgen05 kernel by default, the warp-level mma.sync kernel with
PMMF_TUNE_TC_GRAM = 1) on one set of rows.  Two definitions pin it:

* the split product P = hi hi^T + hi lo^T + lo hi^T, formed here in FP64 from
  the same split (TF32: float32 rounding, then to 10 fraction bits to nearest
  with ties away; BF16: to nearest even).  The products of TF32 or BF16 values
  are exact in FP32, so the kernel may differ from P only by its FP32 chunk
  sums of 48 products, the compensated sum of the chunks and the final FP32
  rounding: |G~ - P| <= (6 * 16 * 2^-24 + 2^-23) (|X||X|^T) with margin.  A
  dropped or doubled product term, a wrong operand layout or a wrong K step
  moves entries by about u |x||y| or more and fails;
* X X^T in FP64 within the certified bound of the shortlist,
  eps sqrt(G_ii G_jj).

Sizes span several 128 x 64 tiles with a ragged tail in rows and in K.
"""

import numpy as np
import pytest

from helpers import gpu, gpu_lib

pytestmark = gpu

EPS_CHUNK = 1.1 * (6 * 16 * 2.0 ** -24 + 2.0 ** -23)
EPS_CERT = {1: 1e-5, 2: 1e-4}   # TF32, BF16: above the certified eps (6.5e-6, 6.3e-5)


def _rna_tf32(f32):
    """float32 -> TF32 (10 fraction bits), to nearest, ties away from zero."""
    b = np.asarray(f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


def _rn_bf16(f32):
    """float32 -> BF16 (7 fraction bits), to nearest even."""
    b = np.asarray(f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _split(x, precision):
    rnd = _rna_tf32 if precision == 1 else _rn_bf16
    hi = rnd(x.astype(np.float32)).astype(np.float64)
    lo = rnd((x - hi).astype(np.float32)).astype(np.float64)
    return hi, lo


def _check(x, precision, kernel):
    pm = gpu_lib()
    L = pm.load()
    assert L.pmmf_set_tuning(pm.TUNE_PARAMS["tc_gram"], 1 << 30, kernel) == 0
    try:
        g = pm.pmmf_gram_reduced(x, precision).astype(np.float64)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)
    hi, lo = _split(x, precision)
    p = hi @ hi.T + hi @ lo.T + lo @ hi.T
    ax = np.abs(x)
    bound = EPS_CHUNK * (ax @ ax.T)
    err = np.abs(g - p)
    assert np.all(err <= bound), (float((err / np.maximum(bound, 1e-300)).max()), kernel)
    exact = x @ x.T
    d = np.sqrt(np.diag(exact))
    assert np.all(np.abs(g - exact) <= EPS_CERT[precision] * np.outer(d, d))
    # both triangles are stored, from one computation per pair
    np.testing.assert_array_equal(g, g.T)
    return g


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("kernel", [2, 1])
def test_split_product_ragged(precision, kernel):
    """200 rows (two row blocks of 128, four column blocks of 64, ragged) and
    300 terms (not a multiple of 8: zero padding, a partial chunk)."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal((200, 300))
    _check(x, precision, kernel)


@pytest.mark.parametrize("precision", [1, 2])
def test_split_product_cluster_shape(precision):
    """512 rows of 4,096 positive terms, the shape of one cluster of the dense
    RBF workload's first stage (values in (0, 1], varied magnitudes)."""
    rng = np.random.default_rng(12)
    x = np.exp(-rng.exponential(2.0, size=(512, 4096)))
    g5 = _check(x, precision, 2)
    g1 = _check(x, precision, 1)
    # the two kernels differ only in FP32 accumulation order inside a chunk
    ax = np.abs(x)
    assert np.all(np.abs(g5 - g1) <= 2 * EPS_CHUNK * (ax @ ax.T))


def test_single_row_and_short_rows():
    """Degenerate shapes: one row; rows of 1 and of 17 terms."""
    rng = np.random.default_rng(13)
    for rows, s in ((1, 64), (5, 1), (130, 17)):
        x = rng.standard_normal((rows, s))
        _check(x, 1, 2)
