"""Measurement aids of the library on the GPU: the FP64 throughput probe
(the roofline denominator of the FP64-bound kernels) returns a plausible rate
for a GB300-class part, and the allocation counter moves with a factorization."""

import pytest

from helpers import gpu, gpu_lib
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu


def test_fp64_probe_is_plausible():
    pm = gpu_lib()
    t = pm.pmmf_probe_fp64()
    # nominal FP64 of GB300 is 1.25 TFLOP/s; B200-class parts reach ~40
    assert 0.2 < t < 100.0, t


def test_alloc_counter_counts_factor_allocations():
    pm = gpu_lib()
    a = I.knn_laplacian(500, seed=1)
    n0 = pm.pmmf_alloc_count()
    pm.factor(a, k=2, eta=0.5, cluster_size=64, core_size=20, seed=0).close()
    assert pm.pmmf_alloc_count() > n0
