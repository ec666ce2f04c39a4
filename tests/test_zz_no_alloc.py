"""pmmf_apply_noalloc: the matrix-free apply for callers that must not allocate
device memory (a solver or serving loop with a fixed memory budget, or a host
program whose allocator belongs to another framework).

Checks, through the C-ABI: two calls in a row give the same results as
pmmf_apply (bit for bit, the tolerance the apply parity tests use for these
ops), the device memory pool records no allocation during those calls, and an
oversize request fails with a clear error.  This file is collected last so
that a run stopping at its first failure has run every other test.
"""

import ctypes as C

import numpy as np
import pytest

from helpers import gpu, gpu_lib
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu

_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8   # CUmemPool_attribute values (cuda.h)


class _Pool:
    """High-water mark of the current device's default memory pool (driver API)."""

    def __init__(self, ordinal):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), ordinal) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, C.byref(z)) == 0


def test_noalloc_apply_matches_apply_twice_without_allocating():
    import torch
    pm = gpu_lib()
    a = I.knn_laplacian(3000, seed=5)
    f = pm.factor(a, k=2, eta=0.5, cluster_size=150, core_size=60, seed=6)
    nrhs = 4
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((a.n, nrhs))).cuda()
    ops = [pm.OP_U, pm.OP_UT, pm.OP_H, pm.OP_A, pm.OP_H_INV, pm.OP_A_INV, pm.OP_H_INV_SQRT,
           pm.OP_A_INV_SQRT]
    ref = {op: f.apply(op, x) for op in ops}   # allocating path; forms inverse, inverse sqrt
    outs = {op: [torch.empty_like(x), torch.empty_like(x)] for op in ops}
    torch.cuda.synchronize()

    pool = _Pool(torch.cuda.current_device())
    used_before = pool.get(_USED_MEM_CURRENT)
    allocs_before = pm.pmmf_alloc_count()
    pool.reset_high()
    for call in range(2):
        for op in ops:
            pm.pmmf_apply_noalloc(f.handle, op, x, outs[op][call], nrhs, nrhs)
    torch.cuda.synchronize()
    assert pool.get(_USED_MEM_HIGH) <= used_before, "the allocation-free apply allocated"
    assert pm.pmmf_alloc_count() == allocs_before, "the allocation-free apply requested memory"

    for op in ops:
        want = ref[op].cpu().numpy()
        for call in range(2):
            got = outs[op][call].cpu().numpy()
            assert np.array_equal(got, want), (op, call)
    # in place, twice
    y = x.clone()
    pm.pmmf_apply_noalloc(f.handle, pm.OP_A, y, y, nrhs, nrhs)
    pm.pmmf_apply_noalloc(f.handle, pm.OP_A, y, y, nrhs, nrhs)
    want = f.apply(pm.OP_A, f.apply(pm.OP_A, x))
    assert torch.equal(y, want)
    f.close()


def test_noalloc_rejects_oversize_and_unformed_inverse():
    import torch
    pm = gpu_lib()
    a = I.knn_laplacian(4096, seed=3)
    f = pm.factor(a, k=2, eta=0.5, cluster_size=256, core_size=2048, seed=1)
    assert f.info().core_size == 2048
    nrhs = 600                                   # 2048 * 600 > 2^20
    x = torch.zeros(a.n, nrhs, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(pm.PmmfError) as e:
        pm.pmmf_apply_noalloc(f.handle, pm.OP_A, x, y, nrhs, nrhs)
    assert e.value.status == pm.ERR_UNSUPPORTED and "1048576" in str(e.value)
    # rotations alone need no scratch and are allowed at any width
    pm.pmmf_apply_noalloc(f.handle, pm.OP_U, x, y, nrhs, nrhs)
    with pytest.raises(pm.PmmfError) as e:
        pm.pmmf_apply_noalloc(f.handle, pm.OP_A_INV, x[:, :2].contiguous(), y[:, :2].contiguous(), 2, 2)
    assert e.value.status == pm.ERR_INVALID_ARG
    with pytest.raises(pm.PmmfError) as e:
        pm.pmmf_apply_noalloc(f.handle, pm.OP_A_INV_SQRT, x[:, :2].contiguous(), y[:, :2].contiguous(), 2, 2)
    assert e.value.status == pm.ERR_INVALID_ARG
    f.close()


def test_noalloc_on_a_second_stream_right_after_forming():
    """The inverse and inverse square root are formed by pmmf_apply on one
    stream; pmmf_apply_noalloc then runs on a new stream with no synchronize
    in between.  Its results must equal the allocating apply's bit for bit
    (the formed reciprocals and core factors are complete once pmmf_apply
    returns from forming them)."""
    import torch
    pm = gpu_lib()
    a = I.knn_laplacian(2500, seed=11)
    f = pm.factor(a, k=2, eta=0.5, cluster_size=128, core_size=50, seed=2)
    nrhs = 8
    x = torch.from_numpy(np.random.default_rng(7).standard_normal((a.n, nrhs))).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        r_inv = f.apply(pm.OP_A_INV, x, stream=s1)        # forms the core inverse on s1
        r_isq = f.apply(pm.OP_A_INV_SQRT, x, stream=s1)   # forms core^{-1/2} on s1
    y_inv = torch.empty_like(x)
    y_isq = torch.empty_like(x)
    allocs_before = pm.pmmf_alloc_count()
    with torch.cuda.stream(s2):
        pm.pmmf_apply_noalloc(f.handle, pm.OP_A_INV, x, y_inv, nrhs, nrhs, s2)
        pm.pmmf_apply_noalloc(f.handle, pm.OP_A_INV_SQRT, x, y_isq, nrhs, nrhs, s2)
    torch.cuda.synchronize()
    assert pm.pmmf_alloc_count() == allocs_before
    assert torch.equal(y_inv, r_inv)
    assert torch.equal(y_isq, r_isq)
    f.close()
