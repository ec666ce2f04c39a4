"""Shared test helpers: library loading and GPU-vs-oracle comparison."""

import numpy as np
import pytest


def gpu_lib():
    """Build (if needed) and load the CUDA library; returns the binding module."""
    from paper_1507_04396_gb300 import build, pmmf
    build.build()
    pmmf.load()
    return pmmf


def factor_both(a, coords="auto", **kw):
    """Factor with the CUDA library and with the oracle on identical inputs."""
    from oracle import oracle as O
    pm = gpu_lib()
    g = pm.factor(a, coords=coords, record_stages=True, **kw)
    if isinstance(coords, str):
        coords = getattr(a, "coords", None)
    o = O.factor(a.n, a.rowptr, a.col, a.val, coords, record=True, **kw)
    assert o.status == 0
    return g, o


def assert_same_factorization(g, o, err_tol=1e-10, check_matrices=True):
    """Selections, rotations, stage matrices and H must match bit for bit;
    the relative Frobenius error within err_tol of the oracle's."""
    info = g.info()
    assert info.stages == len(o.stages), (info.stages, len(o.stages))
    for p, so in enumerate(o.stages):
        sg = g.stage(p)
        assert sg.active == so.active
        assert sg.clusters == len(so.offsets) - 1
        off, mem = g.clusters(p)
        np.testing.assert_array_equal(off, so.offsets)
        np.testing.assert_array_equal(mem, so.members)
        cl, kk, idx, O, el = g.rotations(p)
        assert len(el) == len(so.rot_elim)
        np.testing.assert_array_equal(cl, so.rot_cluster)
        np.testing.assert_array_equal(idx, so.rot_idx)
        np.testing.assert_array_equal(el, so.rot_elim)
        # rotation blocks bit for bit
        assert np.array_equal(O.view(np.uint64), so.rot_O.view(np.uint64)) or \
            np.array_equal(O, so.rot_O)
        if check_matrices and so.matrix is not None:
            rp, col, val = g.stage_matrix(p)
            orp, ocol, oval = so.matrix
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(col, ocol)
            np.testing.assert_array_equal(val, oval)
        assert abs(sg.contrib - so.contrib) <= 1e-10 * max(abs(so.contrib), o.norm_a ** 2 * 1e-16)
    hd, ci, core = g.h()
    np.testing.assert_array_equal(ci, o.core_idx)
    np.testing.assert_array_equal(core, o.core)
    np.testing.assert_array_equal(hd, o.hdiag)
    assert abs(info.error - o.error) <= err_tol * max(o.error, 1e-300) + 1e-15
    assert abs(info.norm_a - o.norm_a) <= 1e-12 * o.norm_a


gpu = pytest.mark.gpu
