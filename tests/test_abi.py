"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pmmf.h declares.  Runs without a GPU: only argument validation is
exercised (it returns before any CUDA call)."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pmmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmmf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_04396_gb300 import build, pmmf
    build.build()
    return pmmf.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pmmf_factor", "pmmf_apply", "pmmf_solve_precond", "pmmf_free"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1507_04396_gb300 import pmmf
    assert sorted(pmmf.EXPORTS) == declared_functions()


def test_invalid_parameters_rejected_without_gpu(lib):
    from paper_1507_04396_gb300 import inputs as I
    from paper_1507_04396_gb300 import pmmf
    a = I.psd_dense(16, 4, seed=1)
    m, keep = pmmf.make_matrix(a)
    bad = [
        pmmf.Params(1, 0.5, 16, 4, 0, 0, 10, None, 0, 0, 0),       # k < 2
        pmmf.Params(2, 1.0, 16, 4, 0, 0, 10, None, 0, 0, 0),       # eta >= 1
        pmmf.Params(2, 0.5, 1, 4, 0, 0, 10, None, 0, 0, 0),        # cluster < k
        pmmf.Params(2, 0.5, 16, 0, 0, 0, 10, None, 0, 0, 0),       # core < 1
        pmmf.Params(2, 0.5, 16, 17, 0, 0, 10, None, 0, 0, 0),      # core > n
    ]
    for prm in bad:
        h = C.c_void_p()
        st = lib.pmmf_factor(C.byref(m), C.byref(prm), C.byref(h), None)
        assert st == pmmf.ERR_INVALID_ARG
        assert h.value is None
        assert lib.pmmf_last_error()
    prm = pmmf.Params(9, 0.5, 16, 4, 0, 0, 10, None, 0, 0, 0)    # k > 8
    h = C.c_void_p()
    assert lib.pmmf_factor(C.byref(m), C.byref(prm), C.byref(h), None) == pmmf.ERR_INVALID_ARG
    lib.pmmf_free(None)   # NULL-safe
    # the reduced-precision Gram diagnostic checks its arguments before any
    # device work
    x = np.ones((4, 8))
    g = np.zeros((4, 4), dtype=np.float32)
    for args in ((None, 4, 8, 1, g.ctypes.data), (x.ctypes.data, 4, 8, 0, g.ctypes.data),
                 (x.ctypes.data, 0, 8, 1, g.ctypes.data), (x.ctypes.data, 4097, 8, 1, g.ctypes.data),
                 (x.ctypes.data, 4, 0, 2, g.ctypes.data), (x.ctypes.data, 4, 8, 2, None)):
        assert lib.pmmf_gram_reduced(*args, None) == pmmf.ERR_INVALID_ARG
        assert lib.pmmf_last_error()


def test_tuning_table_validation_and_json(tmp_path):
    """Launch-shape tuning: argument checks and the JSON the autotuner writes."""
    import json
    from paper_1507_04396_gb300 import pmmf
    lib = pmmf.load()
    assert lib.pmmf_set_tuning(0, 256, 4) == pmmf.OK
    assert lib.pmmf_set_tuning(12, 256, 4) == pmmf.ERR_INVALID_ARG    # unknown parameter
    assert lib.pmmf_set_tuning(11, 256, 1) == pmmf.OK                 # warp-level mma.sync Gram
    assert lib.pmmf_set_tuning(11, 256, 2) == pmmf.OK                 # tcgen05 Gram
    assert lib.pmmf_set_tuning(11, 256, 3) == pmmf.ERR_INVALID_ARG    # only 1 or 2
    assert lib.pmmf_set_tuning(10, 256, 0) == pmmf.OK                 # reduced precision on every stage
    assert lib.pmmf_set_tuning(9, 256, 5) == pmmf.ERR_INVALID_ARG     # 2..4 search CTAs per SM
    assert lib.pmmf_set_tuning(0, 0, 4) == pmmf.ERR_INVALID_ARG       # empty bucket
    assert lib.pmmf_set_tuning(1, 512, 0) == pmmf.ERR_INVALID_ARG     # value out of range
    assert lib.pmmf_set_tuning(2, 512, 16) == pmmf.OK                 # search width
    assert lib.pmmf_set_tuning(2, 512, 12) == pmmf.ERR_INVALID_ARG    # only 8 or 16 warps
    assert lib.pmmf_set_tuning(3, 1, 4) == pmmf.OK                    # pass-1 estimate
    assert lib.pmmf_set_tuning(3, 1, 33) == pmmf.ERR_INVALID_ARG      # above 32
    assert lib.pmmf_set_tuning(4, 1, 1 << 30) == pmmf.OK              # reach threshold
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps({"buckets": {"rows_warps": [[256, 4], [1024, 2]],
                                            "gram_warps": [[512, 8]]}}))
    assert pmmf.apply_tuning(str(path))
    assert not pmmf.apply_tuning(str(tmp_path / "missing.json"))
    lib.pmmf_clear_tuning()
