"""The cluster-sharded stage loop (Sec. 2.3: clusters spread over ranks, the
stage's rotations all-gathered, rows exchanged between the two passes of the
blocked update and reblocked between stages).

With the oracle's own step functions as each rank's compute, the merged
factorization of a 2-rank gloo run (CPU processes) must equal the oracle's
single-process factorization: clusters, rotation tuples, blocks and
eliminations, H (diagonal and core) bit for bit, the error within 1e-12
relative (the residual's sums are added in another order).  A 1-rank run
without any process group checks the same on the loop alone."""

import os
import socket
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import shard_oracle_backend as B  # noqa: E402
from oracle import oracle as O  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _compare(res, o):
    assert res["nst"][0] == len(o.stages)
    for p, so in enumerate(o.stages):
        np.testing.assert_array_equal(res[f"coff{p}"], so.offsets)
        np.testing.assert_array_equal(res[f"mem{p}"], so.members)
        np.testing.assert_array_equal(res[f"cluster{p}"], so.rot_cluster)
        np.testing.assert_array_equal(res[f"kk{p}"], so.rot_k)
        np.testing.assert_array_equal(res[f"idx{p}"], so.rot_idx)
        np.testing.assert_array_equal(res[f"elim{p}"], so.rot_elim)
        assert np.array_equal(res[f"O{p}"].view(np.uint64), so.rot_O.view(np.uint64))
    np.testing.assert_array_equal(res["core_idx"], o.core_idx)
    assert np.array_equal(res["core"], o.core)
    assert np.array_equal(res["hdiag"].view(np.uint64), o.hdiag.view(np.uint64))
    assert abs(res["error"][0] - o.error) <= 1e-12 * o.error


def _oracle(name):
    a, kw, labels = B.make_case(name)
    o = O.factor(a.n, a.rowptr, a.col, a.val, a.coords, labels=labels, **kw)
    assert o.status == 0
    return o


@pytest.mark.parametrize("name", sorted(B.CASES))
def test_one_rank_loop_matches_oracle(name, tmp_path):
    from paper_1507_04396_gb300 import shard
    a, kw, labels = B.make_case(name)
    be = B.OracleStageBackend(a.n, a.coords, labels=labels, **kw)
    f = shard.factor_sharded(be, a.n, a.rowptr, a.col, a.val, core_size=kw["core_size"], k=kw["k"])
    res = {"hdiag": f.hdiag, "core_idx": f.core_idx, "core": f.core, "error": [f.error],
           "nst": [len(f.stages)]}
    for p, s in enumerate(f.stages):
        res[f"coff{p}"], res[f"mem{p}"] = s.coff, s.members
        for nm in ("cluster", "kk", "idx", "O", "elim"):
            res[f"{nm}{p}"] = getattr(s.rot, nm).numpy()
    _compare(res, _oracle(name))


@pytest.mark.parametrize("name", sorted(B.CASES))
def test_two_gloo_ranks_match_oracle(name, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(B.run_rank, args=(2, _free_port(), name, str(tmp_path)), nprocs=2, join=True)
    o = _oracle(name)
    for r in range(2):
        res = dict(np.load(os.path.join(str(tmp_path), f"rank{r}.npz")))
        _compare(res, o)
