"""The sharded stage loop with the GPU stage calls (pmmf_shard_*) as each
rank's compute, against the oracle's single-process factorization: clusters,
rotations and H bit for bit, the error within 1e-12 relative.  One rank on
the GPU, and two ranks (processes) sharing the GPU, their rows and rotations
exchanged over gloo on the host; no kernel of one rank waits for the other."""

import os
import socket
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import shard_oracle_backend as B  # noqa: E402
from helpers import gpu, gpu_lib  # noqa: E402
from test_shard import _compare, _oracle  # noqa: E402

pytestmark = gpu


def _result(f):
    res = {"hdiag": f.hdiag, "core_idx": f.core_idx, "core": f.core, "error": [f.error],
           "nst": [len(f.stages)]}
    for p, s in enumerate(f.stages):
        res[f"coff{p}"], res[f"mem{p}"] = s.coff, s.members
        for nm in ("cluster", "kk", "idx", "O", "elim"):
            res[f"{nm}{p}"] = getattr(s.rot, nm).numpy()
    return res


def _run(name, exchange=None):
    from paper_1507_04396_gb300 import shard
    a, kw, labels = B.make_case(name)
    be = shard.GpuStageBackend(a.n, a.coords, labels=labels, **kw)
    try:
        return shard.factor_sharded(be, a.n, a.rowptr, a.col, a.val, core_size=kw["core_size"],
                                    k=kw["k"], exchange=exchange)
    finally:
        be.close()


@pytest.mark.parametrize("name", sorted(B.CASES))
def test_gpu_stage_calls_one_rank_match_oracle(name):
    gpu_lib()
    _compare(_result(_run(name)), _oracle(name))


def _rank(rank, world, port, name, outdir):
    import torch
    import torch.distributed as dist
    from paper_1507_04396_gb300 import shard
    torch.cuda.set_device(0)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = _run(name, shard.Exchange(comm_device="cpu"))
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), **_result(f))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["knn-k2", "poisson-bricks"])
def test_gpu_stage_calls_two_ranks_match_oracle(name, tmp_path):
    import torch.multiprocessing as mp
    gpu_lib()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.spawn(_rank, args=(2, port, name, str(tmp_path)), nprocs=2, join=True)
    o = _oracle(name)
    for r in range(2):
        _compare(dict(np.load(os.path.join(str(tmp_path), f"rank{r}.npz"))), o)
