"""A CPU backend of the sharded stage loop built from the oracle's own step
functions (test infrastructure): the floating-point steps are the oracle's,
so the sharded run is compared with the oracle's single-process
factorization.  Also the per-rank entry point of the multi-process tests."""

import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

from oracle import oracle as O  # noqa: E402
from paper_1507_04396_gb300.shard import Rows  # noqa: E402


class OracleStageBackend:
    device = torch.device("cpu")

    def __init__(self, n, coords, *, k, eta, cluster_size, core_size, seed, labels=None):
        self.n, self.coords, self.labels = n, coords, labels
        self.kw = dict(k=k, eta=eta, cluster_size=cluster_size, core_size=core_size, seed=seed)
        self.k = k

    def _full_csr(self, rows: Rows):
        """CSR over all n rows, the held rows filled in, the others empty."""
        lens = np.zeros(self.n, dtype=np.int64)
        lens[rows.ids.numpy()] = (rows.rowptr[1:] - rows.rowptr[:-1]).numpy()
        rp = np.zeros(self.n + 1, dtype=np.int64)
        rp[1:] = np.cumsum(lens)
        return rp, rows.col.numpy().astype(np.int32), rows.val.numpy()

    def clusters(self, p, act):
        coff, mem, e = O.step_clusters(self.n, self.coords, act.numpy(), p,
                                       labels=self.labels if p == 1 else None, **self.kw)
        return (torch.from_numpy(coff), torch.from_numpy(mem.astype(np.int64)),
                torch.from_numpy(e))

    def search(self, p, rows, act, coff, members, e, own):
        rp, col, val = self._full_csr(rows)
        rc, rk, ri, ro, re = O.step_search(self.n, rp, col, val, coff.numpy(),
                                           members.numpy().astype(np.int32), e.numpy(),
                                           own.numpy(), p, **self.kw)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x).astype(np.int64))
        return t(rc), t(rk), t(ri), torch.from_numpy(np.ascontiguousarray(ro)), t(re)

    def _transform(self, rows, coff, members, roff, rot):
        return O.step_transform(self.n, rows.rowptr.numpy(), rows.col.numpy().astype(np.int32),
                                rows.val.numpy(), coff.numpy(), members.numpy().astype(np.int32),
                                roff.numpy(), rot.kk.numpy().astype(np.int32),
                                rot.idx.numpy().astype(np.int32), rot.O.numpy(), self.k)

    def pass1(self, p, rows, act, coff, members, roff, rot):
        orp, oc, ov = self._transform(rows, coff, members, roff, rot)
        src = np.repeat(rows.ids.numpy(), np.diff(orp))
        order = np.lexsort((src, oc))                 # by W row y, then source row
        y, x, v = oc[order].astype(np.int64), src[order], ov[order]
        uid, cnt = np.unique(y, return_counts=True)
        rp = np.zeros(len(uid) + 1, dtype=np.int64)
        rp[1:] = np.cumsum(cnt)
        return Rows(torch.from_numpy(uid), torch.from_numpy(rp), torch.from_numpy(x),
                    torch.from_numpy(v))

    def pass2(self, p, wrows, act, coff, members, roff, rot):
        orp, oc, ov = self._transform(wrows, coff, members, roff, rot)
        elim = np.zeros(self.n, dtype=bool)
        elim[rot.elim.numpy()] = True
        ids = wrows.ids.numpy()
        keep_ids, keep_rp, kc, kv = [], [0], [], []
        h_ids, h_vals = [], []
        contrib = 0.0
        for r, y in enumerate(ids):
            c, v = oc[orp[r]:orp[r + 1]], ov[orp[r]:orp[r + 1]]
            if elim[y]:
                d = c == y
                if d.any():
                    h_ids.append(y)
                    h_vals.append(v[d][0])
                contrib += float(np.sum(v[~d] ** 2))
            else:
                ek = elim[c]
                contrib += float(np.sum(v[ek] ** 2))
                keep_ids.append(y)
                kc.append(c[~ek])
                kv.append(v[~ek])
                keep_rp.append(keep_rp[-1] + int((~ek).sum()))
        cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dtype=dt)
        out = Rows(torch.tensor(keep_ids, dtype=torch.int64), torch.tensor(keep_rp, dtype=torch.int64),
                   torch.from_numpy(cat(kc, np.int64)), torch.from_numpy(cat(kv, np.float64)))
        return (out, torch.tensor(h_ids, dtype=torch.int64), torch.tensor(h_vals, dtype=torch.float64),
                contrib)

    def sumsq(self, rows):
        return float(np.sum(rows.val.numpy() ** 2))


CASES = {
    "knn-k2": dict(gen=("knn_laplacian", dict(n=1500, seed=5)),
                   kw=dict(k=2, eta=0.5, cluster_size=100, core_size=40, seed=3)),
    "knn-k3": dict(gen=("knn_laplacian", dict(n=1200, seed=6)),
                   kw=dict(k=3, eta=0.5, cluster_size=90, core_size=40, seed=2)),
    "poisson-bricks": dict(gen=("poisson3d", dict(nx=10, seed=4)),
                           kw=dict(k=2, eta=0.5, cluster_size=50, core_size=30, seed=1),
                           bricks=(10, 10, 10, 5, 5, 2)),
}


def make_case(name):
    from paper_1507_04396_gb300 import inputs as I
    c = CASES[name]
    fn, args = c["gen"]
    a = getattr(I, fn)(**args)
    labels = I.grid_bricks(*c["bricks"]) if "bricks" in c else None
    return a, dict(c["kw"]), labels


def run_rank(rank, world, port, name, outdir):
    """One rank of a world-size `world` gloo run of the sharded stage loop."""
    import torch.distributed as dist
    from paper_1507_04396_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, kw, labels = make_case(name)
        be = OracleStageBackend(a.n, a.coords, labels=labels, **kw)
        f = shard.factor_sharded(be, a.n, a.rowptr, a.col, a.val, core_size=kw["core_size"],
                                 k=kw["k"], exchange=shard.Exchange())
        save = {"hdiag": f.hdiag, "core_idx": f.core_idx, "core": f.core,
                "error": np.array([f.error]), "nst": np.array([len(f.stages)])}
        for p, s in enumerate(f.stages):
            save[f"coff{p}"] = s.coff
            save[f"mem{p}"] = s.members
            for nm in ("cluster", "kk", "idx", "O", "elim"):
                save[f"{nm}{p}"] = getattr(s.rot, nm).numpy()
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), **save)
    finally:
        dist.destroy_process_group()
