"""Offline sweep of the library's tunable launch shapes (run on the target GPU).

For each cluster-size bucket it factors a kNN Laplacian whose clusters fall in
that bucket, times the kernel family each parameter controls (CUDA events,
through the library's profiling hooks) for every candidate value, and writes
the fastest value per bucket to a JSON file keyed by bucket:

    {"device": ..., "buckets": {"rows_warps": [[256, 8], ...], ...},
     "timings_ms": {...}}

The binding applies that file at load time (``tuning.json`` beside it, or the
path in PMMF_TUNING).

    python -m paper_1507_04396_gb300.autotune [--out PATH] [--reps R]
"""

from __future__ import annotations

import argparse
import json
import os
import sys

BUCKETS = [128, 256, 512, 1024]
CANDIDATES = [1, 2, 4, 8]
FAMILY = {"rows_warps": "rows", "gram_warps": "gram"}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    import torch
    from . import build, inputs as I, pmmf
    build.build()
    pmmf.load()
    lib = pmmf.load()
    dev = torch.device("cuda", 0)
    result = {"device": torch.cuda.get_device_name(0), "buckets": {}, "timings_ms": {}}
    for param, family in FAMILY.items():
        table, timings = [], {}
        for bucket in BUCKETS:
            # clusters of about 3/4 of the bucket bound fall inside the bucket
            c = max(16, (3 * bucket) // 4)
            a = I.knn_laplacian(64 * c, 10, seed=5)
            A = I.SymCSR(a.n, torch.from_numpy(a.rowptr).to(dev), torch.from_numpy(a.col).to(dev),
                         torch.from_numpy(a.val).to(dev))
            co = torch.from_numpy(a.coords).to(dev)
            kw = dict(k=2, eta=0.5, cluster_size=c, core_size=c, seed=0, coords=co)
            best, best_ms = None, None
            for v in CANDIDATES:
                lib.pmmf_clear_tuning()
                pmmf._check(lib.pmmf_set_tuning(pmmf.TUNE_PARAMS[param], bucket, v))
                pmmf.factor(A, **kw).close()
                ms = []
                for _ in range(args.reps):
                    pmmf.pmmf_profile_begin([family])
                    pmmf.factor(A, **kw).close()
                    ms.append(pmmf.pmmf_profile_end()[family]["ms"])
                t = sorted(ms)[len(ms) // 2]
                timings[f"{bucket}:{v}"] = round(t, 4)
                if best_ms is None or t < best_ms:
                    best, best_ms = v, t
            table.append([bucket, best])
            print(f"{param} bucket <= {bucket}: best {best} ({best_ms:.3f} ms)", flush=True)
        result["buckets"][param] = table
        result["timings_ms"][param] = timings
    lib.pmmf_clear_tuning()
    out = args.out or pmmf.TUNING_PATH
    with open(out, "w") as fh:
        json.dump(result, fh, indent=1)
    print("wrote", out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
