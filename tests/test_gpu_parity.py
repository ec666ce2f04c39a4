"""CUDA path against the oracle, element by element, on identical seeded inputs.

Bar (integer and index work bit-exact; floating point bit-exact wherever both
sides run the same operation sequence):
  - clusters, selected rotation tuples, eliminated coordinates: identical;
  - rotation blocks (c, s), every stage's compacted A_p, H: identical bits;
  - relative Frobenius error within 1e-10 (relative) of the oracle's (the
    residual sums are accumulated in a different order);
  - U x, U^T x, H x, A~ x: identical bits; A~^{-1} x within 1e-10 relative
    (the core is inverted by Gauss-Jordan on the GPU, by Cholesky in the oracle).
"""

import numpy as np
import pytest

from helpers import assert_same_factorization, factor_both, gpu, gpu_lib
from oracle import oracle as O
from paper_1507_04396_gb300 import inputs as I

pytestmark = gpu


def test_dense_one_cluster_small_case():
    """Dense PSD X X^T/64 + 0.1 I, n = 256, one cluster, core 16 (4 stages, 240 rotations)."""
    a = I.psd_dense(256, 64, seed=0)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=256, core_size=16, seed=0)
    assert o.total_rotations() == 240 and len(o.stages) == 4
    assert_same_factorization(g, o)


@pytest.mark.parametrize("n,c,core", [(4096, 256, 64), (3000, 200, 100), (1500, 97, 31)])
def test_knn_laplacian_clustered(n, c, core):
    """kNN-graph Laplacian with k-means clusters, ragged cluster sizes."""
    a = I.knn_laplacian(n, seed=1)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=c, core_size=core, seed=3)
    assert_same_factorization(g, o)


def test_full_size_bench_workload():
    """The benchmark's own configuration (n = 65,536 kNN Laplacian, clusters of
    ~256, core 256), compared in full: every stage's clusters, rotations and
    A_p, and H."""
    a = I.knn_laplacian(65536, 10, seed=1)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=256, core_size=256, seed=0)
    assert len(o.stages) == 9 and o.total_rotations() == 65280
    assert_same_factorization(g, o)


@pytest.mark.parametrize("eta", [0.25, 0.7])
def test_other_compression_ratios(eta):
    a = I.knn_laplacian(2000, seed=2)
    g, o = factor_both(a, k=2, eta=eta, cluster_size=128, core_size=40, seed=9)
    assert_same_factorization(g, o)


def test_poisson_3d_clusters():
    a = I.poisson3d(12, seed=4)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=64, core_size=50, seed=4)
    assert_same_factorization(g, o)


def test_ties_on_integer_grid_laplacian():
    """Integer-valued grid Laplacian: many equal scores exercise the tie rules."""
    a = I.poisson3d(8, sigma=0.0, seed=0)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=64, core_size=16, seed=1)
    assert_same_factorization(g, o)


def test_edge_cases():
    # n = 1: nothing to rotate, H = A
    a = I.from_dense(np.array([[3.0]]))
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=2, core_size=1, seed=0)
    assert g.info().stages == 0
    assert_same_factorization(g, o)
    # n = 2, core 1: a single rotation
    a = I.from_dense(np.array([[2.0, 0.7], [0.7, 1.0]]))
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=2, core_size=1, seed=0)
    assert_same_factorization(g, o)
    # diagonal: every score 0, identity rotations, zero error
    a = I.from_dense(np.diag(np.arange(1.0, 65.0)))
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=64, core_size=4, seed=5)
    assert_same_factorization(g, o)
    assert g.info().error == 0.0
    # stage limit and a core larger than half of n
    a = I.knn_laplacian(800, seed=7)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=100, core_size=10, seed=2, max_stages=2)
    assert g.info().stages == 2
    assert_same_factorization(g, o)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=100, core_size=700, seed=2)
    assert_same_factorization(g, o)
    # clusters of one coordinate cannot rotate: falls back to one cluster
    a = I.knn_laplacian(40, seed=8)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=2, core_size=39, seed=2)
    assert_same_factorization(g, o)


def test_exact_block_sum():
    a = I.block_pairs(128, k=2, seed=3)
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=256, core_size=128, seed=1)
    assert_same_factorization(g, o)
    assert g.info().error <= 1e-14


def test_input_forms_agree():
    """Host CSR, device CSR and dense input give identical factorizations."""
    import torch
    pm = gpu_lib()
    a = I.psd_dense(96, 20, seed=4)
    kw = dict(k=2, eta=0.5, cluster_size=96, core_size=8, seed=2)
    f1 = pm.factor(a, **kw)
    dev = I.SymCSR(a.n, torch.from_numpy(a.rowptr).cuda(), torch.from_numpy(a.col).cuda(),
                   torch.from_numpy(a.val).cuda())
    f2 = pm.factor(dev, coords=None, **kw)
    f3 = pm.factor(torch.from_numpy(a.to_dense()).cuda(), coords=None, **kw)
    for f in (f2, f3):
        for p in range(f1.info().stages):
            assert np.array_equal(f1.rotations(p)[3], f.rotations(p)[3])
        assert np.array_equal(f1.h()[0], f.h()[0])


def test_apply_matches_oracle():
    import torch
    a = I.knn_laplacian(3000, seed=5)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=150, core_size=60, seed=6)
    x = np.random.default_rng(0).standard_normal((a.n, 3))
    xd = torch.from_numpy(x).cuda()
    for op in (O.OP_U, O.OP_UT, O.OP_H, O.OP_A):
        y = g.apply(op, xd).cpu().numpy()
        assert np.array_equal(y, o.apply(op, x)), op
    for op in (O.OP_A_INV, O.OP_H_INV):
        y = g.apply(op, xd).cpu().numpy()
        want = o.apply(op, x)
        assert np.abs(y - want).max() <= 1e-10 * np.abs(want).max(), op
    # in place and a single vector
    z = xd[:, 0].contiguous()
    g.apply(O.OP_U, z, z)
    assert np.array_equal(z.cpu().numpy(), o.apply(O.OP_U, x[:, :1])[:, 0])


def test_pcg_matches_oracle():
    import torch
    a = I.poisson3d(14, seed=4)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=64, core_size=64, seed=4)
    b = np.random.default_rng(4).standard_normal((a.n, 4))
    st, x, iters, rel = g.solve(a, torch.from_numpy(b).cuda(), rtol=1e-8, maxit=500)
    ost, ox, oit, orel = o.pcg(a, b, 1e-8, 500)
    assert st == 0 and ost == 0
    assert (rel <= 1e-8 * 1.5).all()
    assert (np.abs(iters - oit) <= 2).all(), (iters, oit)
    np.testing.assert_allclose(x.cpu().numpy(), ox, rtol=0, atol=1e-6 * np.abs(ox).max())


def test_rejects_bad_input():
    pm = gpu_lib()
    a = I.psd_dense(32, 8, seed=1)
    val = a.val.copy()
    val[3] += 1.0
    with pytest.raises(pm.PmmfError) as e:
        pm.factor(I.SymCSR(a.n, a.rowptr, a.col, val), k=2, eta=0.5, cluster_size=32, core_size=4)
    assert e.value.status == pm.ERR_NOT_SYMMETRIC
    val = a.val.copy()
    val[0] = np.inf
    with pytest.raises(pm.PmmfError) as e:
        pm.factor(I.SymCSR(a.n, a.rowptr, a.col, val), k=2, eta=0.5, cluster_size=32, core_size=4)
    assert e.value.status == pm.ERR_NONFINITE
    with pytest.raises(pm.PmmfError) as e:
        pm.factor(a, k=9, eta=0.5, cluster_size=32, core_size=4)
    assert e.value.status == pm.ERR_INVALID_ARG
    with pytest.raises(pm.PmmfError) as e:
        pm.factor(a, k=2, eta=1.5, cluster_size=32, core_size=4)
    assert e.value.status == pm.ERR_INVALID_ARG


def test_allocation_failure_is_clean():
    """A failing device allocation returns OOM and leaves no handle behind."""
    import subprocess
    import sys
    import os
    code = (
        "import sys; sys.path.insert(0, '.');"
        "from paper_1507_04396_gb300 import inputs as I, pmmf as pm;"
        "a = I.knn_laplacian(2000, seed=1);"
        "import torch; torch.cuda.init();"
        "\ntry:\n    pm.factor(a, k=2, eta=0.5, cluster_size=128, core_size=40)\n"
        "    print('NOERR')\nexcept pm.PmmfError as e:\n    print('STATUS', e.status)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    gpu_lib()
    for after in (0, 5, 40):
        env = dict(os.environ, PMMF_FAIL_ALLOC_AFTER=str(after))
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                           text=True, timeout=300)
        assert "STATUS 4" in r.stdout, r.stdout + r.stderr


@gpu
def test_given_stage1_bricks():
    """Stage 1 from given clusters (8 x 8 x 4 grid bricks, the structured-grid
    rule), k-means afterwards: bit-identical to the oracle with the same
    labels, from host or device labels; a label out of range is rejected."""
    import torch
    a = I.poisson3d(16, seed=4)
    lab = I.grid_bricks(16, 16, 16, 8, 8, 4)
    kw = dict(k=2, eta=0.5, cluster_size=256, core_size=64, seed=4)
    g, o = factor_both(a, labels=lab, **kw)
    assert_same_factorization(g, o)
    off, mem = g.clusters(0)
    assert len(off) - 1 == 16
    assert np.array_equal(mem[off[3]:off[4]], np.nonzero(lab == 3)[0])
    pm = gpu_lib()
    g2 = pm.factor(a, labels=torch.from_numpy(lab).cuda(), **kw)
    for p in range(g.info().stages):
        assert np.array_equal(g.rotations(p)[3], g2.rotations(p)[3])
    bad = lab.copy()
    bad[100] = 99
    with pytest.raises(pm.PmmfError) as ei:
        pm.pmmf_factor(*_params_with_labels(pm, a, bad, 16, kw))
    assert ei.value.status == pm.ERR_INVALID_ARG


def _params_with_labels(pm, a, lab, num, kw):
    """Raw C-ABI arguments with num_labels fixed (the binding derives it)."""
    m, keep = pm.make_matrix(a)
    co = np.ascontiguousarray(a.coords)
    prm = pm.Params(kw["k"], kw["eta"], kw["cluster_size"], kw["core_size"], kw["seed"], 0, 10,
                    co.ctypes.data, 3, pm.HOST, 0, 0, lab.ctypes.data, pm.HOST, num)
    _params_with_labels.keep = (keep, co, lab)
    return m, prm


@gpu
def test_short_pass1_estimate_retries_exactly():
    """The blocked update allocates its intermediate from an estimate and
    redoes the pass at the exact size when the estimate is short: with the
    first-stage estimate forced to 1x the input the result is still the
    oracle's, bit for bit."""
    pm = gpu_lib()
    L = pm.load()
    a = I.knn_laplacian(3000, seed=5)
    try:
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["pass1_estimate"], 1, 1) == 0
        g, o = factor_both(a, k=2, eta=0.5, cluster_size=150, core_size=60, seed=6)
        assert_same_factorization(g, o)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)


@gpu
@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("mode", ["reach", "levels"])
def test_counting_pass_modes_agree_with_oracle(k, mode):
    """The blocked update's counting passes take the fill pattern either from
    per-cluster reach sets or by running the rotation levels on the pattern
    (chosen by the stage's cluster count); each mode, forced on every stage,
    gives the oracle's factorization bit for bit (k = 2 and k-point)."""
    pm = gpu_lib()
    L = pm.load()
    a = I.knn_laplacian(3000, seed=5)
    try:
        thr = 1 if mode == "reach" else (1 << 30)
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["reach_clusters"], 1, thr) == 0
        g, o = factor_both(a, k=k, eta=0.5, cluster_size=150, core_size=60, seed=6)
        assert_same_factorization(g, o)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)


@gpu
@pytest.mark.parametrize("case", ["gaps", "one-label", "two-stages"])
def test_stage_pipeline_edge_cases(case):
    """Stage-1 labels with unused label values or a single label, and a run
    stopped after two stages (the next stage's clustering is then never
    started): bit-identical to the oracle."""
    a = I.poisson3d(12, seed=3)
    kw = dict(k=2, eta=0.5, cluster_size=96, core_size=40, seed=2)
    if case == "gaps":
        lab = I.grid_bricks(12, 12, 12, 6, 6, 4) * 3 + 1       # values 1, 4, 7, ...
        g, o = factor_both(a, labels=lab, **kw)
        assert len(g.clusters(0)[0]) - 1 == int(lab.max() // 3) + 1
    elif case == "one-label":
        lab = np.zeros(a.n, dtype=np.int32)
        g, o = factor_both(a, labels=lab, **kw)
        assert len(g.clusters(0)[0]) == 2
    else:
        g, o = factor_both(a, max_stages=2, **kw)
        assert g.info().stages == 2
    assert_same_factorization(g, o)


@gpu
def test_concurrent_host_threads_match_oracle():
    """Two host threads factor at the same time, each on its own CUDA stream
    (each thread has its own mapped readback words and its own side stream):
    both factorizations equal the oracle's, bit for bit."""
    import threading
    import torch
    pm = gpu_lib()
    cases = [I.knn_laplacian(3000, seed=5), I.knn_laplacian(2500, seed=7)]
    kw = dict(k=2, eta=0.5, cluster_size=150, core_size=60, seed=6)
    out = [None, None]
    errs = []

    def run(q):
        try:
            s = torch.cuda.Stream()
            f = pm.factor(cases[q], record_stages=True, stream=s, **kw)
            s.synchronize()
            out[q] = f
        except Exception as e:  # reported below, on the main thread
            errs.append(e)

    threads = [threading.Thread(target=run, args=(q,)) for q in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    for q, a in enumerate(cases):
        o = O.factor(a.n, a.rowptr, a.col, a.val, a.coords, record=True, **kw)
        assert o.status == 0
        assert_same_factorization(out[q], o)


@pytest.mark.parametrize("k", [2, 3])
def test_apply_eight_right_hand_sides(k):
    """Eight right-hand sides take the apply kernels' fixed-width
    instantiations (the width the solvers use): U, U^T, H, A~ bit for bit;
    the inverse ops to the tolerance of the other apply tests.  Also a strided
    block (ld > nrhs), which takes the element-wise copy."""
    import torch
    a = I.knn_laplacian(2400, seed=12)
    g, o = factor_both(a, k=k, eta=0.5, cluster_size=120, core_size=48, seed=5)
    x = np.random.default_rng(8).standard_normal((a.n, 8))
    xd = torch.from_numpy(x).cuda()
    for op in (O.OP_U, O.OP_UT, O.OP_H, O.OP_A):
        assert np.array_equal(g.apply(op, xd).cpu().numpy(), o.apply(op, x)), op
    for op, tol in ((O.OP_A_INV, 1e-10), (O.OP_H_INV, 1e-10), (O.OP_A_INV_SQRT, 1e-9),
                    (O.OP_H_INV_SQRT, 1e-9)):
        want = o.apply(op, x)
        got = g.apply(op, xd).cpu().numpy()
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), op
    pm = gpu_lib()
    ld = 11
    wide = torch.zeros(a.n, ld, dtype=torch.float64, device="cuda")
    wide[:, :8] = xd
    out = torch.full_like(wide, 7.0)
    for op in (O.OP_U, O.OP_A):
        pm.pmmf_apply(g.handle, op, wide, out, 8, ld)
        torch.cuda.synchronize()
        assert np.array_equal(out[:, :8].cpu().numpy(), o.apply(op, x)), op
        assert bool((out[:, 8:] == 7.0).all())


def test_wide_search_cta_clusters_above_512():
    """Clusters of ~600 coordinates: the k = 2 search runs its 512-thread CTA
    (12 column warps) on a single factorization, not only in a batch."""
    a = I.knn_laplacian(6000, seed=13)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=600, core_size=100, seed=3)
    sizes = np.diff(o.stages[0].offsets)
    assert sizes.max() > 512 and sizes.max() <= 1536, sizes
    assert_same_factorization(g, o)


def test_generic_search_one_cluster_above_1536():
    """One cluster of 2,048 coordinates (no points: one cluster per stage):
    the first stage runs the generic k = 2 search kernel (beyond 1,536
    coordinates), later stages the 512- and 256-thread ones; U, U^T and A~
    applied bit for bit."""
    import torch
    a = I.knn_laplacian(2048, seed=14)
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=2048, core_size=64, seed=4)
    assert len(o.stages[0].offsets) == 2 and o.stages[0].active == 2048
    assert_same_factorization(g, o)
    # the apply reads a cluster this large's rotations from global memory
    # (they are staged in shared memory up to 1,024 coordinates)
    x = np.random.default_rng(2).standard_normal((a.n, 8))
    xd = torch.from_numpy(x).cuda()
    for op in (O.OP_U, O.OP_UT, O.OP_A):
        assert np.array_equal(g.apply(op, xd).cpu().numpy(), o.apply(op, x)), op


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("case", ["knn-k2", "knn-k3", "poisson-bricks", "small-clusters", "c700"])
def test_update_kernels_agree_with_oracle(kernel, case):
    """The blocked update with one warp per row (1) and with one thread per row
    applying only the rotations that reach each segment's pattern (2), forced
    on every stage: the oracle's factorization bit for bit (every stage's A_p),
    for Givens and 3-point rotations, given bricks, clusters of ~8 (patterns
    within the shared-memory slots) and of ~700 (patterns that spill into the
    global slots)."""
    pm = gpu_lib()
    L = pm.load()
    if case == "knn-k2":
        a, kw = I.knn_laplacian(3000, seed=5), dict(k=2, cluster_size=150, core_size=60)
    elif case == "knn-k3":
        a, kw = I.knn_laplacian(3000, seed=5), dict(k=3, cluster_size=150, core_size=60)
    elif case == "poisson-bricks":
        a, kw = I.poisson3d(16, seed=4), dict(k=2, cluster_size=128, core_size=64,
                                               labels=I.grid_bricks(16, 16, 16, 8, 8, 2))
    elif case == "small-clusters":
        a, kw = I.knn_laplacian(1200, seed=9), dict(k=2, cluster_size=8, core_size=30)
    else:
        a, kw = I.knn_laplacian(4096, seed=3), dict(k=2, cluster_size=700, core_size=256)
    try:
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["rows_kernel"], 1 << 30, kernel) == 0
        g, o = factor_both(a, eta=0.5, seed=6, **kw)
        assert_same_factorization(g, o)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", ["knn-c256", "knn-c300", "poisson-bricks", "small-clusters", "many-clusters"])
def test_search_by_thread_block_clusters_agrees_with_oracle(mode, case):
    """The k = 2 search with G and M in global memory, one CTA per cluster (1),
    and held row-sliced in the shared memory of a thread-block cluster of 8
    CTAs (2), forced on every stage: the oracle's factorization bit for bit.
    Clusters of ~256 and of up to 306 (39 rows per CTA), given bricks,
    clusters of ~8 (CTAs without rows) and a stage of 256 clusters (more
    thread-block clusters than can be resident at once)."""
    pm = gpu_lib()
    L = pm.load()
    if case == "knn-c256":
        a, kw = I.knn_laplacian(4096, seed=3), dict(cluster_size=256, core_size=64)
    elif case == "knn-c300":
        a, kw = I.knn_laplacian(4500, seed=4), dict(cluster_size=265, core_size=100)
    elif case == "poisson-bricks":
        a, kw = I.poisson3d(16, seed=4), dict(cluster_size=128, core_size=64,
                                               labels=I.grid_bricks(16, 16, 16, 8, 8, 2))
    elif case == "small-clusters":
        a, kw = I.knn_laplacian(1200, seed=9), dict(cluster_size=8, core_size=30)
    else:
        a, kw = I.knn_laplacian(65536, seed=1), dict(cluster_size=256, core_size=256, max_stages=1)
    try:
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["select_dsm"], 1 << 30, mode) == 0
        g, o = factor_both(a, k=2, eta=0.5, seed=6, **kw)
        # every stage's clusters within the shared-memory limit of mode 2
        # (up to 318 coordinates: 40 rows of G and M per CTA)
        assert max(int(np.diff(st.offsets).max()) for st in o.stages) <= 318
        if case == "knn-c300":
            assert np.diff(o.stages[0].offsets).max() > 300
        assert_same_factorization(g, o)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", ["knn-k2", "knn-k3", "poisson-bricks"])
@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_apply_passes_agree_with_oracle(mode, case, nrhs):
    """The apply's rotation passes as one launch per stage (1) and as one
    cooperative launch per pass with a grid barrier between stages (2),
    forced: U, U^T, H, A~ bit for bit with the oracle, A~^-1 to the inverse
    ops' tolerance, for 1, 3 and 8 right-hand sides; the PCG solve (its
    iteration replayed as a CUDA graph) agrees with the oracle's."""
    import torch
    pm = gpu_lib()
    L = pm.load()
    if case == "knn-k2":
        a, kw = I.knn_laplacian(5000, seed=2), dict(k=2, cluster_size=200, core_size=64)
    elif case == "knn-k3":
        a, kw = I.knn_laplacian(3000, seed=5), dict(k=3, cluster_size=150, core_size=60)
    else:
        a, kw = I.poisson3d(16, seed=4), dict(k=2, cluster_size=128, core_size=64,
                                               labels=I.grid_bricks(16, 16, 16, 8, 8, 2))
    try:
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["apply_fused"], 1 << 30, mode) == 0
        g, o = factor_both(a, eta=0.5, seed=7, **kw)
        x = np.random.default_rng(nrhs).standard_normal((a.n, nrhs))
        xd = torch.from_numpy(x).cuda()
        for op in (O.OP_U, O.OP_UT, O.OP_H, O.OP_A):
            assert np.array_equal(g.apply(op, xd).cpu().numpy(), o.apply(op, x)), op
        want = o.apply(O.OP_A_INV, x)
        got = g.apply(O.OP_A_INV, xd).cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
        if nrhs == 8 and case != "knn-k3":
            st, xs, iters, rel = g.solve(a, xd, rtol=1e-8, maxit=500)
            ost, ox, oit, orel = o.pcg(a, x, 1e-8, 500)
            assert st == 0 and ost == 0
            assert (rel <= 1e-8 * 1.5).all()
            assert (np.abs(iters - oit) <= 2).all(), (iters, oit)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)


@pytest.mark.parametrize("blocks", [3, 4])
@pytest.mark.parametrize("case", ["c150", "c300", "c8"])
def test_search_occupancy_variants_agree_with_oracle(blocks, case):
    """The k = 2 search with its registers capped for 3 and 4 CTAs per SM
    (the instantiations a stage with many clusters takes), forced on every
    stage: the oracle's factorization bit for bit, for clusters of ~150
    (two columns per thread), ~300 (four) and ~8 (one)."""
    pm = gpu_lib()
    L = pm.load()
    if case == "c150":
        a, kw = I.knn_laplacian(3000, seed=5), dict(cluster_size=150, core_size=60)
    elif case == "c300":
        a, kw = I.knn_laplacian(4800, seed=8), dict(cluster_size=300, core_size=100)
    else:
        a, kw = I.knn_laplacian(1200, seed=9), dict(cluster_size=8, core_size=30)
    try:
        assert L.pmmf_set_tuning(pm.TUNE_PARAMS["select_blocks"], 1 << 30, blocks) == 0
        g, o = factor_both(a, k=2, eta=0.5, seed=6, **kw)
        assert_same_factorization(g, o)
    finally:
        L.pmmf_clear_tuning()
        pm.apply_tuning(pm.TUNING_PATH)


@pytest.mark.parametrize("c", [430, 436, 440])
def test_search_dynamic_shared_memory_just_under_48k(c):
    """One cluster of ~436 coordinates: the search's dynamic shared memory is
    just under 48 KB (48,928 bytes at 436), its static shared memory takes the
    block over the default limit, so the launch must opt in; bit for bit with
    the oracle."""
    a = I.knn_laplacian(c, seed=15)
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=c, core_size=16, seed=80)
    assert o.stages[0].active == c and len(o.stages[0].offsets) == 2
    assert_same_factorization(g, o)
