"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or mathematics fixes:
published generator outputs, closed forms, dense-matrix identities computed with
numpy, brute force on tiny inputs, invariants, and special cases whose exact
answer is known.  None of these runs the CUDA library.
"""

import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_04396_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


# ---------------------------------------------------------------- random picks

def test_splitmix64_known_answer():
    """Counter-based generator (R5) equals the published splitmix64 outputs."""
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.startswith("0x")]
    assert O.splitmix64_stream(0, 3) == want


def test_pick_range_and_uniformity():
    """The pick maps 64-bit draws onto [0, count) and is uniform (chi-square)."""
    assert O.pick(0, 7) == 0
    assert O.pick(2 ** 64 - 1, 7) == 6
    counts = np.zeros(7)
    for t in range(70000):
        counts[O.pick(O.draw(123, 1, 2, t), 7)] += 1
    chi2 = ((counts - 10000.0) ** 2 / 10000.0).sum()
    assert chi2 < 30.0          # 6 dof: P(chi2 > 30) < 1e-4


# ---------------------------------------------------------------- rotations

def _offdiag_after(a, b, d, c, s):
    """Off-diagonal entry of q [[a,b],[b,d]] q^T with q = [[c,-s],[s,c]] (R1)."""
    q = np.array([[c, -s], [s, c]])
    g = np.array([[a, b], [b, d]])
    return (q @ g @ q.T)[0, 1]


@pytest.mark.parametrize("seed", range(20))
def test_jacobi2_zeroes_offdiagonal_smaller_angle(seed):
    """Sec. 2.2: the angle diagonalizes the 2x2 Gram block; |theta| <= pi/4."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((5, 2)) * rng.uniform(0.1, 10.0, 2)
    g = x.T @ x
    a, b, d = g[0, 0], g[0, 1], g[1, 1]
    c, s = O.jacobi2(a, b, d)
    assert abs(c * c + s * s - 1.0) <= 4 * U
    scale = abs(a) + abs(b) + abs(d)
    assert abs(_offdiag_after(a, b, d, c, s)) <= 1e-14 * scale
    assert c > 0 and abs(s) <= c * (1 + 4 * U)
    # theta-grid scan: the chosen angle is the root of smaller magnitude
    th = np.linspace(-np.pi / 2, np.pi / 2, 200001)
    f = np.sin(th) * np.cos(th) * (a - d) + (np.cos(th) ** 2 - np.sin(th) ** 2) * b
    roots = th[:-1][np.sign(f[:-1]) != np.sign(f[1:])]
    best = roots[np.argmin(np.abs(roots))]
    assert abs(math.atan2(s, c) - best) < 1e-4
    # closed form: rotated diagonal = eigenvalues of the block
    q = np.array([[c, -s], [s, c]])
    rot = q @ g @ q.T
    np.testing.assert_allclose(np.sort(np.diag(rot)), np.linalg.eigvalsh(g), rtol=1e-13,
                               atol=1e-14 * scale)


def test_jacobi2_zero_coupling_is_identity():
    assert O.jacobi2(3.0, 0.0, 1.0) == (1.0, 0.0)


@pytest.mark.parametrize("k", [3, 4, 6, 8])
def test_jacobik_orthogonal_and_diagonalizing(k):
    """Sec. 2.2: the k x k block diagonalizes the Gram sub-block."""
    rng = np.random.default_rng(k)
    x = rng.standard_normal((3 * k, k))
    g = I._mirror_upper(x.T @ x)
    st, o = O.jacobik(g)
    assert st == 0
    assert np.abs(o @ o.T - np.eye(k)).max() <= 1e-14
    r = o @ g @ o.T
    off = r - np.diag(np.diag(r))
    assert np.abs(off).max() <= 1e-12 * np.abs(g).max()
    np.testing.assert_allclose(np.sort(np.diag(r)), np.linalg.eigvalsh(g), rtol=1e-12)


@pytest.mark.parametrize("k", [2, 3, 5])
def test_sym_rotate_matches_dense_conjugation(k):
    """The local update equals the dense product O_full X O_full^T (Alg. 2)."""
    rng = np.random.default_rng(10 + k)
    n = 9
    x = I._mirror_upper(rng.standard_normal((n, n)))
    tup = rng.choice(n, k, replace=False)
    z = rng.standard_normal((k, k))
    o, _ = np.linalg.qr(z)
    full = np.eye(n)
    full[np.ix_(tup, tup)] = o
    want = full @ x @ full.T
    got = O.sym_rotate(x, tup, o)
    assert np.array_equal(got, got.T)                    # exactly symmetric
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(x).max())


# ---------------------------------------------------------------- Gram (R9)

def test_gram_exact_on_integer_matrix():
    """Integer entries make every partial sum exact: G must equal A_B^T A_B exactly."""
    a = I.knn_laplacian(300, k=6, seed=9, shift=0.0)
    dense = a.to_dense()
    members = np.sort(np.random.default_rng(0).choice(300, 40, replace=False)).astype(np.int32)
    g, m = O.gram(a, members)
    cols = dense[:, members]
    assert np.array_equal(g, cols.T @ cols)
    assert np.array_equal(m, dense[np.ix_(members, members)])


def test_gram_float_close_to_dense():
    a = I.psd_dense(64, 8, seed=2)
    dense = a.to_dense()
    members = np.arange(0, 64, 3, dtype=np.int32)
    g, _ = O.gram(a, members)
    cols = dense[:, members]
    np.testing.assert_allclose(g, cols.T @ cols, rtol=1e-13, atol=1e-13 * np.abs(g).max())


# ---------------------------------------------------------------- clustering (R10)

def test_partition_recovers_separated_blobs():
    rng = np.random.default_rng(4)
    centres = np.array([[0.1, 0.1], [0.9, 0.1], [0.1, 0.9], [0.9, 0.9]])
    truth = rng.integers(0, 4, 400)
    pts = centres[truth] + rng.uniform(-0.05, 0.05, (400, 2))
    lab = O.partition(pts, np.arange(400), 4)
    # same partition up to a relabelling
    pairs = set(zip(truth.tolist(), lab.tolist()))
    assert len(pairs) == 4 and len({p[0] for p in pairs}) == 4 and len({p[1] for p in pairs}) == 4


def test_partition_one_dimensional_clusters_are_intervals():
    rng = np.random.default_rng(5)
    x = rng.random((500, 1))
    lab = O.partition(x, np.arange(500), 7)
    order = np.argsort(x[:, 0], kind="stable")
    runs = 1 + np.count_nonzero(np.diff(lab[order]))
    assert runs == len(np.unique(lab))
    assert lab.min() >= 0 and lab.max() < 7


def test_quantize_grid():
    pts = np.array([[0.0, 5.0], [1.0, 5.0], [0.5, 5.0]])
    q = O.quantize(pts)
    assert q[:, 0].tolist() == [0, 32767, 16383]
    assert q[:, 1].tolist() == [0, 0, 0]


# ---------------------------------------------------------------- factorization

def _explicit(f, n):
    u = f.apply(O.OP_U, np.eye(n))
    h = np.diag(f.hdiag.copy())
    ci = f.core_idx
    h[np.ix_(ci, ci)] = f.core
    return u, h


CASES = [
    ("dense_k2", lambda: I.psd_dense(96, 24, seed=1), dict(k=2, eta=0.5, cluster_size=96, core_size=8)),
    ("dense_k3", lambda: I.psd_dense(80, 20, seed=2), dict(k=3, eta=0.5, cluster_size=80, core_size=10)),
    ("knn_clustered", lambda: I.knn_laplacian(600, seed=3), dict(k=2, eta=0.5, cluster_size=64, core_size=40)),
    ("knn_clustered_k4", lambda: I.knn_laplacian(400, seed=6), dict(k=4, eta=0.4, cluster_size=50, core_size=30)),
    ("poisson", lambda: I.poisson3d(6, seed=4), dict(k=2, eta=0.5, cluster_size=27, core_size=20)),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def factored(request):
    name, gen, kw = request.param
    a = gen()
    f = O.factor_csr(a, seed=11, **kw)
    assert f.status == 0
    return a, f, kw


def test_reconstruction_matches_accounted_residual(factored):
    """||A - U^T H U||_F^2 equals the accounted sum of contributions (R4, Eq. 1)."""
    a, f, _ = factored
    u, h = _explicit(f, a.n)
    dense = a.to_dense()
    explicit = np.linalg.norm(dense - u.T @ h @ u) ** 2
    accounted = sum(s.contrib for s in f.stages)
    assert abs(explicit - accounted) <= 1e-10 * np.linalg.norm(dense) ** 2
    assert abs(f.error - math.sqrt(accounted) / np.linalg.norm(dense)) < 1e-14


def test_u_orthogonal_and_h_core_diagonal(factored):
    """Every stage is orthogonal; H equals the core of U A U^T plus its diagonal."""
    a, f, _ = factored
    u, _ = _explicit(f, a.n)
    assert np.abs(u @ u.T - np.eye(a.n)).max() <= 1e-13
    b = u @ a.to_dense() @ u.T
    ci = f.core_idx
    scale = np.abs(a.val).max()
    np.testing.assert_allclose(f.core, b[np.ix_(ci, ci)], atol=1e-12 * scale)
    np.testing.assert_allclose(f.hdiag, np.diag(b), atol=1e-12 * scale)


def test_schedule_and_elimination_bookkeeping(factored):
    """Sec. 2: nested active sets, one elimination per rotation, |S_L| <= core size."""
    a, f, kw = factored
    elim = np.concatenate([s.rot_elim for s in f.stages])
    assert len(np.unique(elim)) == len(elim)
    assert len(elim) + len(f.core_idx) == a.n
    assert set(elim.tolist()).isdisjoint(f.core_idx.tolist())
    assert len(f.core_idx) <= kw["core_size"] or len(f.stages) == 0
    s = a.n
    for st in f.stages:
        assert st.active == s
        for r in range(len(st.rot_elim)):
            kk = st.rot_k[r]
            tup = st.rot_idx[r, :kk]
            assert st.rot_elim[r] in tup
            u_ = st.rot_cluster[r]
            mem = st.members[st.offsets[u_]:st.offsets[u_ + 1]]
            assert set(tup.tolist()) <= set(mem.tolist())
            o = st.rot_O[r, :kk * kk].reshape(kk, kk)
            assert np.abs(o @ o.T - np.eye(kk)).max() <= 1e-14
        s -= len(st.rot_elim)


def test_monotone_residual_and_invariants(factored):
    """Residual never decreases with more stages; trace and Frobenius bookkeeping."""
    a, f, _ = factored
    contrib = np.array([s.contrib for s in f.stages])
    assert (contrib >= 0).all()
    dense = a.to_dense()
    assert abs(np.trace(dense) - f.hdiag.sum()) <= 1e-12 * np.abs(dense).sum()
    wave = np.setdiff1d(np.arange(a.n), f.core_idx)
    fro = (f.core ** 2).sum() + contrib.sum() + (f.hdiag[wave] ** 2).sum()
    assert abs(fro - (dense ** 2).sum()) <= 1e-12 * (dense ** 2).sum()


def test_first_step_partner_is_brute_force_argmax():
    """n <= 8: the first partner maximizes |<A_i, A_j>| / ||A_j|| over all j (Sec. 2.2)."""
    for seed in range(12):
        a = I.psd_dense(8, 3, seed=seed)
        for k in (2, 3):
            f = O.factor_csr(a, k=k, eta=0.5, cluster_size=8, core_size=4, seed=seed)
            st = f.stages[0]
            dense = a.to_dense()
            g = dense.T @ dense
            i = st.rot_idx[0, 0]
            score = np.abs(g[i]) / np.sqrt(np.diag(g))
            score[i] = -1
            order = sorted(range(8), key=lambda j: (-score[j], j))
            assert list(st.rot_idx[0, 1:k]) == order[:k - 1]
            # and i is the pick of the counter-based draw among all 8 coordinates
            assert i == O.pick(O.draw(seed, 1, 0, 0), 8)
            # elimination by brute force: rotate G and A densely with the recorded
            # block, then the eliminated member has the smallest off-diagonal norm
            kk = st.rot_k[0]
            tup = st.rot_idx[0, :kk]
            full = np.eye(8)
            full[np.ix_(tup, tup)] = st.rot_O[0, :kk * kk].reshape(kk, kk)
            g2 = full @ g @ full.T
            a2 = full @ dense @ full.T
            off = [g2[x, x] - a2[x, x] ** 2 for x in tup]
            assert st.rot_elim[0] == tup[int(np.argmin(off))]


def test_diagonal_matrix_is_exact():
    a = I.from_dense(np.diag(np.arange(1.0, 33.0)))
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=32, core_size=4, seed=3)
    assert f.error == 0.0
    for st in f.stages:
        assert (st.rot_O[:, 0] == 1.0).all() and (st.rot_O[:, 1] == 0.0).all()


def test_two_by_two_one_rotation_diagonalizes():
    a = I.from_dense(np.array([[2.0, 0.7], [0.7, 1.0]]))
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=2, core_size=1, seed=0)
    assert len(f.stages) == 1 and f.total_rotations() == 1
    assert f.error <= 1e-15
    np.testing.assert_allclose(np.sort(f.hdiag), np.linalg.eigvalsh(a.to_dense()), rtol=1e-14)


@pytest.mark.parametrize("k", [2, 3])
def test_block_direct_sum_factors_exactly(k):
    """A permuted direct sum of k x k SPD blocks has an exact k-point MMF."""
    a = I.block_pairs(24, k=k, seed=7)
    f = O.factor_csr(a, k=k, eta=1.0 / k + 1e-9, cluster_size=a.n, core_size=24, seed=2)
    assert f.status == 0
    assert f.error <= 1e-14


# ---------------------------------------------------------------- apply / inverse / PCG

def test_apply_ops_match_explicit(factored):
    a, f, _ = factored
    u, h = _explicit(f, a.n)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((a.n, 3))
    at = u.T @ h @ u
    np.testing.assert_allclose(f.apply(O.OP_A, x), at @ x, atol=1e-11 * np.abs(at).max())
    np.testing.assert_allclose(f.apply(O.OP_UT, f.apply(O.OP_U, x)), x, atol=1e-13)
    np.testing.assert_allclose(f.apply(O.OP_H, x), h @ x, atol=1e-12 * np.abs(h).max())


def test_inverse_is_inverse_of_factorization():
    a = I.poisson3d(5, seed=1)
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=25, core_size=12, seed=5)
    u, h = _explicit(f, a.n)
    at = u.T @ h @ u
    x = np.random.default_rng(2).standard_normal((a.n, 2))
    np.testing.assert_allclose(at @ f.apply(O.OP_A_INV, x), x, atol=1e-9)


def test_pcg_converges_and_exact_preconditioner_takes_one_step():
    a = I.poisson3d(6, seed=2)
    b = np.random.default_rng(3).standard_normal((a.n, 2))
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=27, core_size=20, seed=1)
    st, x, iters, rel = f.pcg(a, b, 1e-10, 500)
    assert st == 0 and (rel <= 1e-9).all()
    np.testing.assert_allclose(a.to_dense() @ x, b, atol=1e-8 * np.abs(b).max())
    # no stages: U = I, H = A, so M^{-1} = A^{-1} and CG converges in one step
    f0 = O.factor_csr(a, k=2, eta=0.5, cluster_size=27, core_size=a.n, seed=1)
    st, x, iters, rel = f0.pcg(a, b, 1e-10, 10)
    assert st == 0 and (iters == 1).all()


# ---------------------------------------------------------------- validation

def test_rejects_bad_inputs():
    a = I.psd_dense(16, 4, seed=1)
    val = a.val.copy()
    val[1] += 1.0
    assert O.factor(a.n, a.rowptr, a.col, val, k=2, core_size=4).status == O.ERR_NOT_SYMMETRIC
    val = a.val.copy()
    val[0] = np.nan
    assert O.factor(a.n, a.rowptr, a.col, val, k=2, core_size=4).status == O.ERR_NONFINITE
    assert O.factor(a.n, a.rowptr, a.col, a.val, k=1, core_size=4).status == O.ERR_INVALID_ARG
    assert O.factor(a.n, a.rowptr, a.col, a.val, k=2, eta=1.0, core_size=4).status == O.ERR_INVALID_ARG


# ---------------------------------------------------------------- xi = 1/2 preconditioner

def test_inverse_square_root_operator():
    """Sec. 4 (xi = 1/2): A~^{-1/2} = U^T H^{-1/2} U squares to A~^{-1}, is
    symmetric, and H^{-1/2} equals the dense inverse square root of H."""
    a = I.poisson3d(6, seed=2)
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=27, core_size=20, seed=1)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((a.n, 2))
    y = f.apply(O.OP_A_INV_SQRT, f.apply(O.OP_A_INV_SQRT, x))
    want = f.apply(O.OP_A_INV, x)
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-10 * np.abs(want).max())
    z = rng.standard_normal((a.n, 2))
    lhs = np.sum(z * f.apply(O.OP_A_INV_SQRT, x))
    rhs = np.sum(f.apply(O.OP_A_INV_SQRT, z) * x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # H^{-1/2} against numpy on the dense H (wavelet diagonal plus symmetric core)
    h = np.diag(f.hdiag.copy())
    ci = np.asarray(f.core_idx)
    c = np.tril(f.core) + np.tril(f.core, -1).T
    h[np.ix_(ci, ci)] = c
    ev, vec = np.linalg.eigh(h)
    hs = vec @ np.diag(ev ** -0.5) @ vec.T
    np.testing.assert_allclose(f.apply(O.OP_H_INV_SQRT, x), hs @ x, rtol=0, atol=1e-10 * np.abs(hs @ x).max())


def test_inverse_square_root_of_diagonal_is_exact():
    a = I.from_dense(np.diag(np.arange(1.0, 33.0)))
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=32, core_size=4, seed=3)
    x = np.ones((32, 1))
    got = f.apply(O.OP_A_INV_SQRT, x)[:, 0]
    np.testing.assert_allclose(got, 1.0 / np.sqrt(np.arange(1.0, 33.0)), rtol=1e-15)


def test_split_cg_matches_pcg_iterates_and_exact_split_takes_one_step():
    """Sec. 4 (xi = 1/2): CG on W A W y = W b with x = W y, W^2 = M^{-1}, runs
    the same iterates as PCG with M^{-1} in exact arithmetic; with no stages
    (H = A) the split system is the identity and CG stops after one step."""
    a = I.poisson3d(6, seed=2)
    b = np.random.default_rng(5).standard_normal((a.n, 3))
    f = O.factor_csr(a, k=2, eta=0.5, cluster_size=27, core_size=20, seed=1)
    for it in (1, 3, 6):
        st1, x1, i1, _ = f.pcg(a, b, 1e-300, it)
        st2, x2, i2, _ = f.pcg_sym(a, b, 1e-300, it)
        assert st1 == st2 == O.ERR_NOT_CONVERGED and (i1 == it).all() and (i2 == it).all()
        np.testing.assert_allclose(x2, x1, rtol=0, atol=1e-9 * np.abs(x1).max())
    st, x, iters, rel = f.pcg_sym(a, b, 1e-10, 500)
    assert st == 0 and (rel <= 1e-8).all()
    np.testing.assert_allclose(a.to_dense() @ x, b, atol=1e-8 * np.abs(b).max())
    f0 = O.factor_csr(a, k=2, eta=0.5, cluster_size=27, core_size=a.n, seed=1)
    st, x, iters, rel = f0.pcg_sym(a, b, 1e-10, 10)
    assert st == 0 and (iters == 1).all() and (rel <= 1e-10).all()


# ---------------------------------------------------------------- given stage-1 clusters

def test_stage1_labels_reproduce_kmeans_and_bricks():
    """R10: stage 1 may take given clusters (grid bricks for structured grids).
    Labels equal to the k-means labels give the k-means factorization; brick
    labels give stage-1 clusters that are exactly the bricks, in brick order,
    members ascending."""
    a = I.poisson3d(8, seed=3)
    kw = dict(k=2, eta=0.5, cluster_size=32, core_size=24, seed=2)
    f0 = O.factor_csr(a, **kw)
    km = O.partition(a.coords, np.arange(a.n, dtype=np.int32), (a.n + 16) // 32)
    f1 = O.factor_csr(a, labels=km, **kw)
    assert f0.status == f1.status == 0
    for s0, s1 in zip(f0.stages, f1.stages):
        assert np.array_equal(s0.members, s1.members) and np.array_equal(s0.rot_idx, s1.rot_idx)
    assert f0.error == f1.error
    lab = I.grid_bricks(8, 8, 8, 4, 4, 2)
    assert lab.max() == 2 * 2 * 4 - 1
    fb = O.factor_csr(a, labels=lab, **kw)
    assert fb.status == 0
    st = fb.stages[0]
    assert len(st.offsets) - 1 == 16
    for u in range(16):
        want = np.nonzero(lab == u)[0]
        assert np.array_equal(st.members[st.offsets[u]:st.offsets[u + 1]], want)
    x, y, z = np.unravel_index(st.members[st.offsets[5]:st.offsets[6]], (8, 8, 8))
    assert (x // 4 == 0).all() and (y // 4 == 1).all() and (z // 2 == 1).all()   # brick (0, 1, 1)
    bad = lab.copy()
    bad[7] = -1
    assert O.factor_csr(a, labels=bad, **kw).status == O.ERR_INVALID_ARG


# ---------------------------------------------------------------- the multi-core timing build

def test_openmp_build_gives_the_same_factorization():
    """The OpenMP build (clusters and rows spread over the host's cores; used
    only for the multi-core CPU timing) must give the single-thread build's
    factorization: the same error and H diagonal, bit for bit, on clustered
    k = 2 and k = 3 cases."""
    import os
    if O.build_openmp() is None:
        pytest.skip("gcc without OpenMP")
    os.environ.setdefault("OMP_NUM_THREADS", "4")
    for a, kw in ((I.knn_laplacian(3000, seed=4), dict(k=2, cluster_size=128, core_size=40)),
                  (I.rbf_mixture(600, components=6, seed=2), dict(k=3, cluster_size=64, core_size=30))):
        kw = dict(kw, eta=0.5, seed=5)
        f = O.factor_csr(a, **kw)
        assert f.status == 0
        hd = np.empty(a.n)
        t, err, threads = O.time_factor_openmp(a.n, a.rowptr, a.col, a.val, a.coords,
                                               hdiag_out=hd, **kw)
        assert threads >= 1
        assert err == f.error
        assert np.array_equal(hd.view(np.uint64), f.hdiag.view(np.uint64))


# ---------------------------------------------------------------- all rows in the Gram (R2 variant)

@pytest.mark.parametrize("make,kw", [
    (lambda: I.knn_laplacian(300, seed=3), dict(k=2, cluster_size=60, core_size=20)),
    (lambda: I.psd_dense(96, 24, seed=2), dict(k=3, cluster_size=96, core_size=12)),
    (lambda: I.rbf_mixture(200, components=4, seed=1), dict(k=2, cluster_size=50, core_size=16)),
], ids=["knn300", "psd96-k3", "rbf200"])
def test_rows_all_reconstruction_and_first_stage(make, kw):
    """The variant whose Grams sum over all n rows of the uncompacted matrix:
    its reported error is ||A - U^T H U||_F / ||A||_F computed explicitly
    (U^T H U applied to the identity), its rotations are orthogonal, and its
    first stage equals the default reading's (at stage 1 every row is
    active)."""
    a = make()
    kw = dict(kw, eta=0.5, seed=4)
    f = O.factor_csr(a, rows_all=True, **kw)
    g = O.factor_csr(a, **kw)
    assert f.status == 0 and g.status == 0
    A = a.to_dense()
    At = f.apply(O.OP_A, np.eye(a.n))
    err = np.linalg.norm(A - At) / np.linalg.norm(A)
    assert abs(err - f.error) <= 1e-12 * max(f.error, 1e-300) + 1e-15
    for st in f.stages:
        for t in range(len(st.rot_elim)):
            kk = st.rot_k[t]
            Ob = st.rot_O[t][:kk * kk].reshape(kk, kk)
            assert np.abs(Ob @ Ob.T - np.eye(kk)).max() <= 1e-14
    s0, t0 = f.stages[0], g.stages[0]
    assert np.array_equal(s0.rot_idx, t0.rot_idx) and np.array_equal(s0.rot_elim, t0.rot_elim)
    assert np.array_equal(s0.rot_O, t0.rot_O)
    assert f.total_rotations() == g.total_rotations()
