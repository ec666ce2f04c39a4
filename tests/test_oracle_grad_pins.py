"""Pins of the oracle's gradient of the factorized operator.

L = sum(g * op(x)) with op(x) = U^T M U x, M = H or H^{-1}, the greedy
selections held fixed.  The oracle's backward is checked against things that
do not come from it: central finite differences of the oracle's own forward
apply in every parameter (rotation angles, the diagonal of H, the core, x),
and dL/dH against U built densely in numpy from the exported rotation blocks.
None of this runs the CUDA library.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_04396_gb300 import inputs as I

OP_A, OP_A_INV = 0, 1


def _small(kind):
    if kind == "dense":
        a = I.psd_dense(24, 6, seed=3)
        f = O.factor_csr(a, k=2, eta=0.5, cluster_size=24, core_size=4, seed=1)
    else:
        a = I.knn_laplacian(160, k=5, seed=4, shift=0.05)
        f = O.factor_csr(a, k=2, eta=0.5, cluster_size=40, core_size=10, seed=2)
    assert f.status == 0
    return a, f


def _loss(f, op, x, g):
    return float(np.sum(g * f.apply(op, x)))


def _rotations(f):
    out = []
    for p, s in enumerate(f.stages):
        for t in range(len(s.rot_elim)):
            out.append((p, t, s.rot_O[t, :4].copy()))
    return out


def _dense_u(f, n):
    """U as a dense n x n matrix, composed in numpy from the exported blocks."""
    u = np.eye(n)
    for s in f.stages:
        for t in range(len(s.rot_elim)):
            i, j = s.rot_idx[t, 0], s.rot_idx[t, 1]
            c, sn = s.rot_O[t, 0], s.rot_O[t, 2]
            q = np.eye(n)
            q[i, i], q[i, j], q[j, i], q[j, j] = c, -sn, sn, c
            u = q @ u
    return u


@pytest.mark.parametrize("kind", ["dense", "clustered"])
@pytest.mark.parametrize("op", [OP_A, OP_A_INV])
def test_angle_gradient_matches_finite_differences(kind, op):
    a, f = _small(kind)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((a.n, 3))
    g = rng.standard_normal((a.n, 3))
    grad = f.apply_grad(op, x, g)
    rots = _rotations(f)
    assert len(grad["dtheta"]) == len(rots) > 0
    eps = 1e-5
    picks = range(len(rots)) if len(rots) <= 40 else rng.choice(len(rots), 40, replace=False)
    scale = max(1.0, float(np.max(np.abs(grad["dtheta"]))))
    for q in picks:
        p, t, o = rots[q]
        th = np.arctan2(o[2], o[0])
        vals = []
        for sgn in (1.0, -1.0):
            c, s = np.cos(th + sgn * eps), np.sin(th + sgn * eps)
            f.set_rotation(p, t, np.array([c, -s, s, c]))
            vals.append(_loss(f, op, x, g))
        f.set_rotation(p, t, np.array([np.cos(th), -np.sin(th), np.sin(th), np.cos(th)]))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad["dtheta"][q]) <= 1e-6 * scale, (q, fd, grad["dtheta"][q])
        f.set_rotation(p, t, o)


def test_block_gradient_matches_finite_differences():
    """dL/dO per block entry (k = 3 blocks, no angle parameterisation)."""
    a = I.psd_dense(18, 6, seed=8)
    f = O.factor_csr(a, k=3, eta=0.5, cluster_size=18, core_size=4, seed=3)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((a.n, 2))
    g = rng.standard_normal((a.n, 2))
    grad = f.apply_grad(OP_A, x, g)
    s0 = f.stages[0]
    kk = int(s0.rot_k[0])
    o = s0.rot_O[0, :kk * kk].copy()
    eps = 1e-6
    for e in range(kk * kk):
        vals = []
        for sgn in (1.0, -1.0):
            oo = o.copy()
            oo[e] += sgn * eps
            f.set_rotation(0, 0, oo)
            vals.append(_loss(f, OP_A, x, g))
        f.set_rotation(0, 0, o)
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad["dO"][0, e]) <= 1e-7 * max(1.0, abs(fd)), (e, fd, grad["dO"][0, e])


@pytest.mark.parametrize("op", [OP_A, OP_A_INV])
def test_h_gradient_matches_finite_differences(op):
    a, f = _small("clustered")
    rng = np.random.default_rng(9)
    x = rng.standard_normal((a.n, 2))
    g = rng.standard_normal((a.n, 2))
    grad = f.apply_grad(op, x, g)
    h0, c0 = f.hdiag.copy(), f.core.copy()
    core = set(int(i) for i in f.core_idx)
    eps = 1e-6
    wav = [i for i in range(a.n) if i not in core]
    for i in rng.choice(wav, 12, replace=False):
        vals = []
        for sgn in (1.0, -1.0):
            h = h0.copy()
            h[i] += sgn * eps * max(1.0, abs(h0[i]))
            f.set_h(hdiag=h)
            vals.append(_loss(f, op, x, g))
        f.set_h(hdiag=h0)
        fd = (vals[0] - vals[1]) / (2 * eps * max(1.0, abs(h0[i])))
        assert abs(fd - grad["dhdiag"][i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad["dhdiag"][i])
    for i in core:
        assert grad["dhdiag"][i] == 0.0
    # core: directional derivative along a random (not symmetric) direction
    d = rng.standard_normal(c0.shape)
    vals = []
    for sgn in (1.0, -1.0):
        f.set_h(core=c0 + sgn * eps * d)
        vals.append(_loss(f, op, x, g))
    f.set_h(core=c0)
    fd = (vals[0] - vals[1]) / (2 * eps)
    an = float(np.sum(grad["dcore"] * d))
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (fd, an)


@pytest.mark.parametrize("op", [OP_A, OP_A_INV])
def test_x_gradient_is_exact_directional_derivative(op):
    a, f = _small("dense")
    rng = np.random.default_rng(2)
    x = rng.standard_normal((a.n, 2))
    g = rng.standard_normal((a.n, 2))
    grad = f.apply_grad(op, x, g)
    d = rng.standard_normal(x.shape)
    # L is linear in x: the central difference is exact up to rounding
    fd = (_loss(f, op, x + d, g) - _loss(f, op, x - d, g)) / 2.0
    assert abs(fd - float(np.sum(grad["dx"] * d))) <= 1e-10 * max(1.0, abs(fd))


def test_h_gradient_against_dense_u():
    """dL/dH = (U g)(U x)^T on H's structure, U composed densely in numpy."""
    a, f = _small("clustered")
    rng = np.random.default_rng(4)
    x = rng.standard_normal((a.n, 3))
    g = rng.standard_normal((a.n, 3))
    grad = f.apply_grad(OP_A, x, g)
    u = _dense_u(f, a.n)
    outer = (u @ g) @ (u @ x).T
    ci = np.asarray(f.core_idx)
    core = np.zeros(a.n, bool)
    core[ci] = True
    np.testing.assert_allclose(grad["dcore"], outer[np.ix_(ci, ci)], rtol=1e-12, atol=1e-12)
    want = np.where(core, 0.0, np.diag(outer))
    np.testing.assert_allclose(grad["dhdiag"], want, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- k-point angles

@pytest.mark.parametrize("kk", [2, 3, 4, 6, 8])
def test_block_angles_round_trip(kk):
    """Givens elimination of an orthogonal block and its rebuild: O is
    recovered to rounding, the signs are +-1 with det(D) = det(O), the
    identity has zero angles, and a 2 x 2 rotation R(t) = [[c, -s], [s, c]]
    has the single angle t (the k = 2 parameterisation)."""
    rng = np.random.default_rng(kk)
    for _ in range(5):
        q, _r = np.linalg.qr(rng.standard_normal((kk, kk)))
        th, D = O.block_angles(q)
        assert th.shape == (kk * (kk - 1) // 2,) and set(np.abs(D)) == {1.0}
        assert np.prod(D) == np.sign(np.linalg.det(q))
        np.testing.assert_allclose(O.block_from_angles(th, D), q, rtol=0, atol=1e-14)
    th, D = O.block_angles(np.eye(kk))
    assert np.all(th == 0.0) and np.all(D == 1.0)
    if kk == 2:
        for t in (0.3, -2.1, 3.0):
            R = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
            th, D = O.block_angles(R)
            assert abs(th[0] - t) <= 1e-15 and np.all(D == 1.0)


@pytest.mark.parametrize("kk", [3, 5])
def test_block_angle_gradient_finite_differences(kk):
    """d<W, O(theta)>/dtheta against central differences in every angle."""
    rng = np.random.default_rng(10 + kk)
    q, _r = np.linalg.qr(rng.standard_normal((kk, kk)))
    th, D = O.block_angles(q)
    W = rng.standard_normal((kk, kk))
    grad = O.block_angle_grad(th, D, W)
    eps = 1e-6
    for i in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (np.sum(W * O.block_from_angles(tp, D)) - np.sum(W * O.block_from_angles(tm, D))) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-8 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_operator_angle_gradient_kpoint():
    """dL/dtheta of the operator for k = 3 (block gradient, then the angle
    chain rule) against central differences of the forward apply with the
    block rebuilt from perturbed angles."""
    a = I.psd_dense(18, 6, seed=8)
    f = O.factor_csr(a, k=3, eta=0.5, cluster_size=18, core_size=4, seed=3)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((a.n, 2))
    g = rng.standard_normal((a.n, 2))
    grad = f.apply_grad(OP_A, x, g)
    s0 = f.stages[0]
    for t in (0, 1):
        kk = int(s0.rot_k[t])
        o = s0.rot_O[t, :kk * kk].copy()
        th, D = O.block_angles(o.reshape(kk, kk))
        dth = O.block_angle_grad(th, D, grad["dO"][t, :kk * kk].reshape(kk, kk))
        eps = 1e-6
        for i in range(len(th)):
            vals = []
            for sgn in (1.0, -1.0):
                tt = th.copy()
                tt[i] += sgn * eps
                f.set_rotation(0, t, O.block_from_angles(tt, D).ravel())
                vals.append(_loss(f, OP_A, x, g))
            f.set_rotation(0, t, o)
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(fd - dth[i]) <= 1e-7 * max(1.0, abs(fd)), (t, i, fd, dth[i])
