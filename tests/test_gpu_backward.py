"""GPU gradient of the factorized operator against the oracle's gradient.

The CUDA factorization is first checked bit-identical to the oracle's, then
pmmf_apply_backward's dx, dtheta, dhdiag and dcore are compared with the
oracle's (pinned by finite differences on the CPU).  The two sum the same
terms in different orders, so the bar is a relative tolerance: 1e-11 of the
largest entry of each gradient.  The autograd wrapper is checked with
torch.autograd.gradcheck (finite differences of the CUDA forward).
"""

import numpy as np
import pytest

from helpers import assert_same_factorization, factor_both, gpu
from paper_1507_04396_gb300 import inputs as I

OP_A, OP_A_INV = 0, 1
TOL = 1e-11


def _close(got, want, what):
    scale = max(float(np.max(np.abs(want))) if want.size else 0.0, 1e-300)
    err = float(np.max(np.abs(got - want))) if want.size else 0.0
    assert err <= TOL * scale, f"{what}: max error {err:.3e} vs scale {scale:.3e}"


def _compare(g, o, op, nrhs, seed):
    import torch
    n = g.info().n
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, nrhs))
    gy = rng.standard_normal((n, nrhs))
    want = o.apply_grad(op, x, gy)
    got = g.backward(op, torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda())
    _close(got["dx"].cpu().numpy(), want["dx"], "dx")
    _close(got["dtheta"].cpu().numpy(), want["dtheta"], "dtheta")
    _close(got["dhdiag"].cpu().numpy(), want["dhdiag"], "dhdiag")
    _close(got["dcore"].cpu().numpy(), want["dcore"], "dcore")


@gpu
@pytest.mark.parametrize("op", [OP_A, OP_A_INV])
@pytest.mark.parametrize("nrhs", [1, 3, 11])
def test_backward_matches_oracle_clustered(op, nrhs):
    """Several clusters per stage, ragged cluster sizes; nrhs = 11 runs two
    column chunks."""
    a = I.knn_laplacian(3000, seed=5)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=96, core_size=40, seed=4)
    assert_same_factorization(g, o)
    _compare(g, o, op, nrhs, seed=nrhs)


@gpu
def test_backward_matches_oracle_dense_one_cluster():
    a = I.psd_dense(256, 64, seed=0)
    g, o = factor_both(a, coords=None, k=2, eta=0.5, cluster_size=256, core_size=16, seed=0)
    assert_same_factorization(g, o)
    for op in (OP_A, OP_A_INV):
        _compare(g, o, op, 8, seed=op)


@gpu
@pytest.mark.parametrize("k", [3, 4])
def test_backward_kpoint_block_gradient(k):
    """k-point rotations parameterised by their blocks: dL/dO per rotation
    (k * k slots), dx, dH against the oracle; two stages of several clusters,
    nrhs = 10 runs two column chunks."""
    import torch
    a = I.knn_laplacian(1500, seed=8)
    g, o = factor_both(a, k=k, eta=0.5, cluster_size=80, core_size=60, seed=2)
    assert_same_factorization(g, o)
    assert g.info().stages >= 2
    rng = np.random.default_rng(k)
    for op, nrhs in ((OP_A, 10), (OP_A_INV, 3)):
        x = rng.standard_normal((a.n, nrhs))
        gy = rng.standard_normal((a.n, nrhs))
        want = o.apply_grad(op, x, gy)
        got = g.backward(op, torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda())
        _close(got["dx"].cpu().numpy(), want["dx"], "dx")
        _close(got["dO"].cpu().numpy(), want["dO"].reshape(got["dO"].shape), "dO")
        _close(got["dhdiag"].cpu().numpy(), want["dhdiag"], "dhdiag")
        _close(got["dcore"].cpu().numpy(), want["dcore"], "dcore")


@gpu
def test_backward_full_size_workload():
    """The bench workload (65,536 coordinates, 9 stages), 8 right-hand sides."""
    a = I.knn_laplacian(65536, seed=1)
    g, o = factor_both(a, k=2, eta=0.5, cluster_size=256, core_size=256, seed=0)
    assert_same_factorization(g, o, check_matrices=False)
    _compare(g, o, OP_A, 8, seed=7)


@gpu
def test_angles_roundtrip_and_set_parameters():
    import torch
    from paper_1507_04396_gb300 import pmmf as P
    a = I.knn_laplacian(800, seed=2)
    g = P.factor(a, k=2, eta=0.5, cluster_size=64, core_size=20, seed=1)
    th = g.angles()
    rots = [g.rotations(p)[3] for p in range(g.info().stages)]
    O = np.concatenate(rots)
    np.testing.assert_allclose(np.cos(th.cpu().numpy()), O[:, 0], atol=1e-15)
    np.testing.assert_allclose(np.sin(th.cpu().numpy()), O[:, 2], atol=1e-15)
    x = torch.from_numpy(np.random.default_rng(0).standard_normal((a.n, 2))).cuda()
    y0 = g.apply(OP_A, x)
    # a new angle set changes the operator; writing the old one back restores it
    g.set_parameters(theta=th + 0.01)
    y1 = g.apply(OP_A, x)
    assert float((y1 - y0).abs().max()) > 1e-6
    g.set_parameters(theta=th)
    y2 = g.apply(OP_A, x)
    assert float((y2 - y0).abs().max()) <= 1e-13 * float(y0.abs().max())
    hd, core = g.h_tensors()
    g.set_parameters(hdiag=2 * hd, core=2 * core)
    y3 = g.apply(OP_A, x)
    assert float((y3 - 2 * y0).abs().max()) <= 1e-12 * float(y0.abs().max())


@gpu
@pytest.mark.parametrize("op", [OP_A, OP_A_INV])
def test_autograd_gradcheck(op):
    import torch
    from paper_1507_04396_gb300 import pmmf as P
    a = I.knn_laplacian(96, k=5, seed=3, shift=0.1)
    g = P.factor(a, k=2, eta=0.5, cluster_size=24, core_size=8, seed=2)
    th = g.angles().clone().requires_grad_(True)
    hd, core = g.h_tensors()
    hd = hd.clone().requires_grad_(True)
    core = core.clone().requires_grad_(True)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((a.n, 2))).cuda().requires_grad_(True)
    fn = lambda x_, t_, h_, c_: P.pmmf_operator(g, x_, t_, h_, c_, op)
    assert torch.autograd.gradcheck(fn, (x, th, hd, core), eps=1e-6, atol=1e-7, rtol=1e-5)


@gpu
def test_kpoint_angles_against_oracle():
    """k >= 3 angle parameterisation on the GPU: every block's Givens angles
    equal the oracle's decomposition of the same block, set(get()) leaves the
    operator unchanged, and dL/dtheta equals the oracle's chain rule applied
    to the oracle's dL/dO."""
    import torch
    from oracle import oracle as O
    a = I.knn_laplacian(1200, seed=9)
    g, o = factor_both(a, k=3, eta=0.5, cluster_size=80, core_size=50, seed=5)
    assert_same_factorization(g, o)
    th = g.angles().cpu().numpy()
    blocks = np.concatenate([s.rot_O for s in o.stages])
    kks = np.concatenate([s.rot_k for s in o.stages])
    want_th, want_D = [], []
    for t in range(len(kks)):
        kk = int(kks[t])
        w, d = O.block_angles(blocks[t, :kk * kk].reshape(kk, kk))
        want_th.append(np.pad(w, (0, 3 - len(w))))
        want_D.append(d)
    np.testing.assert_allclose(th, np.array(want_th), rtol=0, atol=1e-13)
    x = np.random.default_rng(0).standard_normal((a.n, 2))
    xd = torch.from_numpy(x).cuda()
    y0 = g.apply(0, xd).cpu().numpy()
    g.set_parameters(theta=torch.from_numpy(th.ravel()).cuda())
    y1 = g.apply(0, xd).cpu().numpy()
    np.testing.assert_allclose(y1, y0, rtol=0, atol=1e-13 * np.abs(y0).max())
    gy = np.random.default_rng(1).standard_normal((a.n, 2))
    got = g.backward(0, xd, torch.from_numpy(gy).cuda())
    want = o.apply_grad(0, x, gy)
    dth = got["dtheta"].cpu().numpy()
    ref = []
    for t in range(len(kks)):
        kk = int(kks[t])
        r = O.block_angle_grad(want_th[t][:kk * (kk - 1) // 2], want_D[t],
                               want["dO"][t, :kk * kk].reshape(kk, kk))
        ref.append(np.pad(r, (0, 3 - len(r))))
    _close(dth, np.array(ref), "dtheta (k = 3)")
