"""Differentiable TSQR: tsqr_backward behind a torch.autograd.Function.

Checked against (a) the FP64 CPU reference gradient: the published QR adjoint
M = R Rbar^T - Qbar^T Q, Abar = (Qbar + Q copyltu(M)) R^-T evaluated in numpy on the oracle's
Q and R, and (b) central finite differences of the GPU forward (h = 1e-6, FP64) along random
unit directions and per entry on a slice.  Loss: sum(W1 * Q) + sum(W2 * R), W iid N(0, 1).
"""
import numpy as np
import pytest

import oracle
from paper_0809_2407_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    tsqr.load()
    return tsqr


def reference_grad(A, W1, W2):
    """FP64 CPU gradient of sum(W1*Q) + sum(W2*R) from the oracle's factors."""
    f = oracle.qr(A)
    Q, R = f["Q"], f["R"]
    Rb = np.triu(W2)
    M = R @ Rb.T - W1.T @ Q
    C = np.tril(M) + np.tril(M, -1).T
    B = W1 + Q @ C
    return np.linalg.solve(R, B.T).T  # B R^-T


def loss_and_grad(T, A_h, W1, W2, keep="tree", precision=0):
    import torch

    A = torch.from_numpy(A_h.copy()).cuda().requires_grad_(True)
    Q, R = T.qr_autograd(A, keep=keep, precision=precision)
    w1 = torch.from_numpy(W1).cuda()
    w2 = torch.from_numpy(W2).cuda()
    L = (w1 * Q).sum() + (w2 * R).sum()
    L.backward()
    return L.item(), A.grad.cpu().numpy()


def loss_only(T, A_h, W1, W2):
    import torch

    A = torch.from_numpy(A_h.copy()).cuda()
    f = T.Factorization(A)
    Q = f.form_q()
    L = (torch.from_numpy(W1).cuda() * Q).sum() + (torch.from_numpy(W2).cuda() * f.R).sum()
    return L.item()


@pytest.mark.parametrize("m,n,prec", [(300, 7, 0), (2000, 16, 0), (5000, 40, 0), (3000, 32, 1), (4096, 64, 2),
                                      (6000, 128, 0), (3000 + 7, 100, 1), (2500, 154, 0)])
def test_against_cpu_reference(T, m, n, prec):
    A_h = inputs.usv(m, n, 2.0, 700 + m)
    rng = np.random.default_rng(m + n)
    W1, W2 = rng.standard_normal((m, n)), rng.standard_normal((n, n))
    _, g = loss_and_grad(T, A_h, W1, W2, precision=prec)
    ref = reference_grad(A_h, W1, W2)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= (1e-11 if prec != 1 else 1e-9)


def test_finite_differences(T):
    m, n = 512, 8
    A_h = inputs.usv(m, n, 1.0, 71)
    rng = np.random.default_rng(72)
    W1, W2 = rng.standard_normal((m, n)), rng.standard_normal((n, n))
    _, g = loss_and_grad(T, A_h, W1, W2)
    h = 1e-6
    for k in range(8):
        E = rng.standard_normal((m, n))
        E /= np.linalg.norm(E)
        fd = (loss_only(T, A_h + h * E, W1, W2) - loss_only(T, A_h - h * E, W1, W2)) / (2 * h)
        assert abs(fd - np.sum(g * E)) <= 1e-7 * max(1.0, abs(fd))
    # per entry on a 16 x 8 slice
    for i in range(100, 116):
        for j in range(n):
            E = np.zeros((m, n))
            E[i, j] = 1.0
            fd = (loss_only(T, A_h + h * E, W1, W2) - loss_only(T, A_h - h * E, W1, W2)) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(fd))


def test_tree_and_recompute_agree(T):
    A_h = inputs.gaussian(20000, 32, 73)
    rng = np.random.default_rng(74)
    W1, W2 = rng.standard_normal((20000, 32)), rng.standard_normal((32, 32))
    L1, g1 = loss_and_grad(T, A_h, W1, W2, keep="tree")
    L2, g2 = loss_and_grad(T, A_h, W1, W2, keep="recompute")
    assert L1 == L2 and np.array_equal(g1, g2)


def test_one_sided_losses_and_batch(T):
    import torch

    A_h = np.stack([inputs.gaussian(3000, 12, 80 + i) for i in range(3)])
    A = torch.from_numpy(A_h.copy()).cuda().requires_grad_(True)
    Q, R = T.qr_autograd(A)
    (Q ** 2).sum().backward()  # depends on Q only; Q^T Q = I makes the gradient vanish in theory
    assert torch.linalg.norm(A.grad).item() <= 1e-10 * torch.linalg.norm(A).item()
    A.grad = None
    Q, R = T.qr_autograd(A)
    R.diagonal(dim1=1, dim2=2).sum().backward()  # R only: d trace(R) / dA
    for b in range(3):
        W1 = np.zeros((3000, 12))
        W2 = np.eye(12)
        assert np.abs(A.grad[b].cpu().numpy() - reference_grad(A_h[b], W1, W2)).max() <= 1e-11


@pytest.mark.parametrize("m,n", [(4096, 16), (20000, 64), (6000, 100)])
def test_f32_against_cpu_reference(T, m, n):
    """FP32 storage: the float32 gradient against the FP64 reference gradient of the float32 A,
    within the FP32 perturbation bound 50 kappa n u, u = 2^-24 (kappa(A) = 10)."""
    import torch

    A32 = inputs.usv(m, n, 1.0, 800 + m).astype(np.float32)
    rng = np.random.default_rng(m + n + 1)
    W1 = rng.standard_normal((m, n)).astype(np.float32)
    W2 = rng.standard_normal((n, n)).astype(np.float32)
    A = torch.from_numpy(A32.copy()).cuda().requires_grad_(True)
    Q, R = T.qr_autograd(A)
    assert Q.dtype == torch.float32 and R.dtype == torch.float32
    L = (torch.from_numpy(W1).cuda() * Q).sum() + (torch.from_numpy(W2).cuda() * R).sum()
    L.backward()
    assert A.grad.dtype == torch.float32
    g = A.grad.double().cpu().numpy()
    ref = reference_grad(A32.astype(np.float64), W1.astype(np.float64), W2.astype(np.float64))
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 50 * 10 * n * 2.0 ** -24


@pytest.mark.parametrize("dtype,keep", [("float64", "tree"), ("float32", "tree"), ("float64", "recompute")])
def test_batch_matches_single(T, dtype, keep):
    """The batched function (matrices spread over CUDA streams) gives the per-matrix results
    bitwise: forward Q, R and the gradient."""
    import torch

    tdt = getattr(torch, dtype)
    A_h = np.stack([inputs.gaussian(4000 + 0, 24, 90 + i) for i in range(5)])
    W = np.random.default_rng(91).standard_normal(A_h.shape)
    A = torch.from_numpy(A_h).to(tdt).cuda().requires_grad_(True)
    w = torch.from_numpy(W).to(tdt).cuda()
    Q, R = T.qr_autograd(A, keep=keep)
    ((w * Q).sum() + R.sum()).backward()
    g_batch = A.grad.clone()
    for i in range(A.shape[0]):
        Ai = A.detach()[i].clone().requires_grad_(True)
        Qi, Ri = T.qr_autograd(Ai, keep=keep)
        ((w[i] * Qi).sum() + Ri.sum()).backward()
        assert torch.equal(Qi, Q[i]) and torch.equal(Ri, R[i])
        assert torch.equal(Ai.grad, g_batch[i])
