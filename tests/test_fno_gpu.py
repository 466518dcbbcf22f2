"""The surrogate's tensor-core GEMM (tcgen05, bf16 operands, float32
accumulators in tensor memory) and network against the float64 oracle.

Tolerances: the GEMM rounds its inputs to bfloat16 and accumulates in float32,
so against float64 products of the same rounded inputs it agrees to ~1e-6
relative.  The network also rounds activations and DFT matrices to bfloat16
(8-bit mantissa, unit roundoff 2^-9 ~ 2e-3) in every contraction, so outputs and
gradients are compared with relative L2 bounds of a few percent.
"""
import numpy as np
import pytest

from oracle import fno_oracle as F

pytestmark = pytest.mark.gpu


def bf16(a):
    import torch
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("M,N,K,ta,tb,ksplit", [(64, 64, 32, False, False, 1), (100, 37, 53, True, False, 1),
                                                 (33, 130, 260, False, True, 1), (32, 32, 4096, False, True, 8),
                                                 (5, 7, 3, True, True, 1), (300, 24, 64, False, False, 1),
                                                 (257, 200, 129, True, True, 1), (1000, 300, 72, False, False, 3),
                                                 (24, 2000, 12, False, True, 1)])
def test_gemm_bf16_against_numpy(lib, M, N, K, ta, tb, ksplit):
    import torch
    rng = np.random.default_rng(M * N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    At = torch.tensor(A.T.copy(), device="cuda").t() if ta else torch.tensor(A, device="cuda")
    Bt = torch.tensor(B.T.copy(), device="cuda").t() if tb else torch.tensor(B, device="cuda")
    Ct = torch.tensor(C0, device="cuda")
    lib.gemm_bf16(At, Bt, Ct, alpha=0.5, beta=0.25, ksplit=ksplit)
    torch.cuda.synchronize()
    want = 0.5 * bf16(A) @ bf16(B) + 0.25 * C0
    got = Ct.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5


def _model(lib, c, B, seed=1):
    return lib.Fno(c.NP, width=c.C, layers=c.L, patch=c.P, modes=c.m, hidden=c.H, out_channels=c.NO, max_batch=B,
                   seed=seed)


@pytest.mark.parametrize("cfg", [(6, 4, 2, 8, 2, 8, 3), (6, 8, 4, 16, 4, 16, 3)])
def test_fno_forward_matches_oracle(lib, cfg):
    import torch
    c = F.FnoConfig(*cfg)
    B = 2
    net = _model(lib, c, B)
    assert net.n_params == F.num_params(c)
    rng = np.random.default_rng(7)
    theta = rng.standard_normal(F.num_params(c)) * 0.2
    net.params.copy_(torch.tensor(theta, dtype=torch.float32))
    prm = rng.uniform(-1, 1, (B, c.NP))
    got = net.forward(torch.tensor(prm, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = F.forward(theta, prm, c)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 3e-2
    net.close()


def test_fno_gradients_match_finite_differences(lib):
    import torch
    c = F.FnoConfig(6, 4, 2, 8, 2, 8, 3)
    B = 2
    net = _model(lib, c, B)
    rng = np.random.default_rng(11)
    theta = rng.standard_normal(F.num_params(c)) * 0.2
    net.params.copy_(torch.tensor(theta, dtype=torch.float32))
    prm = rng.uniform(-1, 1, (B, c.NP))
    target = rng.standard_normal((B, c.NO, c.P, c.P, c.P)) * 0.1
    loss = net.loss_backward(torch.tensor(prm, dtype=torch.float32, device="cuda"),
                             torch.tensor(target, dtype=torch.float32, device="cuda"))
    assert abs(loss / F.loss(theta, prm, target, c) - 1) <= 3e-2
    g = net.grads.cpu().numpy().astype(np.float64)
    # a sample of every parameter group
    n = F.num_params(c)
    idx = np.unique(np.concatenate([rng.choice(n, 80, replace=False), np.arange(0, 40), np.arange(n - 30, n)]))
    fd = F.finite_difference_grad(theta, prm, target, c, idx)
    assert np.linalg.norm(g[idx] - fd) / np.linalg.norm(fd) <= 5e-2
    assert np.dot(g[idx], fd) / (np.linalg.norm(g[idx]) * np.linalg.norm(fd)) >= 0.998
    net.close()


def test_fno_training_reduces_loss(lib):
    import torch
    c = F.FnoConfig(3, 8, 2, 16, 4, 16, 2)
    B = 4
    net = _model(lib, c, B, seed=3)
    rng = np.random.default_rng(5)
    prm = rng.uniform(-1, 1, (16, c.NP)).astype(np.float32)
    x = -1 + 2 * np.arange(c.P) / c.P
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    tgt = np.stack([np.stack([p[0] * np.cos(np.pi * X) + p[1] * np.sin(np.pi * Y) * np.cos(np.pi * Z),
                              p[2] * np.sin(np.pi * (X + Y))]) for p in prm]).astype(np.float32)
    P_t = torch.tensor(prm, device="cuda")
    T_t = torch.tensor(tgt, device="cuda")
    losses = []
    for it in range(200):
        sel = slice((it % 4) * B, (it % 4) * B + B)
        losses.append(net.loss_backward(P_t[sel].contiguous(), T_t[sel].contiguous()))
        net.adam_step(2e-3)
    first, last = np.mean(losses[:4]), np.mean(losses[-4:])
    assert last < 0.4 * first, (first, last)
    net.close()
