"""Pins of the oracle's MLP, MSE and Adam (not GPU).

The oracle is checked against an independent float64 implementation built
from torch CPU autograd (test only), central finite differences, GELU
special values, torch's bfloat16 rounding and torch's Adam.
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp
from synth.bunch import mlp_init

WIDTHS = [6, 128, 128, 128, 128, 6]


def _net(seed=3, widths=WIDTHS):
    return mlp_init(widths, seed)


def _torch_forward(Ws, bs, X):
    h = X
    for l, (W, b) in enumerate(zip(Ws, bs)):
        h = h @ W.T + b
        if l < len(Ws) - 1:
            h = torch.nn.functional.gelu(h, approximate="tanh")
    return h


def test_forward_backward_match_torch_autograd():
    Ws, bs = _net()
    rng = np.random.default_rng(0)
    X = rng.normal(size=(37, 6))
    dY = rng.normal(size=(37, 6))
    Y, cache = mlp.forward(Ws, bs, X, keep=True)
    dX, dWs, dbs = mlp.backward(Ws, cache, dY)
    tW = [torch.tensor(W, requires_grad=True) for W in Ws]
    tb = [torch.tensor(b, requires_grad=True) for b in bs]
    tX = torch.tensor(X, requires_grad=True)
    tY = _torch_forward(tW, tb, tX)
    tY.backward(torch.tensor(dY))
    assert np.max(np.abs(Y - tY.detach().numpy())) < 1e-13
    assert np.max(np.abs(dX - tX.grad.numpy())) < 1e-13
    for a, b in zip(dWs, tW):
        assert np.max(np.abs(a - b.grad.numpy())) < 1e-12
    for a, b in zip(dbs, tb):
        assert np.max(np.abs(a - b.grad.numpy())) < 1e-12


def test_backward_central_differences():
    Ws, bs = _net(widths=[6, 16, 16, 6])
    rng = np.random.default_rng(2)
    X = rng.normal(size=(5, 6))
    dY = rng.normal(size=(5, 6))
    loss = lambda W, b, x: float(np.sum(mlp.forward(W, b, x) * dY))
    _, cache = mlp.forward(Ws, bs, X, keep=True)
    dX, dWs, dbs = mlp.backward(Ws, cache, dY)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 5), (4, 2)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, j] += h
        Xm[i, j] -= h
        fd = (loss(Ws, bs, Xp) - loss(Ws, bs, Xm)) / (2 * h)
        assert abs(fd - dX[i, j]) < 1e-8 * max(1, abs(fd))
    for l, (i, j) in [(0, (3, 4)), (1, (7, 2)), (2, (5, 15))]:
        Wp = [W.copy() for W in Ws]
        Wm = [W.copy() for W in Ws]
        Wp[l][i, j] += h
        Wm[l][i, j] -= h
        fd = (loss(Wp, bs, X) - loss(Wm, bs, X)) / (2 * h)
        assert abs(fd - dWs[l][i, j]) < 1e-8 * max(1, abs(fd))


def test_gelu_special_values_and_derivative():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    big = np.array([12.0, 30.0])
    assert np.allclose(mlp.gelu(big), big, rtol=0, atol=1e-15)
    assert np.all(np.abs(mlp.gelu(-big)) < 1e-15)
    x = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-9
    # tanh-form GELU stays within 5e-4 of the exact erf form
    from scipy.special import erf
    exact = 0.5 * x * (1 + erf(x / math.sqrt(2)))
    assert np.max(np.abs(mlp.gelu(x) - exact)) < 5e-4


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(5)
    x = rng.normal(size=10000).astype(np.float32).astype(np.float64) * 10.0 ** rng.integers(-8, 8, 10000)
    x = x.astype(np.float32).astype(np.float64)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert mlp.bf16_round(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16_round(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    # the input pair hi + lo: exact for 16 significant bits, 2^-16 relative beyond
    x = np.array([1 + 2.0 ** -10, 1 + 2.0 ** -10 + 2.0 ** -20, -3.0 * (1 + 2.0 ** -12), 0.75])
    p = mlp.bf16_pair(x)
    assert p[0] == x[0] and p[2] == x[2] and p[3] == x[3]
    assert p[1] == 1 + 2.0 ** -10
    r = np.random.default_rng(4).normal(size=10000) * 3
    assert np.max(np.abs(mlp.bf16_pair(r) - r) / np.abs(r)) <= 2.0 ** -16 + 2.0 ** -24
    # the split is of the FP32 value the normalisation stores
    r32 = r.astype(np.float32).astype(np.float64)
    assert np.array_equal(mlp.bf16_pair(r), mlp.bf16_pair(r32))


def test_identity_layers():
    # widths 6 -> 6 -> 6 with identity weights: F(x) = gelu(x)
    Ws = [np.eye(6), np.eye(6)]
    bs = [np.zeros(6), np.zeros(6)]
    X = np.linspace(-3, 3, 36).reshape(6, 6)
    assert np.max(np.abs(mlp.forward(Ws, bs, X) - mlp.gelu(X))) == 0.0


def test_mse_matches_torch():
    rng = np.random.default_rng(9)
    P, Y = rng.normal(size=(50, 6)), rng.normal(size=(50, 6))
    ref = torch.nn.functional.mse_loss(torch.tensor(P), torch.tensor(Y)).item()
    assert abs(mlp.mse(P, Y) - ref) < 1e-15
    tP = torch.tensor(P, requires_grad=True)
    torch.nn.functional.mse_loss(tP, torch.tensor(Y)).backward()
    assert np.max(np.abs(mlp.mse_grad(P, Y) - tP.grad.numpy())) < 1e-16


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    p = rng.normal(size=100)
    g = rng.normal(size=100) * 10.0 ** rng.integers(-6, 3, 100)
    opt = mlp.Adam([p], lr=1e-3, eps=1e-8)
    new = opt.step([p], [g])[0]
    expect = p - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(new - expect)) < 1e-15


def test_adam_matches_torch_over_steps():
    rng = np.random.default_rng(6)
    p0 = rng.normal(size=(8, 5))
    tp = torch.tensor(p0.copy(), requires_grad=True)
    topt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    opt = mlp.Adam([p0], lr=1e-2)
    p = [p0.copy()]
    for s in range(20):
        g = rng.normal(size=(8, 5))
        p = opt.step(p, [g])
        tp.grad = torch.tensor(g)
        topt.step()
    assert np.max(np.abs(p[0] - tp.detach().numpy())) < 1e-14


def test_prelu_network_matches_torch():
    """The paper's PReLU networks (one slope per layer) against torch's prelu,
    including a BF16-emulating pass whose rounding points torch reproduces
    with explicit casts."""
    Ws, bs = _net(widths=[6, 40, 40, 40, 6])
    slopes = [0.25, -0.1, 0.6]
    rng = np.random.default_rng(5)
    X = rng.normal(size=(53, 6))
    Y = mlp.forward(Ws, bs, X, slopes=slopes)
    h = torch.tensor(X)
    for l, (W, b) in enumerate(zip(Ws, bs)):
        h = h @ torch.tensor(W).T + torch.tensor(b)
        if l < len(Ws) - 1:
            h = torch.nn.functional.prelu(h, torch.tensor([slopes[l]], dtype=torch.float64))
    assert np.max(np.abs(Y - h.numpy())) < 1e-13
    # BF16 emulation: the input as a BF16 hi + lo pair, every hidden
    # activation rounded once
    Yb = mlp.forward(Ws, bs, X, bf16=True, slopes=slopes)
    tx = torch.tensor(X).float().double()
    hi = tx.to(torch.bfloat16).double()
    h = hi + (tx - hi).to(torch.bfloat16).double()
    for l, (W, b) in enumerate(zip(Ws, bs)):
        h = h @ torch.tensor(W).T + torch.tensor(b)
        if l < len(Ws) - 1:
            h = torch.nn.functional.prelu(h, torch.tensor([slopes[l]], dtype=torch.float64))
            h = h.to(torch.bfloat16).double()
    assert np.max(np.abs(Yb - h.numpy())) < 1e-13
    # closed form on special values
    assert np.array_equal(mlp.prelu(np.array([-2.0, 0.0, 3.0]), 0.25), np.array([-0.5, 0.0, 3.0]))


def test_prelu_backward_matches_torch_autograd_and_differences():
    """PReLU reverse mode (weights, biases, input and the per-layer slopes)
    against torch float64 autograd through torch's prelu, and the slope
    gradient against central differences of the network output."""
    Ws, bs = _net(seed=8, widths=[6, 24, 24, 24, 6])
    slopes = [0.25, -0.1, 0.6]
    rng = np.random.default_rng(9)
    X = rng.normal(size=(41, 6))
    dY = rng.normal(size=(41, 6))
    Y, cache = mlp.forward(Ws, bs, X, keep=True, slopes=slopes)
    dX, dWs, dbs, dsl = mlp.backward(Ws, cache, dY, slopes=slopes)
    tW = [torch.tensor(W, requires_grad=True) for W in Ws]
    tb = [torch.tensor(b, requires_grad=True) for b in bs]
    ta = [torch.tensor([a], dtype=torch.float64, requires_grad=True) for a in slopes]
    tX = torch.tensor(X, requires_grad=True)
    h = tX
    for l in range(len(Ws)):
        h = h @ tW[l].T + tb[l]
        if l < len(Ws) - 1:
            h = torch.nn.functional.prelu(h, ta[l])
    h.backward(torch.tensor(dY))
    assert np.max(np.abs(dX - tX.grad.numpy())) < 1e-13
    for a, b in zip(dWs, tW):
        assert np.max(np.abs(a - b.grad.numpy())) < 1e-12
    for a, b in zip(dbs, tb):
        assert np.max(np.abs(a - b.grad.numpy())) < 1e-12
    for a, b in zip(dsl, ta):
        assert abs(a - b.grad.item()) < 1e-11 * max(1.0, abs(a))
    eps = 1e-6
    for l in range(3):
        sp, sm = list(slopes), list(slopes)
        sp[l] += eps
        sm[l] -= eps
        fd = (np.sum(mlp.forward(Ws, bs, X, slopes=sp) * dY)
              - np.sum(mlp.forward(Ws, bs, X, slopes=sm) * dY)) / (2 * eps)
        assert abs(fd - dsl[l]) < 1e-7 * max(1.0, abs(fd))
