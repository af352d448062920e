"""Pins of the FP64 reference network (oracle/mlp.py) against finite
differences, closed forms and an independent bfloat16 conversion."""
import numpy as np
import pytest

from oracle import mlp as M


def small_problem(seed=3, n=6):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed).astype(np.float64)
    p[M.B_OFF[0]:M.B_OFF[0] + 256] = rng.normal(size=256) * 0.1   # nonzero biases
    x = rng.uniform(-1, 1, size=(n, 4))
    y = np.zeros((n, 8))
    y[:, 0] = rng.integers(0, 2, size=n)
    y[:, 1:] = rng.normal(size=(n, 7)) * 0.5
    m = (rng.uniform(size=(n, 8)) > 0.3).astype(np.float64)
    m[:, 0] = 1.0
    return p, x, y, m


def test_gradient_matches_central_differences():
    p, x, y, m = small_problem()
    L, g = M.grad(p, x, y, m)
    assert abs(L - M.loss(M.forward(p, x, keep=True)[0], y, m)) < 1e-14
    rng = np.random.default_rng(9)
    # sample coordinates in every live block of every layer
    idx = []
    for l in range(M.LAYERS):
        n_out = M.OUT if l == M.LAYERS - 1 else M.HID
        fan = M.IN if l == 0 else M.HID
        for _ in range(6):
            idx.append(M.W_OFF[l] + rng.integers(n_out) * M.in_dim(l) + rng.integers(fan))
            idx.append(M.B_OFF[l] + rng.integers(n_out))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        Lp = M.loss(M.forward(p + e, x, keep=True)[0], y, m)
        Lm = M.loss(M.forward(p - e, x, keep=True)[0], y, m)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_padding_receives_no_gradient():
    p, x, y, m = small_problem()
    _, g = M.grad(p, x, y, m)
    Ws, bs = M.unpack(g)
    assert np.all(Ws[0][:, M.IN:] == 0)                # padded inputs
    assert np.all(Ws[-1][M.OUT:, :] == 0) and np.all(bs[-1][M.OUT:] == 0)


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 101)
    assert np.allclose(M.silu(z), z * 0.5 * (1 + np.tanh(z / 2)), rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.allclose(M.silu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_loss_definition():
    out = np.zeros((2, 64))
    out[0, 0], out[1, 0] = 2.0, -1.0
    out[:, 1] = 0.5
    y = np.zeros((2, 8))
    y[0, 0] = 1.0
    m = np.zeros((2, 8))
    m[:, 0] = 1.0
    m[1, 1] = 1.0
    # row 0: softplus(2) - 2; row 1: softplus(-1) + 0.25
    want = 0.5 * ((np.log1p(np.exp(2.0)) - 2.0) + (np.log1p(np.exp(-1.0)) + 0.25))
    assert abs(M.loss(out, y, m) - want) < 1e-15


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005, -3.1415926, 65504.0, 1e-30, 0.0])
    want = np.array([1.0, 1.0, 1.0078125, -3.140625, 65536.0])
    got = M.bf16(vals)
    assert np.array_equal(got[:5], want)
    assert got[6] == 0.0
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = rng.normal(size=10000).astype(np.float32) * 10 ** rng.uniform(-5, 5, size=10000)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)
