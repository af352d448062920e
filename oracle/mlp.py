"""Plain FP64 reference of the surrogate network (numpy).

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU leg.

The network (this project's surrogate; the paper has none):
  inputs x = (alpha/25, beta/25, a, cos i),
  h_1..h_4 = silu(W_l h_{l-1} + b_l) with 256 units, silu(z) = z / (1 + e^-z),
  out = W_5 h_4 + b_5 (8 values: capture logit, (ln r1 - 2)/2, cos phi1,
        sin phi1, (ln r2 - 2)/2, cos phi2, sin phi2, g1 - 1),
  loss per row = softplus(o0) - y0 o0 + sum_{j>=1} m_j (o_j - y_j)^2,
  batch loss = mean over rows.
Parameters use the padded layout of the C ABI: for l = 0..4, W_l [out][in]
then b_l [out], in = 16, 256, 256, 256, 256 and out = 256, 256, 256, 256, 64.

`quantize=True` rounds to bfloat16 (round to nearest even) where the GPU
path stores bfloat16: the weights, every layer input and the backward
signals dZ / dOut; accumulation stays exact here (FP64).
"""
from __future__ import annotations

import numpy as np

IN, IN_PAD, HID, LAYERS, OUT, OUT_PAD = 4, 16, 256, 5, 8, 64


def in_dim(l: int) -> int:
    return IN_PAD if l == 0 else HID


def out_dim(l: int) -> int:
    return OUT_PAD if l == LAYERS - 1 else HID


def layout():
    off, w, b = 0, [], []
    for l in range(LAYERS):
        w.append(off)
        off += out_dim(l) * in_dim(l)
        b.append(off)
        off += out_dim(l)
    return w, b, off


W_OFF, B_OFF, NUM_PARAMS = layout()


def unpack(p: np.ndarray):
    Ws, bs = [], []
    for l in range(LAYERS):
        Ws.append(p[W_OFF[l]:W_OFF[l] + out_dim(l) * in_dim(l)].reshape(out_dim(l), in_dim(l)))
        bs.append(p[B_OFF[l]:B_OFF[l] + out_dim(l)])
    return Ws, bs


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters (uniform +-1/sqrt(fan_in) on the live block,
    zero padding and biases) as float32."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NUM_PARAMS, dtype=np.float64)
    Ws, bs = unpack(p)
    for l in range(LAYERS):
        fan_in = IN if l == 0 else HID
        n_out = OUT if l == LAYERS - 1 else HID
        lim = 1.0 / np.sqrt(fan_in)
        Ws[l][:n_out, :fan_in] = rng.uniform(-lim, lim, size=(n_out, fan_in))
    return p.astype(np.float32)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest even) and return as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    out[nan] = np.nan
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p: np.ndarray, x: np.ndarray, quantize: bool = False, keep: bool = False):
    """Network outputs (n, 8) for inputs x (n, 4)."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    Ws, bs = unpack(np.asarray(p, dtype=np.float64))
    a = np.zeros((x.shape[0], IN_PAD))
    a[:, :IN] = x
    a = q(a)
    acts, pre = [a], []
    for l in range(LAYERS):
        z = a @ q(Ws[l]).T + bs[l]
        if l < LAYERS - 1:
            pre.append(z)
            a = q(silu(z))
            acts.append(a)
        else:
            out = z
    if keep:
        return out, acts, pre
    return out[:, :OUT]


def loss(out: np.ndarray, y: np.ndarray, m: np.ndarray) -> float:
    z = out[:, 0]
    sp = np.where(z > 0, z + np.log1p(np.exp(-z)), np.log1p(np.exp(z)))
    row = sp - y[:, 0] * z + np.sum(m[:, 1:] * (out[:, 1:OUT] - y[:, 1:]) ** 2, axis=1)
    return float(np.mean(row))


def grad(p: np.ndarray, x: np.ndarray, y: np.ndarray, m: np.ndarray,
         quantize: bool = False) -> tuple[float, np.ndarray]:
    """Batch loss and its gradient with respect to the parameter vector."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    n = x.shape[0]
    out, acts, pre = forward(p, x, quantize, keep=True)
    L = loss(out, y, m)
    Ws, _ = unpack(np.asarray(p, dtype=np.float64))
    g = np.zeros(NUM_PARAMS)
    gW, gb = unpack(g)
    d = np.zeros((n, OUT_PAD))
    z0 = out[:, 0]
    d[:, 0] = (1.0 / (1.0 + np.exp(-z0)) - y[:, 0]) / n
    d[:, 1:OUT] = 2.0 * m[:, 1:] * (out[:, 1:OUT] - y[:, 1:]) / n
    d = q(d)
    for l in range(LAYERS - 1, -1, -1):
        gW[l][...] = d.T @ acts[l]
        gb[l][...] = d.sum(axis=0)
        if l > 0:
            dA = d @ q(Ws[l])
            d = q(dA * silu_grad(pre[l - 1]))
    return L, g
