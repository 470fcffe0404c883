"""fp64 reference of the surrogate network -- TEST INFRASTRUCTURE.

The network (no counterpart in the paper; it predicts the steady-state
velocity and the jam probability of a BML run, Sec. 2 describing the
free-flowing and jammed phases it distinguishes):

    x (in_dim) -> [Linear 128, ReLU] x 3 -> Linear 2 -> (v_hat, z)

with parameters W1 (128 x in_dim), b1, W2, b2, W3, b3 (128 x 128, 128),
W4 (2 x 128), b4 (2), stored flat in that order, each W row-major
[out][in].  Per-sample loss (v_hat - v)^2 + BCE(z, jam), BCE with logits
(max(z, 0) - z*jam + log(1 + exp(-|z|))); the batch loss is the mean.
AdamW (Loshchilov & Hutter, decoupled weight decay) with bias-corrected
moments.

Everything here is plain fp64 numpy: matrix products are the only library
primitive used.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128
N_HIDDEN = 3
N_OUT = 2


def shapes(in_dim: int):
    dims = [in_dim] + [HIDDEN] * N_HIDDEN + [N_OUT]
    out = []
    for l in range(len(dims) - 1):
        out.append((dims[l + 1], dims[l]))  # W
        out.append((dims[l + 1],))          # b
    return out


def num_params(in_dim: int) -> int:
    return int(sum(np.prod(s) for s in shapes(in_dim)))


def unflatten(flat: np.ndarray, in_dim: int):
    ps, off = [], 0
    for s in shapes(in_dim):
        n = int(np.prod(s))
        ps.append(np.asarray(flat[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return ps


def flatten(ps) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in ps])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as
    fp64.  bfloat16 keeps the top 16 bits of the IEEE binary32 pattern."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(ps, x: np.ndarray):
    """Returns (outputs (B, 2), cache of pre-activations and activations)."""
    h = np.asarray(x, dtype=np.float64)
    acts, pres = [h], []
    nl = len(ps) // 2
    for l in range(nl):
        W, b = ps[2 * l], ps[2 * l + 1]
        z = h @ W.T + b
        pres.append(z)
        h = np.maximum(z, 0.0) if l < nl - 1 else z
        acts.append(h)
    return h, (acts, pres)


def bce_with_logits(z, y):
    return np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    """Logistic function, 1/(1+e^-z) for z >= 0 and e^z/(1+e^z) below, so
    neither branch cancels."""
    z = np.asarray(z, dtype=np.float64)
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def loss(ps, x, v, jam) -> float:
    out, _ = forward(ps, x)
    per = (out[:, 0] - v) ** 2 + bce_with_logits(out[:, 1], jam)
    return float(per.mean())


def backward(ps, x, v, jam):
    """Gradients of the mean loss, in the layout of `ps`; and the loss."""
    out, (acts, pres) = forward(ps, x)
    B = x.shape[0]
    d = np.zeros_like(out)
    d[:, 0] = 2.0 * (out[:, 0] - v) / B
    d[:, 1] = (sigmoid(out[:, 1]) - jam) / B
    nl = len(ps) // 2
    grads = [None] * len(ps)
    for l in range(nl - 1, -1, -1):
        W = ps[2 * l]
        grads[2 * l] = d.T @ acts[l]
        grads[2 * l + 1] = d.sum(axis=0)
        if l > 0:
            d = (d @ W) * (pres[l - 1] > 0)
    per = (out[:, 0] - v) ** 2 + bce_with_logits(out[:, 1], jam)
    return grads, float(per.mean())


class AdamW:
    """AdamW state for a flat parameter vector."""

    def __init__(self, n: int, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, w: np.ndarray, g: np.ndarray, lr: float, wd: float) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w - lr * (mh / (np.sqrt(vh) + self.eps) + wd * w)
