"""FP64 oracle of the learned Newton warm start (test infrastructure only).

The warm start predicts, for every node, the increment of its velocity and pressure over the next
backward-Euler step (Remark of Section 4.1: the transient term), so that Newton (Section 4.2)
starts from u^n + increment instead of u^n; Newton then converges to the same tolerance, so the
network only changes the starting point.

Network (plain definition, written out here):
  features  x = [u^n (4), d = u^n - u^{n-1} (4), mean of d over the node's 1-ring (4)] (12)
  H1 = tanh(x W1 + b1)          W1 (12 x 128)
  H2 = tanh(H1 W2 + b2)         W2 (128 x 128)
  y  = H2 W3 + b3               W3 (128 x 4)
  loss = mean over nodes and components of (y - t)^2
The weights are stored in BF16 (round to nearest, ties to even); the oracle computes in FP64 with
the same BF16-rounded weights, so only the kernels' FP32 rounding separates the two.
Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, w -= lr mhat / (sqrt(vhat) + eps) with the
bias corrections mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).

Parity status: pinned (finite differences of the loss, closed forms, BF16 rounding of known values).
"""
from __future__ import annotations

import numpy as np

N_IN, WIDTH, N_OUT = 12, 128, 4
SHAPES = [("W1", (N_IN, WIDTH)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def unpack(flat) -> dict:
    """Split a flat parameter vector (order W1, b1, W2, b2, W3, b3; row-major) into arrays."""
    flat = np.asarray(flat, np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[k:k + n].reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def stored(flat) -> dict:
    """The parameters the kernels use: weights rounded to BF16, biases in FP32."""
    p = unpack(flat)
    return {k: (bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
            for k, v in p.items()}


def forward(p: dict, x):
    """Returns (y, cache) for features x (N x 12)."""
    x = np.asarray(x, np.float64)
    h1 = np.tanh(x @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    y = h2 @ p["W3"] + p["b3"]
    return y, (x, h1, h2)


def loss_and_grad(p: dict, x, t):
    """Mean squared error and its gradient with respect to every parameter (backpropagation)."""
    y, (x, h1, h2) = forward(p, x)
    t = np.asarray(t, np.float64)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = 2.0 * (y - t) / n
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = (dy @ p["W3"].T) * (1.0 - h2 ** 2)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"].T) * (1.0 - h1 ** 2)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return loss, g


def adam_step(w, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of flat arrays w (master weights), m, v with gradient g at step t >= 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    w = w - lr * mhat / (np.sqrt(vhat) + eps)
    return w, m, v


def ring_mean(conn, n_nodes, u):
    """Mean of u over each node's 1-ring: the other nodes of the elements that contain it."""
    conn = np.asarray(conn)
    rows = np.repeat(conn, conn.shape[1], axis=1).ravel()
    cols = np.tile(conn, (1, conn.shape[1])).ravel()
    keep = rows != cols
    pairs = np.unique(np.stack([rows[keep], cols[keep]], axis=1), axis=0)
    s = np.zeros((n_nodes, u.shape[1]))
    np.add.at(s, pairs[:, 0], u[pairs[:, 1]])
    cnt = np.bincount(pairs[:, 0], minlength=n_nodes).astype(np.float64)
    return s / np.maximum(cnt, 1.0)[:, None]


def features(conn, u_n, u_nm1, scale_in=None):
    """x = [u^n, d, ring mean of d] with d = u^n - u^{n-1}, each column divided by scale_in (12)
    if given."""
    u_n = np.asarray(u_n, np.float64)
    d = u_n - np.asarray(u_nm1, np.float64)
    x = np.concatenate([u_n, d, ring_mean(conn, u_n.shape[0], d)], axis=1)
    if scale_in is not None:
        x = x / np.asarray(scale_in, np.float64)[None, :]
    return x
