"""CPU reference of the learned-pruning MLP (test infrastructure only).

16 -> 128 -> 128 -> 1 with ReLU, loss mean((y - t)^2).  The parameter
vector (18817 values) is W1[16][128], b1[128], W2[128][128], b2[128], w3[128],
b3, W[k][n] mapping input k to output n.

`bf16=True` reproduces the library's mixed precision: the inputs, W1, W2,
w3, the hidden activation fed to layer 2 and, in the backward pass, the GEMM
operands dh2 and dh1 are rounded to bfloat16 (round to nearest even); sums are
FP64 here.  Rounding is treated as the identity in the derivative
(straight-through), so the gradients are those of the same formulas.
`bf16=False` is plain FP64 and is pinned by finite differences.
"""
from __future__ import annotations

import numpy as np

F, H = 16, 128
OFF = {"W1": 0, "b1": 2048, "W2": 2176, "b2": 18560, "w3": 18688, "b3": 18816}
N_PARAMS = 18817


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[0:2048].reshape(F, H), p[2048:2176], p[2176:18560].reshape(H, H),
            p[18560:18688], p[18688:18816], p[18816])


def forward(p, X, use_bf16=True):
    r = bf16 if use_bf16 else (lambda v: np.asarray(v, np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(p)
    Xr = r(X)
    h1p = Xr @ r(W1) + b1
    h1 = r(np.maximum(h1p, 0.0))
    h2p = h1 @ r(W2) + b2
    h2 = np.maximum(h2p, 0.0)
    y = h2 @ r(w3) + b3
    return y, (Xr, h1p, h1, h2p, h2)


def loss_and_grad(p, X, T, use_bf16=True):
    r = bf16 if use_bf16 else (lambda v: np.asarray(v, np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, (Xr, h1p, h1, h2p, h2) = forward(p, X, use_bf16)
    n = len(y)
    e = y - np.asarray(T, np.float64)
    loss = float(np.sum(e * e) / n)
    dy = 2.0 * e / n
    g = np.zeros(N_PARAMS)
    g[OFF["b3"]] = dy.sum()
    g[OFF["w3"]:OFF["w3"] + H] = h2.T @ dy
    dh2 = np.outer(dy, r(w3)) * (h2p > 0)
    g[OFF["b2"]:OFF["b2"] + H] = dh2.sum(axis=0)
    dh2r = r(dh2)
    g[OFF["W2"]:OFF["W2"] + H * H] = (h1.T @ dh2r).reshape(-1)
    dh1 = (dh2r @ r(W2).T) * (h1p > 0)
    g[OFF["b1"]:OFF["b1"] + H] = dh1.sum(axis=0)
    g[OFF["W1"]:OFF["W1"] + F * H] = (Xr.T @ r(dh1)).reshape(-1)
    return loss, g
