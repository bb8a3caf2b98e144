"""FP64 reference of the warm-start network (oracle; test infrastructure only).

The paper has no learned component; this is the plain definition of the small network
the library trains: a tanh multilayer perceptron from standardised run parameters to a
phase field on a uniform grid (x periodic on [x0, x1), cells starting at
x0 + i (x1 - x0)/gnx; y on [y0, y1] with both ends), carried to the GLL nodes by bilinear
interpolation, with the mean squared error to target node fields as the loss.
Parameters are laid out layer by layer: W (dims[l] x dims[l+1], row-major), then b.

``bf16=True`` rounds the weight matrices (not the biases) to bfloat16 with
round-to-nearest-even before every product, as the GPU stores them.

Pinned by tests/test_oracle_neural.py: gradients equal central finite differences.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (8 exponent, 7 mantissa bits), nearest-even."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bilinear_map(gnx, gny, box, node_x, node_y):
    """Dense (nq x gnx*gny) interpolation matrix from the grid to the nodes ([y][x] order)."""
    x0, x1, y0, y1 = box
    nq = len(node_x) * len(node_y)
    R = np.zeros((nq, gnx * gny))
    for qy, Y in enumerate(node_y):
        ty = (Y - y0) / (y1 - y0) * (gny - 1)
        j0 = int(min(max(np.floor(ty), 0), gny - 2))
        wy = ty - j0
        for qx, X in enumerate(node_x):
            tx = (X - x0) / (x1 - x0) * gnx
            i0 = int(np.floor(tx))
            wx = tx - i0
            i0 %= gnx
            i1 = (i0 + 1) % gnx
            q = qy * len(node_x) + qx
            R[q, j0 * gnx + i0] += (1 - wx) * (1 - wy)
            R[q, j0 * gnx + i1] += wx * (1 - wy)
            R[q, (j0 + 1) * gnx + i0] += (1 - wx) * wy
            R[q, (j0 + 1) * gnx + i1] += wx * wy
    return R


def unpack(params, dims):
    out, off = [], 0
    for l in range(len(dims) - 1):
        k, n = dims[l], dims[l + 1]
        W = params[off:off + k * n].reshape(k, n)
        off += k * n
        b = params[off:off + n]
        off += n
        out.append((W, b))
    return out


def loss_and_grad(params, dims, feat_mean, feat_std, R, feat, target, bf16=False):
    """MSE over all (row, node) pairs and its gradient with respect to params."""
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    x = (np.asarray(feat, dtype=np.float64) - feat_mean) / feat_std
    acts = [x]
    Ws = []
    for W, b in layers:
        Wp = bf16_round(W) if bf16 else W
        Ws.append(Wp)
        acts.append(np.tanh(acts[-1] @ Wp + b))
    pred = acts[-1] @ R.T
    err = pred - target
    n = err.size
    loss = float(np.sum(err ** 2) / n)
    d = (2.0 / n) * err @ R                       # gradient with respect to the grid output
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        dz = d * (1.0 - acts[l + 1] ** 2)
        grads.append((acts[l].T @ dz, dz.sum(axis=0)))
        d = dz @ Ws[l].T
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat, pred
