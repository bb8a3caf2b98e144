"""Gauss-Lobatto-Legendre tables (oracle; test infrastructure only).

The paper discretises with C0 spectral elements of order K (Sec. 3.2.1) and
does not spell the quadrature out; the standard nodal choice is the K+1
Gauss-Lobatto-Legendre (GLL) points with their quadrature weights, which is
what this module computes:

* nodes:   -1, +1 and the K-1 roots of P_K'(x) (P_K = Legendre polynomial),
* weights: w_j = 2 / (K (K+1) P_K(x_j)^2),
* D[i, j] = l_j'(x_i), the derivative of the j-th Lagrange cardinal
  polynomial at node i, computed with barycentric weights.

Pinned by tests/test_oracle_gll.py: quadrature exact to degree 2K-1, D exact
on polynomials of degree <= K, closed-form nodes/weights for K = 2, 3, 4.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def gll(K: int):
    """Return (nodes, weights, D) for the K+1 point GLL rule on [-1, 1]."""
    if K < 1:
        raise ValueError("order K must be >= 1")
    cK = np.zeros(K + 1)
    cK[K] = 1.0                                  # coefficients of P_K
    interior = L.legroots(L.legder(cK)) if K > 1 else np.zeros(0)
    x = np.concatenate(([-1.0], np.sort(np.real(interior)), [1.0]))
    # one Newton polish of the interior roots of P_K' in extended arithmetic
    dcK = L.legder(cK)
    ddcK = L.legder(dcK)
    for _ in range(3):
        xi = x[1:-1]
        x[1:-1] = xi - L.legval(xi, dcK) / L.legval(xi, ddcK)
    PK = L.legval(x, cK)
    w = 2.0 / (K * (K + 1) * PK ** 2)
    # barycentric weights and the differentiation matrix
    n = K + 1
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    bw = 1.0 / np.prod(diff, axis=1)             # lambda_j = 1 / prod_{k != j}(x_j - x_k)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (bw[j] / bw[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return x, w, D


def lagrange_eval(x_nodes: np.ndarray, xq: np.ndarray) -> np.ndarray:
    """Matrix B[q, j] = l_j(xq[q]) of the Lagrange cardinal functions."""
    n = len(x_nodes)
    B = np.ones((len(xq), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                B[:, j] *= (xq - x_nodes[k]) / (x_nodes[j] - x_nodes[k])
    return B
