"""Pins for the oracle's GLL tables against textbook closed forms and exactness."""
import math

import numpy as np
import pytest

from oracle.gll import gll, lagrange_eval


def test_closed_forms():
    x, w, _ = gll(2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-14)
    x, w, _ = gll(3)
    s = 1 / math.sqrt(5)
    np.testing.assert_allclose(x, [-1, -s, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)
    x, w, _ = gll(4)
    s = math.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [0.1, 49 / 90, 32 / 45, 49 / 90, 0.1], rtol=1e-14)


@pytest.mark.parametrize("K", [1, 2, 3, 5, 8, 10, 12, 15])
def test_quadrature_exact_to_2K_minus_1(K):
    x, w, _ = gll(K)
    for deg in range(0, 2 * K):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(w, x ** deg) - exact) < 1e-13
    if K >= 1:
        # degree 2K is NOT integrated exactly by a (K+1)-point Lobatto rule
        assert abs(np.dot(w, x ** (2 * K)) - 2.0 / (2 * K + 1)) > 1e-10


@pytest.mark.parametrize("K", [2, 4, 6, 9, 12])
def test_differentiation_exact_on_polynomials(K):
    x, _, D = gll(K)
    rng = np.random.default_rng(K)
    c = rng.standard_normal(K + 1)
    p = np.polynomial.Polynomial(c)
    np.testing.assert_allclose(D @ p(x), p.deriv()(x), atol=1e-11 * np.abs(c).sum() * K * K)
    # rows annihilate constants; the corner entries have the closed form -+K(K+1)/4
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12)
    assert abs(D[0, 0] + K * (K + 1) / 4) < 1e-11
    assert abs(D[K, K] - K * (K + 1) / 4) < 1e-11


def test_lagrange_cardinal():
    x, _, _ = gll(6)
    np.testing.assert_allclose(lagrange_eval(x, x), np.eye(7), atol=1e-14)
