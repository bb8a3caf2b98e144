"""Pins for the oracle's assembled spectral-element operators."""
import math

import numpy as np
import pytest

from oracle.sem import Mesh2D


def mesh(K=6, graded=False):
    yb = np.linspace(0.0, 1.0, 4)
    if graded:
        yb = 0.5 * (1 - np.cos(np.pi * yb))
    return Mesh2D(np.linspace(0.0, 2.0, 5), yb, K)


@pytest.mark.parametrize("graded", [False, True])
def test_mass_and_area(graded):
    m = mesh(graded=graded)
    assert abs(m.Mdiag.sum() - 2.0) < 1e-13
    assert np.all(m.Mdiag > 0)
    # GLL quadrature integrates y^q exactly for q <= 2K - 1 (x-independent, periodic in x)
    Yg = np.repeat(m.Y, m.nx)
    for q in range(2 * m.K):
        assert abs(m.Mdiag @ Yg ** q - 2.0 / (q + 1)) < 1e-12


@pytest.mark.parametrize("graded", [False, True])
def test_stiffness(graded):
    m = mesh(graded=graded)
    Kd = m.Kmat.toarray()
    np.testing.assert_allclose(Kd, Kd.T, atol=1e-10)
    np.testing.assert_allclose(Kd @ np.ones(m.n2), 0.0, atol=1e-10)
    ev = np.linalg.eigvalsh(Kd)
    assert ev[0] > -1e-9 and abs(ev[0]) < 1e-9 and ev[1] > 1e-3   # one zero mode (constants)
    Yg = np.repeat(m.Y, m.nx)
    for a in range(1, 4):
        for b in range(1, 4):
            exact = 2.0 * a * b / (a + b - 1)            # int_0^2 int_0^1 (a y^{a-1})(b y^{b-1})
            assert abs((Yg ** a) @ (m.Kmat @ Yg ** b) - exact) < 1e-10


def test_gradients_spectral_in_x():
    m = mesh(K=10)
    Xg = np.tile(m.X, m.ny)
    f = np.sin(np.pi * Xg)
    np.testing.assert_allclose(m.Gx @ f, np.pi * np.cos(np.pi * m.XL), atol=1e-7)
    # energy of sin(pi x): int |d/dx|^2 = pi^2 * int_0^2 cos^2 = pi^2
    assert abs(f @ (m.Kmat @ f) - math.pi ** 2) < 1e-7


def test_projection_and_weak_derivatives():
    m = mesh()
    Yg = np.repeat(m.Y, m.nx)
    # the L2 projection of an element-local gradient of a polynomial is the polynomial gradient
    Ey = (m.ZW @ (m.Gy @ Yg ** 3)) / m.Mdiag
    np.testing.assert_allclose(Ey, 3 * Yg ** 2, atol=1e-11)
    # int f dw/dx summed over all test functions w is int f d(1)/dx = 0
    rng = np.random.default_rng(0)
    fL = rng.standard_normal(m.nL)
    assert abs(np.sum(m.WDx @ fL)) < 1e-12 and abs(np.sum(m.WDy @ fL)) < 1e-12
    # int f * 1 = sum WL f
    assert abs(np.sum(m.ZW @ fL) - m.WL @ fL) < 1e-12


def test_faces():
    m = mesh()
    for name, y0 in (("bottom", 0.0), ("top", 1.0)):
        F = m.face[name]
        assert abs(np.sum(F["FM"] @ (F["RZ"] @ np.ones(m.nx))) - 2.0) < 1e-13
        # face nodes sit on the side
        rows = F["FZ"].indices
        np.testing.assert_allclose(np.repeat(m.Y, m.nx)[rows], y0, atol=1e-15)
        # int_side sin(pi x) d w/dx summed against w = cos(pi x) -> int sin(pi x) (-pi sin(pi x)) = -pi
        Xg = np.tile(m.X, m.ny)
        fF = F["RZ"] @ np.sin(np.pi * m.X)
        val = np.cos(np.pi * Xg) @ (F["FDx"] @ fF)
        assert abs(val + math.pi) < 1e-7
