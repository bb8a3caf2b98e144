"""Pins for the oracle's discrete energy E(t) of eq. (14) and for the mixture laws of eq.
(interpolation), each against a closed form or a continuum integral computed independently
(adaptive quadrature), so that a dropped factor, a wrong sign or a swapped term in any of the
four parts of E(t) (kinetic, mixing, electric, wall) fails one of them."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.scheme import DIRICHLET, NEUMANN, Params, Solver, VBC
from oracle.sem import Mesh2D

LX = 2.0
FLUID = dict(rho1=3.0, rho2=1.0, mu1=2.0, mu2=1.0, eps1=5.0, eps2=1.0, sigma=1.3, gamma1=1e-3)


def _solver(eta, K=12, ey=8, ex=2, theta=90.0, vb=0.0, vt=0.0, top=DIRICHLET, nz=1):
    prm = Params(eta=eta, dt=1e-4, theta_s_deg=theta, **FLUID)
    mesh = Mesh2D(np.linspace(0.0, LX, ex + 1), np.linspace(0.0, 1.0, ey + 1), K)
    return Solver(mesh, prm, VBC(DIRICHLET, top, vb, vt), nz=nz, lz=1.0)


def _layer(sol, h, width):
    """phi = tanh((h - y) / (sqrt 2 width)) at the nodes (fluid 1 below y = h), all planes."""
    Yg = np.repeat(sol.mesh.Y, sol.mesh.nx)
    return np.repeat(np.tanh((h - Yg) / (math.sqrt(2.0) * width))[None, :], sol.nz, axis=0)


def _quad(f, a=0.0, b=1.0, pts=None):
    return integrate.quad(f, a, b, points=pts, epsabs=1e-13, epsrel=1e-13, limit=400)[0]


def test_mixture_laws_and_derivatives():
    """eq. (interpolation): rho, mu linear and eps the cubic Hermite blend with the pure values at
    phi = +-1; eps' (used in Q2, T and J) is d eps / d phi; lambda h = dF/dphi for the double
    well F = lambda (phi^2 - 1)^2 / (4 eta^2) of eq. (double_well); Theta' is the derivative of
    the wall energy sigma cos(theta_s) phi (phi^2 - 3) / 4 of eq. (theta_def)."""
    p = Params(eta=0.07, dt=1e-4, theta_s_deg=63.0, **FLUID)
    assert p.rho(1.0) == p.rho1 and p.rho(-1.0) == p.rho2
    assert p.mu(1.0) == p.mu1 and p.mu(-1.0) == p.mu2
    assert abs(p.eps(1.0) - p.eps1) < 1e-15 and abs(p.eps(-1.0) - p.eps2) < 1e-15
    assert p.deps(1.0) == 0.0 and p.deps(-1.0) == 0.0          # flat at the pure phases
    phis = np.linspace(-1.3, 1.3, 27)
    hstep = 1e-5
    fd = lambda f, x: (f(x + hstep) - f(x - hstep)) / (2 * hstep)
    np.testing.assert_allclose(p.deps(phis), fd(p.eps, phis), rtol=0, atol=1e-8)
    F = lambda x: p.lam * (x ** 2 - 1.0) ** 2 / (4.0 * p.eta ** 2)
    np.testing.assert_allclose(p.lam * p.h(phis), fd(F, phis), rtol=1e-8, atol=1e-8)
    Th = lambda x: p.sigma * math.cos(math.radians(63.0)) * x * (x ** 2 - 3.0) / 4.0
    np.testing.assert_allclose(p.dTheta(phis), fd(Th, phis), rtol=0, atol=1e-9)
    # eps is monotone between the phases and never leaves [eps2, eps1] on [-1, 1]
    e = p.eps(np.linspace(-1, 1, 201))
    assert np.all(np.diff(e) > 0) and e.min() >= p.eps2 - 1e-15 and e.max() <= p.eps1 + 1e-15


@pytest.mark.parametrize("ratio", [1.0, 2.0])
def test_mixing_energy_of_a_flat_interface(ratio):
    """Mixing part of eq. (14): for phi = tanh((h - y)/(sqrt 2 eta w)) the energy per unit length
    of interface is (sigma/2)(1/w + w) with lambda = 3 sigma eta / (2 sqrt 2) (Sec. 2.1); w = 1 is
    the equilibrium profile whose energy is the surface tension sigma itself.  The gradient and
    double-well halves enter with different powers of w, so a wrong factor in either fails."""
    eta = 0.04
    sol = _solver(eta)
    sol.set_initial(_layer(sol, 0.5, eta * ratio))
    e = sol.energy()
    closed = LX * 0.5 * sol.prm.sigma * (1.0 / ratio + ratio)
    # the profile's tails beyond the domain ([0, 1], interface at 0.5) carry ~exp(-sqrt(2)/(eta w))
    tail = 8.0 * math.exp(-math.sqrt(2.0) / (eta * ratio)) * closed
    assert abs(e - closed) < 1e-9 * closed + tail, (e, closed, tail)


def test_mixing_energy_3d_counts_the_z_period():
    """The same flat interface in Alg. 2's 3D setting (z-period 1): E is sigma times the area
    L_x L_z of the interface."""
    eta = 0.05
    sol = _solver(eta, nz=4)
    sol.set_initial(_layer(sol, 0.5, eta))
    assert abs(sol.energy() - LX * sol.prm.sigma) < 1e-9 * LX


@pytest.mark.parametrize("dv", [1.0, 2.0])
def test_electric_energy_of_flat_layers_is_the_series_capacitor(dv):
    """Electric part of eq. (14), (1/2) D.E = (1/2) eps |E|^2: for flat layers between two
    electrodes the potential solves (eps V')' = 0, so the energy per unit wall length is
    (1/2) dV^2 / int_0^1 eps(phi)^-1 dy (the series capacitor).  E(t) at voltage dV minus E(t) at
    zero voltage on the same phi isolates it; it must scale with dV^2."""
    eta, h = 0.05, 0.4
    sol0 = _solver(eta)
    sol0.set_initial(_layer(sol0, h, eta))
    sol = _solver(eta, vb=dv, vt=0.0)
    sol.set_initial(_layer(sol, h, eta))
    inv_eps = lambda y: 1.0 / sol.prm.eps(math.tanh((h - y) / (math.sqrt(2.0) * eta)))
    closed = LX * 0.5 * dv ** 2 / _quad(inv_eps, pts=[h])
    got = sol.energy() - sol0.energy()
    assert abs(got - closed) < 1e-9 * closed, (got, closed)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_wall_energy_of_a_sessile_drop(theta):
    """Wall part of eq. (14) with Theta of eq. (theta_def) (constant dropped): for a drop sitting
    on the wall, E(theta_s) - E(90 deg) = sigma cos(theta_s) int_wall phi (phi^2 - 3)/4 dx, the
    wall trace phi(x, 0) = tanh((r0 - |x - 1|)/(sqrt 2 eta)); sign and factor flip with cos."""
    eta, r0 = 0.05, 0.45
    ph = lambda X, Y: np.tanh((r0 - np.sqrt((X - 1.0) ** 2 + Y ** 2)) / (math.sqrt(2.0) * eta))
    vals = {}
    for th in (90.0, theta):
        sol = _solver(eta, K=12, ey=4, ex=16, theta=th)
        X = np.tile(sol.mesh.X, sol.mesh.ny)
        Y = np.repeat(sol.mesh.Y, sol.mesh.nx)
        sol.set_initial(ph(X, Y)[None, :])
        vals[th] = sol.energy()
    trace = lambda x: math.tanh((r0 - abs(x - 1.0)) / (math.sqrt(2.0) * eta))
    wall = _quad(lambda x: (lambda f: f * (f * f - 3.0) / 4.0)(trace(x)), 0.0, LX, pts=[1.0 - r0, 1.0, 1.0 + r0])
    closed = FLUID["sigma"] * math.cos(math.radians(theta)) * wall
    got = vals[theta] - vals[90.0]
    assert abs(got - closed) < 1e-8 * abs(closed), (got, closed)


def test_kinetic_energy_with_variable_density():
    """Kinetic part of eq. (14), (1/2) rho(phi) |u|^2: with a shear flow u = (sin(pi y), 0) over
    flat layers (rho1 = 3 below, rho2 = 1 above) it is L_x int (1/2) rho(phi(y)) sin^2(pi y) dy."""
    eta, h = 0.05, 0.5
    sol0 = _solver(eta)
    sol0.set_initial(_layer(sol0, h, eta))
    sol = _solver(eta)
    Yg = np.repeat(sol.mesh.Y, sol.mesh.nx)[None, :]
    z = np.zeros_like(Yg)
    sol.set_initial(_layer(sol, h, eta), u0=[np.sin(np.pi * Yg), z, z])
    rho = lambda y: sol.prm.rho(math.tanh((h - y) / (math.sqrt(2.0) * eta)))
    closed = LX * _quad(lambda y: 0.5 * rho(y) * math.sin(math.pi * y) ** 2, pts=[h])
    got = sol.energy() - sol0.energy()
    assert abs(got - closed) < 1e-9 * closed, (got, closed)
