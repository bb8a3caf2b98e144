"""Pins for the oracle's time step (Alg. 1 / Alg. 2) against facts fixed by the paper
and by mathematics, independent of the oracle's own formulas."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads
from oracle import manufactured as mf
from oracle.runner import solver_of
from oracle.scheme import DIRICHLET, NEUMANN, Params, Solver, VBC
from oracle.sem import Mesh2D

# Physical parameters for the manufactured-solution runs (the paper does not list
# the values it used in Sec. 4.1; any consistent set exercises every term).
MMS = dict(rho1=1.0, rho2=3.0, mu1=0.01, mu2=0.02, eps1=1.0, eps2=3.0, sigma=0.05, eta=0.1,
           gamma1=1e-2, theta_s_deg=75.0)


def mms_run(case, K, dt, tf, S=0.0, nz=1):
    prm = Params(dt=dt, S=S, **MMS)
    if case == "2d":
        mesh, lz = Mesh2D([0, 1, 2], [0, 1], K), 1.0
    else:
        mesh, lz = Mesh2D([0, 1, 2], [-1, 1], K), 2.0
    exact, sfor = mf.build(case, prm)
    sol = Solver(mesh, prm, VBC(DIRICHLET, NEUMANN), nz=nz, lz=lz)
    sol.sources = sfor(sol)
    ex0 = mf.nodal_exact(sol, exact, 0.0)
    sol.set_initial(ex0["phi"], u0=ex0["u"], P0=ex0["P"])
    for _ in range(int(round(tf / dt))):
        sol.step()
    ex = mf.nodal_exact(sol, exact, sol.t)
    return np.array([max(np.max(np.abs(sol.u[c] - ex["u"][c])) for c in range(3)),
                     np.max(np.abs(sol.P - ex["P"])), np.max(np.abs(sol.phi - ex["phi"])),
                     np.max(np.abs(sol.V - ex["V"]))])


def test_fourier_conventions():
    """f_hat_k = (1/Nz) sum f_j exp(-i beta_k z_j) (Sec. 3.2.2) and d/dz <-> i beta_k."""
    mesh = Mesh2D([0, 2], [0, 1], 2)
    sol = Solver(mesh, Params(dt=1e-3, **MMS), VBC(), nz=8, lz=2.0)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((8, mesh.n2))
    z = sol.zc
    naive = np.array([[np.sum(f[:, i] * np.exp(-1j * 2 * np.pi * k / 2.0 * z)) / 8 for i in range(mesh.n2)]
                      for k in range(5)])
    np.testing.assert_allclose(sol.fft(f), naive, atol=1e-14)
    np.testing.assert_allclose(sol.ifft(sol.fft(f)), f, atol=1e-14)
    g = np.sin(3 * np.pi * z)[:, None] * np.ones((1, mesh.n2))
    np.testing.assert_allclose(sol.dz(g), 3 * np.pi * np.cos(3 * np.pi * z)[:, None] * np.ones((1, mesh.n2)),
                               atol=1e-12)
    # Nyquist mode cos(4 pi z) on 8 points (beta = 4 pi): its first derivative is dropped
    gn = np.cos(4 * np.pi * z)[:, None] * np.ones((1, mesh.n2))
    np.testing.assert_allclose(sol.dz(gn), 0.0, atol=1e-12)


def test_manufactured_2d_spatial():
    """eq. (80): errors decay exponentially in the element order (Fig. 2b shape)."""
    e4, e6, e8 = (mms_run("2d", K, 1e-3, 0.05) for K in (4, 6, 8))
    assert np.all(e6 < e4 / 5) and np.all(e8 < e6 / 5), (e4, e6, e8)
    assert np.all(e8 < 3e-4)


def test_manufactured_2d_temporal():
    """eq. (80): second order in dt (Fig. 2c shape).  S is held at the bound of the
    smallest dt: S scaling like dt^{-1/2} would make the stabiliser term O(dt^{3/2})."""
    S = Params(dt=2e-3, **MMS).S
    e = [mms_run("2d", 12, dt, 0.2, S=S) for dt in (8e-3, 4e-3, 2e-3)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert np.all(r1 > 3.5) and np.all(r2 > 3.5), (r1, r2)


def test_manufactured_3d_spatial():
    """eq. (81) with the whole wall Dirichlet for V: exponential in K (Fig. 3b shape)."""
    e4, e6, e8 = (mms_run("3d", K, 1e-3, 0.02, nz=8) for K in (4, 6, 8))
    assert np.all(e6 < e4 / 3) and np.all(e8 < e6 / 3), (e4, e6, e8)


def test_manufactured_3d_temporal():
    S = Params(dt=2e-3, **MMS).S
    e = [mms_run("3d", 12, dt, 0.08, S=S, nz=8) for dt in (8e-3, 4e-3)]
    r = e[0] / e[1]
    assert np.all(r > 2.7), r


@pytest.mark.parametrize("phival", [1.0, -1.0])
def test_reduction_consistency(phival):
    """Sec. 2.2: phi = +-1 is an exact solution; the run is single-phase NS plus Laplace,
    so with u0 = 0 and whole-side voltages, u stays 0 and V is the linear profile."""
    wl = workloads.small2d(ex=4, ey=3, order=5, theta_s_deg=60.0)
    sol = solver_of(wl, init=False)
    sol.set_initial(np.full((1, sol.mesh.n2), phival))
    for _ in range(4):
        sol.step()
    np.testing.assert_allclose(sol.phi, phival, atol=1e-12)
    assert sol.umax() < 1e-12
    Yg = np.repeat(sol.mesh.Y, sol.mesh.nx)
    np.testing.assert_allclose(sol.V[0], 1.0 - Yg, atol=1e-12)
    np.testing.assert_allclose(sol.E[1][0], -1.0, atol=1e-11)


def _layer_potential_exact(prm, eta, h, vb, vt, y):
    inv_eps = lambda s: 1.0 / prm.eps(math.tanh((h - s) / (math.sqrt(2) * eta)))
    tot = integrate.quad(inv_eps, 0, 1, points=[h], epsabs=1e-14, epsrel=1e-14, limit=200)[0]
    return np.array([vb + (vt - vb) * integrate.quad(inv_eps, 0, yy, points=[h] if yy > h else None,
                                                     epsabs=1e-14, epsrel=1e-14, limit=200)[0] / tot
                     for yy in y])


def test_flat_layers_series_capacitor():
    """Flat layered dielectrics (fluid 1 below y = h): the exact potential solves
    (eps V')' = 0, V = V_b + (V_t - V_b) int_0^y 1/eps / int_0^1 1/eps.  The discrete
    initial potential converges to it spectrally; phi stays x-independent and u_x = 0."""
    eta, h = 0.1, 0.4
    errs = []
    for K in (4, 8, 12):
        wl = workloads.small2d(ex=2, ey=8, order=K)
        wl.fluid.eta = eta
        sol = solver_of(wl, init=False)
        Yg = np.repeat(sol.mesh.Y, sol.mesh.nx)
        sol.set_initial(np.tanh((h - Yg) / (math.sqrt(2) * eta))[None, :])
        ex = _layer_potential_exact(sol.prm, eta, h, 1.0, 0.0, sol.mesh.Y)
        errs.append(np.max(np.abs(sol.V[0].reshape(sol.mesh.ny, sol.mesh.nx) - ex[:, None])))
    assert errs[1] < errs[0] / 100 and errs[2] < errs[1] / 100 and errs[2] < 1e-9, errs
    for _ in range(3):
        sol.step()
    assert np.max(np.abs(sol.u[0])) < 1e-12
    phi2 = sol.phi[0].reshape(sol.mesh.ny, sol.mesh.nx)
    assert np.max(np.abs(phi2 - phi2[:, :1])) < 1e-12


def test_phase_mass_identity():
    """Taking the test function 1 in eq. (56)/(57) and alpha (alpha + S/eta^2) =
    -gamma0/(lambda gamma1 dt) gives  gamma0 int phi^{n+1} - int phi_hat =
    -dt int u* . grad phi*  exactly (wall terms cancel), for any contact angle."""
    wl = workloads.small2d(ex=4, ey=2, order=5, theta_s_deg=60.0)
    sol = solver_of(wl)
    m = sol.mesh
    for n in range(4):
        J = 1 if n == 0 else 2
        g0 = 1.0 if J == 1 else 1.5
        ph, pho = sol.phi.copy(), sol.phi_old.copy()
        u, uo = [c.copy() for c in sol.u], [c.copy() for c in sol.u_old]
        phs = ph if J == 1 else 2 * ph - pho
        phh = ph if J == 1 else 2 * ph - 0.5 * pho
        us = [c if J == 1 else 2 * c - co for c, co in zip(u, uo)]
        adv = sum(sol.loc(us[c]) * sol.grad(phs)[c] for c in range(3))
        sol.step()
        lhs = g0 * sol.phi[0] @ m.Mdiag - phh[0] @ m.Mdiag
        rhs = -sol.prm.dt * float(adv[0] @ m.WL)
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(sol.phi[0] @ m.Mdiag))
    assert sol.umax() > 1e-8          # the identity was checked with a moving fluid


def test_mass_conserved_from_rest():
    """First step from rest: u* = u^0 = 0, so int phi is conserved to round-off."""
    wl = workloads.small2d(ex=4, ey=2, order=6, theta_s_deg=60.0)
    sol = solver_of(wl)
    m0 = sol.phase_mass()
    sol.step()
    assert abs(sol.phase_mass() - m0) < 1e-13 * abs(m0)


def test_energy_decays_at_zero_voltage():
    """Eq. (a15) with V = 0 and a drop far from the open side: E(t) is non-increasing."""
    wl = workloads.small2d(ex=6, ey=3, order=6, eta=0.05)
    wl.vbc.v_bottom = 0.0
    wl.phi0 = lambda x, y, z: np.tanh((0.25 - np.sqrt(((x - 1.0) / 1.4) ** 2 + ((y - 0.35) / 0.8) ** 2))
                                      / (math.sqrt(2) * 0.05))
    sol = solver_of(wl, dt=2e-4)
    e = [sol.energy()]
    for _ in range(30):
        sol.step()
        e.append(sol.energy())
    d = np.diff(e)
    assert np.all(d <= 1e-10 * abs(e[0])), d
    assert e[-1] < e[0] - 1e-6 * abs(e[0])


def test_3d_z_independent_reduces_to_2d():
    """Alg. 2 with z-independent data reduces to Alg. 1: only mode 0 is excited and the
    3D fields equal the 2D ones plane by plane (u_z stays 0)."""
    wl2 = workloads.small2d(ex=4, ey=2, order=4)
    s2 = solver_of(wl2)
    wl3 = workloads.small2d(ex=4, ey=2, order=4)
    wl3.mesh.nz, wl3.mesh.lz = 4, 1.0
    s3 = solver_of(wl3)
    for _ in range(3):
        s2.step()
        s3.step()
    for a, b in ((s2.V, s3.V), (s2.phi, s3.phi), (s2.P, s3.P), (s2.u[0], s3.u[0]), (s2.u[1], s3.u[1])):
        np.testing.assert_allclose(b, np.repeat(a, 4, axis=0), atol=1e-11)
    assert np.max(np.abs(s3.u[2])) < 1e-14


def test_equilibrium_system_conserves_mass_and_keeps_u_zero():
    """Sec. 2.4 simpler system: u = 0 throughout, so the phase-mass identity gives exact
    conservation at every step (and the pseudo-time march lowers the free energy)."""
    wl = workloads.small2d(ex=4, ey=2, order=6, theta_s_deg=60.0)
    wl.scheme.equilibrium = True
    sol = solver_of(wl)
    m0 = sol.phase_mass()
    for _ in range(8):
        sol.step()
        assert abs(sol.phase_mass() - m0) < 1e-13 * abs(m0)
    assert sol.umax() == 0.0 and np.all(sol.P == 0.0)


def test_equilibrium_system_matches_full_model_steps_for_phi_and_v():
    """The simpler system's V and phi sub-steps are the full model's with u* = 0: on the
    first step from rest (u^0 = 0) both give the same V^1 and phi^1."""
    wl = workloads.small2d(ex=4, ey=2, order=5)
    full = solver_of(wl)
    wl.scheme.equilibrium = True
    eq = solver_of(wl)
    full.step()
    eq.step()
    np.testing.assert_allclose(eq.phi, full.phi, atol=1e-14)
    np.testing.assert_allclose(eq.V, full.V, atol=1e-14)
