"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This module holds only *inputs*: mesh breakpoints, fluid parameters, boundary
voltages, time-step settings and the initial phase-field profiles evaluated at
caller-supplied coordinates.  It contains none of the numerical method (no GLL
tables, no operators, no time stepping), so both the CPU oracle and the CUDA
path can import it without sharing any arithmetic of the method.

Workloads (all quantities in the normalised units of the paper's Table 1,
with rho2 = mu2 = eps2 = 1, sigma = 1 unless stated):

* ``droplet2d``  -- 2D plain method, [0,2]x[0,1], 8x4 elements, order 6,
  droplet phi = tanh((0.25 - r)/(sqrt(2)*0.01)) centred at (1, 0.25),
  permittivity ratio 5, density/viscosity ratios 1, mobility 1e-4,
  V = 1 on the bottom electrode and V = 0 on the top, dt = 1e-4, 100 steps.
* ``droplet3d``  -- 3D hybrid, 16x8 elements of order 8 times Nz = 64
  Fourier planes on z in [0,1); sphere of radius 0.25 at (1, 0.25, 0.5)
  touching the bottom electrode; ratios eps 10, rho 2, mu 5; V = 2 on the
  bottom, 0 on top; eta = 0.01; dt = 5e-5, 1000 steps.
* ``layers3d``   -- 3D hybrid large, 32x16 elements of order 10 times
  Nz = 256; two stacked layers (fluid 1 below y = 0.3) plus a fluid-1 drop of
  radius 0.15 at (1, 0.65, 0.5); eta = 0.005; ratios eps 20, rho 10, mu 10;
  V = 2; dt = 5e-5; 500 steps.
* ``ensemble2d`` -- 256 independent 2D runs drawn with a fixed seed: element
  counts Ex in {4,6,...,24}, Ey = Ex/2, order in {4..10}, V ~ U(0,3),
  permittivity ratio ~ logU(2,20), drop radius ~ U(0.15,0.35) sitting on the
  wall; eta = 0.02, dt = 1e-4.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Fluid:
    rho1: float = 1.0
    rho2: float = 1.0
    mu1: float = 1.0
    mu2: float = 1.0
    eps1: float = 1.0
    eps2: float = 1.0
    sigma: float = 1.0
    eta: float = 0.01
    gamma1: float = 1e-4
    theta_s_deg: float = 90.0


# Boundary-condition kinds for the potential on a side of the domain.  BC_PATCHES (wall only):
# electrodes on parts of the wall (Dirichlet, one voltage per electrode), zero normal derivative on
# the gaps between them; electrodes are x-intervals, uniform in z (stripes along z in 3D).
BC_DIRICHLET = 0
BC_NEUMANN = 1
BC_PATCHES = 2


@dataclasses.dataclass
class VoltageBC:
    bottom_kind: int = BC_DIRICHLET
    top_kind: int = BC_NEUMANN
    v_bottom: float = 0.0
    v_top: float = 0.0
    patches: tuple = ()     # with BC_PATCHES: ((x0, x1, voltage), ...), closed x-intervals


@dataclasses.dataclass
class Mesh:
    xb: np.ndarray          # Ex+1 breakpoints in x (periodic in x)
    yb: np.ndarray          # Ey+1 breakpoints in y
    order: int              # element order K
    nz: int = 1             # Fourier planes in z; 1 means 2D
    lz: float = 1.0         # period in z

    @property
    def ex(self) -> int:
        return len(self.xb) - 1

    @property
    def ey(self) -> int:
        return len(self.yb) - 1


@dataclasses.dataclass
class Scheme:
    dt: float
    bdf: int = 2
    S: float = 0.0          # 0 -> default from the stability bound
    nu_m: float = 0.0       # 0 -> default max(mu)/min(rho)
    rho0: float = 0.0       # 0 -> default min(rho)
    eps0: float = 0.0       # 0 -> default max(eps)
    equilibrium: bool = False   # march the simpler equilibrium system (u = 0) instead


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    fluid: Fluid
    vbc: VoltageBC
    scheme: Scheme
    steps: int
    phi0: Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray]
    seed: int = 0

    def dof(self) -> int:
        """Real values per scalar field: n_x * n_y * Nz."""
        m = self.mesh
        return (m.ex * m.order) * (m.ey * m.order + 1) * m.nz


def _tanh_profile(dist: np.ndarray, eta: float) -> np.ndarray:
    return np.tanh(dist / (math.sqrt(2.0) * eta))


def droplet2d() -> Workload:
    eta = 0.01

    def phi0(x, y, z):
        r = np.sqrt((x - 1.0) ** 2 + (y - 0.25) ** 2)
        return _tanh_profile(0.25 - r, eta)

    return Workload(
        name="droplet2d",
        mesh=Mesh(xb=np.linspace(0.0, 2.0, 9), yb=np.linspace(0.0, 1.0, 5), order=6),
        fluid=Fluid(rho1=1.0, rho2=1.0, mu1=1.0, mu2=1.0, eps1=5.0, eps2=1.0,
                    sigma=1.0, eta=eta, gamma1=1e-4),
        vbc=VoltageBC(BC_DIRICHLET, BC_DIRICHLET, v_bottom=1.0, v_top=0.0),
        scheme=Scheme(dt=1e-4),
        steps=100,
        phi0=phi0,
    )


def droplet3d() -> Workload:
    eta = 0.01

    def phi0(x, y, z):
        r = np.sqrt((x - 1.0) ** 2 + (y - 0.25) ** 2 + (z - 0.5) ** 2)
        return _tanh_profile(0.25 - r, eta)

    return Workload(
        name="droplet3d",
        mesh=Mesh(xb=np.linspace(0.0, 2.0, 17), yb=np.linspace(0.0, 1.0, 9), order=8,
                  nz=64, lz=1.0),
        fluid=Fluid(rho1=2.0, rho2=1.0, mu1=5.0, mu2=1.0, eps1=10.0, eps2=1.0,
                    sigma=1.0, eta=eta, gamma1=1e-4),
        vbc=VoltageBC(BC_DIRICHLET, BC_DIRICHLET, v_bottom=2.0, v_top=0.0),
        scheme=Scheme(dt=5e-5),
        steps=1000,
        phi0=phi0,
    )


def layers3d() -> Workload:
    eta = 0.005

    def phi0(x, y, z):
        layer = _tanh_profile(0.3 - y, eta)
        r = np.sqrt((x - 1.0) ** 2 + (y - 0.65) ** 2 + (z - 0.5) ** 2)
        drop = _tanh_profile(0.15 - r, eta)
        return np.maximum(layer, drop)

    return Workload(
        name="layers3d",
        mesh=Mesh(xb=np.linspace(0.0, 2.0, 33), yb=np.linspace(0.0, 1.0, 17), order=10,
                  nz=256, lz=1.0),
        fluid=Fluid(rho1=10.0, rho2=1.0, mu1=10.0, mu2=1.0, eps1=20.0, eps2=1.0,
                    sigma=1.0, eta=eta, gamma1=1e-4),
        vbc=VoltageBC(BC_DIRICHLET, BC_DIRICHLET, v_bottom=2.0, v_top=0.0),
        scheme=Scheme(dt=5e-5),
        steps=500,
        phi0=phi0,
    )


def small3d(ex: int = 4, ey: int = 2, order: int = 4, nz: int = 8, eta: float = 0.08,
            theta_s_deg: float = 90.0, v_top_kind: int = BC_DIRICHLET) -> Workload:
    """A small 3D droplet case (same physics as ``droplet3d``) for element-by-element parity."""

    def phi0(x, y, z):
        r = np.sqrt((x - 1.0) ** 2 + (y - 0.3) ** 2 + (z - 0.5) ** 2)
        return _tanh_profile(0.35 - r, eta)

    return Workload(
        name=f"small3d_{ex}x{ey}_K{order}_Nz{nz}",
        mesh=Mesh(xb=np.linspace(0.0, 2.0, ex + 1), yb=np.linspace(0.0, 1.0, ey + 1),
                  order=order, nz=nz, lz=1.0),
        fluid=Fluid(rho1=2.0, rho2=1.0, mu1=5.0, mu2=1.0, eps1=10.0, eps2=1.0,
                    sigma=1.0, eta=eta, gamma1=1e-3, theta_s_deg=theta_s_deg),
        vbc=VoltageBC(BC_DIRICHLET, v_top_kind, v_bottom=2.0, v_top=0.0),
        scheme=Scheme(dt=1e-3),
        steps=10,
        phi0=phi0,
    )


def small2d(ex: int = 4, ey: int = 2, order: int = 5, eta: float = 0.08,
            theta_s_deg: float = 90.0, graded: bool = False,
            v_top_kind: int = BC_DIRICHLET) -> Workload:
    """A small 2D droplet case for element-by-element parity (optionally graded in y)."""

    def phi0(x, y, z):
        r = np.sqrt((x - 1.0) ** 2 + (y - 0.3) ** 2)
        return _tanh_profile(0.35 - r, eta)

    yb = np.linspace(0.0, 1.0, ey + 1)
    if graded:
        yb = 0.5 * (1.0 - np.cos(np.pi * yb))
    return Workload(
        name=f"small2d_{ex}x{ey}_K{order}",
        mesh=Mesh(xb=np.linspace(0.0, 2.0, ex + 1), yb=yb, order=order),
        fluid=Fluid(rho1=3.0, rho2=1.0, mu1=2.0, mu2=1.0, eps1=5.0, eps2=1.0,
                    sigma=1.0, eta=eta, gamma1=1e-3, theta_s_deg=theta_s_deg),
        vbc=VoltageBC(BC_DIRICHLET, v_top_kind, v_bottom=1.0, v_top=0.0),
        scheme=Scheme(dt=1e-3),
        steps=10,
        phi0=phi0,
    )


def patches2d(ex: int = 16, ey: int = 4, order: int = 8, nz: int = 1, v0: float = 0.5,
              eta: float = 0.02, top_kind: int = BC_NEUMANN, dt: float = 1e-4) -> Workload:
    """Electrodes on part of the wall (the four-electrode drop of Sec. 4 in normalised units):
    domain [0, 1.6] x [0, 0.5] (x [0, 1) in 3D), electrodes on x in [0.1, 0.2], [0.3, 0.4],
    [0.5, 0.6], [0.7, 0.8] at -v0, +v0, -v0, +v0, zero normal derivative of V on the gaps and on
    the open top; a half-disc (3D: half-ball) drop of radius 0.35 centred on the wall at x = 1.2.
    The default v0 = 0.5 keeps the flow gentle: the tanh profile has not saturated over the
    electrodes (phi ~ -0.95 there), and at v0 = 1.5 the electric stress eps'(phi)/2 |E|^2 grad phi
    at the electrode edges, where |E|^2 is singular, drives max|u| to ~1 within ten steps."""

    def phi0(x, y, z):
        r2 = (x - 1.2) ** 2 + y ** 2
        if nz > 1:
            r2 = r2 + (z - 0.5) ** 2
        return _tanh_profile(0.35 - np.sqrt(r2), eta)

    pats = ((0.1, 0.2, -v0), (0.3, 0.4, v0), (0.5, 0.6, -v0), (0.7, 0.8, v0))
    return Workload(
        name=f"patches_{ex}x{ey}_K{order}_nz{nz}",
        mesh=Mesh(xb=np.linspace(0.0, 1.6, ex + 1), yb=np.linspace(0.0, 0.5, ey + 1), order=order,
                  nz=nz, lz=1.0),
        fluid=Fluid(rho1=2.0, rho2=1.0, mu1=2.0, mu2=1.0, eps1=5.0, eps2=1.0,
                    sigma=1.0, eta=eta, gamma1=1e-3, theta_s_deg=90.0),
        vbc=VoltageBC(BC_PATCHES, top_kind, v_bottom=0.0, v_top=0.0, patches=pats),
        scheme=Scheme(dt=dt),
        steps=10,
        phi0=phi0,
    )


def electrode_array3d(ex: int = 20, ey: int = 6, order: int = 12, nz: int = 120, volts: float = 150.0,
                      eta: float = 0.02, dt: float = 2e-6, grading: float = 1.0) -> Workload:
    """The 3D electrode-array drop of Sec. 4, normalised as the paper's table for the equilibrium
    system (lengths by L0 = 1.2 mm, V by V_d = 150 V, permittivities by L0 gamma / V_d^2 with
    gamma = 3.857e-2 kg/s^2, so eps_air = 4.30e-3 and the liquid's 32 times that): domain
    [0, 5/3] x [0, 2/3] x [0, 7/2], ten electrode stripes along z of width 1/12 spaced 1/12 apart
    (on x in [i/6, i/6 + 1/12], +V0 and -V0 alternating, V0 = volts / 150), dV/dn = 0 on the gaps
    and on the open top; a hemispherical liquid drop (fluid 1) of radius 1/2 centred on the wall at
    (5/6, 0, 7/4); eta = 0.02, lambda gamma1 = 0.1, pseudo-time step 2e-6; the equilibrium system
    of Sec. 2.4 (u = 0).  Mesh: 20 uniform elements in x, 6 in y (grading 1: uniform; g > 1:
    each element g times the one below), order 12, Nz = 120 Fourier planes."""

    def phi0(x, y, z):
        r = np.sqrt((x - 5.0 / 6.0) ** 2 + y ** 2 + (z - 1.75) ** 2)
        return _tanh_profile(0.5 - r, eta)

    lam = 3.0 * 1.0 * eta / (2.0 * np.sqrt(2.0))          # lambda with the normalised gamma = 1
    e_air = 8.854e-12 * 150.0 ** 2 / (1.2e-3 * 3.857e-2)
    h = grading ** np.arange(ey)
    yb = (2.0 / 3.0) * np.concatenate([[0.0], np.cumsum(h) / np.sum(h)])
    v0 = volts / 150.0
    pats = tuple((i / 6.0, i / 6.0 + 1.0 / 12.0, v0 if i % 2 == 0 else -v0) for i in range(10))
    return Workload(
        name=f"electrode_array3d_{ex}x{ey}_K{order}_nz{nz}",
        mesh=Mesh(xb=np.linspace(0.0, 5.0 / 3.0, ex + 1), yb=yb, order=order, nz=nz, lz=3.5),
        fluid=Fluid(rho1=1.0, rho2=1.0, mu1=1.0, mu2=1.0, eps1=32.0 * e_air, eps2=e_air,
                    sigma=1.0, eta=eta, gamma1=0.1 / lam, theta_s_deg=90.0),
        vbc=VoltageBC(BC_PATCHES, BC_NEUMANN, patches=pats),
        scheme=Scheme(dt=dt, equilibrium=True),
        steps=10,
        phi0=phi0,
    )


@dataclasses.dataclass
class EnsembleMember:
    ex: int
    ey: int
    order: int
    v: float
    eps_ratio: float
    radius: float


def ensemble2d(n: int = 256, seed: int = 20230515) -> List[Workload]:
    """Independent 2D runs of uneven size drawn with a fixed seed."""
    rng = np.random.default_rng(seed)
    out = []
    eta = 0.02
    for i in range(n):
        ex = int(rng.choice(np.arange(4, 25, 2)))
        ey = ex // 2
        order = int(rng.integers(4, 11))
        v = float(rng.uniform(0.0, 3.0))
        eps_ratio = float(math.exp(rng.uniform(math.log(2.0), math.log(20.0))))
        radius = float(rng.uniform(0.15, 0.35))

        def phi0(x, y, z, r0=radius):
            r = np.sqrt((x - 1.0) ** 2 + (y - 0.0) ** 2)
            return _tanh_profile(r0 - r, eta)

        out.append(Workload(
            name=f"ensemble2d_{i}",
            mesh=Mesh(xb=np.linspace(0.0, 2.0, ex + 1), yb=np.linspace(0.0, 1.0, ey + 1),
                      order=order),
            fluid=Fluid(rho1=1.0, rho2=1.0, mu1=1.0, mu2=1.0, eps1=eps_ratio, eps2=1.0,
                        sigma=1.0, eta=eta, gamma1=1e-4),
            vbc=VoltageBC(BC_DIRICHLET, BC_DIRICHLET, v_bottom=v, v_top=0.0),
            scheme=Scheme(dt=1e-4),
            steps=200000,
            phi0=phi0,
            seed=seed,
        ))
    return out


def by_name(name: str) -> Workload:
    return {"droplet2d": droplet2d, "droplet3d": droplet3d, "layers3d": layers3d}[name]()


def eval_on_grid(fn: Callable, x: np.ndarray, y: np.ndarray, z: Optional[np.ndarray]) -> np.ndarray:
    """Evaluate ``fn(x, y, z)`` on the tensor grid ``[z][y][x]`` (x fastest).

    ``x``, ``y``, ``z`` are 1D coordinate arrays supplied by the caller (each
    side computes its own node coordinates).  ``z=None`` means a 2D field
    returned with shape ``[1][y][x]``.
    """
    zz = np.zeros(1) if z is None else np.asarray(z, dtype=np.float64)
    Z, Y, X = np.meshgrid(zz, np.asarray(y, dtype=np.float64), np.asarray(x, dtype=np.float64),
                          indexing="ij")
    return np.ascontiguousarray(fn(X, Y, Z), dtype=np.float64)


def warmstart2d(n: int, seed: int, ex: int = 16, ey: int = 8, order: int = 8) -> List[Workload]:
    """Runs for the learned warm start: one fixed mesh (ex x ey elements on [0,2] x [0,1], default
    16x8 of order 8) so that only the voltage V ~ U(0,3), the permittivity ratio ~ logU(2,20) and
    the drop radius ~ U(0.15,0.35) (drop centred on the wall, hence its volume) vary; eta = 0.02,
    dt = 1e-4."""
    rng = np.random.default_rng(seed)
    eta = 0.02
    out = []
    for i in range(n):
        v = float(rng.uniform(0.0, 3.0))
        eps_ratio = float(math.exp(rng.uniform(math.log(2.0), math.log(20.0))))
        radius = float(rng.uniform(0.15, 0.35))

        def phi0(x, y, z, r0=radius):
            r = np.sqrt((x - 1.0) ** 2 + y ** 2)
            return _tanh_profile(r0 - r, eta)

        out.append(Workload(
            name=f"warmstart2d_{seed}_{i}",
            mesh=Mesh(xb=np.linspace(0.0, 2.0, ex + 1), yb=np.linspace(0.0, 1.0, ey + 1), order=order),
            fluid=Fluid(rho1=1.0, rho2=1.0, mu1=1.0, mu2=1.0, eps1=eps_ratio, eps2=1.0,
                        sigma=1.0, eta=eta, gamma1=1e-4),
            vbc=VoltageBC(BC_DIRICHLET, BC_DIRICHLET, v_bottom=v, v_top=0.0),
            scheme=Scheme(dt=1e-4),
            steps=200000,
            phi0=phi0,
            seed=seed,
        ))
    return out


def warmstart_features(wl: Workload) -> np.ndarray:
    """(V, permittivity ratio, drop area) of a warm-start run: the network's three inputs."""
    # the drop is a half disc on the wall: area pi r^2 / 2, recovered from the initial profile's
    # parameters stored in the closure default
    r0 = wl.phi0.__defaults__[0]
    return np.array([wl.vbc.v_bottom, wl.fluid.eps1 / wl.fluid.eps2, 0.5 * math.pi * r0 ** 2])
