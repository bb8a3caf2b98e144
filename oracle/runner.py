"""Build an oracle ``Solver`` from a synthetic workload (oracle; test infrastructure only)."""
from __future__ import annotations

import numpy as np

from .scheme import Params, Solver, VBC
from .sem import Mesh2D


def params_of(wl, dt=None, bdf=None) -> Params:
    f, s = wl.fluid, wl.scheme
    return Params(rho1=f.rho1, rho2=f.rho2, mu1=f.mu1, mu2=f.mu2, eps1=f.eps1, eps2=f.eps2,
                  sigma=f.sigma, eta=f.eta, gamma1=f.gamma1, theta_s_deg=f.theta_s_deg,
                  dt=s.dt if dt is None else dt, bdf=s.bdf if bdf is None else bdf,
                  S=s.S, nu_m=s.nu_m, rho0=s.rho0, eps0=s.eps0,
                  equilibrium=bool(getattr(s, "equilibrium", False)))


def solver_of(wl, init=True, **kw) -> Solver:
    m = wl.mesh
    mesh = Mesh2D(m.xb, m.yb, m.order)
    v = wl.vbc
    sol = Solver(mesh, params_of(wl, **kw), VBC(v.bottom_kind, v.top_kind, v.v_bottom, v.v_top, tuple(getattr(v, 'patches', ()))),
                 nz=m.nz, lz=m.lz)
    if init:
        Zg, Yg, Xg = np.meshgrid(sol.zc, mesh.Y, mesh.X, indexing="ij")
        phi0 = wl.phi0(Xg, Yg, Zg).reshape(sol.nz, mesh.n2)
        sol.set_initial(phi0)
    return sol
