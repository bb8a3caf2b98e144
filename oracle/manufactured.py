"""Manufactured solutions of Sec. 4.1 (oracle; test infrastructure only).

eq. (80) (2D, [0,2]x[0,1], wall at y = 0, open side at y = 1):
    u = cos(pi y) sin(pi x) sin t,  v = -sin(pi y) cos(pi x) sin t,
    P = sin(pi y) cos(pi x) cos t,  phi = cos(pi x) cos(pi y) sin t,
    V = sin(pi x) cos(pi y).
eq. (81) (3D, [0,2]x[-1,1]x[0,2], wall at y = -1, open side at y = 1):
    u = cos(pi x) cos(pi y) cos(pi z) sin t, v = 0,
    w = sin(pi x) cos(pi y) sin(pi z) sin t,
    P = sin(pi x) sin(pi y) sin(pi z) cos t,
    phi = cos(pi x) cos(pi y) cos(pi z) sin t, V = sin(pi x) cos(pi y) cos(pi z).

The source terms are derived symbolically (sympy) so that the fields satisfy
eqs. (a27), (a28), (28) [read as div(eps grad V) = f_V] with E = grad V, and
the boundary conditions (29)-(33) in the forms the scheme uses, (phia) for g1
and (phic) for g3:
    g   = phi_t + u.grad phi - gamma1 lap(lambda h - lambda lap phi - eps'/2 |E|^2)
    f   = rho (u_t + u.grad u) + Jt.grad u + lambda lap(phi) grad phi
          + eps'/2 |E|^2 grad phi - mu lap u - grad(mu).D(u) + grad P,
          Jt = -gamma1 (rho1 - rho2)/2 grad(lambda h - lambda lap phi - eps'/2 |E|^2)
    f_V = div(eps(phi) grad V)
    g1  = n.grad(lap phi - h + eps' |E|^2 / (2 lambda))   on the open side and the wall
    g2  = n.grad phi                                      on the open side
    g3  = -n.grad phi - Theta'(phi)/lambda                on the wall
    f1  = du/dn on the open side, f2 = P there, w = u on the wall.
The potential is Dirichlet (its exact value) on the whole wall in both cases
(the 3D test of the paper splits the wall into Dirichlet and Neumann halves;
the whole-side variant is used here) and homogeneous Neumann on the open side,
which eq. (80) and eq. (81) satisfy exactly.
"""
from __future__ import annotations

import numpy as np
import sympy as sp

X, Y, Zs, T = sp.symbols("x y z t", real=True)


def _fields(case: str):
    pi, s, c = sp.pi, sp.sin, sp.cos
    if case == "2d":
        u = [c(pi * Y) * s(pi * X) * s(T), -s(pi * Y) * c(pi * X) * s(T), sp.Integer(0)]
        P = s(pi * Y) * c(pi * X) * c(T)
        phi = c(pi * X) * c(pi * Y) * s(T)
        V = s(pi * X) * c(pi * Y)
    elif case == "3d":
        u = [c(pi * X) * c(pi * Y) * c(pi * Zs) * s(T), sp.Integer(0),
             s(pi * X) * c(pi * Y) * s(pi * Zs) * s(T)]
        P = s(pi * X) * s(pi * Y) * s(pi * Zs) * c(T)
        phi = c(pi * X) * c(pi * Y) * c(pi * Zs) * s(T)
        V = s(pi * X) * c(pi * Y) * c(pi * Zs)
    else:
        raise ValueError(case)
    return u, P, phi, V


def build(case: str, prm):
    """Return (exact, sources) callables for the oracle Solver.

    ``exact(t, x, y, z)`` returns dict(u=[3], P, phi, V) arrays;
    ``sources_for(solver)`` returns the ``sources(t)`` callable that evaluates
    every term at the solver's nodes.
    """
    u, P, phi, V = _fields(case)
    co = [X, Y, Zs]

    def grad(f):
        return [sp.diff(f, v) for v in co]

    def lap(f):
        return sum(sp.diff(f, v, 2) for v in co)

    rho1, rho2, mu1, mu2 = prm.rho1, prm.rho2, prm.mu1, prm.mu2
    eps1, eps2, lam, eta, g1c = prm.eps1, prm.eps2, prm.lam, prm.eta, prm.gamma1
    rho = (rho1 + rho2) / 2 + (rho1 - rho2) / 2 * phi
    mu = (mu1 + mu2) / 2 + (mu1 - mu2) / 2 * phi
    eps = (eps1 + eps2) / 2 + (eps1 - eps2) / 2 * phi * (3 - phi ** 2) / 2
    deps = (eps2 - eps1) / 2 * 3 * (phi ** 2 - 1) / 2
    h = phi * (phi ** 2 - 1) / eta ** 2
    E = grad(V)
    E2 = sum(e ** 2 for e in E)
    muc = lam * h - lam * lap(phi) - deps / 2 * E2
    g = sp.diff(phi, T) + sum(u[i] * sp.diff(phi, co[i]) for i in range(3)) - g1c * lap(muc)
    Jt = [-g1c * (rho1 - rho2) / 2 * gm for gm in grad(muc)]
    gphi = grad(phi)
    gmu = grad(mu)
    f = []
    for c in range(3):
        du = grad(u[c])
        conv = sum(u[d] * du[d] for d in range(3))
        jt = sum(Jt[d] * du[d] for d in range(3))
        visc = sum(gmu[d] * (sp.diff(u[c], co[d]) + sp.diff(u[d], co[c])) for d in range(3))
        f.append(rho * (sp.diff(u[c], T) + conv) + jt + lam * lap(phi) * gphi[c]
                 + deps / 2 * E2 * gphi[c] - mu * lap(u[c]) - visc + sp.diff(P, co[c]))
    fV = sum(sp.diff(eps * E[i], co[i]) for i in range(3))
    chem = lap(phi) - h + deps * E2 / (2 * lam)
    dTheta = prm.sigma * prm.cos_theta * 3 * (phi ** 2 - 1) / 4
    # outward normals: open side n = +e_y, wall n = -e_y
    g1_top = sp.diff(chem, Y)
    g1_bot = -sp.diff(chem, Y)
    g2_top = sp.diff(phi, Y)
    g3_bot = -(-sp.diff(phi, Y)) - dTheta / lam
    f1_top = [sp.diff(uc, Y) for uc in u]

    args = (T, X, Y, Zs)

    def lf(e):
        fn = sp.lambdify(args, e, "numpy")
        return lambda t, x, y, z: np.broadcast_to(np.asarray(fn(t, x, y, z), dtype=np.float64),
                                                  np.broadcast(x, y, z).shape).copy()

    ex_fn = dict(u=[lf(c) for c in u], P=lf(P), phi=lf(phi), V=lf(V))
    src_fn = dict(g=lf(g), f=[lf(c) for c in f], fV=lf(fV), g1_top=lf(g1_top), g1_bot=lf(g1_bot),
                  g2_top=lf(g2_top), g3_bot=lf(g3_bot), f1_top=[lf(c) for c in f1_top],
                  f2_top=lf(P), w_bot=[lf(c) for c in u], V_bot=lf(V))

    def exact(t, x, y, z):
        return dict(u=[fn(t, x, y, z) for fn in ex_fn["u"]], P=ex_fn["P"](t, x, y, z),
                    phi=ex_fn["phi"](t, x, y, z), V=ex_fn["V"](t, x, y, z))

    def sources_for(solver):
        m = solver.mesh
        zc = solver.zc
        Zg, Yg, Xg = np.meshgrid(zc, m.Y, m.X, indexing="ij")
        shp = (solver.nz, m.n2)
        Zb, Xb = np.meshgrid(zc, m.X, indexing="ij")
        yb0 = np.full_like(Xb, m.Y[0])
        yb1 = np.full_like(Xb, m.Y[-1])

        def vol(fn, t):
            return fn(t, Xg, Yg, Zg).reshape(shp)

        def row(fn, t, yy):
            return fn(t, Xb, yy, Zb)

        def sources(t):
            return dict(
                g=vol(src_fn["g"], t), f=[vol(fn, t) for fn in src_fn["f"]], fV=vol(src_fn["fV"], t),
                g1_top=row(src_fn["g1_top"], t, yb1), g1_bot=row(src_fn["g1_bot"], t, yb0),
                g2_top=row(src_fn["g2_top"], t, yb1), g3_bot=row(src_fn["g3_bot"], t, yb0),
                f1_top=[row(fn, t, yb1) for fn in src_fn["f1_top"]],
                f2_top=row(src_fn["f2_top"], t, yb1),
                w_bot=[row(fn, t, yb0) for fn in src_fn["w_bot"]],
                V_bot=row(src_fn["V_bot"], t, yb0))
        return sources

    return exact, sources_for


def nodal_exact(solver, exact, t):
    m = solver.mesh
    Zg, Yg, Xg = np.meshgrid(solver.zc, m.Y, m.X, indexing="ij")
    ex = exact(t, Xg, Yg, Zg)
    shp = (solver.nz, m.n2)
    return dict(u=[c.reshape(shp) for c in ex["u"]], P=ex["P"].reshape(shp),
                phi=ex["phi"].reshape(shp), V=ex["V"].reshape(shp))
