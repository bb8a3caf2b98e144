"""The decoupled semi-implicit time step of Sec. 3 (oracle; test infrastructure only).

One step follows Algorithm 1 (2D, eqs. 54-59) and Algorithm 2 (3D, eqs. 74-78)
in the paper's order  V -> E -> psi -> phi -> P -> u,  with

* BDF-J time derivative and J-th order extrapolation (Sec. 3.1, J = 1 for the
  first step and J = 2 afterwards),
* constant algorithmic parameters eps0 = max(eps), rho0 = min(rho),
  nu_m = max(mu)/min(rho), S from the stability bound of Sec. 3.1,
* the split of the Cahn-Hilliard step into two Helmholtz equations, eq. (44),
  with alpha from the closed form under eq. (44) and Q1, Q2 defined there,
* T from eq. (49), G, Y, K, L from the definitions above eq. (3D_u),
* the Fourier reduction of Sec. 3.2.2 with numpy's real FFT:
  f_hat_k = (1/Nz) sum_j f(z_j) exp(-i beta_k z_j), beta_k = 2 pi k / Lz,
  modes k = 0..Nz/2; the first z-derivative of the Nyquist mode is set to 0.

Every linear system is the assembled sparse matrix of ``sem.Mesh2D`` (plus
beta_k^2 M for mode k) solved by SuperLU with Dirichlet rows eliminated.

Readings of the paper taken here (each also listed in the design notes):
* eq. (28) "div(eps V) = f_V" is read as div(eps grad V) = f_V (eq. 9, eq. 41);
* eq. (69)/(76) "+ int psi omega" is read as "- int psi omega" (eq. 47/57 and
  the derivation from eq. 44b);
* E_z = dV/dz, i.e. i beta_k V_hat_k in mode k (eq. a8); the minus sign in
  eq. (70)/(78) is read as coming from the conjugated test function;
* the boundary integral of (mu/rho) n x omega in the pressure equation runs
  over the whole boundary as in eq. (48)/(58a); on the open side it vanishes
  identically, so eq. (3D_u)/(77a) writing only the open side is read as
  that; the wall contributes;
* grad(mu/rho) is taken by the chain rule on phi^{n+1};
* g1 and g3 enter as in (phia) and (phic) (the forms the weak forms use);
* the initial pressure is P^0 = 0 unless the caller supplies one;
* the initial-potential fixed point ("upon convergence") starts from V^(0) = 0
  and runs to the FP64 stagnation point: it stops when max|V^(k+1) - V^(k)| <=
  1e-15 vmax, or once the update is below 1e-11 vmax and no longer decreases
  (vmax = max(1, max|V_D|)); cap 20000 iterations;
* the stability parameter defaults to S = eta^2 sqrt(4 gamma0 / (lambda
  gamma1 dt)) with gamma0 of the run's BDF order; a discriminant below 1e-10
  in the formula for alpha is set to 0.

Electrode patches (eq. 21, NEXT to the whole-side conditions): with VBC(bottom_kind=PATCHES) the
wall nodes whose x lies on an electrode interval (closed, or its periodic image) are Dirichlet
nodes holding that electrode's voltage, and the other wall nodes are free (the natural condition
dV/dn = 0 of the gaps); the electrodes are uniform in z (stripes along z, as in Sec. 4's set-up),
so in 3D only mode 0 carries the electrode voltages.

With ``Params(equilibrium=True)`` the step is that of the simpler equilibrium system of Sec. 2.4
(eq. 16 with eq. 15c, 15d): the V and phi sub-steps with u = 0; P and u are not computed.

Parity status: pinned by tests/test_oracle_scheme.py (manufactured solutions
of eq. 80/81 converge spectrally in K and at second order in dt; reduction
consistency for phi = 1; series-capacitor potential of flat layers; discrete
phase-mass identity; energy decay at zero voltage; zero velocity for a flat
interface at rest) and tests/test_oracle_patches.py (patches reduce to whole-side conditions;
symmetries of an alternating array; a manufactured potential with dV/dy = 0 on the gaps converges
spectrally).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, Optional

import numpy as np
import scipy.sparse.linalg as spla

from .sem import Mesh2D

DIRICHLET = 0
NEUMANN = 1
PATCHES = 2     # wall only: electrodes (Dirichlet) on x-intervals, natural condition on the gaps


@dataclass
class Params:
    rho1: float
    rho2: float
    mu1: float
    mu2: float
    eps1: float
    eps2: float
    sigma: float
    eta: float
    gamma1: float
    dt: float
    theta_s_deg: float = 90.0
    bdf: int = 2
    S: float = 0.0
    nu_m: float = 0.0
    rho0: float = 0.0
    eps0: float = 0.0
    equilibrium: bool = False   # Sec. 2.4 simpler system: eq. (16) + eq. (15c, d), u = 0

    def __post_init__(self):
        # Sec. 2.1: lambda = 3 sigma eta / (2 sqrt 2)
        self.lam = 3.0 * self.sigma * self.eta / (2.0 * math.sqrt(2.0))
        # Sec. 3.1: constants that make every coefficient matrix time-independent
        if self.eps0 == 0.0:
            self.eps0 = max(self.eps1, self.eps2)
        if self.rho0 == 0.0:
            self.rho0 = min(self.rho1, self.rho2)
        if self.nu_m == 0.0:
            self.nu_m = max(self.mu1, self.mu2) / min(self.rho1, self.rho2)
        if self.S == 0.0:
            g0 = 1.5 if self.bdf == 2 else 1.0
            self.S = self.eta ** 2 * math.sqrt(4.0 * g0 / (self.lam * self.gamma1 * self.dt))
        self.cos_theta = math.cos(math.radians(self.theta_s_deg))

    def gamma0(self, J: int) -> float:
        return 1.0 if J == 1 else 1.5

    def alpha(self, J: int) -> float:
        """alpha of eq. (44): -S/(2 eta^2) (1 + sqrt(1 - 4 gamma0 eta^4 / (lambda gamma1 dt S^2)))."""
        g0 = self.gamma0(J)
        disc = 1.0 - 4.0 * g0 * self.eta ** 4 / (self.lam * self.gamma1 * self.dt * self.S ** 2)
        if disc < 1e-10:
            disc = 0.0
        return -self.S / (2.0 * self.eta ** 2) * (1.0 + math.sqrt(disc))

    # ---- mixture laws, eq. (interpolation); free energy pieces, Sec. 2.1 ----------------
    def rho(self, phi):
        return 0.5 * (self.rho1 + self.rho2) + 0.5 * (self.rho1 - self.rho2) * phi

    def mu(self, phi):
        return 0.5 * (self.mu1 + self.mu2) + 0.5 * (self.mu1 - self.mu2) * phi

    def eps(self, phi):
        return 0.5 * (self.eps1 + self.eps2) + 0.5 * (self.eps1 - self.eps2) * phi * (3.0 - phi ** 2) / 2.0

    def deps(self, phi):
        """eps'(phi) = (eps2 - eps1)/2 * 3 (phi^2 - 1)/2."""
        return 0.5 * (self.eps2 - self.eps1) * 3.0 * (phi ** 2 - 1.0) / 2.0

    def h(self, phi):
        """h(phi) = phi (phi^2 - 1) / eta^2."""
        return phi * (phi ** 2 - 1.0) / self.eta ** 2

    def dTheta(self, phi):
        """Theta'(phi) for Theta = sigma cos(theta_s) phi (phi^2 - 3)/4 + const, eq. (theta_def)."""
        return self.sigma * self.cos_theta * 3.0 * (phi ** 2 - 1.0) / 4.0


@dataclass
class VBC:
    """Potential boundary conditions of eq. (21) and (a25): each side Dirichlet or Neumann as a
    whole, or (wall only) PATCHES: V = V_e on the electrodes, dV/dn = 0 on the gaps between them.
    ``patches`` lists (x0, x1, V_e) per electrode; a wall node is on an electrode when its x lies
    in the closed interval (to 1e-9 of the interval length plus 1e-12; x or its periodic image)."""
    bottom_kind: int = DIRICHLET
    top_kind: int = NEUMANN
    v_bottom: float = 0.0
    v_top: float = 0.0
    patches: tuple = ()


def electrode_of(x, patches, period):
    """Index of the electrode (x0, x1, V) holding wall coordinate x (or its periodic image
    x + period), or -1 on a gap."""
    for e, (x0, x1, _) in enumerate(patches):
        tol = 1e-9 * abs(x1 - x0) + 1e-12
        if x0 - tol <= x <= x1 + tol or x0 - tol <= x + period <= x1 + tol:
            return e
    return -1


def _zeros_like_rows(nz, nx):
    return np.zeros((nz, nx))


class Solver:
    """State and time stepping of the two-phase dielectric scheme.

    Fields are stored at the unique GLL nodes with shape (Nz, n2), n2 = n_y n_x,
    x fastest; Nz = 1 is the 2D algorithm.  Velocity is a list of 3 components
    (the third is identically zero and never solved in 2D).

    ``sources(t)`` may return a dict with any of the manufactured-solution
    terms of Sec. 3.1 evaluated at time t:
      'g' (Nz,n2), 'f' [3 x (Nz,n2)], 'fV' (Nz,n2),
      'g1_top','g1_bot','g2_top','g3_bot' (Nz,nx),
      'f1_top' [3 x (Nz,nx)], 'f2_top' (Nz,nx), 'w_bot' [3 x (Nz,nx)],
      'V_bot','V_top' (Nz,nx) Dirichlet data of the potential.
    Missing terms are zero (constant electrode voltages come from ``vbc``).
    """

    def __init__(self, mesh: Mesh2D, prm: Params, vbc: VBC, nz: int = 1, lz: float = 1.0,
                 sources: Optional[Callable[[float], Dict]] = None):
        if nz != 1 and nz % 2 != 0:
            raise ValueError("Nz must be 1 (2D) or even")
        self.mesh, self.prm, self.vbc = mesh, prm, vbc
        self.nz, self.lz = nz, lz
        self.d3 = nz > 1
        self.sources = sources
        nm = nz // 2 + 1 if self.d3 else 1
        self.nm = nm
        k = np.arange(nm)
        self.beta = 2.0 * math.pi * k / lz if self.d3 else np.zeros(1)
        ib = 1j * self.beta
        if self.d3:
            ib[-1] = 0.0                       # Nyquist: first derivative dropped
        self.ibeta = ib
        self.zc = np.arange(nz) * lz / nz if self.d3 else np.zeros(1)
        self._lu = {}
        n2 = mesh.n2
        self.t = 0.0
        self.nstep = 0
        z = np.zeros((nz, n2))
        self.V, self.V_old = z.copy(), z.copy()
        self.phi, self.phi_old = z.copy(), z.copy()
        self.P, self.P_old = z.copy(), z.copy()
        self.u = [z.copy() for _ in range(3)]
        self.u_old = [z.copy() for _ in range(3)]
        self.E = [z.copy() for _ in range(3)]
        self.psi = z.copy()
        self.v_iters = 0

    # ---- Fourier helpers (Sec. 3.2.2) ------------------------------------------------------
    def fft(self, a):
        if not self.d3:
            return a.astype(np.complex128)
        return np.fft.rfft(a, axis=0, norm="forward")

    def ifft(self, A):
        if not self.d3:
            return np.real(A).copy()
        return np.fft.irfft(A, n=self.nz, axis=0, norm="forward")

    def dz(self, f):
        if not self.d3:
            return np.zeros_like(f)
        return self.ifft(self.ibeta[:, None] * self.fft(f))

    # ---- element-local evaluation --------------------------------------------------------
    def loc(self, f):
        return (self.mesh.Z @ f.T).T

    def gx(self, f):
        return (self.mesh.Gx @ f.T).T

    def gy(self, f):
        return (self.mesh.Gy @ f.T).T

    def grad(self, f):
        """Element-local gradient (d/dx, d/dy at element nodes; d/dz spectral)."""
        return [self.gx(f), self.gy(f), self.loc(self.dz(f))]

    # ---- linear solves ---------------------------------------------------------------------
    def _electrode_columns(self):
        """x-indices of the wall nodes on electrodes, and their voltages (PATCHES only)."""
        m = self.mesh
        period = m.xb[-1] - m.xb[0]
        cols, vals = [], []
        for j, x in enumerate(m.X):
            e = electrode_of(x, self.vbc.patches, period)
            if e >= 0:
                cols.append(j)
                vals.append(self.vbc.patches[e][2])
        return np.array(cols, dtype=int), np.array(vals)

    def _dirichlet_nodes(self, kind):
        m = self.mesh
        if kind == "V":
            nodes = []
            if self.vbc.bottom_kind == DIRICHLET:
                nodes.append(m.bottom_nodes)
            elif self.vbc.bottom_kind == PATCHES:
                nodes.append(m.bottom_nodes[self._electrode_columns()[0]])
            if self.vbc.top_kind == DIRICHLET:
                nodes.append(m.top_nodes)
            return np.concatenate(nodes) if nodes else np.zeros(0, dtype=int)
        if kind == "P":
            return m.top_nodes
        if kind == "u":
            return m.bottom_nodes
        return np.zeros(0, dtype=int)

    def solve(self, kind: str, shift: float, key, rhs: np.ndarray, xD: Optional[np.ndarray] = None,
              scale: float = 1.0):
        """Solve scale*(K + shift M) x = rhs with Dirichlet nodes of ``kind`` set to xD."""
        m = self.mesh
        Dn = self._dirichlet_nodes(kind)
        free = np.setdiff1d(np.arange(m.n2), Dn)
        ck = (kind, key)
        if ck not in self._lu:
            A = scale * m.helmholtz(shift)
            A = A.tocsr()
            self._lu[ck] = (spla.splu(A[free][:, free].tocsc()), A[free][:, Dn].tocsr())
        lu, AFD = self._lu[ck]
        x = np.zeros(m.n2, dtype=np.complex128)
        b = rhs[free].astype(np.complex128)
        if len(Dn) and xD is not None:
            x[Dn] = xD
            b = b - AFD @ xD
        sol = lu.solve(np.ascontiguousarray(b.real)) + 1j * lu.solve(np.ascontiguousarray(b.imag))
        x[free] = sol
        return x

    # ---- sources -------------------------------------------------------------------------
    def _src(self, t):
        s = self.sources(t) if self.sources is not None else {}
        m = self.mesh
        z2 = np.zeros((self.nz, m.n2))
        zr = np.zeros((self.nz, m.nx))
        out = dict(g=s.get("g", z2), fV=s.get("fV", z2),
                   f=s.get("f", [z2, z2, z2]),
                   g1_top=s.get("g1_top", zr), g1_bot=s.get("g1_bot", zr),
                   g2_top=s.get("g2_top", zr), g3_bot=s.get("g3_bot", zr),
                   f1_top=s.get("f1_top", [zr, zr, zr]), f2_top=s.get("f2_top", zr),
                   w_bot=s.get("w_bot", [zr, zr, zr]))
        if self.vbc.bottom_kind == PATCHES:
            cols, vals = self._electrode_columns()
            vb0 = np.zeros((self.nz, m.nx))
            vb0[:, cols] = vals
        else:
            vb0 = np.full((self.nz, m.nx), self.vbc.v_bottom)
        vb = s.get("V_bot", vb0)
        vt = s.get("V_top", np.full((self.nz, m.nx), self.vbc.v_top))
        out["V_bot"], out["V_top"] = vb, vt
        return out

    def _vD(self, s):
        """Per-mode Dirichlet values of V on its Dirichlet nodes (same order as _dirichlet_nodes)."""
        parts = []
        if self.vbc.bottom_kind == DIRICHLET:
            parts.append(self.fft(s["V_bot"]))
        elif self.vbc.bottom_kind == PATCHES:
            parts.append(self.fft(s["V_bot"][:, self._electrode_columns()[0]]))
        if self.vbc.top_kind == DIRICHLET:
            parts.append(self.fft(s["V_top"]))
        if not parts:
            return None
        return np.concatenate(parts, axis=1)

    # ---- setup ---------------------------------------------------------------------------
    def set_initial(self, phi0: np.ndarray, u0=None, P0=None, tol: float = 1e-15, max_iter: int = 20000):
        """phi^0, u^0 (eq. a26/a27), P^0, and V^0 by the fixed point of the Remark in Sec. 3.1."""
        self.phi = np.array(phi0, dtype=np.float64).reshape(self.nz, self.mesh.n2)
        self.phi_old = self.phi.copy()
        if u0 is not None:
            self.u = [np.array(c, dtype=np.float64).reshape(self.nz, -1) for c in u0]
        self.u_old = [c.copy() for c in self.u]
        if P0 is not None:
            self.P = np.array(P0, dtype=np.float64).reshape(self.nz, -1)
        self.P_old = self.P.copy()
        self.V = self.initial_potential(self.phi, tol=tol, max_iter=max_iter)
        self.V_old = self.V.copy()
        self.E = self.project_E(self.V)
        self.t = 0.0
        self.nstep = 0

    def potential_rhs(self, phi_s, V_s, fV):
        """RHS of eq. (54a)/(74a) per mode: -int (eps(phi*) - eps0) grad V* . grad w - int f_V w."""
        m, p = self.mesh, self.prm
        epsL = p.eps(self.loc(phi_s)) - p.eps0
        gV = self.grad(V_s)
        R = [epsL * g for g in gV]
        Rh = [self.fft(r) for r in R]
        fVh = self.fft(fV)
        rhs = np.zeros((self.nm, m.n2), dtype=np.complex128)
        for k in range(self.nm):
            rhs[k] = (-(m.WDx @ Rh[0][k] + m.WDy @ Rh[1][k]) + self.ibeta[k] * (m.ZW @ Rh[2][k])
                      - m.Mdiag * fVh[k])
        return rhs

    def solve_potential(self, rhs, vD):
        out = np.zeros((self.nm, self.mesh.n2), dtype=np.complex128)
        for k in range(self.nm):
            out[k] = self.solve("V", self.beta[k] ** 2, ("V", k), rhs[k],
                                None if vD is None else vD[k], scale=self.prm.eps0)
        return out

    def initial_potential(self, phi0, tol=1e-15, max_iter=20000):
        """Fixed point of the Remark in Sec. 3.1, run to the FP64 stagnation point:
        stop when max|V^(k+1) - V^(k)| <= tol * vmax, or when the update has fallen below
        1e-11 * vmax and no longer decreases (round-off floor), or after max_iter."""
        s = self._src(0.0)
        vD = self._vD(s)
        V = np.zeros((self.nz, self.mesh.n2))
        vmax = 1.0
        if vD is not None:
            vmax = max(1.0, float(np.max(np.abs(np.concatenate([s["V_bot"].ravel(), s["V_top"].ravel()])))))
        prev = math.inf
        for it in range(1, max_iter + 1):
            rhs = self.potential_rhs(phi0, V, s["fV"])
            Vn = self.ifft(self.solve_potential(rhs, vD))
            diff = float(np.max(np.abs(Vn - V)))
            V = Vn
            if diff <= tol * vmax or (diff <= 1e-11 * vmax and diff >= prev):
                break
            prev = diff
        self.v_iters = it
        return V

    def project_E(self, V):
        """E = grad V by the L2 projection of eq. (55)/(78); E_z = dV/dz."""
        m = self.mesh
        Ex = (m.ZW @ self.gx(V).T).T / m.Mdiag
        Ey = (m.ZW @ self.gy(V).T).T / m.Mdiag
        return [Ex, Ey, self.dz(V)]

    # ---- one time step: Algorithm 1 / Algorithm 2 -------------------------------------------
    def step(self):
        m, p = self.mesh, self.prm
        J = 1 if (self.nstep == 0 or p.bdf == 1) else 2
        g0 = p.gamma0(J)
        al = p.alpha(J)
        dt = p.dt
        t1 = self.t + dt
        s = self._src(t1)
        d = 3 if self.d3 else 2
        nm = self.nm

        def star(a, b):
            return a.copy() if J == 1 else 2.0 * a - b

        def hat(a, b):
            return a.copy() if J == 1 else 2.0 * a - 0.5 * b

        phi_s = star(self.phi, self.phi_old)
        phi_h = hat(self.phi, self.phi_old)
        V_s = star(self.V, self.V_old)
        P_s = star(self.P, self.P_old)
        u_s = [star(self.u[c], self.u_old[c]) for c in range(3)]
        u_h = [hat(self.u[c], self.u_old[c]) for c in range(3)]
        bot, top = m.face["bottom"], m.face["top"]

        # ---- V^{n+1}: eq. (54) / (74)
        rhs = self.potential_rhs(phi_s, V_s, s["fV"])
        Vh = self.solve_potential(rhs, self._vD(s))
        V1 = self.ifft(Vh)

        # ---- E^{n+1}: eq. (55) / (78)
        E = self.project_E(V1)
        E2 = E[0] ** 2 + E[1] ** 2 + E[2] ** 2

        # ---- psi^{n+1}: eq. (56) / (75)
        gphs = self.grad(phi_s)
        usL = [self.loc(c) for c in u_s]
        Q1 = (self.loc(s["g"]) - sum(usL[c] * gphs[c] for c in range(3)) + self.loc(phi_h) / dt) \
            / (p.lam * p.gamma1)
        Q2 = p.h(phi_s) - (p.S / p.eta ** 2) * phi_s - p.deps(phi_s) / (2.0 * p.lam) * E2
        phis_bot = phi_s[:, :m.nx]
        U = -s["g3_bot"] - p.dTheta(phis_bot) / p.lam            # n . grad phi on the wall (phic)
        Q1h, Q2h, Uh = self.fft(Q1), self.fft(Q2), self.fft(U)
        g1t, g1b, g2t = self.fft(s["g1_top"]), self.fft(s["g1_bot"]), self.fft(s["g2_top"])
        cpsi = al + p.S / p.eta ** 2
        psih = np.zeros((nm, m.n2), dtype=np.complex128)
        for k in range(nm):
            gQx = m.Gx @ Q2h[k]
            gQy = m.Gy @ Q2h[k]
            r = (self.beta[k] ** 2 * m.Mdiag * Q2h[k] - m.ZW @ Q1h[k]
                 + m.WDx @ gQx + m.WDy @ gQy
                 + top["FM"] @ (top["RZ"] @ (g1t[k] + cpsi * g2t[k]))
                 + bot["FM"] @ (bot["RZ"] @ (g1b[k] + cpsi * Uh[k])))
            psih[k] = self.solve("psi", cpsi + self.beta[k] ** 2, ("psi", J, k), r)

        # ---- phi^{n+1}: eq. (57) / (76)
        phih = np.zeros_like(psih)
        for k in range(nm):
            r = (-m.Mdiag * psih[k] + top["FM"] @ (top["RZ"] @ g2t[k])
                 + bot["FM"] @ (bot["RZ"] @ Uh[k]))
            phih[k] = self.solve("phi", -al + self.beta[k] ** 2, ("phi", J, k), r)
        phi1 = self.ifft(phih)
        psi1 = self.ifft(psih)

        if p.equilibrium:
            # Sec. 2.4: the equilibrium solution has u = 0; eq. (16) is marched in pseudo-time with
            # the same V and phi steps (u* = 0 in Q1), and neither P nor u is computed
            self.V_old, self.V = self.V, V1
            self.phi_old, self.phi = self.phi, phi1
            self.E = E
            self.psi = psi1
            self.t = t1
            self.nstep += 1
            return

        # ---- P^{n+1}: eq. (58) / (77), T from eq. (49)
        phiL = self.loc(phi1)
        rhoL, muL = p.rho(phiL), p.mu(phiL)
        gphi = self.grad(phi1)
        lap_phi = psi1 - al * phi1                                  # eq. (44b)
        Wf = lap_phi - (p.S / p.eta ** 2) * (phi1 - phi_s) - p.h(phi_s) + p.deps(phi_s) / (2.0 * p.lam) * E2
        gW = self.grad(Wf)
        Jt = [0.5 * (p.rho1 - p.rho2) * p.lam * p.gamma1 * gw for gw in gW]
        gu = [self.grad(u_s[c]) for c in range(3)]                 # gu[c][d] = d u_c / d x_d
        uhL = [self.loc(c) for c in u_h]
        gPs = self.grad(P_s)
        fL = [self.loc(c) for c in s["f"]]
        E2L = self.loc(E2)
        lapL = self.loc(lap_phi)
        gmu = [0.5 * (p.mu1 - p.mu2) * g for g in gphi]
        depsL = p.deps(phiL)
        T = []
        for c in range(3):
            visc = sum(gmu[dd] * (gu[c][dd] + gu[dd][c]) for dd in range(3))
            jgu = sum(Jt[dd] * gu[c][dd] for dd in range(3))
            conv = sum(usL[dd] * gu[c][dd] for dd in range(3))
            T.append((fL[c] - p.lam * lapL * gphi[c] - 0.5 * depsL * E2L * gphi[c] + visc - jgu) / rhoL
                     + uhL[c] / dt - conv + (1.0 / p.rho0 - 1.0 / rhoL) * gPs[c])
        om = [gu[2][1] - gu[1][2], gu[0][2] - gu[2][0], gu[1][0] - gu[0][1]]
        mr = muL / rhoL
        dmr_dphi = (0.5 * (p.mu1 - p.mu2) * rhoL - muL * 0.5 * (p.rho1 - p.rho2)) / rhoL ** 2
        gmr = [dmr_dphi * g for g in gphi]
        cross = [gmr[1] * om[2] - gmr[2] * om[1], gmr[2] * om[0] - gmr[0] * om[2],
                 gmr[0] * om[1] - gmr[1] * om[0]]
        G = [T[c] + cross[c] for c in range(3)]
        Gh = [self.fft(g) for g in G]
        # boundary term -rho0 oint (mu/rho) (n x omega) . grad q on bottom (n_y=-1) and top (n_y=+1)
        faceJ = {}
        for name, ny in (("bottom", -1.0), ("top", 1.0)):
            F = m.face[name]
            mrF = (F["FL"] @ mr.T).T
            omxF = (F["FL"] @ om[0].T).T
            omzF = (F["FL"] @ om[2].T).T
            faceJ[name] = (self.fft(mrF * ny * omzF), self.fft(-mrF * ny * omxF))
        wyh = self.fft(s["w_bot"][1])
        f2h = self.fft(s["f2_top"])
        Ph = np.zeros((nm, m.n2), dtype=np.complex128)
        for k in range(nm):
            r = p.rho0 * (m.WDx @ Gh[0][k] + m.WDy @ Gh[1][k]) - self.ibeta[k] * p.rho0 * (m.ZW @ Gh[2][k])
            for name in ("bottom", "top"):
                F = m.face[name]
                Jxh, Jzh = faceJ[name]
                r = r - p.rho0 * (F["FDx"] @ Jxh[k] - self.ibeta[k] * (F["FM"] @ Jzh[k]))
            # -(rho0 gamma0/dt) int_wall n . w q  with n = (0,-1,0)
            r = r + (p.rho0 * g0 / dt) * (bot["FM"] @ (bot["RZ"] @ wyh[k]))
            Ph[k] = self.solve("P", self.beta[k] ** 2, ("P", k), r, xD=f2h[k])
        P1 = self.ifft(Ph)

        # ---- u^{n+1}: eq. (59) / (78)
        gP1 = self.grad(P1)
        Y = [G[c] - gP1[c] / p.rho0 for c in range(3)]
        Kv = [(mr - p.nu_m) * o for o in om]
        Yh = [self.fft(y) for y in Y]
        Kh = [self.fft(kv) for kv in Kv]
        Ft = m.face["top"]
        mrT = (Ft["FL"] @ mr.T).T
        Ltop = [(mrT - p.nu_m) * (Ft["FL"] @ om[2].T).T, None,
                -(mrT - p.nu_m) * (Ft["FL"] @ om[0].T).T]           # (mu/rho - nu_m) n x omega, n = e_y
        Lh = [self.fft(l) if l is not None else None for l in Ltop]
        f1h = [self.fft(c) for c in s["f1_top"]]
        wh = [self.fft(c) for c in s["w_bot"]]
        cu = g0 / (p.nu_m * dt)
        inu = 1.0 / p.nu_m
        u1 = [np.zeros((self.nz, m.n2)) for _ in range(3)]
        for c in range(d):
            uh = np.zeros((nm, m.n2), dtype=np.complex128)
            for k in range(nm):
                ib = self.ibeta[k]
                r = inu * (m.ZW @ Yh[c][k])
                # -(1/nu_m) int K x grad v, grad v = (dv/dx, dv/dy, -i beta v)
                if c == 0:
                    r = r + inu * (m.WDy @ Kh[2][k] + ib * (m.ZW @ Kh[1][k]))
                elif c == 1:
                    r = r - inu * (m.WDx @ Kh[2][k] + ib * (m.ZW @ Kh[0][k]))
                else:
                    r = r - inu * (m.WDy @ Kh[0][k] - m.WDx @ Kh[1][k])
                r = r + Ft["FM"] @ (Ft["RZ"] @ f1h[c][k])
                if Lh[c] is not None:
                    r = r - inu * (Ft["FM"] @ Lh[c][k])
                uh[k] = self.solve("u", cu + self.beta[k] ** 2, ("u", J, k), r, xD=wh[c][k])
            u1[c] = self.ifft(uh)

        # ---- advance the history
        self.V_old, self.V = self.V, V1
        self.phi_old, self.phi = self.phi, phi1
        self.P_old, self.P = self.P, P1
        self.u_old, self.u = self.u, u1
        self.E = E
        self.psi = psi1
        self.t = t1
        self.nstep += 1

    # ---- diagnostics ------------------------------------------------------------------------
    def plane_weight(self):
        return self.lz / self.nz if self.d3 else 1.0

    def phase_mass(self, phi=None):
        phi = self.phi if phi is None else phi
        return float(np.sum(phi @ self.mesh.Mdiag) * self.plane_weight())

    def energy(self):
        """Discrete E(t) of eq. (14) with GLL quadrature (wall-energy constant dropped)."""
        m, p = self.mesh, self.prm
        phiL = self.loc(self.phi)
        g = self.grad(self.phi)
        kin = 0.5 * p.rho(phiL) * sum(self.loc(c) ** 2 for c in self.u)
        free = 0.5 * p.lam * sum(gg ** 2 for gg in g) + p.lam / (4 * p.eta ** 2) * (phiL ** 2 - 1) ** 2
        E2L = self.loc(sum(e ** 2 for e in self.E))
        elec = 0.5 * p.eps(phiL) * E2L
        vol = float(np.sum((kin + free + elec) @ m.WL))
        pb = self.phi[:, :m.nx]
        theta = p.sigma * p.cos_theta * pb * (pb ** 2 - 3.0) / 4.0
        wall = float(np.sum((m.face["bottom"]["RZ"] @ theta.T).T @ m.face["bottom"]["FW"]))
        return (vol + wall) * self.plane_weight()

    def umax(self):
        return float(max(np.max(np.abs(c)) for c in self.u))
