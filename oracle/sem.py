"""Tensor-product C0 spectral-element mesh and assembled sparse operators
(oracle; test infrastructure only).

Follows Sec. 3.2.1: the 2D domain (the xy plane in 3D) is partitioned into
Ex x Ey quadrilateral elements; every element carries the (K+1)^2 GLL nodes of
order K; x is periodic (Sec. 2.4: periodic in the horizontal directions), so
the unique nodes form an n_y x n_x grid with n_x = Ex K and n_y = Ey K + 1.

Every operator is built from its quadrature definition, element by element:

* ``Z``   (nL x n2)  gather of global nodal values into element-local slots,
* ``Gx``, ``Gy`` (nL x n2)  element-local derivatives d/dx, d/dy at the
  element's own GLL nodes (discontinuous across element edges),
* ``WL``  (nL)  quadrature weight x Jacobian of every element-local slot,
* ``M = Z^T WL Z`` (diagonal GLL mass), ``K = Gx^T WL Gx + Gy^T WL Gy``,
* ``ZW = Z^T diag(WL)``:     integral of an element-local field f times omega_i,
* ``WDx = Gx^T diag(WL)``:   integral of f * d omega_i / dx  (same for y),
* face operators on the bottom (wall) and top (open) sides:
  ``FZ`` gathers nodal values on the side into face slots, ``FL`` picks the
  face slots out of an element-local array, ``FM = FZ^T diag(FW)`` integrates
  f * omega_i along the side and ``FDx = FGx^T diag(FW)`` integrates
  f * d omega_i / dx along the side.

Pinned by tests/test_oracle_sem.py (exact integration of polynomials,
K annihilates constants, symmetric positive semi-definite K, M sums to the
area, face operators integrate known functions).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .gll import gll


class Mesh2D:
    def __init__(self, xb, yb, K: int):
        self.xb = np.asarray(xb, dtype=np.float64)
        self.yb = np.asarray(yb, dtype=np.float64)
        self.K = int(K)
        self.Ex = len(self.xb) - 1
        self.Ey = len(self.yb) - 1
        if self.Ex < 1 or self.Ey < 1:
            raise ValueError("need at least one element per direction")
        self.hx = np.diff(self.xb)
        self.hy = np.diff(self.yb)
        self.nx = self.Ex * self.K
        self.ny = self.Ey * self.K + 1
        self.n2 = self.nx * self.ny
        self.p = self.K + 1
        self.nL = self.Ex * self.Ey * self.p * self.p
        self.xi, self.w, self.D = gll(self.K)
        self._coords()
        self._build()

    # ---- numbering -----------------------------------------------------------------------
    def gid(self, ex, ey, a, b):
        """Global node of local GLL node (a in x, b in y) of element (ex, ey)."""
        return (ey * self.K + b) * self.nx + (ex * self.K + a) % self.nx

    def lid(self, ex, ey, a, b):
        """Slot of (a, b) of element (ex, ey) in an element-local array."""
        return ((ey * self.Ex + ex) * self.p + b) * self.p + a

    def _coords(self):
        K = self.K
        X = np.zeros(self.nx)
        for ex in range(self.Ex):
            for a in range(K):
                X[ex * K + a] = self.xb[ex] + 0.5 * (self.xi[a] + 1.0) * self.hx[ex]
        Y = np.zeros(self.ny)
        for ey in range(self.Ey):
            for b in range(K + 1):
                Y[ey * K + b] = self.yb[ey] + 0.5 * (self.xi[b] + 1.0) * self.hy[ey]
        self.X, self.Y = X, Y
        # coordinates of element-local slots (x is the unwrapped element coordinate)
        xl = np.zeros(self.nL)
        yl = np.zeros(self.nL)
        for ey in range(self.Ey):
            for ex in range(self.Ex):
                for b in range(self.p):
                    for a in range(self.p):
                        l = self.lid(ex, ey, a, b)
                        xl[l] = self.xb[ex] + 0.5 * (self.xi[a] + 1.0) * self.hx[ex]
                        yl[l] = self.yb[ey] + 0.5 * (self.xi[b] + 1.0) * self.hy[ey]
        self.XL, self.YL = xl, yl

    # ---- operators -----------------------------------------------------------------------
    def _build(self):
        p, D, w = self.p, self.D, self.w
        zr, zc = [], []
        gxr, gxc, gxv = [], [], []
        gyr, gyc, gyv = [], [], []
        WL = np.zeros(self.nL)
        for ey in range(self.Ey):
            for ex in range(self.Ex):
                jx = 0.5 * self.hx[ex]
                jy = 0.5 * self.hy[ey]
                for b in range(p):
                    for a in range(p):
                        l = self.lid(ex, ey, a, b)
                        zr.append(l)
                        zc.append(self.gid(ex, ey, a, b))
                        WL[l] = jx * jy * w[a] * w[b]
                        for m in range(p):
                            gxr.append(l)
                            gxc.append(self.gid(ex, ey, m, b))
                            gxv.append(D[a, m] / jx)
                            gyr.append(l)
                            gyc.append(self.gid(ex, ey, a, m))
                            gyv.append(D[b, m] / jy)
        shp = (self.nL, self.n2)
        self.Z = sp.csr_matrix((np.ones(len(zr)), (zr, zc)), shape=shp)
        self.Gx = sp.csr_matrix((gxv, (gxr, gxc)), shape=shp)   # duplicates are summed
        self.Gy = sp.csr_matrix((gyv, (gyr, gyc)), shape=shp)
        self.WL = WL
        Wd = sp.diags(WL)
        self.ZW = (self.Z.T @ Wd).tocsr()
        self.WDx = (self.Gx.T @ Wd).tocsr()
        self.WDy = (self.Gy.T @ Wd).tocsr()
        self.Mdiag = np.asarray(self.ZW @ np.ones(self.nL)).ravel()
        self.M = sp.diags(self.Mdiag).tocsr()
        self.Kmat = (self.WDx @ self.Gx + self.WDy @ self.Gy).tocsr()
        self.face = {"bottom": self._face(0, 0), "top": self._face(self.Ey - 1, self.K)}
        self.bottom_nodes = np.arange(self.nx)
        self.top_nodes = (self.ny - 1) * self.nx + np.arange(self.nx)

    def _face(self, ey, b):
        """Operators for the side y = const made of local row b of element row ey."""
        p, D, w = self.p, self.D, self.w
        nF = self.Ex * p
        fz_r, fz_c, fgx_r, fgx_c, fgx_v, fl_r, fl_c = [], [], [], [], [], [], []
        FW = np.zeros(nF)
        for ex in range(self.Ex):
            jx = 0.5 * self.hx[ex]
            for a in range(p):
                f = ex * p + a
                FW[f] = jx * w[a]
                fz_r.append(f)
                fz_c.append(self.gid(ex, ey, a, b))
                fl_r.append(f)
                fl_c.append(self.lid(ex, ey, a, b))
                for m in range(p):
                    fgx_r.append(f)
                    fgx_c.append(self.gid(ex, ey, m, b))
                    fgx_v.append(D[a, m] / jx)
        FZ = sp.csr_matrix((np.ones(nF), (fz_r, fz_c)), shape=(nF, self.n2))
        FGx = sp.csr_matrix((fgx_v, (fgx_r, fgx_c)), shape=(nF, self.n2))
        FL = sp.csr_matrix((np.ones(nF), (fl_r, fl_c)), shape=(nF, self.nL))
        Fd = sp.diags(FW)
        # face rows of the global grid, so nodal row data (length nx) maps to face slots
        RZ = sp.csr_matrix((np.ones(nF), (np.arange(nF),
                                          [(ex * self.K + a) % self.nx
                                           for ex in range(self.Ex) for a in range(p)])),
                           shape=(nF, self.nx))
        return dict(FZ=FZ, FL=FL, FW=FW, RZ=RZ,
                    FM=(FZ.T @ Fd).tocsr(), FDx=(FGx.T @ Fd).tocsr(), FGx=FGx)

    def helmholtz(self, shift: float) -> sp.csr_matrix:
        """Assembled K + shift * M."""
        return (self.Kmat + shift * self.M).tocsr()
