"""Electrode patches on the wall (eq. 21: V = V_e on the electrodes, dV/dn = 0 on the gaps) in
the oracle, pinned by cases that reduce to whole-side conditions, by the symmetries of an
alternating electrode array, and by a manufactured potential that satisfies the gap condition."""
import math

import numpy as np
import pytest

import workloads
from oracle.runner import solver_of
from oracle.scheme import PATCHES, electrode_of

FIELDS = ("V", "phi", "P")


def _fields(sol):
    return {"V": sol.V, "phi": sol.phi, "P": sol.P, "ux": sol.u[0], "uy": sol.u[1]}


def test_electrode_classification_closed_intervals_and_periodic_image():
    pats = ((0.1, 0.2, -1.0), (1.5, 1.6, 2.0))
    assert electrode_of(0.1, pats, 1.6) == 0 and electrode_of(0.2, pats, 1.6) == 0
    assert electrode_of(0.2 + 1e-6, pats, 1.6) == -1
    assert electrode_of(0.0, pats, 1.6) == 1          # x = 0 is the periodic image of 1.6
    assert electrode_of(0.7, pats, 1.6) == -1


def test_patch_over_the_whole_wall_is_the_dirichlet_wall():
    a = workloads.small2d(ex=4, ey=2, order=5)
    b = workloads.small2d(ex=4, ey=2, order=5)
    b.vbc.bottom_kind = workloads.BC_PATCHES
    b.vbc.patches = ((0.0, 2.0, a.vbc.v_bottom),)
    sa, sb = solver_of(a), solver_of(b)
    for _ in range(3):
        sa.step()
        sb.step()
    fa, fb = _fields(sa), _fields(sb)
    for k in fa:
        assert np.max(np.abs(fa[k] - fb[k])) <= 1e-12 * max(1.0, np.max(np.abs(fa[k]))), k


def test_no_patch_is_the_neumann_wall():
    a = workloads.small2d(ex=4, ey=2, order=5)
    a.vbc.bottom_kind = workloads.BC_NEUMANN
    a.vbc.v_top = 1.0
    b = workloads.small2d(ex=4, ey=2, order=5)
    b.vbc.bottom_kind = workloads.BC_PATCHES
    b.vbc.patches = ()
    b.vbc.v_top = 1.0
    sa, sb = solver_of(a), solver_of(b)
    np.testing.assert_allclose(sa.V, 1.0, atol=1e-12)      # one Dirichlet side, no charge: V = V_top
    for _ in range(2):
        sa.step()
        sb.step()
    fa, fb = _fields(sa), _fields(sb)
    for k in fa:
        assert np.max(np.abs(fa[k] - fb[k])) <= 1e-12 * max(1.0, np.max(np.abs(fa[k]))), k


def test_alternating_electrodes_shift_antisymmetry_and_mirror_symmetry():
    """Uniform permittivity, electrodes [0.05, 0.15] at -V and [0.25, 0.35] at +V on a period of
    0.4 with an open (Neumann) top: V(x + 0.2) = -V(x) and V(0.2 - x) = V(x); V equals the
    electrode voltage on electrode nodes and is not constant along the gaps."""
    wl = workloads.small2d(ex=4, ey=3, order=6)
    wl.mesh.xb = np.linspace(0.0, 0.4, 5)
    wl.vbc.bottom_kind, wl.vbc.top_kind = workloads.BC_PATCHES, workloads.BC_NEUMANN
    wl.vbc.patches = ((0.05, 0.15, -1.3), (0.25, 0.35, 1.3))
    sol = solver_of(wl, init=False)
    sol.set_initial(np.ones((1, sol.mesh.n2)))
    m = sol.mesh
    V = sol.V[0].reshape(m.ny, m.nx)
    X = m.X
    h = 1e-12
    def node(target):   # index of the node at periodic coordinate target
        d = np.abs((X - target + 0.2) % 0.4 - 0.2)
        j = int(np.argmin(d))
        assert d[j] < 1e-12
        return j

    shift = [node(x + 0.2) for x in X]
    mirror = [node(0.2 - x) for x in X]
    assert np.max(np.abs(V[:, shift] + V)) <= 1e-11
    assert np.max(np.abs(V[:, mirror] - V)) <= 1e-11
    wall = V[0]
    for j, x in enumerate(X):
        e = electrode_of(x, wl.vbc.patches, 0.4)
        if e >= 0:
            assert abs(wall[j] - wl.vbc.patches[e][2]) <= h
    gaps = [j for j, x in enumerate(X) if electrode_of(x, wl.vbc.patches, 0.4) < 0]
    assert np.ptp(wall[gaps]) > 0.5


@pytest.mark.parametrize("nz", [1, 4])
def test_manufactured_potential_with_gaps_converges_spectrally(nz):
    """V_m = cos(2 pi x / L) cos(pi y / H) (cos(2 pi z / Lz) in 3D) has dV/dy = 0 on the wall and
    on the top, so with f_V = eps lap V_m, phi = 1 and the electrode nodes held at V_m it is the
    exact solution of the patch problem; the discrete potential converges to it spectrally."""
    L, H, lz = 2.0, 1.0, 1.0
    errs = []
    for K in (4, 6, 8, 10):
        wl = workloads.small2d(ex=4, ey=2, order=K)
        wl.mesh.nz, wl.mesh.lz = nz, lz
        wl.vbc.bottom_kind, wl.vbc.top_kind = workloads.BC_PATCHES, workloads.BC_NEUMANN
        wl.vbc.patches = ((0.2, 0.65, 0.0), (1.1, 1.5, 0.0))
        sol = solver_of(wl, init=False)
        m = sol.mesh
        zc = sol.zc if nz > 1 else np.zeros(1)
        Xg, Yg = np.tile(m.X, m.ny), np.repeat(m.Y, m.nx)
        fz = np.cos(2 * math.pi * zc / lz) if nz > 1 else np.ones(1)
        Vm = np.cos(2 * math.pi * Xg / L) * np.cos(math.pi * Yg / H)
        lap = -((2 * math.pi / L) ** 2 + (math.pi / H) ** 2 + ((2 * math.pi / lz) ** 2 if nz > 1 else 0.0))
        eps = sol.prm.eps(1.0)
        fV = eps * lap * fz[:, None] * Vm[None, :]
        Vbot = fz[:, None] * np.cos(2 * math.pi * m.X / L)[None, :]
        sol.sources = lambda t: {"fV": fV, "V_bot": Vbot}
        sol.set_initial(np.ones((nz, m.n2)))
        errs.append(np.max(np.abs(sol.V - fz[:, None] * Vm[None, :])))
    assert errs[1] < errs[0] / 20 and errs[2] < errs[1] / 20 and errs[3] < 1e-7, errs
