"""CPU checks of the C-ABI library: it loads without a GPU, exports every symbol that
include/pf.h declares, and its host-side set-up (GLL tables, 1D operators, eigenbases)
agrees with the oracle's independently assembled operators."""
import os
import re

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads

from oracle.gll import gll as oracle_gll
from oracle.sem import Mesh2D
from paper_2305_09020_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = native.load()
    syms = declared_symbols()
    assert "pf_create" in syms and "pf_step" in syms and "pf_solve_helmholtz" in syms
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


@pytest.mark.parametrize("K", [2, 4, 7, 10, 15])
def test_gll_matches_oracle(K):
    x, w, D = native.gll(K)
    xo, wo, Do = oracle_gll(K)
    np.testing.assert_allclose(x, xo, atol=1e-15)
    np.testing.assert_allclose(w, wo, rtol=1e-13)
    np.testing.assert_allclose(D, Do, atol=1e-11 * K * K)


def test_bad_arguments_rejected():
    L = native.load()
    with pytest.raises(native.PfError):
        native.gll(0)
    with pytest.raises(native.PfError):
        native.operators_1d([0.0, 1.0, 0.5], 4, False)      # decreasing breakpoints


@pytest.mark.parametrize("graded", [False, True])
def test_tensor_operators_match_oracle_assembly(graded):
    """K2D = Kx (x) My + Mx (x) Ky and M2D = Mx (x) My reproduce the oracle's element-by-
    element assembled matrices (the separability behind the fast-diagonalisation solve)."""
    xb = np.linspace(0.0, 2.0, 4)
    yb = np.linspace(0.0, 1.0, 4)
    if graded:
        yb = 0.5 * (1 - np.cos(np.pi * yb))
    K = 5
    m = Mesh2D(xb, yb, K)
    Kx, Mx = native.operators_1d(xb, K, True)
    Ky, My = native.operators_1d(yb, K, False)
    K2 = np.kron(Ky, np.diag(Mx)) + np.kron(np.diag(My), Kx)   # index (i, j) -> i*nx + j
    np.testing.assert_allclose(K2, m.Kmat.toarray(), atol=1e-11)
    np.testing.assert_allclose(np.kron(My, Mx), m.Mdiag, rtol=1e-14)
    np.testing.assert_allclose(native.nodes_1d(xb, K, True), m.X, atol=1e-15)
    np.testing.assert_allclose(native.nodes_1d(yb, K, False), m.Y, atol=1e-15)


@pytest.mark.parametrize("mask", ["none", "bottom", "top", "both"])
def test_fdm_1d_generalised_eigenbasis(mask):
    Ky, My = native.operators_1d(np.linspace(0, 1, 6), 6, False)
    n = len(My)
    d = np.zeros(n, dtype=np.uint8)
    if mask in ("bottom", "both"):
        d[0] = 1
    if mask in ("top", "both"):
        d[-1] = 1
    S, lam = native.fdm_1d(Ky, My, d)
    nf = n - int(d.sum())
    Sf = S[:, :nf]
    np.testing.assert_allclose(Sf.T @ np.diag(My) @ Sf, np.eye(nf), atol=1e-11)
    free = d == 0
    Kf = Ky[np.ix_(free, free)]
    np.testing.assert_allclose(Kf @ Sf[free], np.diag(My[free]) @ Sf[free] @ np.diag(lam[:nf]),
                               atol=1e-8 * lam.max())
    assert np.all(S[~free] == 0) and np.all(S[:, nf:] == 0)
    assert np.all(np.diff(lam[:nf]) >= -1e-9)


@pytest.mark.parametrize("bc", ["P", "U", "V"])
def test_fast_diagonalisation_equals_direct_solve(bc):
    """With the library's factors, S_y [(S_y^T (M f) S_x) / (L_y + L_x + c)] S_x^T is the
    solution of the oracle's assembled (K + c M) u = M f with homogeneous Dirichlet rows."""
    xb, yb, K, c = np.linspace(0, 2, 4), np.linspace(0, 1, 4), 4, 3.7
    m = Mesh2D(xb, yb, K)
    Kx, Mx = native.operators_1d(xb, K, True)
    Ky, My = native.operators_1d(yb, K, False)
    Sx, Lx = native.fdm_1d(Kx, Mx)
    ny = len(My)
    d = np.zeros(ny, dtype=np.uint8)
    if bc == "P":
        d[-1] = 1
    elif bc == "U":
        d[0] = 1
    else:
        d[0] = d[-1] = 1
    Sy, Ly = native.fdm_1d(Ky, My, d)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((ny, len(Mx)))
    b = np.outer(My, Mx) * f
    t = Sy.T @ b @ Sx / (Ly[:, None] + Lx[None, :] + c)
    u = Sy @ t @ Sx.T
    Dn = np.where(np.repeat(d, len(Mx)) == 1)[0]
    free = np.setdiff1d(np.arange(m.n2), Dn)
    A = m.helmholtz(c).tocsr()
    ref = np.zeros(m.n2)
    ref[free] = spla.spsolve(A[free][:, free].tocsc(), (m.Mdiag * f.ravel())[free])
    np.testing.assert_allclose(u.ravel(), ref, atol=1e-12 * np.abs(ref).max())


def _create(**over):
    """pf_create with one descriptor field changed; the validation happens before any CUDA call."""
    import ctypes
    L = native.load()
    xb = np.linspace(0, 2, 3)
    yb = np.linspace(0, 1, 3)
    m = dict(ex=2, ey=2, order=4, nz=1, lz=1.0)
    m.update({k: v for k, v in over.items() if k in m})
    xbv = np.ascontiguousarray(over.get("xb", xb), dtype=np.float64)
    mesh = native.PfMesh(m["ex"], m["ey"], native._dp(xbv), native._dp(yb), m["order"], m["nz"], m["lz"])
    fl = dict(rho1=1.0, rho2=1.0, mu1=1.0, mu2=1.0, eps1=2.0, eps2=1.0, sigma=1.0, eta=0.1, gamma1=1e-3,
              theta_s_deg=90.0)
    fl.update({k: v for k, v in over.items() if k in fl})
    fluid = native.PfFluid(**fl)
    vb = dict(bottom_kind=0, top_kind=0, v_bottom=1.0, v_top=0.0)
    vb.update({k: v for k, v in over.items() if k in vb})
    pats = over.get("patches")
    if pats is not None:
        arrs = [np.ascontiguousarray([p[c] for p in pats], dtype=np.float64) for c in range(3)]
        null = over.get("null_patch", False)
        vbc = native.PfVbc(**vb, n_patch=over.get("n_patch", len(pats)),
                           **{n: (None if null else native._dp(a)) for n, a in zip(("patch_x0", "patch_x1", "patch_v"), arrs)})
    else:
        vbc = native.PfVbc(**vb)
    sc = dict(dt=1e-3, bdf=2, precision=0, model=0)
    sc.update({k: v for k, v in over.items() if k in sc})
    scheme = native.PfScheme(sc["dt"], sc["bdf"], sc["precision"], 0.0, 0.0, 0.0, 0.0, sc.get("model", 0))
    phi = np.zeros(10000)
    h = ctypes.c_void_p()
    rc = L.pf_create(ctypes.byref(mesh), ctypes.byref(fluid), ctypes.byref(vbc), ctypes.byref(scheme),
                     native._dp(phi) if not over.get("null_phi") else None, None, None, ctypes.byref(h))
    return rc, L.pf_last_error(None).decode(), h.value


@pytest.mark.parametrize("over,needle", [
    (dict(order=1), "order"), (dict(order=16), "order"), (dict(nz=3), "nz"), (dict(nz=2048), "nz"),
    (dict(ex=0), "element"), (dict(xb=np.array([0.0, 1.5, 1.0])), "xb"),
    (dict(bottom_kind=1, top_kind=1), "electrode"), (dict(bottom_kind=7), "bottom_kind"),
    (dict(dt=-1.0), "dt"), (dict(bdf=3), "bdf"), (dict(precision=9), "precision"),
    (dict(eta=0.0), "positive"), (dict(model=5), "model"), (dict(rho2=-1.0), "positive"), (dict(null_phi=True), "null"),
    (dict(bottom_kind=2, patches=[(0.1, 0.2, 1.0)], n_patch=-1), "patch"),
    (dict(bottom_kind=2, patches=[(0.1, 0.2, 1.0)], null_patch=True), "patch"),
    (dict(bottom_kind=2, patches=[(0.3, 0.2, 1.0)]), "x0 <= x1"),
    (dict(bottom_kind=2, patches=[(0.1, float("nan"), 1.0)]), "finite"),
    (dict(top_kind=2), "top_kind"),
    (dict(bottom_kind=2, top_kind=1, patches=[(0.3, 0.3, 1.0)]), "undetermined"),
])
def test_create_rejects_bad_descriptors_without_gpu(over, needle):
    rc, msg, h = _create(**over)
    assert rc == native.PF_EINVAL and h is None
    assert needle in msg, msg


def test_null_handles_are_rejected():
    L = native.load()
    assert L.pf_step(None, 1) == native.PF_EINVAL
    assert L.pf_sync(None) == native.PF_EINVAL
    assert L.pf_diagnostics(None, None) == native.PF_EINVAL
    L.pf_destroy(None)          # no-op


def test_ensembles_reject_electrode_patches_without_gpu():
    """Ensembles take whole-side conditions only; the check happens before any CUDA call."""
    import ctypes
    L = native.load()
    wl = workloads.patches2d(ex=4, ey=2, order=4)
    m = wl.mesh
    xb, yb = np.ascontiguousarray(m.xb), np.ascontiguousarray(m.yb)
    mesh = (native.PfMesh * 1)(native.PfMesh(m.ex if hasattr(m, "ex") else len(xb) - 1, len(yb) - 1,
                                             native._dp(xb), native._dp(yb), m.order, 1, 1.0))
    f = wl.fluid
    fluid = (native.PfFluid * 1)(native.PfFluid(f.rho1, f.rho2, f.mu1, f.mu2, f.eps1, f.eps2, f.sigma, f.eta,
                                                f.gamma1, f.theta_s_deg))
    arrs = [np.ascontiguousarray([p[c] for p in wl.vbc.patches]) for c in range(3)]
    vbc = (native.PfVbc * 1)(native.PfVbc(2, 1, 0.0, 0.0, len(wl.vbc.patches), *(native._dp(a) for a in arrs)))
    scheme = native.PfScheme(1e-4, 2, 0, 0.0, 0.0, 0.0, 0.0, 0)
    phi = np.zeros(len(xb) * len(yb) * m.order * m.order)
    phis = (ctypes.POINTER(ctypes.c_double) * 1)(native._dp(phi))
    h = ctypes.c_void_p()
    rc = L.pf_batch_create(1, mesh, fluid, vbc, ctypes.byref(scheme), phis, None, ctypes.byref(h))
    assert rc == native.PF_EINVAL and h.value is None
    assert "patch" in L.pf_last_error(None).decode()
