"""The allocation-free solve pf_fdm_solve_static against the handle's pf_solve_helmholtz.

It is for callers that cannot allocate device memory where they need a solve; its
scratch lives in a static device array.  This file is collected last on purpose: it
must pass both alone in a fresh process and after every other test."""
import numpy as np
import pytest

import workloads
from paper_2305_09020_gb300 import native

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 Helmholtz parity tolerance of the other GPU tests


def _factors(wl, dirichlet_bottom, dirichlet_top):
    m = wl.mesh
    Kx, Mx = native.operators_1d(m.xb, m.order, True)
    Ky, My = native.operators_1d(m.yb, m.order, False)
    Sx, Lx = native.fdm_1d(Kx, Mx)
    d = np.zeros(len(My), dtype=np.uint8)
    d[0], d[-1] = int(dirichlet_bottom), int(dirichlet_top)
    Sy, Ly = native.fdm_1d(Ky, My, d)
    Lx[np.abs(Lx) < 1e-11] = 0.0
    Ly[np.abs(Ly) < 1e-11] = 0.0
    return Sx, Lx, Sy, Ly, Mx, My


def test_static_solve_matches_handle_twice():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    wl = workloads.small3d(ex=4, ey=3, order=5, nz=8)
    h = native.from_workload(wl, precision=native.PF_FP64)
    Sx, Lx, Sy, Ly, Mx, My = _factors(wl, dirichlet_bottom=False, dirichlet_top=True)   # pressure set
    nx, ny = len(Mx), len(My)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    dSx, dSxT, dLx, dSy, dSyT, dLy = t(Sx), t(Sx.T), t(Lx), t(Sy), t(Sy.T), t(Ly)
    lam, mode = 1.75, 3
    beta = 2 * np.pi * mode / wl.mesh.lz
    shift = t(np.full(2, lam + beta ** 2))
    out = torch.empty(2 * ny * nx, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(11)
    for call in range(2):                       # two calls in a row share the static scratch
        f = rng.standard_normal((2, ny, nx))
        ref = h.solve_helmholtz(native.PF_BCSET_P, mode, lam, f).reshape(2, ny, nx)
        rhs = t(np.outer(My, Mx)[None, :, :] * f)      # weak-form (mass-weighted) right-hand side
        native.fdm_solve_static(nx, ny, 2, dSx.data_ptr(), dSxT.data_ptr(), dLx.data_ptr(), dSy.data_ptr(),
                                dSyT.data_ptr(), dLy.data_ptr(), shift.data_ptr(), rhs.data_ptr(),
                                out.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy().reshape(2, ny, nx)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL, f"call {call}: relative error {err:.3e}"
    h.close()


def test_static_solve_rejects_oversize():
    big = native.PF_STATIC_MAX_VALUES + 1
    with pytest.raises(native.PfError) as ei:
        native.fdm_solve_static(big, 1, 1, *([1] * 9))
    assert ei.value.code == native.PF_EINVAL
