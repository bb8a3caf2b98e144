"""Degenerate and extreme cases of the GPU path against the oracle."""
import numpy as np
import pytest

import workloads
from oracle.runner import solver_of
from paper_2305_09020_gb300 import native

from gpu_util import ALL, oracle_fields, rel_errors, run_pair

pytestmark = pytest.mark.gpu


def _check(res, tol=1e-11):
    for step, errs in res:
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, f"step {step}: {bad}"


@pytest.mark.parametrize("phival", [1.0, -1.0])
@pytest.mark.parametrize("nz", [1, 4])
def test_reduction_consistency_on_gpu(phival, nz):
    """Sec. 2.2: with one fluid only, phi stays exactly +-1, u stays 0, V is the linear profile."""
    wl = workloads.small2d(ex=4, ey=3, order=5, theta_s_deg=60.0) if nz == 1 else \
        workloads.small3d(ex=4, ey=3, order=5, nz=nz, theta_s_deg=60.0)
    wl.phi0 = lambda x, y, z: np.full_like(x, phival)
    h = native.from_workload(wl, precision=native.PF_FP64)
    h.step(4)
    f = h.get(ALL)
    _, y, _ = h.geometry()
    h.close()
    np.testing.assert_allclose(f["phi"], phival, atol=1e-12)
    for k in ("ux", "uy", "uz"):
        assert np.max(np.abs(f[k])) < 1e-12
    vb = wl.vbc.v_bottom
    np.testing.assert_allclose(f["V"], (vb * (1.0 - y))[None, :, None] * np.ones_like(f["V"]), atol=1e-12)


@pytest.mark.parametrize("ex,ey,K", [(1, 1, 2), (1, 2, 3), (2, 1, 15), (3, 2, 12)])
def test_small_and_high_order_meshes(ex, ey, K):
    wl = workloads.small2d(ex=ex, ey=ey, order=K, eta=0.15)
    _check(run_pair(wl, 3, check_every=1))


def test_smallest_3d():
    wl = workloads.small3d(ex=2, ey=2, order=4, nz=2, eta=0.15)
    _check(run_pair(wl, 3, check_every=1))


def test_3d_with_z_independent_data_equals_2d():
    """Algorithm 2 on z-independent data reduces to Algorithm 1 plane by plane (GPU vs GPU)."""
    w2 = workloads.small2d(ex=4, ey=2, order=5)
    w3 = workloads.small2d(ex=4, ey=2, order=5)
    w3.mesh.nz, w3.mesh.lz = 8, 1.0
    a = native.from_workload(w2, precision=native.PF_FP64)
    b = native.from_workload(w3, precision=native.PF_FP64)
    a.step(5)
    b.step(5)
    fa, fb = a.get(ALL), b.get(ALL)
    a.close()
    b.close()
    for k in ("V", "phi", "P", "ux", "uy", "Ex", "Ey"):
        np.testing.assert_allclose(fb[k], np.repeat(fa[k], 8, axis=0), atol=1e-11 * max(1.0, np.abs(fa[k]).max()))
    assert np.max(np.abs(fb["uz"])) < 1e-14 and np.max(np.abs(fb["Ez"])) < 1e-12
