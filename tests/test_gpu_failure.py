"""Failure detection and restart through the C-ABI (no GPU fault is provoked):
* a non-finite value written into the state is reported by pf_sync as PF_EDIVERGED;
* a bounded device wait of the tensor-core transforms that runs out (a test hook makes one wait
  on a barrier that nothing arrives at) is reported as PF_ETIMEOUT, and the handle stays usable;
* a run restarted from both history levels plus its step count and time continues exactly."""
import numpy as np
import pytest

import workloads
from gpu_util import ALL
from paper_2305_09020_gb300 import native

pytestmark = pytest.mark.gpu

STATE = native.PF_FIELD_V | native.PF_FIELD_PHI | native.PF_FIELD_P | native.PF_FIELD_U


@pytest.mark.parametrize("precision", [native.PF_FP64, native.PF_MIXED])
def test_nan_in_state_is_reported_as_diverged(precision):
    wl = workloads.small3d(ex=4, ey=2, order=4, nz=8)
    h = native.from_workload(wl, precision=precision)
    h.step(2)
    h.sync()
    phi = h.get(native.PF_FIELD_PHI)["phi"].copy()
    phi[3, 4, 5] = np.nan
    h.set(native.PF_FIELD_PHI, phi)
    with pytest.raises(native.PfError) as ei:
        h.sync()
    assert ei.value.code == native.PF_EDIVERGED
    assert h.diagnostics()[5] == 1.0
    h.close()


def test_tensor_core_timeout_is_reported_and_handle_stays_usable():
    wl = workloads.small3d(ex=4, ey=2, order=4, nz=8)
    h = native.from_workload(wl, precision=native.PF_MIXED)
    n2 = 16 * 9
    f = np.random.default_rng(3).standard_normal(n2)
    good = h.solve_helmholtz(native.PF_BCSET_NN, 0, 1.5, f)
    h.debug_tc_stall(20_000_000)                       # 20 ms
    with pytest.raises(native.PfError) as ei:
        h.solve_helmholtz(native.PF_BCSET_NN, 0, 1.5, f)
    assert ei.value.code == native.PF_ETIMEOUT
    again = h.solve_helmholtz(native.PF_BCSET_NN, 0, 1.5, f)   # the context is intact
    assert np.array_equal(again, good)
    h.step(2)
    h.debug_tc_stall(20_000_000)
    h.step(1)
    with pytest.raises(native.PfError) as ei:
        h.sync()
    assert ei.value.code == native.PF_ETIMEOUT
    h.sync()                                           # reported once, then cleared
    h.close()


def _restart(wl, precision, n1, n2):
    a = native.from_workload(wl, precision=precision)
    a.step(n1 + n2)
    ref = a.get(ALL)
    a.close()
    b = native.from_workload(wl, precision=precision)
    b.step(n1)
    d = b.diagnostics()
    cur = b.get(STATE)
    old = b.get(STATE | native.PF_FIELD_OLD)
    b.close()
    c = native.from_workload(wl, precision=precision)
    pack = lambda f: np.concatenate([f[k].ravel() for k in ("V", "phi", "P", "ux", "uy", "uz")])
    c.set(STATE | native.PF_FIELD_OLD, pack(old))
    c.set(STATE, pack(cur))
    c.set_step(int(d[3]), float(d[2]))
    c.step(n2)
    out = c.get(ALL)
    assert c.diagnostics()[3] == n1 + n2
    c.close()
    return ref, out


@pytest.mark.parametrize("precision", [native.PF_FP64, native.PF_MIXED])
def test_restart_2d_is_bit_exact(precision):
    """2 x 50 steps through pf_get_fields / pf_set_fields of both levels = 100 steps."""
    ref, out = _restart(workloads.small2d(ex=4, ey=2, order=5, theta_s_deg=60.0), precision, 50, 50)
    for k in ref:
        assert np.array_equal(ref[k], out[k]), k


def test_restart_3d_continues_the_run():
    """3D: the z-derivatives are recomputed from the restored fields by the transforms, so the
    continuation agrees to round-off rather than bit for bit."""
    ref, out = _restart(workloads.small3d(ex=4, ey=2, order=4, nz=8, theta_s_deg=70.0), native.PF_FP64, 20, 20)
    for k in ref:
        nrm = np.linalg.norm(ref[k])
        assert np.linalg.norm(out[k] - ref[k]) <= 1e-12 * max(nrm, 1e-30) + 1e-300, k
