"""The discrete energy E(t) of eq. (14) computed on the GPU (pf_diagnostics out[7], FP64
reduction) against the oracle's Solver.energy (pinned term by term in test_oracle_energy.py),
with a voltage, a contact angle other than 90 degrees and a moving fluid."""
import numpy as np
import pytest

import workloads
from oracle.runner import solver_of
from paper_2305_09020_gb300 import native

pytestmark = pytest.mark.gpu


def _energies(wl, steps, precision):
    ora = solver_of(wl)
    gpu = native.from_workload(wl, precision=precision)
    out = [(ora.energy(), gpu.diagnostics()[7])]
    for _ in range(steps):
        ora.step()
    gpu.step(steps)
    out.append((ora.energy(), gpu.diagnostics()[7]))
    um = gpu.diagnostics()[1]
    gpu.close()
    return out, um


@pytest.mark.parametrize("wl", [workloads.small2d(ex=4, ey=3, order=6, theta_s_deg=60.0),
                                workloads.small3d(ex=4, ey=2, order=5, nz=8, theta_s_deg=70.0)],
                         ids=["2d", "3d"])
def test_energy_fp64_matches_oracle(wl):
    res, um = _energies(wl, 4, native.PF_FP64)
    assert um > 1e-8                                  # the kinetic term is exercised
    for e_ora, e_gpu in res:
        assert abs(e_gpu - e_ora) <= 1e-11 * abs(e_ora), (e_gpu, e_ora)


def test_energy_mixed_within_single_precision():
    wl = workloads.small3d(ex=4, ey=2, order=4, nz=8, theta_s_deg=70.0)
    res, _ = _energies(wl, 3, native.PF_MIXED)
    for e_ora, e_gpu in res:
        assert abs(e_gpu - e_ora) <= 1e-5 * abs(e_ora), (e_gpu, e_ora)
