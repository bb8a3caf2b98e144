"""Shared helpers of the GPU parity tests (the oracle runs on the host CPU)."""
import numpy as np

import workloads
from oracle.runner import solver_of
from paper_2305_09020_gb300 import native

FIELDS = ("V", "Ex", "Ey", "Ez", "phi", "psi", "P", "ux", "uy", "uz")
ALL = native.PF_FIELD_V | native.PF_FIELD_E | native.PF_FIELD_PHI | native.PF_FIELD_PSI | \
    native.PF_FIELD_P | native.PF_FIELD_U


def oracle_fields(sol):
    m = sol.mesh
    shp = (sol.nz, m.ny, m.nx)
    return dict(V=sol.V.reshape(shp), Ex=sol.E[0].reshape(shp), Ey=sol.E[1].reshape(shp),
                Ez=sol.E[2].reshape(shp), phi=sol.phi.reshape(shp), psi=sol.psi.reshape(shp),
                P=sol.P.reshape(shp), ux=sol.u[0].reshape(shp), uy=sol.u[1].reshape(shp),
                uz=sol.u[2].reshape(shp))


def rel_errors(gpu: dict, ref: dict, skip=()):
    out = {}
    for k in FIELDS:
        if k in skip:
            continue
        r = ref[k]
        if np.max(np.abs(r)) < 1e-9:
            # an identically-zero field (e.g. E when V is constant): compare absolutely
            out[k] = float(np.max(np.abs(gpu[k] - r)))
        else:
            out[k] = float(np.linalg.norm(gpu[k] - r) / np.linalg.norm(r))
    return out


def run_pair(wl, steps, precision=native.PF_FP64, check_every=None):
    """Advance the oracle and the GPU path side by side; returns (errors per checkpoint)."""
    ora = solver_of(wl)
    gpu = native.from_workload(wl, precision=precision)
    res = []
    skip = ("psi",)   # psi is defined after the first step only
    res.append((0, rel_errors(gpu.get(ALL), oracle_fields(ora), skip=skip + (("Ez", "uz") if wl.mesh.nz == 1 else ()))))
    done = 0
    marks = sorted(set([steps] + ([] if check_every is None else list(range(check_every, steps, check_every)))))
    for mk in marks:
        for _ in range(mk - done):
            ora.step()
        gpu.step(mk - done)
        done = mk
        sk = ("Ez", "uz") if wl.mesh.nz == 1 else ()
        res.append((mk, rel_errors(gpu.get(ALL), oracle_fields(ora), skip=sk)))
    gpu.close()
    return res
