"""Learned warm start for equilibrium runs: data generation, training and evaluation.

Orchestration only: every time step runs in the ensemble engine (pf_batch_*), every network
forward/backward/update in the library's kernels (pf_no_*); this module moves arrays.

* ``equilibrium_runs`` switches runs to the pseudo-time march of the equilibrium system (Sec. 2.4).
* ``generate``   runs batches of independent 2D runs on one fixed mesh until every run meets the
  criterion (max|u|, or for the equilibrium system the pseudo-time rate, below tol; each run
  exits on the device at its own step) or the step cap, and returns the run features (V,
  permittivity ratio, drop area), the phase field at the exit (the equilibrium target) and the
  steps each run needed.
* ``make_operator`` / ``train``  the network of ``native.NeuralOperator``: 3 -> 128 -> 384 ->
  128x64 grid (tanh), bilinear to the GLL nodes, BF16 weights.
* ``evaluate``  runs held-out cases from the usual initial profile (cold) and from the network's
  prediction shifted to the run's phase mass (warm) to the same criterion, and a third time cold to
  a tighter tolerance (the judge); it reports steps and wall time to the criterion and the error of
  both final states against the judge.
"""
from __future__ import annotations

import time
from typing import List, Optional

import numpy as np

import workloads
from . import native

GRID = (128, 64)
BOX = (0.0, 2.0, 0.0, 1.0)
DIMS = [3, 128, 384, GRID[0] * GRID[1]]


def equilibrium_runs(runs: List[workloads.Workload], dt: float = 1e-3, gamma1: float = 3e-3):
    """The runs marched with the simpler equilibrium system of Sec. 2.4 (eq. 16 with eq. 15c, 15d,
    u = 0) in pseudo-time.  Its steady states do not depend on the mobility or the time step, so
    both are taken larger than in the full model (faster relaxation; at mobility 1e-2 some runs
    of this family diverge)."""
    for w in runs:
        w.scheme.equilibrium = True
        w.scheme.dt = dt
        w.fluid.gamma1 = gamma1
    return runs


def _chunks(seq, n):
    for i in range(0, len(seq), n):
        yield seq[i:i + n]


def generate(runs: List[workloads.Workload], tol: float, max_steps: int, check_every: int = 200,
             precision: int = native.PF_MIXED, stream: Optional[int] = None, batch: int = 256):
    feats, finals, steps = [], [], []
    for chunk in _chunks(runs, batch):
        b = native.Batch(chunk, precision=precision, stream=stream)
        st = b.run_to_equilibrium(tol, max_steps, check_every)
        for r in range(len(chunk)):
            finals.append(b.get(r, native.PF_FIELD_PHI)["phi"].ravel())
        b.close()
        feats.extend(workloads.warmstart_features(w) for w in chunk)
        steps.extend(st.tolist())
    feats, finals, steps = np.array(feats), np.array(finals), np.array(steps)
    ok = (steps != -2) & np.all(np.isfinite(finals), axis=1)     # drop runs that diverged
    return feats[ok], finals[ok], steps[ok]


def make_operator(feats: np.ndarray, mesh: workloads.Mesh, seed: int = 0, stream: Optional[int] = None):
    node_x = native.nodes_1d(mesh.xb, mesh.order, True)
    node_y = native.nodes_1d(mesh.yb, mesh.order, False)
    return native.NeuralOperator(DIMS, feats.mean(axis=0), feats.std(axis=0) + 1e-12, GRID, BOX, node_x, node_y,
                                 seed=seed, stream=stream)


def node_weights(mesh: workloads.Mesh):
    """Quadrature weights of the GLL node grid (the assembled 1D masses in x and y)."""
    _, wx = native.operators_1d(mesh.xb, mesh.order, True)
    _, wy = native.operators_1d(mesh.yb, mesh.order, False)
    return wx, wy


def evaluate(no, runs: List[workloads.Workload], tol: float, max_steps: int, check_every: int = 200,
             precision: int = native.PF_MIXED, stream: Optional[int] = None, judge_tol: Optional[float] = None,
             judge_steps: Optional[int] = None):
    """Held-out runs, cold (the usual initial profile) and warm (the network's field, shifted on the
    device to the run's own phase mass), each to the same criterion; both final states are compared
    with a judge: the cold start run to the tighter tolerance judge_tol (default tol / 10)."""
    feats = np.array([workloads.warmstart_features(w) for w in runs])
    judge_tol = tol / 10.0 if judge_tol is None else judge_tol
    judge_steps = 4 * max_steps if judge_steps is None else judge_steps
    out, finals, steps = {}, {}, {}
    b = native.Batch(runs, precision=precision, stream=stream)
    _, mass0 = b.umax()                       # phase mass of every run's initial profile (FP64)
    b.close()
    wx, wy = node_weights(runs[0].mesh)
    pred = no.predict_mass(feats, mass0, wx, wy)
    for mode in ("cold", "warm", "judge"):
        t0 = time.perf_counter()
        b = native.Batch(runs, precision=precision, stream=stream, phi0_list=list(pred) if mode == "warm" else None)
        t1 = time.perf_counter()
        st = b.run_to_equilibrium(judge_tol if mode == "judge" else tol,
                                  judge_steps if mode == "judge" else max_steps, check_every)
        t2 = time.perf_counter()
        finals[mode] = np.array([b.get(r, native.PF_FIELD_PHI)["phi"].ravel() for r in range(len(runs))])
        b.close()
        steps[mode] = st
        out[mode] = {"setup_s": t1 - t0, "run_s": t2 - t1, "diverged": int((st == -2).sum()),
                     "capped": int((st == -1).sum())}
    # the runs that no side lost to divergence; capped runs count as the cap
    ok = (steps["cold"] != -2) & (steps["warm"] != -2) & (steps["judge"] != -2)
    ref = finals["judge"][ok]
    for mode in ("cold", "warm"):
        cap = max_steps
        s = np.where(steps[mode] == -1, cap, steps[mode])[ok]
        err = np.linalg.norm(finals[mode][ok] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        out[mode].update({"steps_mean": float(s.mean()), "steps_median": float(np.median(s)), "runs": int(ok.sum()),
                          "err_vs_judge_median": float(np.median(err)), "err_vs_judge_max": float(err.max()),
                          "steps": s.tolist(), "err": err.tolist()})
    out["judge"].update({"tol": judge_tol, "capped": int((steps["judge"] == -1).sum())})
    diff = np.linalg.norm(finals["warm"][ok] - finals["cold"][ok], axis=1) / np.linalg.norm(finals["cold"][ok], axis=1)
    out["final_phi_rel_diff_warm_vs_cold"] = {"median": float(np.median(diff)), "max": float(diff.max())}
    return out
