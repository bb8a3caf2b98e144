"""Ensembles of independent 2D runs (pf_batch_*) against the FP64 oracle, run by run."""
import numpy as np
import pytest

import workloads
from tolerances import mixed_bar
from oracle.runner import solver_of
from paper_2305_09020_gb300 import native

from gpu_util import ALL, oracle_fields, rel_errors

pytestmark = pytest.mark.gpu


def uneven_runs():
    """Five runs in three mesh groups, each with its own permittivity ratio and voltage."""
    runs = []
    for (ex, ey, K, eps, v) in [(4, 2, 5, 5.0, 1.0), (4, 2, 5, 12.0, 2.5), (4, 2, 5, 2.0, 0.5),
                                (6, 3, 4, 7.0, 1.5), (2, 2, 6, 3.0, 2.0)]:
        wl = workloads.small2d(ex=ex, ey=ey, order=K)
        wl.fluid.eps1 = eps
        wl.vbc.v_bottom = v
        runs.append(wl)
    return runs


def _compare(batch, runs, oras, tol, steps):
    for r, (wl, ora) in enumerate(zip(runs, oras)):
        got = batch.get(r, ALL)
        errs = rel_errors(got, oracle_fields(ora), skip=("Ez", "uz") + (("psi",) if steps == 0 else ()))
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, f"run {r} after {steps} steps: {bad}"


def test_batch_fp64_matches_oracle_per_run():
    runs = uneven_runs()
    b = native.Batch(runs, precision=native.PF_FP64)
    assert b.groups()[0] == 3
    oras = [solver_of(wl) for wl in runs]
    _compare(b, runs, oras, 1e-11, 0)
    for _ in range(6):
        for o in oras:
            o.step()
    b.step(6)
    _compare(b, runs, oras, 1e-11, 6)
    umax, mass = b.umax()
    for r, o in enumerate(oras):
        assert abs(umax[r] - o.umax()) <= 1e-11 * max(o.umax(), 1e-30)
        assert abs(mass[r] - o.phase_mass()) <= 1e-12 * abs(o.phase_mass())
    b.close()


def test_batch_mixed_and_graph_stream():
    torch = pytest.importorskip("torch")
    runs = uneven_runs()
    s = torch.cuda.Stream()
    b = native.Batch(runs, precision=native.PF_MIXED, stream=s.cuda_stream)
    oras = [solver_of(wl) for wl in runs]
    for _ in range(3):
        for o in oras:
            o.step()
    b.step(3)                     # steps 2 and 3 replay the ensemble graph
    for r, ora in enumerate(oras):
        errs = rel_errors(b.get(r, ALL), oracle_fields(ora), skip=("Ez", "uz"))
        for k, v in errs.items():
            assert v <= mixed_bar(k, 100), (r, k, v)
    b.close()


def test_batch_autotune_keeps_lockstep():
    runs = uneven_runs()
    b = native.Batch(runs, precision=native.PF_FP64)
    ms = b.autotune(steps=1)      # one BDF1 step, then 6 x 2 = 12 steps per group
    assert len(ms) == 3 and np.all(ms > 0)
    oras = [solver_of(wl) for wl in runs]
    for _ in range(13):
        for o in oras:
            o.step()
    _compare(b, runs, oras, 1e-11, 13)
    b.close()


def test_batch_run_to_equilibrium_reports_steps():
    runs = uneven_runs()
    b = native.Batch(runs, precision=native.PF_FP64)
    steps = b.run_to_equilibrium(tol=1e30, max_steps=10, check_every=4)
    assert np.all(steps == 1)            # the exit is checked on the device after every step
    steps = b.run_to_equilibrium(tol=0.0, max_steps=10, check_every=4)   # never below 0
    assert np.all(steps == -1)
    b.close()


def test_per_run_exit_is_exact_and_freezes_the_run():
    """Equilibrium system (pseudo-time rate max|phi^{n+1} - phi^n| / dt, which decays): each run of
    an uneven ensemble stops at the first step its own rate falls below the tolerance, found on
    the device whatever check_every is, and its fields stay those of that step while the other runs
    go on.  The reference is each run alone on a handle of its own."""
    runs = uneven_runs()
    for w in runs:
        w.scheme.equilibrium = True
    nmax = 40
    rates, states = [], []
    for wl in runs:
        h = native.from_workload(wl, precision=native.PF_FP64)
        r, st = [], []
        for _ in range(nmax):
            h.step(1)
            r.append(h.diagnostics()[6])
            st.append(h.get(ALL))
        h.close()
        rates.append(np.array(r))
        states.append(st)
    # a tolerance halfway (geometrically) between two well separated rates at step 15
    vals = np.sort(np.array([r[14] for r in rates]))
    gaps = vals[1:] / vals[:-1]
    i = int(np.argmax(gaps))
    tol = float(np.sqrt(vals[i] * vals[i + 1]))
    expect = []
    for r in rates:
        below = np.nonzero(r < tol)[0]
        expect.append(int(below[0]) + 1 if below.size else -1)
        assert np.all(np.abs(r / tol - 1.0) > 1e-6)        # no rate sits on the tolerance
    assert len(set(expect)) > 1                           # the runs stop at different steps
    b = native.Batch(runs, precision=native.PF_FP64)
    steps = b.run_to_equilibrium(tol=tol, max_steps=nmax, check_every=7)
    assert list(steps) == expect, (list(steps), expect)
    for r, s in enumerate(expect):
        ref = states[r][(s if s > 0 else nmax) - 1]
        errs = rel_errors(b.get(r, ALL), ref, skip=("Ez", "uz", "P", "ux", "uy", "psi"))
        assert all(v <= 1e-11 for v in errs.values()), (r, s, errs)
    b.close()



def test_batch_equilibrium_model_stops_on_rate():
    runs = uneven_runs()
    for w in runs:
        w.scheme.equilibrium = True
    b = native.Batch(runs, precision=native.PF_FP64)
    oras = [solver_of(wl) for wl in runs]
    b.step(4)
    for o in oras:
        for _ in range(4):
            o.step()
    _compare(b, runs, oras, 1e-11, 4)
    rate, _ = b.umax()
    for r, o in enumerate(oras):
        ref = np.max(np.abs(o.phi - o.phi_old)) / o.prm.dt
        assert abs(rate[r] - ref) <= 1e-9 * ref
    b.close()
