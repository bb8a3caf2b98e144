"""Host-side pieces of bench.py and the workload generators it times (no GPU)."""
import math

import numpy as np
import pytest

import bench
import workloads


def test_fdm_flop_count_per_solve_set():
    nx, ny, nz = 128, 65, 64
    per_solve = 4.0 * nx * ny * (nx + ny) * nz
    assert bench.fdm_flops_per_step(nx, ny, nz, True) == pytest.approx(7 * per_solve)          # V, psi, phi, P, u x3
    assert bench.fdm_flops_per_step(nx, ny, 1, False) == pytest.approx(6 * per_solve / nz)     # 2D: u x2
    assert bench.fdm_flops_per_step(nx, ny, nz, True, equilibrium=True) == pytest.approx(3 * per_solve)
    assert bench.fdm_flops_per_step(nx, ny, nz, True, equilibrium=True, patches=True) == pytest.approx(4 * per_solve)


def test_transform_kernel_labels_and_traffic_table():
    assert bench.transform_kernel(3, 0) == "k_gemm_cp"
    assert bench.transform_kernel(64, 1) == "k_gemm + k_fdm_y"
    assert bench.transform_kernel(0, 1) == "k_gemm_tc"
    assert bench.transform_kernel(6, 1) == "k_fdm_cluster<4>"
    assert bench.transform_kernel(8, 1) == "k_gemm_tc + k_gemm_cp"
    # only captured (precision, variant, fused y) triples carry a DRAM traffic figure
    assert set(bench.TRANSFORM_DRAM_BYTES_PER_LAUNCH) == {("droplet3d", "mixed", 3, 0), ("layers3d", "mixed", 0, 0)}
    # the layers3d figure is at least the planes read once (13.19M FP32 values) and at most twice that
    assert 4 * 13189120 <= bench.TRANSFORM_DRAM_BYTES_PER_LAUNCH[("layers3d", "mixed", 0, 0)] <= 8 * 13189120
    assert bench.transform_bytes_per_launch(128, 65, 64, 1) == pytest.approx(4 * (2 * 128 * 65 * 64 + 128 ** 2))


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_every_bench_workload_builds(name):
    wls = bench.make_workload(name)
    for wl in (wls if isinstance(wls, list) else [wls]):
        assert wl.mesh.order >= 2 and wl.scheme.dt > 0
        x = np.linspace(0.0, 1.0, 7)
        phi = wl.phi0(x, 0.1 + 0 * x, 0.5 + 0 * x)
        assert np.all(np.abs(phi) <= 1.0)
    if name == "ensemble2d":
        assert len(wls) == 256 and len({(w.mesh.ex, w.mesh.order) for w in wls}) > 20


def test_electrode_array_normalisation():
    """Permittivities normalised by L0 gamma / V_d^2 (L0 = 1.2 mm, gamma = 3.857e-2, V_d = 150 V)."""
    wl = workloads.electrode_array3d()
    e_air = 8.854e-12 * 150.0 ** 2 / (1.2e-3 * 3.857e-2)
    assert wl.fluid.eps2 == pytest.approx(e_air) and wl.fluid.eps1 == pytest.approx(32 * e_air)
    assert e_air == pytest.approx(4.30e-3, rel=2e-3)
    lam = 3.0 * wl.fluid.sigma * wl.fluid.eta / (2.0 * math.sqrt(2.0))
    assert lam * wl.fluid.gamma1 == pytest.approx(0.1)
    pats = wl.vbc.patches
    assert len(pats) == 10 and all(abs(b - a - 1.0 / 12.0) < 1e-15 for a, b, _ in pats)
    assert [v for _, _, v in pats] == [1.0, -1.0] * 5
    assert wl.mesh.nz == 120 and wl.scheme.equilibrium


def test_bench_functions_name_only_defined_globals():
    """Every global a function of bench.py reads is defined at module level or is a builtin (the
    GPU-only legs never run on the CPU, so a missing helper would otherwise surface on a GPU machine)."""
    import builtins
    import symtable
    src = open(bench.__file__).read()
    top = symtable.symtable(src, bench.__file__, "exec")
    missing = []

    def walk(t):
        for ch in t.get_children():
            if ch.get_type() == "function":
                for sym in ch.get_symbols():
                    if sym.is_global() and sym.is_referenced() and not hasattr(bench, sym.get_name()) \
                            and not hasattr(builtins, sym.get_name()):
                        missing.append((ch.get_name(), sym.get_name()))
            walk(ch)

    walk(top)
    assert not missing, missing
