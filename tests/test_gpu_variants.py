"""Every transform variant of the fast-diagonalisation solves (tensor cores, whole plane in shared
memory, SIMT tiles; y pair fused or separate; z-transform tiles) against the oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from tolerances import mixed_bar
from oracle.sem import Mesh2D
from paper_2305_09020_gb300 import native

from gpu_util import ALL, oracle_fields, rel_errors, run_pair

pytestmark = pytest.mark.gpu

FP32_VARIANTS = [(native.PF_GEMM_TC, 1), (native.PF_GEMM_PLANE, 1), (native.PF_GEMM_SIMT32, 0),
                 (native.PF_GEMM_SIMT32, 1), (native.PF_GEMM_SIMT64, 1), (native.PF_GEMM_SIMT32X64, 0),
                 (native.PF_GEMM_PIPE64, 0), (native.PF_GEMM_PIPE32, 1), (native.PF_GEMM_PIPE32X64, 0),
                 (native.PF_GEMM_CLUSTER4, 1), (native.PF_GEMM_CLUSTER2, 1), (native.PF_GEMM_TC_HYBRID, 1)]
SIMT = (native.PF_GEMM_SIMT32, native.PF_GEMM_SIMT64, native.PF_GEMM_SIMT32X64, native.PF_GEMM_PIPE64,
        native.PF_GEMM_PIPE32, native.PF_GEMM_PIPE32X64)


def _direct(m, bcset, shift, f):
    """(K + shift M) x = M f with the Dirichlet rows of the bcset eliminated (x = 0 there)."""
    Dn = []
    if bcset == native.PF_BCSET_V:
        Dn = list(m.bottom_nodes) + list(m.top_nodes)
    elif bcset == native.PF_BCSET_U:
        Dn = list(m.bottom_nodes)
    free = np.setdiff1d(np.arange(m.n2), Dn)
    lu = spla.splu(m.helmholtz(shift).tocsr()[free][:, free].tocsc())
    out = np.zeros_like(f)
    for pl in range(f.shape[0]):
        out[pl, free] = lu.solve((m.Mdiag * f[pl])[free])
    return out


@pytest.mark.parametrize("gemm,fuse_y", FP32_VARIANTS)
@pytest.mark.parametrize("mesh", [(6, 5, 6), (16, 8, 8)])
@pytest.mark.parametrize("bcset", [native.PF_BCSET_V, native.PF_BCSET_U])
def test_helmholtz_variant(gemm, fuse_y, mesh, bcset):
    """A ragged plane (36 x 31 nodes) and the 128 x 65 plane of the 16 x 8, order-8 mesh, one
    Fourier mode pair, each variant within the FP32 bar of the assembled direct solve."""
    ex, ey, K = mesh
    wl = workloads.small3d(ex=ex, ey=ey, order=K, nz=4)
    g = native.from_workload(wl, precision=native.PF_MIXED)
    g.set_variant(gemm, fuse_y=fuse_y)
    m = Mesh2D(wl.mesh.xb, wl.mesh.yb, wl.mesh.order)
    mode, lam = 1, 3.0
    beta = 2 * np.pi * mode / wl.mesh.lz
    f = np.random.default_rng(7 + bcset).standard_normal((2, m.n2))
    x = g.solve_helmholtz(bcset, mode, lam, f).reshape(2, m.n2)
    g.close()
    ref = _direct(m, bcset, lam + beta ** 2, f)
    for pl in range(2):
        assert np.linalg.norm(x[pl] - ref[pl]) <= 2e-6 * np.linalg.norm(ref[pl])


@pytest.mark.parametrize("gemm,fuse_y", FP32_VARIANTS)
def test_step_variant_3d(gemm, fuse_y):
    """Ten mixed-precision steps of a small 3D run with each variant pinned, against the oracle
    (the bars of the mixed path: 5e-5 on V, phi, psi and 5e-4 on the derived fields)."""
    from oracle.runner import solver_of
    wl = workloads.small3d(ex=4, ey=2, order=5, nz=8)
    ora = solver_of(wl)
    g = native.from_workload(wl, precision=native.PF_MIXED)
    g.set_variant(gemm, fuse_y=fuse_y, tile=8)
    for _ in range(10):
        ora.step()
    g.step(10)
    errs = rel_errors(g.get(ALL), oracle_fields(ora))
    g.close()
    for k, v in errs.items():
        assert v <= mixed_bar(k, 100), (k, v)


def test_set_variant_rejects_what_the_run_cannot_use():
    wl = workloads.small3d(ex=2, ey=2, order=4, nz=4)
    g64 = native.from_workload(wl, precision=native.PF_FP64)
    gs = native.from_workload(wl, precision=native.PF_MIXED_SIMT)
    for h, args in [(g64, (native.PF_GEMM_PLANE, True, 0)), (g64, (native.PF_GEMM_TC, True, 0)),
                    (g64, (native.PF_GEMM_TC_HYBRID, True, 0)), (gs, (native.PF_GEMM_TC, True, 0)),
                    (gs, (native.PF_GEMM_TC_HYBRID, True, 0)), (gs, (48, True, 0)), (gs, (native.PF_GEMM_SIMT32, True, 6))]:
        with pytest.raises(native.PfError) as e:
            h.set_variant(*args)
        assert e.value.code == native.PF_EINVAL
    with pytest.raises(native.PfError):
        g64.set_variant(native.PF_GEMM_CLUSTER4)
    # the tensor-core transforms need n_x % 4 == 0 (16-byte rows for TMA): 30 x 25 nodes cannot
    odd = native.from_workload(workloads.small3d(ex=5, ey=4, order=6, nz=4), precision=native.PF_MIXED)
    with pytest.raises(native.PfError) as e:
        odd.set_variant(native.PF_GEMM_TC)
    assert e.value.code == native.PF_EINVAL
    odd.step(2)                                       # the default variant is a CUDA-core one there
    odd.close()
    gs.set_variant(native.PF_GEMM_CLUSTER2)
    gs.set_variant(native.PF_GEMM_PLANE, tile=16)    # FP32 without tensor cores can take the plane solves
    gs.step(3)
    g64.set_variant(native.PF_GEMM_SIMT64, fuse_y=False, tile=4)
    g64.step(3)
    g64.close()
    gs.close()


@pytest.mark.parametrize("gemm", [native.PF_GEMM_PLANE, native.PF_GEMM_CLUSTER4])
def test_batch_plane_variant_matches_oracle(gemm):
    from oracle.runner import solver_of
    from test_gpu_batch import uneven_runs
    runs = uneven_runs()
    b = native.Batch(runs, precision=native.PF_MIXED)
    b.set_variant(gemm)
    oras = [solver_of(wl) for wl in runs]
    for _ in range(4):
        for o in oras:
            o.step()
    b.step(4)
    for r, ora in enumerate(oras):
        errs = rel_errors(b.get(r, ALL), oracle_fields(ora), skip=("Ez", "uz"))
        for k, v in errs.items():
            assert v <= mixed_bar(k, 100), (r, k, v)
    b.close()
    bf = native.Batch(runs, precision=native.PF_FP64)
    with pytest.raises(native.PfError):
        bf.set_variant(native.PF_GEMM_PLANE)
    bf.close()


@pytest.mark.parametrize("with_stream", [True, False])
def test_autotune_advances_the_stated_steps_and_keeps_parity(with_stream):
    """pf_autotune times every variant (graph replays on a stream of its own, eager launches on the
    legacy stream), advances the run by 16 (steps + 2) steps, and the run stays on the FP64 oracle."""
    from oracle.runner import solver_of
    torch = pytest.importorskip("torch")
    wl = workloads.small3d(ex=4, ey=2, order=4, nz=8)
    s = torch.cuda.Stream() if with_stream else None
    g = native.from_workload(wl, precision=native.PF_FP64, stream=s.cuda_stream if s is not None else None)
    choice, ms = g.autotune(steps=1)
    assert ms > 0 and choice % 1000 in SIMT
    assert (choice // 1000) % 100 in (0, 4, 8, 16, 32) and choice // 100000 in (0, 1)
    g.step(3)
    ora = solver_of(wl)
    for _ in range(1 + 16 * 3 + 3):
        ora.step()
    errs = rel_errors(g.get(ALL), oracle_fields(ora))
    g.close()
    assert all(v <= 1e-11 for v in errs.values()), errs


@pytest.mark.parametrize("nz", [1, 8, 2])
def test_fp64_cuda_core_variants_agree_bit_for_bit(nz):
    """In FP64 every CUDA-core transform variant sums in sequential k order: identical bits (for
    each choice of the y pair, whose fused form adds the eigenvalue sum in another order)."""
    if nz == 2:   # n_y = 73: the y transforms take the 80-wide column tiles of the pipelined variants
        wl = workloads.small3d(ex=3, ey=9, order=8, nz=nz)
    else:
        wl = workloads.small3d(ex=5, ey=3, order=5, nz=nz) if nz > 1 else workloads.small2d(ex=5, ey=3, order=5)
    for fuse_y in (0, 1):
        ref = None
        for gemm in SIMT:
            g = native.from_workload(wl, precision=native.PF_FP64)
            g.set_variant(gemm, fuse_y=bool(fuse_y))
            g.step(4)
            f = g.get(ALL)
            g.close()
            if ref is None:
                ref = f
            for k in f:
                assert np.array_equal(f[k], ref[k]), (gemm, fuse_y, k)


@pytest.mark.parametrize("gemm", [native.PF_GEMM_TC, native.PF_GEMM_TC_HYBRID, native.PF_GEMM_CLUSTER4,
                                  native.PF_GEMM_PLANE, native.PF_GEMM_PIPE32])
def test_variant_graph_replay_is_bit_identical(gemm):
    """A pinned variant replayed from the captured graphs gives the bits of eager launches."""
    torch = pytest.importorskip("torch")
    wl = workloads.small3d(ex=4, ey=2, order=4, nz=8)
    s = torch.cuda.Stream()
    a = native.from_workload(wl, precision=native.PF_MIXED, stream=s.cuda_stream)
    b = native.from_workload(wl, precision=native.PF_MIXED)
    for h in (a, b):
        h.set_variant(gemm, tile=8)
        h.step(6)
    fa, fb = a.get(ALL), b.get(ALL)
    a.close()
    b.close()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.fixture(scope="module")
def droplet2d_100():
    """The FP64 oracle's 2D droplet after 50 and 100 steps."""
    from oracle.runner import solver_of
    wl = workloads.droplet2d()
    ora = solver_of(wl)
    out = {}
    for n in range(1, 101):
        ora.step()
        if n in (50, 100):
            out[n] = oracle_fields(ora)
    return wl, out


@pytest.mark.parametrize("gemm,acc", [(native.PF_GEMM_TC, None), (native.PF_GEMM_TC, ((1, 0), (1, 0))),
                                      (native.PF_GEMM_TC, ((2, 1), (2, 1))), (native.PF_GEMM_TC_HYBRID, None),
                                      (native.PF_GEMM_TC_HYBRID, ((4, 0), (8, 1)))])
def test_tc_accumulation(droplet2d_100, gemm, acc):
    """The tensor-core transforms with each accumulation layout (slices per TMEM group, correction
    products in their own region, per solve family; None: the defaults) hold the mixed bars of the
    2D droplet over 100 steps against the oracle: 5e-5 on V, phi, psi and 5e-4 on E, P, u."""
    wl, ref = droplet2d_100
    g = native.from_workload(wl, precision=native.PF_MIXED)
    g.set_variant(gemm, fuse_y=False)
    if acc is not None:
        for fam, (slices, sep) in enumerate(acc):
            g.set_tc_accum(gemm, fam, slices, sep)
    for n in (50, 100):
        g.step(50)
        errs = rel_errors(g.get(ALL), ref[n], skip=("Ez", "uz"))
        for k, v in errs.items():
            assert v <= mixed_bar(k, n), (n, k, v)
    g.close()


def test_tc_accumulation_rejects():
    wl = workloads.small3d(ex=2, ey=2, order=4, nz=4)
    g = native.from_workload(wl, precision=native.PF_MIXED)
    for args in [(1, 0, 1, 0), (native.PF_GEMM_TC, 2, 1, 0), (native.PF_GEMM_TC, 0, 0, 0),
                 (native.PF_GEMM_TC, 1, 65, 0), (native.PF_GEMM_TC, 1, 2, 2)]:
        with pytest.raises(RuntimeError):
            g.set_tc_accum(*args)
    g.close()
    g64 = native.from_workload(wl, precision=native.PF_FP64)
    with pytest.raises(RuntimeError):
        g64.set_tc_accum(native.PF_GEMM_TC, 1, 2, 1)
    g64.close()
