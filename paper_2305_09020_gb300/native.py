"""Thin ctypes binding of the C-ABI declared in include/pf.h (argument marshalling only).

Every step of the time-stepping path runs in the CUDA library ``libpf.so``;
this module converts numpy arrays and Python numbers to the C structs and
pointers of the ABI and turns negative status codes into exceptions.  If the
library cannot be loaded the import fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_size_t, c_uint, c_void_p, c_char_p, c_ubyte
from typing import Optional, Sequence

import numpy as np

from . import _build

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENOTSEPARABLE, PF_EDIVERGED, PF_ETIMEOUT, PF_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
PF_BC_DIRICHLET, PF_BC_NEUMANN, PF_BC_PATCHES = 0, 1, 2
PF_FP64, PF_MIXED, PF_MIXED_SIMT = 0, 1, 2
PF_BCSET_V, PF_BCSET_NN, PF_BCSET_P, PF_BCSET_U = 0, 1, 2, 3
PF_MODEL_FULL, PF_MODEL_EQUILIBRIUM = 0, 1
PF_GEMM_TC, PF_GEMM_PLANE, PF_GEMM_SIMT32, PF_GEMM_SIMT64, PF_GEMM_SIMT32X64 = 0, 1, 32, 64, 2
PF_GEMM_PIPE64, PF_GEMM_PIPE32, PF_GEMM_PIPE32X64 = 3, 4, 5
PF_GEMM_CLUSTER4, PF_GEMM_CLUSTER2 = 6, 7
PF_GEMM_TC_HYBRID = 8
PF_FIELD_V, PF_FIELD_E, PF_FIELD_PHI, PF_FIELD_PSI, PF_FIELD_P, PF_FIELD_U, PF_FIELD_OLD = \
    1, 2, 4, 8, 16, 32, 64
KERNEL_CLASSES = ["gemm", "fwd", "inv", "potential", "chem", "momentum", "ugradp", "efield", "other"]
_BLOCKS = [(PF_FIELD_V, ["V"]), (PF_FIELD_E, ["Ex", "Ey", "Ez"]), (PF_FIELD_PHI, ["phi"]),
           (PF_FIELD_PSI, ["psi"]), (PF_FIELD_P, ["P"]), (PF_FIELD_U, ["ux", "uy", "uz"])]


class PfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pf error {code}: {msg}")
        self.code = code


class PfMesh(ctypes.Structure):
    _fields_ = [("ex", c_int), ("ey", c_int), ("xb", POINTER(c_double)), ("yb", POINTER(c_double)),
                ("order", c_int), ("nz", c_int), ("lz", c_double)]


class PfFluid(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("rho1", "rho2", "mu1", "mu2", "eps1", "eps2", "sigma", "eta",
                                        "gamma1", "theta_s_deg")]


class PfVbc(ctypes.Structure):
    _fields_ = [("bottom_kind", c_int), ("top_kind", c_int), ("v_bottom", c_double), ("v_top", c_double),
                ("n_patch", c_int), ("patch_x0", POINTER(c_double)), ("patch_x1", POINTER(c_double)),
                ("patch_v", POINTER(c_double))]


class PfScheme(ctypes.Structure):
    _fields_ = [("dt", c_double), ("bdf", c_int), ("precision", c_int), ("S", c_double),
                ("nu_m", c_double), ("rho0", c_double), ("eps0", c_double), ("model", c_int)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpf.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    dp = POINTER(c_double)
    L.pf_gll.argtypes = [c_int, dp, dp, dp]
    L.pf_nodes_1d.argtypes = [c_int, dp, c_int, c_int, dp]
    L.pf_operators_1d.argtypes = [c_int, dp, c_int, c_int, dp, dp]
    L.pf_fdm_1d.argtypes = [c_int, dp, dp, POINTER(c_ubyte), dp, dp]
    L.pf_create.argtypes = [POINTER(PfMesh), POINTER(PfFluid), POINTER(PfVbc), POINTER(PfScheme), dp, dp,
                            c_void_p, POINTER(c_void_p)]
    L.pf_step.argtypes = [c_void_p, c_int]
    L.pf_sync.argtypes = [c_void_p]
    L.pf_get_fields.argtypes = [c_void_p, c_uint, dp, c_size_t]
    L.pf_set_fields.argtypes = [c_void_p, c_uint, dp, c_size_t, c_int]
    L.pf_diagnostics.argtypes = [c_void_p, dp]
    L.pf_solve_helmholtz.argtypes = [c_void_p, c_int, c_int, c_double, dp, dp]
    L.pf_geometry.argtypes = [c_void_p, dp, dp, POINTER(c_int)]
    L.pf_profile.argtypes = [c_void_p, c_int]
    L.pf_autotune.argtypes = [c_void_p, c_int, POINTER(c_int), dp]
    L.pf_set_variant.argtypes = [c_void_p, c_int, c_int, c_int]
    L.pf_set_step.argtypes = [c_void_p, c_int, c_double]
    L.pf_measure_peaks.argtypes = [POINTER(c_double)]
    L.pf_set_tc_accum.argtypes = [c_void_p, c_int, c_int, c_int, c_int]
    L.pf_debug_tc_stall.argtypes = [c_void_p, ctypes.c_ulonglong]
    L.pf_fdm_solve_static.argtypes = [c_int, c_int, c_int] + [c_void_p] * 10
    L.pf_batch_create.argtypes = [c_int, POINTER(PfMesh), POINTER(PfFluid), POINTER(PfVbc), POINTER(PfScheme),
                                  POINTER(POINTER(c_double)), c_void_p, POINTER(c_void_p)]
    L.pf_batch_step.argtypes = [c_void_p, c_int]
    L.pf_batch_umax.argtypes = [c_void_p, dp, dp]
    L.pf_batch_run_to_equilibrium.argtypes = [c_void_p, c_double, c_int, c_int, POINTER(c_int)]
    L.pf_batch_get_fields.argtypes = [c_void_p, c_int, c_uint, dp, c_size_t]
    L.pf_batch_autotune.argtypes = [c_void_p, c_int, dp]
    L.pf_batch_set_variant.argtypes = [c_void_p, c_int, c_int]
    L.pf_batch_last_error.argtypes = [c_void_p]
    L.pf_batch_last_error.restype = c_char_p
    L.pf_batch_groups.argtypes = [c_void_p, POINTER(c_int)]
    L.pf_batch_destroy.argtypes = [c_void_p]
    L.pf_batch_destroy.restype = None
    L.pf_no_create.argtypes = [c_int, POINTER(c_int), dp, dp, c_int, c_int, c_double, c_double, c_double, c_double,
                               c_int, c_int, dp, dp, ctypes.c_uint64, c_void_p, POINTER(c_void_p)]
    L.pf_no_param_count.argtypes = [c_void_p]
    L.pf_no_param_count.restype = ctypes.c_longlong
    L.pf_no_get_params.argtypes = [c_void_p, dp, c_size_t]
    L.pf_no_set_params.argtypes = [c_void_p, dp, c_size_t]
    L.pf_no_predict.argtypes = [c_void_p, c_int, dp, dp]
    L.pf_no_predict_mass.argtypes = [c_void_p, c_int, dp, dp, dp, dp, dp]
    L.pf_no_loss_grad.argtypes = [c_void_p, c_int, dp, dp, dp, dp]
    L.pf_no_train.argtypes = [c_void_p, c_int, dp, dp, c_int, c_int, c_double, ctypes.c_uint64, dp]
    L.pf_no_destroy.argtypes = [c_void_p]
    L.pf_no_destroy.restype = None
    L.pf_profile_read.argtypes = [c_void_p, dp, POINTER(ctypes.c_longlong)]
    L.pf_destroy.argtypes = [c_void_p]
    L.pf_destroy.restype = None
    L.pf_last_error.argtypes = [c_void_p]
    L.pf_last_error.restype = c_char_p
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, handle=None):
    if rc != PF_OK:
        msg = load().pf_last_error(handle)
        raise PfError(rc, msg.decode() if msg else "")


# ---- host-only helpers ----------------------------------------------------------------------
def gll(K: int):
    L = load()
    x, w, D = np.zeros(K + 1), np.zeros(K + 1), np.zeros((K + 1) * (K + 1))
    _check(L.pf_gll(K, _dp(x), _dp(w), _dp(D)))
    return x, w, D.reshape(K + 1, K + 1)


def nodes_1d(br, K: int, periodic: bool):
    L = load()
    br = _f64(br)
    ne = len(br) - 1
    n = ne * K if periodic else ne * K + 1
    out = np.zeros(n)
    _check(L.pf_nodes_1d(ne, _dp(br), K, int(periodic), _dp(out)))
    return out


def operators_1d(br, K: int, periodic: bool):
    L = load()
    br = _f64(br)
    ne = len(br) - 1
    n = ne * K if periodic else ne * K + 1
    Km, M = np.zeros((n, n)), np.zeros(n)
    _check(L.pf_operators_1d(ne, _dp(br), K, int(periodic), _dp(Km), _dp(M)))
    return Km, M


def fdm_1d(Kmat, Mdiag, dirichlet=None):
    L = load()
    Kmat, Mdiag = _f64(Kmat), _f64(Mdiag)
    n = len(Mdiag)
    mask = np.zeros(n, dtype=np.uint8) if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
    S, lam = np.zeros((n, n)), np.zeros(n)
    _check(L.pf_fdm_1d(n, _dp(Kmat), _dp(Mdiag), mask.ctypes.data_as(POINTER(c_ubyte)), _dp(S), _dp(lam)))
    return S, lam


PF_STATIC_MAX_VALUES = 1 << 20


def fdm_solve_static(nx: int, ny: int, nplanes: int, Sx, SxT, lam_x, Sy, SyT, lam_y, shift, rhs, out,
                     stream: Optional[int] = None):
    """Allocation-free FP64 fast-diagonalisation solve; every array argument is a device
    pointer (int), e.g. ``tensor.data_ptr()`` of a float64 CUDA tensor."""
    L = load()
    ptrs = [c_void_p(int(p)) for p in (Sx, SxT, lam_x, Sy, SyT, lam_y, shift, rhs, out)]
    rc = L.pf_fdm_solve_static(int(nx), int(ny), int(nplanes), *ptrs, c_void_p(stream or 0))
    _check(rc, None)


def measure_peaks() -> dict:
    """Measured TF32 tensor, FP32 FFMA and FP64 DFMA peaks of the current device (TFLOP/s)."""
    out = np.zeros(3)
    _check(load().pf_measure_peaks(_dp(out)))
    return {"tf32_tflops": float(out[0]), "fp32_tflops": float(out[1]), "fp64_tflops": float(out[2])}


# ---- the time stepper -------------------------------------------------------------------------
class Solver:
    """Owner of one ``pf_handle``: the device state of one two-phase dielectric run."""

    def __init__(self, xb, yb, order: int, nz: int, lz: float, fluid: dict, vbc: dict, scheme: dict,
                 phi0: np.ndarray, u0: Optional[np.ndarray] = None, stream: Optional[int] = None):
        L = load()
        self._xb, self._yb = _f64(xb), _f64(yb)
        self.mesh = PfMesh(len(self._xb) - 1, len(self._yb) - 1, _dp(self._xb), _dp(self._yb), int(order),
                           int(nz), float(lz))
        self.fluid = PfFluid(**{k: float(v) for k, v in fluid.items()})
        pats = tuple(vbc.get("patches", ()))
        self._patch = [_f64([p[c] for p in pats]) for c in range(3)]   # kept alive for pf_create
        self.vbc = PfVbc(int(vbc["bottom_kind"]), int(vbc["top_kind"]), float(vbc["v_bottom"]),
                         float(vbc["v_top"]), len(pats), *(_dp(a) for a in self._patch))
        self.scheme = PfScheme(float(scheme["dt"]), int(scheme.get("bdf", 2)), int(scheme.get("precision", PF_FP64)),
                               float(scheme.get("S", 0.0)), float(scheme.get("nu_m", 0.0)),
                               float(scheme.get("rho0", 0.0)), float(scheme.get("eps0", 0.0)),
                               int(scheme.get("model", PF_MODEL_FULL)))
        self.nx = self.mesh.ex * order
        self.ny = self.mesh.ey * order + 1
        self.nz = nz
        self.n = self.nx * self.ny * nz
        phi0 = _f64(phi0).ravel()
        if phi0.size != self.n:
            raise ValueError(f"phi0 has {phi0.size} values, expected {self.n}")
        u0p = None
        if u0 is not None:
            u0 = _f64(u0).ravel()
            if u0.size != 3 * self.n:
                raise ValueError("u0 must hold 3 blocks")
            u0p = _dp(u0)
        h = c_void_p()
        rc = L.pf_create(ctypes.byref(self.mesh), ctypes.byref(self.fluid), ctypes.byref(self.vbc),
                         ctypes.byref(self.scheme), _dp(phi0), u0p, c_void_p(stream or 0), ctypes.byref(h))
        _check(rc, None)
        self._h = h

    @property
    def handle(self):
        return self._h

    def step(self, n: int = 1):
        _check(load().pf_step(self._h, int(n)), self._h)

    def sync(self):
        _check(load().pf_sync(self._h), self._h)

    def get(self, mask: int) -> dict:
        names = [nm for bit, nms in _BLOCKS if mask & bit for nm in nms]
        out = np.zeros(len(names) * self.n)
        _check(load().pf_get_fields(self._h, int(mask), _dp(out), out.size), self._h)
        shp = (self.nz, self.ny, self.nx)
        return {nm: out[i * self.n:(i + 1) * self.n].reshape(shp) for i, nm in enumerate(names)}

    def get_into(self, mask: int, out: np.ndarray):
        """Copy fields into a caller-provided (e.g. pinned) float64 buffer, no allocation."""
        if out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array")
        _check(load().pf_get_fields(self._h, int(mask), _dp(out), out.size), self._h)
        return out

    def set(self, mask: int, data: np.ndarray, reset_history: bool = False):
        data = _f64(data).ravel()
        _check(load().pf_set_fields(self._h, int(mask), _dp(data), data.size, int(reset_history)), self._h)

    def set_step(self, nstep: int, t: float):
        """Restart bookkeeping: step count (BDF order of the next step) and time."""
        _check(load().pf_set_step(self._h, int(nstep), float(t)), self._h)

    def set_tc_accum(self, gemm: int, family: int, slices: int, sep: int):
        """Accumulation of the tensor-core transforms of variant gemm for a solve family (0: psi
        and phi, 1: V, P, u): K slices per TMEM group, and whether the correction products chain
        in a region of their own."""
        _check(load().pf_set_tc_accum(self._h, int(gemm), int(family), int(slices), int(sep)), self._h)

    def debug_tc_stall(self, wait_ns: int):
        """Test hook: the next tensor-core transform launch reports a time-out after wait_ns."""
        _check(load().pf_debug_tc_stall(self._h, int(wait_ns)), self._h)

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(8)
        _check(load().pf_diagnostics(self._h, _dp(out)), self._h)
        return out

    def solve_helmholtz(self, bcset: int, mode: int, lam: float, rhs: np.ndarray) -> np.ndarray:
        rhs = _f64(rhs).ravel()
        out = np.zeros_like(rhs)
        _check(load().pf_solve_helmholtz(self._h, int(bcset), int(mode), float(lam), _dp(rhs), _dp(out)), self._h)
        return out

    def autotune(self, steps: int = 5):
        """Pick the fastest transform variant, y pair and z-transform tile; returns
        (gemm + 1000 * tile + 100000 * fused_y, ms/step)."""
        ch = c_int()
        ms = np.zeros(1)
        _check(load().pf_autotune(self._h, int(steps), ctypes.byref(ch), _dp(ms)), self._h)
        return int(ch.value), float(ms[0])

    def set_variant(self, gemm: int, fuse_y: bool = True, tile: int = 0):
        """Pin the transform variant (a PF_GEMM_* code), the fused y pair and the z-transform tile."""
        _check(load().pf_set_variant(self._h, int(gemm), int(bool(fuse_y)), int(tile)), self._h)

    def profile(self, enable: bool):
        _check(load().pf_profile(self._h, int(bool(enable))), self._h)

    def profile_read(self):
        ms = np.zeros(len(KERNEL_CLASSES))
        ln = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        _check(load().pf_profile_read(self._h, _dp(ms), ln), self._h)
        return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def geometry(self):
        x, y = np.zeros(self.nx), np.zeros(self.ny)
        dims = (c_int * 4)()
        _check(load().pf_geometry(self._h, _dp(x), _dp(y), dims), self._h)
        return x, y, list(dims)

    def close(self):
        if getattr(self, "_h", None):
            load().pf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(wl, precision: int = PF_FP64, stream: Optional[int] = None, dt: Optional[float] = None,
                  phi0: Optional[np.ndarray] = None) -> Solver:
    """Create a Solver for a ``workloads.Workload`` (initial phi evaluated at this library's nodes)."""
    import workloads
    m, f, v, s = wl.mesh, wl.fluid, wl.vbc, wl.scheme
    x = nodes_1d(m.xb, m.order, True)
    y = nodes_1d(m.yb, m.order, False)
    z = None if m.nz == 1 else np.arange(m.nz) * m.lz / m.nz
    if phi0 is None:
        phi0 = workloads.eval_on_grid(wl.phi0, x, y, z)
    fluid = dict(rho1=f.rho1, rho2=f.rho2, mu1=f.mu1, mu2=f.mu2, eps1=f.eps1, eps2=f.eps2, sigma=f.sigma,
                 eta=f.eta, gamma1=f.gamma1, theta_s_deg=f.theta_s_deg)
    vbc = dict(bottom_kind=v.bottom_kind, top_kind=v.top_kind, v_bottom=v.v_bottom, v_top=v.v_top,
               patches=tuple(getattr(v, "patches", ())))
    scheme = dict(dt=s.dt if dt is None else dt, bdf=s.bdf, precision=precision, S=s.S, nu_m=s.nu_m,
                  rho0=s.rho0, eps0=s.eps0,
                  model=PF_MODEL_EQUILIBRIUM if getattr(s, "equilibrium", False) else PF_MODEL_FULL)
    return Solver(m.xb, m.yb, m.order, m.nz, m.lz, fluid, vbc, scheme, phi0, stream=stream)


# ---- ensembles of independent 2D runs --------------------------------------------------------
class Batch:
    """Owner of one ``pf_batch``: independent 2D runs advanced together (grouped by mesh)."""

    def __init__(self, workloads_list, precision: int = PF_FP64, stream: Optional[int] = None,
                 phi0_list=None):
        import workloads as _wl
        L = load()
        n = len(workloads_list)
        self.n = n
        self._keep = []
        meshes = (PfMesh * n)()
        fluids = (PfFluid * n)()
        vbcs = (PfVbc * n)()
        phis = (POINTER(c_double) * n)()
        self.shapes = []
        s0 = workloads_list[0].scheme
        for r, wl in enumerate(workloads_list):
            m, f, v = wl.mesh, wl.fluid, wl.vbc
            if m.nz != 1:
                raise ValueError("ensemble runs must be 2D")
            xb, yb = _f64(m.xb), _f64(m.yb)
            x = nodes_1d(xb, m.order, True)
            y = nodes_1d(yb, m.order, False)
            phi = _f64(_wl.eval_on_grid(wl.phi0, x, y, None) if phi0_list is None else phi0_list[r]).ravel()
            self._keep += [xb, yb, phi]
            meshes[r] = PfMesh(m.ex, m.ey, _dp(xb), _dp(yb), m.order, 1, 1.0)
            fluids[r] = PfFluid(f.rho1, f.rho2, f.mu1, f.mu2, f.eps1, f.eps2, f.sigma, f.eta, f.gamma1, f.theta_s_deg)
            vbcs[r] = PfVbc(v.bottom_kind, v.top_kind, v.v_bottom, v.v_top)
            phis[r] = _dp(phi)
            self.shapes.append((len(y), len(x)))
        self.scheme = PfScheme(s0.dt, s0.bdf, int(precision), s0.S, s0.nu_m, s0.rho0, s0.eps0,
                               PF_MODEL_EQUILIBRIUM if getattr(s0, "equilibrium", False) else PF_MODEL_FULL)
        h = c_void_p()
        _check(L.pf_batch_create(n, meshes, fluids, vbcs, ctypes.byref(self.scheme), phis, c_void_p(stream or 0),
                                 ctypes.byref(h)))
        self._h = h

    def step(self, n: int = 1):
        _check_b(load().pf_batch_step(self._h, int(n)), self._h)

    def umax(self):
        u, m = np.zeros(self.n), np.zeros(self.n)
        _check_b(load().pf_batch_umax(self._h, _dp(u), _dp(m)), self._h)
        return u, m

    def run_to_equilibrium(self, tol: float, max_steps: int, check_every: int = 100):
        out = (c_int * self.n)()
        _check_b(load().pf_batch_run_to_equilibrium(self._h, float(tol), int(max_steps), int(check_every), out), self._h)
        return np.array(list(out))

    def get(self, run: int, mask: int) -> dict:
        ny, nx = self.shapes[run]
        names = [nm for bit, nms in _BLOCKS if mask & bit for nm in nms]
        out = np.zeros(len(names) * nx * ny)
        _check_b(load().pf_batch_get_fields(self._h, int(run), int(mask), _dp(out), out.size), self._h)
        return {nm: out[i * nx * ny:(i + 1) * nx * ny].reshape(1, ny, nx) for i, nm in enumerate(names)}

    def groups(self):
        g = (c_int * self.n)()
        ng = load().pf_batch_groups(self._h, g)
        return ng, np.array(list(g))

    def set_variant(self, gemm: int, fuse_y: bool = True):
        rc = load().pf_batch_set_variant(self._h, int(gemm), int(bool(fuse_y)))
        if rc < 0:
            _check_b(rc, self._h)

    def autotune(self, steps: int = 5):
        ng, _ = self.groups()
        ms = np.zeros(max(1, ng))
        rc = load().pf_batch_autotune(self._h, int(steps), _dp(ms))
        if rc < 0:
            _check_b(rc, self._h)
        return ms[:ng]

    def close(self):
        if getattr(self, "_h", None):
            load().pf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_b(rc: int, h=None):
    if rc < 0:
        msg = load().pf_batch_last_error(h).decode() if h else ""
        raise PfError(rc, msg or "ensemble call failed")


# ---- neural operator (learned warm start) -------------------------------------------------------
class NeuralOperator:
    """tanh MLP: run parameters -> phase field on a uniform grid -> bilinear map to GLL nodes."""

    def __init__(self, dims, feat_mean, feat_std, grid, box, node_x, node_y, seed: int = 0,
                 stream: Optional[int] = None):
        L = load()
        self.dims = [int(d) for d in dims]
        d = (c_int * len(self.dims))(*self.dims)
        fm, fs = _f64(feat_mean), _f64(feat_std)
        nxv, nyv = _f64(node_x), _f64(node_y)
        self.nq = len(nxv) * len(nyv)
        h = c_void_p()
        _check(L.pf_no_create(len(self.dims), d, _dp(fm), _dp(fs), int(grid[0]), int(grid[1]), float(box[0]),
                              float(box[1]), float(box[2]), float(box[3]), len(nxv), len(nyv), _dp(nxv), _dp(nyv),
                              ctypes.c_uint64(seed), c_void_p(stream or 0), ctypes.byref(h)), None)
        self._h = h
        self.nparam = int(L.pf_no_param_count(h))

    def params(self):
        out = np.zeros(self.nparam)
        _check(load().pf_no_get_params(self._h, _dp(out), out.size), None)
        return out

    def set_params(self, p):
        p = _f64(p)
        _check(load().pf_no_set_params(self._h, _dp(p), p.size), None)

    def predict(self, feat):
        feat = _f64(feat).reshape(-1, self.dims[0])
        out = np.zeros((feat.shape[0], self.nq))
        _check(load().pf_no_predict(self._h, feat.shape[0], _dp(feat), _dp(out)), None)
        return out

    def predict_mass(self, feat, mass, wx, wy):
        """Predictions shifted to the phase masses ``mass`` (quadrature weights wx, wy)."""
        feat = _f64(feat).reshape(-1, self.dims[0])
        mass, wx, wy = _f64(mass).ravel(), _f64(wx).ravel(), _f64(wy).ravel()
        if mass.size != feat.shape[0]:
            raise ValueError("one target mass per feature row")
        out = np.zeros((feat.shape[0], self.nq))
        _check(load().pf_no_predict_mass(self._h, feat.shape[0], _dp(feat), _dp(mass), _dp(wx), _dp(wy),
                                         _dp(out)), None)
        return out

    def loss_grad(self, feat, target):
        feat = _f64(feat).reshape(-1, self.dims[0])
        target = _f64(target).reshape(feat.shape[0], self.nq)
        loss = np.zeros(1)
        grad = np.zeros(self.nparam)
        _check(load().pf_no_loss_grad(self._h, feat.shape[0], _dp(feat), _dp(target), _dp(loss), _dp(grad)), None)
        return float(loss[0]), grad

    def train(self, feat, target, batch: int = 64, epochs: int = 100, lr: float = 1e-3, seed: int = 0):
        feat = _f64(feat).reshape(-1, self.dims[0])
        target = _f64(target).reshape(feat.shape[0], self.nq)
        losses = np.zeros(max(1, epochs))
        _check(load().pf_no_train(self._h, feat.shape[0], _dp(feat), _dp(target), int(batch), int(epochs), float(lr),
                                  ctypes.c_uint64(seed), _dp(losses)), None)
        return losses[:epochs]

    def close(self):
        if getattr(self, "_h", None):
            load().pf_no_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
