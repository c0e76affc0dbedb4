"""Thin ctypes binding of libebpoisson (include/ebpoisson.h).

Argument marshalling only: every step of the geometry pass, the operator
construction, the multigrid solve and the field evaluation runs in the CUDA
library.  PyTorch provides device memory and streams.  There is no CPU
fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

EB_OK, EB_ERR_INVALID, EB_ERR_OOM, EB_ERR_NOT_CONVERGED, EB_ERR_CUDA, EB_ERR_TIMEOUT, EB_ERR_UNSUPPORTED, \
    EB_ERR_BUSY = range(8)
EB_PREC_FP64, EB_PREC_MIXED = 0, 1
EB_BOTTOM_RELAX, EB_BOTTOM_INV64, EB_BOTTOM_INV32, EB_BOTTOM_KRYLOV = 1, 2, 3, 4
BOTTOM_NAMES = {EB_BOTTOM_RELAX: "relax", EB_BOTTOM_INV64: "inverse_fp64", EB_BOTTOM_INV32: "inverse_fp32",
                EB_BOTTOM_KRYLOV: "bicgstab"}


class EBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Prim(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 10)]


class _Csg(C.Structure):
    _fields_ = [("op", C.c_int), ("a", C.c_int), ("b", C.c_int)]


class GeomDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("h", C.c_double),
                ("prims", C.POINTER(_Prim)), ("n_prims", C.c_int), ("nodes", C.POINTER(_Csg)), ("n_nodes", C.c_int),
                ("electrode_root", C.c_int), ("n_electrodes", C.c_int), ("electrode_node", C.c_int * 4),
                ("electrode_phi", C.c_double * 4), ("dielectric_root", C.c_int), ("eps_gas", C.c_double),
                ("eps_diel", C.c_double), ("bc_type", C.c_int * 6), ("bc_value", C.c_double * 6),
                ("bc_robin", C.c_double * 12), ("electrode_robin", C.c_int), ("electrode_robin_a", C.c_double * 2),
                ("helmholtz_lam", C.c_double * 2)]


class GeomInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_phase", C.c_int), ("n_cells", C.c_longlong), ("n_dof", C.c_longlong),
                ("n_eb", C.c_longlong), ("n_irregular", C.c_longlong), ("n_levels", C.c_int),
                ("level_n", (C.c_int * 3) * 16), ("stencil_order", C.c_longlong * 3), ("device_bytes", C.c_longlong)]


class GeomArrays(C.Structure):
    _fields_ = [("flags", C.c_void_p), ("kappa", C.c_void_p), ("eb_cell", C.c_void_p), ("eb_area", C.c_void_p),
                ("eb_normal", C.c_void_p), ("eb_centroid", C.c_void_p), ("eb_kind", C.c_void_p),
                ("stencil_order", C.c_void_p)]


class SolverOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("precision", C.c_int), ("inner_cycles", C.c_int), ("bottom_sweeps", C.c_int), ("launch_mode", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("vcycles", C.c_int), ("rel_res", C.c_double),
                ("bnorm", C.c_double), ("kernel_launches", C.c_longlong), ("kernel_ms", C.c_double),
                ("bottom", C.c_int), ("levels", C.c_int), ("sweep_levels", C.c_int)]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("max_slots", C.c_int), ("queue_cap", C.c_int),
                ("step_iters", C.c_int), ("device", C.c_int), ("solver", SolverOpts)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("queued", C.c_longlong), ("active", C.c_longlong), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("cells_per_s", C.c_double), ("cells_completed", C.c_longlong), ("hbm_budget", C.c_longlong),
                ("hbm_used", C.c_longlong), ("hbm_peak", C.c_longlong), ("steps", C.c_longlong),
                ("estimate_misses", C.c_longlong)]


EXPORTS = ["eb_status_str", "eb_last_error", "eb_geom_build", "eb_geom_query", "eb_geom_destroy", "eb_geom_export",
           "eb_solver_opts_default", "eb_poisson_setup", "eb_poisson_destroy", "eb_poisson_residual",
           "eb_poisson_solve", "eb_field_eval", "eb_poisson_profile", "eb_poisson_trace",
           "eb_poisson_residual_noalloc", "eb_poisson_solve_batched", "eb_server_opts_default", "eb_server_create",
           "eb_server_submit", "eb_server_poll", "eb_server_wait", "eb_server_query", "eb_server_destroy",
           "eb_amr_setup", "eb_amr_query", "eb_amr_residual", "eb_amr_solve", "eb_amr_kernel_stats",
           "eb_amr_destroy", "eb_amr_setup_levels", "eb_amr_level_query", "eb_amr_level_geom",
           "eb_amr_residual_levels", "eb_amr_solve_levels", "eb_amr_field_eval", "eb_tag_cells", "eb_regrid_box",
           "eb_device_fma_rates", "eb_tga_coefficients", "eb_tga_create",
           "eb_tga_step", "eb_tga_destroy"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libebpoisson.so; raises if it is not built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {path} is not built: run __graft_entry__.build()")
            _build.build()
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.eb_status_str.restype = C.c_char_p
        lib.eb_status_str.argtypes = [C.c_int]
        lib.eb_last_error.restype = C.c_char_p
        lib.eb_geom_build.restype = C.c_int
        lib.eb_geom_build.argtypes = [C.POINTER(GeomDesc), P, C.POINTER(P)]
        lib.eb_geom_query.restype = C.c_int
        lib.eb_geom_query.argtypes = [P, C.POINTER(GeomInfo)]
        lib.eb_geom_destroy.argtypes = [P]
        lib.eb_geom_export.restype = C.c_int
        lib.eb_geom_export.argtypes = [P, C.POINTER(GeomArrays), P]
        lib.eb_solver_opts_default.argtypes = [C.POINTER(SolverOpts)]
        lib.eb_poisson_setup.restype = C.c_int
        lib.eb_poisson_setup.argtypes = [P, C.POINTER(SolverOpts), P, C.POINTER(P)]
        lib.eb_poisson_destroy.argtypes = [P]
        lib.eb_poisson_residual.restype = C.c_int
        lib.eb_poisson_residual.argtypes = [P, P, P, P, P, P]
        lib.eb_poisson_solve.restype = C.c_int
        lib.eb_poisson_solve.argtypes = [P, P, P, P, C.POINTER(SolveInfo), P]
        lib.eb_field_eval.restype = C.c_int
        lib.eb_field_eval.argtypes = [P, P, P, P, P, P]
        lib.eb_poisson_solve_batched.restype = C.c_int
        lib.eb_poisson_solve_batched.argtypes = [P, C.c_int, P, P, P, C.POINTER(SolveInfo), P]
        lib.eb_poisson_residual_noalloc.restype = C.c_int
        lib.eb_poisson_residual_noalloc.argtypes = [P, P, P, P, P, P]
        lib.eb_poisson_trace.restype = C.c_int
        lib.eb_poisson_trace.argtypes = [P, C.POINTER(C.c_double), C.c_int]
        lib.eb_poisson_profile.restype = C.c_int
        lib.eb_poisson_profile.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), P]
        lib.eb_amr_setup.restype = C.c_int
        lib.eb_amr_setup.argtypes = [C.POINTER(GeomDesc), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(SolverOpts), P, C.POINTER(P)]
        lib.eb_amr_query.restype = C.c_int
        lib.eb_amr_query.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                     C.POINTER(C.c_longlong)]
        lib.eb_amr_residual.restype = C.c_int
        lib.eb_amr_residual.argtypes = [P] + [P] * 8 + [P]
        lib.eb_amr_solve.restype = C.c_int
        lib.eb_amr_solve.argtypes = [P] + [P] * 6 + [C.POINTER(SolveInfo), P]
        lib.eb_amr_destroy.argtypes = [P]
        lib.eb_amr_kernel_stats.restype = C.c_int
        lib.eb_amr_kernel_stats.argtypes = [P, C.POINTER(C.c_double)]
        lib.eb_amr_setup_levels.restype = C.c_int
        lib.eb_amr_setup_levels.argtypes = [C.POINTER(GeomDesc), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(SolverOpts), P, C.POINTER(P)]
        lib.eb_amr_level_query.restype = C.c_int
        lib.eb_amr_level_query.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                           C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                           C.POINTER(C.c_longlong)]
        lib.eb_amr_level_geom.restype = C.c_int
        lib.eb_amr_level_geom.argtypes = [P, C.c_int, C.POINTER(P)]
        lib.eb_amr_residual_levels.restype = C.c_int
        lib.eb_amr_residual_levels.argtypes = [P, P, P, P, P, P]
        lib.eb_amr_solve_levels.restype = C.c_int
        lib.eb_amr_solve_levels.argtypes = [P, P, P, P, C.POINTER(SolveInfo), P]
        lib.eb_amr_field_eval.restype = C.c_int
        lib.eb_amr_field_eval.argtypes = [P, C.c_int, P, P, P, P, P]
        lib.eb_tag_cells.restype = C.c_int
        lib.eb_tag_cells.argtypes = [P, P, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int), P,
                                     C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                     C.POINTER(C.c_double), P]
        lib.eb_regrid_box.restype = C.c_int
        lib.eb_regrid_box.argtypes = [C.c_int] + [C.POINTER(C.c_int)] * 5 + [C.c_longlong, C.c_int, C.c_int,
                                                                            C.POINTER(C.c_int), C.POINTER(C.c_int),
                                                                            C.POINTER(C.c_int)]
        lib.eb_device_fma_rates.restype = C.c_int
        lib.eb_device_fma_rates.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.eb_tga_coefficients.restype = C.c_int
        lib.eb_tga_coefficients.argtypes = [C.c_double, C.POINTER(C.c_double)]
        lib.eb_tga_create.restype = C.c_int
        lib.eb_tga_create.argtypes = [P] * 6 + [C.c_double, P, C.POINTER(P)]
        lib.eb_tga_step.restype = C.c_int
        lib.eb_tga_step.argtypes = [P, P, P, P, C.c_double, C.POINTER(SolveInfo), P]
        lib.eb_tga_destroy.argtypes = [P]
        lib.eb_server_opts_default.argtypes = [C.POINTER(ServerOpts)]
        lib.eb_server_create.restype = C.c_int
        lib.eb_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(P)]
        lib.eb_server_submit.restype = C.c_int
        lib.eb_server_submit.argtypes = [P, C.POINTER(GeomDesc), P, P, C.POINTER(C.c_ulonglong)]
        lib.eb_server_poll.restype = C.c_int
        lib.eb_server_poll.argtypes = [P, C.c_ulonglong, P, C.POINTER(SolveInfo)]
        lib.eb_server_wait.restype = C.c_int
        lib.eb_server_wait.argtypes = [P, C.c_ulonglong, C.c_double, P, C.POINTER(SolveInfo)]
        lib.eb_server_query.restype = C.c_int
        lib.eb_server_query.argtypes = [P, C.POINTER(ServerStats)]
        lib.eb_server_destroy.argtypes = [P]
        _lib = lib
        return lib


def _check(st: int, what: str):
    if st != EB_OK:
        lib = load()
        raise EBError(st, f"{what}: {lib.eb_status_str(st).decode()}: {lib.eb_last_error().decode()}")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _dev(t, dtype, device):
    if t is None:
        return None
    t = torch.as_tensor(t)
    return t.to(device=device, dtype=dtype).contiguous()


def make_desc(desc: dict):
    """Problem dict (see workloads.py) -> GeomDesc plus the arrays it points to."""
    prims = (_Prim * max(1, len(desc["prims"])))()
    for i, (k, p) in enumerate(desc["prims"]):
        prims[i].kind = int(k)
        for j, v in enumerate(p):
            prims[i].p[j] = float(v)
    nodes = (_Csg * max(1, len(desc["nodes"])))()
    for i, (op, a, b) in enumerate(desc["nodes"]):
        nodes[i].op, nodes[i].a, nodes[i].b = int(op), int(a), int(b)
    d = GeomDesc()
    d.dim = int(desc["dim"])
    for k in range(3):
        d.n[k] = int(desc["n"][k]) if k < len(desc["n"]) else 1
        d.lo[k] = float(desc["lo"][k]) if k < len(desc["lo"]) else 0.0
    d.h = float(desc["h"])
    d.prims = C.cast(prims, C.POINTER(_Prim))
    d.n_prims = len(desc["prims"])
    d.nodes = C.cast(nodes, C.POINTER(_Csg))
    d.n_nodes = len(desc["nodes"])
    d.electrode_root = int(desc.get("root_E", -1))
    elec = desc.get("electrodes")
    if elec is None:
        elec = [(d.electrode_root, desc.get("phi_E", 0.0))] if d.electrode_root >= 0 else []
    d.n_electrodes = len(elec)
    for i, (r, v) in enumerate(elec):
        d.electrode_node[i] = int(r)
        d.electrode_phi[i] = float(v)
    d.dielectric_root = int(desc.get("root_D", -1))
    d.eps_gas, d.eps_diel = float(desc["eps"][0]), float(desc["eps"][1])
    for k in range(6):
        d.bc_type[k] = int(desc["bc"][k])
        d.bc_value[k] = float(desc.get("phi_wall", [0.0] * 6)[k])
    rob = desc.get("robin")
    if rob is not None:  # Robin walls: a1, a2 per side (phi_wall holds a3)
        for k in range(6):
            d.bc_robin[2 * k], d.bc_robin[2 * k + 1] = float(rob[k][0]), float(rob[k][1])
    ebr = desc.get("eb_robin")
    if ebr is not None:  # Robin electrodes: a1, a2 (the electrode values are a3)
        d.electrode_robin = 1
        d.electrode_robin_a[0], d.electrode_robin_a[1] = float(ebr[0]), float(ebr[1])
    lam = desc.get("lam", (0.0, 0.0))
    d.helmholtz_lam[0], d.helmholtz_lam[1] = float(lam[0]), float(lam[1])
    return d, (prims, nodes)


# ------------------------------------------------------------- C-ABI mirrors

def eb_geom_build(desc: dict, stream=None):
    lib = load()
    d, keep = make_desc(desc)
    h = C.c_void_p()
    _check(lib.eb_geom_build(C.byref(d), _stream(stream), C.byref(h)), "eb_geom_build")
    del keep
    return h


def eb_geom_query(handle) -> dict:
    lib = load()
    info = GeomInfo()
    _check(lib.eb_geom_query(handle, C.byref(info)), "eb_geom_query")
    return dict(dim=info.dim, n_phase=info.n_phase, n_cells=info.n_cells, n_dof=info.n_dof, n_eb=info.n_eb,
                n_irregular=info.n_irregular, n_levels=info.n_levels,
                level_n=[tuple(info.level_n[l]) for l in range(info.n_levels)],
                stencil_order=dict(order2=info.stencil_order[0], order1=info.stencil_order[1],
                                   ls=info.stencil_order[2]), device_bytes=info.device_bytes)


def eb_solver_opts_default() -> SolverOpts:
    o = SolverOpts()
    load().eb_solver_opts_default(C.byref(o))
    return o


def eb_poisson_setup(geom_handle, opts: SolverOpts | None = None, stream=None):
    lib = load()
    h = C.c_void_p()
    _check(lib.eb_poisson_setup(geom_handle, C.byref(opts) if opts is not None else None, _stream(stream),
                                C.byref(h)), "eb_poisson_setup")
    return h


def eb_poisson_residual(handle, rhs, sigma, phi, out, stream=None):
    _check(load().eb_poisson_residual(handle, _ptr(rhs), _ptr(sigma), _ptr(phi), _ptr(out), _stream(stream)),
           "eb_poisson_residual")


def eb_poisson_residual_noalloc(geom_handle, rhs, sigma, phi, out, stream=None):
    """Residual b - A phi without any device allocation (static scratch, see the header)."""
    _check(load().eb_poisson_residual_noalloc(geom_handle, _ptr(rhs), _ptr(sigma), _ptr(phi), _ptr(out),
                                              _stream(stream)), "eb_poisson_residual_noalloc")


def eb_poisson_solve(handle, rhs, sigma, phi, stream=None) -> dict:
    info = SolveInfo()
    st = load().eb_poisson_solve(handle, _ptr(rhs), _ptr(sigma), _ptr(phi), C.byref(info), _stream(stream))
    if st not in (EB_OK, EB_ERR_NOT_CONVERGED):
        _check(st, "eb_poisson_solve")
    return dict(status=info.status, outer_iters=info.outer_iters, vcycles=info.vcycles, rel_res=info.rel_res,
                bnorm=info.bnorm, kernel_launches=info.kernel_launches, kernel_ms=info.kernel_ms,
                bottom=BOTTOM_NAMES.get(info.bottom, "none"), levels=info.levels,
                sweep_levels=info.sweep_levels)


def device_fma_rates(device: int = 0):
    """Measured FP64 and FP32 fused multiply-add rates of a device, TFLOP/s."""
    f64, f32 = C.c_double(), C.c_double()
    _check(load().eb_device_fma_rates(int(device), C.byref(f64), C.byref(f32)), "eb_device_fma_rates")
    return f64.value, f32.value


def eb_poisson_profile(handle, kernel: int, reps: int, stream=None):
    ms, by = C.c_double(), C.c_double()
    _check(load().eb_poisson_profile(handle, kernel, reps, C.byref(ms), C.byref(by), _stream(stream)),
           "eb_poisson_profile")
    return ms.value, by.value


def _info_dict(info):
    return dict(status=info.status, outer_iters=info.outer_iters, vcycles=info.vcycles, rel_res=info.rel_res,
                bnorm=info.bnorm, kernel_launches=info.kernel_launches, kernel_ms=info.kernel_ms,
                bottom=BOTTOM_NAMES.get(info.bottom, "none"), levels=info.levels,
                sweep_levels=info.sweep_levels)


def eb_poisson_solve_batched(handles, rhs, sigma, phi, stream=None) -> list:
    """n independent solves in one persistent launch; lists of handles and device tensors."""
    n = len(handles)
    arr = lambda xs: (C.c_void_p * max(n, 1))(*[(x.value if isinstance(x, C.c_void_p) else  # noqa: E731
                                                  (x.data_ptr() if x is not None else 0)) for x in xs])
    hs, rs, ss, ps = arr(handles), arr(rhs), arr(sigma if sigma is not None else [None] * n), arr(phi)
    infos = (SolveInfo * max(n, 1))()
    st = load().eb_poisson_solve_batched(C.cast(hs, C.c_void_p), n, C.cast(rs, C.c_void_p), C.cast(ss, C.c_void_p),
                                         C.cast(ps, C.c_void_p), infos, _stream(stream))
    if st not in (EB_OK, EB_ERR_NOT_CONVERGED):
        _check(st, "eb_poisson_solve_batched")
    return [_info_dict(infos[i]) for i in range(n)]


def eb_field_eval(handle, phi, sigma, E, En, stream=None):
    _check(load().eb_field_eval(handle, _ptr(phi), _ptr(sigma), _ptr(E), _ptr(En), _stream(stream)),
           "eb_field_eval")


def eb_tga_coefficients(dt):
    mu = (C.c_double * 4)()
    _check(load().eb_tga_coefficients(float(dt), mu), "eb_tga_coefficients")
    return [mu[k] for k in range(4)]


def eb_tga_create(g0, g1, g2, p0, p1, p2, dt, stream=None):
    h = C.c_void_p()
    _check(load().eb_tga_create(g0, g1, g2, p0, p1, p2, float(dt), _stream(stream), C.byref(h)), "eb_tga_create")
    return h


def eb_tga_step(handle, phi, rho, out, tol, stream=None):
    infos = (SolveInfo * 2)()
    st = load().eb_tga_step(handle, _ptr(phi), _ptr(rho), _ptr(out), float(tol), infos, _stream(stream))
    if st not in (EB_OK, EB_ERR_NOT_CONVERGED):
        _check(st, "eb_tga_step")
    return [_info_dict(infos[k]) for k in range(2)]


# ------------------------------------------------------------- convenience

class Geometry:
    """Cut-cell geometry and the multigrid hierarchy of one problem (owns an eb_geom)."""

    def __init__(self, desc: dict, device="cuda", stream=None):
        self.desc = desc
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self._h = eb_geom_build(desc, stream)
        self.info = eb_geom_query(self._h)
        self.ncell = int(self.info["n_cells"])
        self.dim = int(desc["dim"])

    def export(self, stream=None) -> dict:
        n, neb = self.ncell, int(self.info["n_eb"])
        dev = self.device
        out = dict(flags=torch.empty(n, dtype=torch.uint8, device=dev),
                   kappa=torch.empty(2, n, dtype=torch.float64, device=dev),
                   eb_cell=torch.empty(max(neb, 1), dtype=torch.int32, device=dev),
                   eb_area=torch.empty(max(neb, 1), dtype=torch.float64, device=dev),
                   eb_normal=torch.empty(max(neb, 1), 3, dtype=torch.float64, device=dev),
                   eb_centroid=torch.empty(max(neb, 1), 3, dtype=torch.float64, device=dev),
                   eb_kind=torch.empty(max(neb, 1), dtype=torch.uint8, device=dev),
                   stencil_order=torch.empty(max(neb, 1), 2, dtype=torch.int32, device=dev))
        a = GeomArrays(*[C.c_void_p(out[k].data_ptr()) for k in
                         ("flags", "kappa", "eb_cell", "eb_area", "eb_normal", "eb_centroid", "eb_kind",
                          "stencil_order")])
        _check(load().eb_geom_export(self._h, C.byref(a), _stream(stream)), "eb_geom_export")
        for k in list(out):
            if k.startswith("eb_") or k == "stencil_order":
                out[k] = out[k][:neb]
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().eb_geom_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(solvers, rhs, sigma=None, phi=None, stream=None):
    """Batched solve over Poisson objects; returns (phis, infos)."""
    rhs_d, sig_d, phis = [], [], []
    for k, P in enumerate(solvers):
        r, s = P._fields(rhs[k], None if sigma is None else sigma[k])
        rhs_d.append(r)
        sig_d.append(s)
        phis.append(torch.zeros(2, P.geom.ncell, dtype=torch.float64, device=P.geom.device) if phi is None
                    else phi[k])
    infos = eb_poisson_solve_batched([P._h for P in solvers], rhs_d, sig_d, phis, stream)
    return phis, infos


class Poisson:
    """Multigrid solver bound to a Geometry (owns an eb_poisson)."""

    def __init__(self, geom: Geometry, *, precision="mixed", tol=1e-10, max_cycles=100, nu1=-1, nu2=-1,
                 inner_cycles=2, bottom_sweeps=64, launch_mode=0, stream=None):
        self.geom = geom
        o = eb_solver_opts_default()
        o.tol, o.max_cycles, o.nu1, o.nu2 = tol, max_cycles, nu1, nu2
        o.precision = EB_PREC_MIXED if precision == "mixed" else EB_PREC_FP64
        o.inner_cycles, o.bottom_sweeps, o.launch_mode = inner_cycles, bottom_sweeps, int(launch_mode)
        self.opts = o
        with torch.cuda.device(geom.device):
            self._h = eb_poisson_setup(geom._h, o, stream)

    def _fields(self, rhs, sigma):
        n, dev = self.geom.ncell, self.geom.device
        rhs = _dev(rhs, torch.float64, dev)
        if rhs.dim() == 1:
            rhs = torch.stack([rhs, torch.zeros_like(rhs)])
        rhs = rhs.reshape(2, n).contiguous()
        sigma = _dev(sigma, torch.float64, dev)
        if sigma is not None:
            sigma = sigma.reshape(n).contiguous()
        return rhs, sigma

    def residual(self, rhs, sigma, phi, stream=None):
        rhs, sigma = self._fields(rhs, sigma)
        phi = _dev(phi, torch.float64, self.geom.device).reshape(2, -1).contiguous()
        out = torch.empty_like(phi)
        eb_poisson_residual(self._h, rhs, sigma, phi, out, stream)
        return out

    def solve(self, rhs, sigma=None, phi=None, stream=None):
        rhs, sigma = self._fields(rhs, sigma)
        if phi is None:
            phi = torch.zeros(2, self.geom.ncell, dtype=torch.float64, device=self.geom.device)
        info = eb_poisson_solve(self._h, rhs, sigma, phi, stream)
        return phi, info

    def field(self, phi, sigma=None, stream=None):
        n, neb = self.geom.ncell, int(self.geom.info["n_eb"])
        dev = self.geom.device
        phi = _dev(phi, torch.float64, dev).reshape(2, n).contiguous()
        sigma = _dev(sigma, torch.float64, dev)
        E = torch.empty(self.geom.dim, 2, n, dtype=torch.float64, device=dev)
        En = torch.empty(max(neb, 1), 2, dtype=torch.float64, device=dev)
        eb_field_eval(self._h, phi, sigma, E, En, stream)
        return E, En[:neb]

    def profile(self, kernel: int, reps: int = 50, stream=None):
        """(ms per launch, algorithmic bytes per launch) of a finest-level kernel."""
        return eb_poisson_profile(self._h, kernel, reps, stream)

    def trace(self):
        """Phases of the first V-cycle of the last solve: list of (level, kind, ms)."""
        cap = 2 * 4096 + 1
        v = (C.c_double * cap)()
        _check(load().eb_poisson_trace(self._h, v, cap), "eb_poisson_trace")
        m = int(v[0])
        return [(int(v[1 + 2 * i]) >> 4, int(v[1 + 2 * i]) & 15, v[2 + 2 * i]) for i in range(m)]

    def close(self):
        if getattr(self, "_h", None):
            load().eb_poisson_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (owns an eb_server and its worker thread).

    submit() copies the request and returns a ticket at once; poll() returns
    None until the result is ready, then (phi [2][n_cells] numpy, info)."""

    def __init__(self, *, hbm_budget_bytes=0.0, max_slots=64, queue_cap=1 << 16, step_iters=1, device=0,
                 precision="mixed", tol=1e-10, max_cycles=200, nu1=-1, nu2=-1, inner_cycles=2):
        lib = load()
        o = ServerOpts()
        lib.eb_server_opts_default(C.byref(o))
        o.hbm_budget_bytes, o.max_slots, o.queue_cap = float(hbm_budget_bytes), max_slots, queue_cap
        o.step_iters, o.device = step_iters, device
        o.solver.tol, o.solver.max_cycles, o.solver.nu1, o.solver.nu2 = tol, max_cycles, nu1, nu2
        o.solver.precision = EB_PREC_MIXED if precision == "mixed" else EB_PREC_FP64
        o.solver.inner_cycles = inner_cycles
        h = C.c_void_p()
        _check(lib.eb_server_create(C.byref(o), C.byref(h)), "eb_server_create")
        self._h = h
        self._n = {}

    def submit(self, desc: dict, rhs, sigma=None):
        """Queue one solve; rhs [2][n_cells] (or [n_cells]) and sigma [n_cells] as host arrays.
        Raises EBError(EB_ERR_BUSY) when the queue is full."""
        import numpy as np
        d, keep = make_desc(desc)
        n = int(np.prod([int(desc["n"][k]) for k in range(int(desc["dim"]))]))
        r = np.ascontiguousarray(np.asarray(rhs, dtype=np.float64))
        if r.ndim == 1:
            r = np.stack([r, np.zeros_like(r)])
        r = np.ascontiguousarray(r.reshape(2, n))
        sg = None if sigma is None else np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(n))
        t = C.c_ulonglong()
        _check(load().eb_server_submit(self._h, C.byref(d), C.c_void_p(r.ctypes.data),
                                       C.c_void_p(sg.ctypes.data) if sg is not None else C.c_void_p(0),
                                       C.byref(t)), "eb_server_submit")
        self._n[t.value] = n
        return t.value

    def _take(self, fn, ticket, *extra):
        import numpy as np
        n = self._n.get(ticket, 0)  # unknown tickets: the library reports them
        phi = np.zeros((2, n))
        info = SolveInfo()
        st = fn(self._h, C.c_ulonglong(ticket), *extra, C.c_void_p(phi.ctypes.data), C.byref(info))
        if st == EB_ERR_BUSY:
            return None
        _check(st, "eb_server_poll")
        self._n.pop(ticket, None)
        return phi, _info_dict(info)

    def poll(self, ticket):
        return self._take(load().eb_server_poll, ticket)

    def wait(self, ticket, timeout_s=600.0):
        return self._take(load().eb_server_wait, ticket, C.c_double(timeout_s))

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().eb_server_query(self._h, C.byref(s)), "eb_server_query")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().eb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Composite:
    """Composite grid: one ratio-2 refined box over coarse cells [box_lo, box_hi) (owns an eb_amr)."""

    def __init__(self, desc: dict, box_lo, box_hi, *, precision="mixed", tol=1e-10, max_cycles=100, nu1=-1, nu2=-1,
                 inner_cycles=2, bottom_sweeps=64, device=None, stream=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        d, keep = make_desc(desc)
        o = eb_solver_opts_default()
        o.tol, o.max_cycles, o.nu1, o.nu2 = tol, max_cycles, nu1, nu2
        o.precision = EB_PREC_MIXED if precision == "mixed" else EB_PREC_FP64
        o.inner_cycles, o.bottom_sweeps = inner_cycles, bottom_sweeps
        lo = (C.c_int * 3)(*[int(v) for v in (list(box_lo) + [0] * 3)[:3]])
        hi = (C.c_int * 3)(*[int(v) for v in (list(box_hi) + [1] * 3)[:3]])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(load().eb_amr_setup(C.byref(d), lo, hi, C.byref(o), _stream(stream), C.byref(h)), "eb_amr_setup")
        self._h = h
        nc, nf, nfa = C.c_longlong(), C.c_longlong(), C.c_longlong()
        fn = (C.c_int * 3)()
        _check(load().eb_amr_query(h, C.byref(nc), C.byref(nf), fn, C.byref(nfa)), "eb_amr_query")
        self.n_coarse, self.n_fine, self.fine_n, self.cf_faces = nc.value, nf.value, tuple(fn), nfa.value

    def _f(self, x, n):
        if x is None:
            return None
        x = _dev(x, torch.float64, self.device)
        if x.dim() == 1 and x.numel() == n:
            return x.contiguous()
        return x.reshape(2, n).contiguous()

    def residual(self, rhs_c, sig_c, rhs_f, sig_f, phi_c, phi_f, stream=None):
        nc, nf = self.n_coarse, self.n_fine
        args = [self._f(rhs_c, nc), self._f(sig_c, nc), self._f(rhs_f, nf), self._f(sig_f, nf),
                self._f(phi_c, nc), self._f(phi_f, nf)]
        rc = torch.empty(2, nc, dtype=torch.float64, device=self.device)
        rf = torch.empty(2, nf, dtype=torch.float64, device=self.device)
        _check(load().eb_amr_residual(self._h, *[_ptr(a) for a in args], _ptr(rc), _ptr(rf), _stream(stream)),
               "eb_amr_residual")
        return rc, rf

    def solve(self, rhs_c, rhs_f, sig_c=None, sig_f=None, phi_c=None, phi_f=None, stream=None):
        nc, nf = self.n_coarse, self.n_fine
        pc = torch.zeros(2, nc, dtype=torch.float64, device=self.device) if phi_c is None else self._f(phi_c, nc)
        pf = torch.zeros(2, nf, dtype=torch.float64, device=self.device) if phi_f is None else self._f(phi_f, nf)
        info = SolveInfo()
        # keep the converted inputs alive until the call returns
        ins = [self._f(rhs_c, nc), self._f(sig_c, nc), self._f(rhs_f, nf), self._f(sig_f, nf)]
        st = load().eb_amr_solve(self._h, *[_ptr(a) for a in ins], _ptr(pc), _ptr(pf), C.byref(info),
                                 _stream(stream))
        if st not in (EB_OK, EB_ERR_NOT_CONVERGED):
            _check(st, "eb_amr_solve")
        return pc, pf, _info_dict(info)

    def kernel_stats(self):
        """Persistent multigrid launches of the last solve: {"coarse": ..., "fine": ...}, each with
        launches, kernel_ms, vcycles, outer."""
        out = (C.c_double * 8)()
        _check(load().eb_amr_kernel_stats(self._h, out), "eb_amr_kernel_stats")
        keys = ("launches", "kernel_ms", "vcycles", "outer")
        return {w: {k: out[4 * i + j] for j, k in enumerate(keys)} for i, w in enumerate(("coarse", "fine"))}

    def close(self):
        if getattr(self, "_h", None):
            load().eb_amr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Composite grid of nested ratio-2 boxes, one per level (owns an eb_amr).

    boxes: [(lo, hi), ...] for levels 1.., each over cells of its parent level's grid counted from
    that grid's lower corner."""

    def __init__(self, desc: dict, boxes, *, precision="mixed", tol=1e-10, max_cycles=100, nu1=-1, nu2=-1,
                 inner_cycles=2, device=None, stream=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.desc = desc
        self.dim = int(desc["dim"])
        d, keep = make_desc(desc)
        o = eb_solver_opts_default()
        o.tol, o.max_cycles, o.nu1, o.nu2 = tol, max_cycles, nu1, nu2
        o.precision = EB_PREC_MIXED if precision == "mixed" else EB_PREC_FP64
        o.inner_cycles = inner_cycles
        self.boxes = [([int(v) for v in (list(lo) + [0] * 3)[:3]], [int(v) for v in (list(hi) + [1] * 3)[:3]])
                      for lo, hi in boxes]
        nb_ = len(self.boxes)
        lo = (C.c_int * (3 * max(nb_, 1)))(*[v for b in self.boxes for v in b[0]])
        hi = (C.c_int * (3 * max(nb_, 1)))(*[v for b in self.boxes for v in b[1]])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(load().eb_amr_setup_levels(C.byref(d), nb_ + 1, lo, hi, C.byref(o), _stream(stream),
                                              C.byref(h)), "eb_amr_setup_levels")
        self._h = h
        self.levels = []
        for l in range(nb_ + 1):
            nl, nc, faces = C.c_int(), C.c_longlong(), C.c_longlong()
            n3, lo3, hh = (C.c_int * 3)(), (C.c_double * 3)(), C.c_double()
            _check(load().eb_amr_level_query(h, l, C.byref(nl), C.byref(nc), n3, lo3, C.byref(hh), C.byref(faces)),
                   "eb_amr_level_query")
            self.levels.append(dict(n_cells=nc.value, n=tuple(n3), lo=tuple(lo3), h=hh.value, cf_faces=faces.value))
        self.L = nb_ + 1

    def level_desc(self, l):
        """The level's grid as a description (for cell centres)."""
        out = dict(self.desc)
        out.update(n=self.levels[l]["n"], lo=self.levels[l]["lo"], h=self.levels[l]["h"])
        return out

    def level_geom(self, l):
        g = C.c_void_p()
        _check(load().eb_amr_level_geom(self._h, l, C.byref(g)), "eb_amr_level_geom")
        return g

    def _f(self, x, l):
        n = self.levels[l]["n_cells"]
        if x is None:
            return None
        x = _dev(x, torch.float64, self.device)
        return x.reshape(2, n).contiguous()

    @staticmethod
    def _arr(ts):
        return (C.c_void_p * len(ts))(*[(t.data_ptr() if t is not None else 0) for t in ts])

    def residual(self, rhs, sig, phi, stream=None):
        L = self.L
        ins = [[self._f(v[l] if v is not None else None, l) for l in range(L)] for v in (rhs, sig, phi)]
        r = [torch.empty(2, self.levels[l]["n_cells"], dtype=torch.float64, device=self.device) for l in range(L)]
        _check(load().eb_amr_residual_levels(self._h, C.cast(self._arr(ins[0]), C.c_void_p),
                                             C.cast(self._arr(ins[1]), C.c_void_p),
                                             C.cast(self._arr(ins[2]), C.c_void_p), C.cast(self._arr(r), C.c_void_p),
                                             _stream(stream)), "eb_amr_residual_levels")
        return r

    def solve(self, rhs, sig=None, phi=None, stream=None):
        L = self.L
        rs = [self._f(rhs[l], l) for l in range(L)]
        ss = [self._f(sig[l] if sig is not None else None, l) for l in range(L)]
        ps = [torch.zeros(2, self.levels[l]["n_cells"], dtype=torch.float64, device=self.device) if phi is None
              else self._f(phi[l], l).clone() for l in range(L)]
        info = SolveInfo()
        st = load().eb_amr_solve_levels(self._h, C.cast(self._arr(rs), C.c_void_p), C.cast(self._arr(ss), C.c_void_p),
                                        C.cast(self._arr(ps), C.c_void_p), C.byref(info), _stream(stream))
        if st not in (EB_OK, EB_ERR_NOT_CONVERGED):
            _check(st, "eb_amr_solve_levels")
        return ps, _info_dict(info)

    def field(self, l, phi, sigma=None, stream=None):
        """E [D][2][n] on level l's grid (and the EB normal field)."""
        n = self.levels[l]["n_cells"]
        lev_geom = self.level_geom(l)
        gi = GeomInfo()
        _check(load().eb_geom_query(lev_geom, C.byref(gi)), "eb_geom_query")
        E = torch.empty(self.dim, 2, n, dtype=torch.float64, device=self.device)
        En = torch.empty(max(int(gi.n_eb), 1), 2, dtype=torch.float64, device=self.device)
        ph = self._f(phi, l)
        sg = self._f(sigma, l) if sigma is not None else None
        _check(load().eb_amr_field_eval(self._h, l, _ptr(ph), _ptr(sg), _ptr(E), _ptr(En), _stream(stream)),
               "eb_amr_field_eval")
        return E, En

    def kernel_stats(self):
        out = (C.c_double * 8)()
        _check(load().eb_amr_kernel_stats(self._h, out), "eb_amr_kernel_stats")
        keys = ("launches", "kernel_ms", "vcycles", "outer")
        return {w: {k: out[4 * i + j] for j, k in enumerate(keys)} for i, w in enumerate(("coarse", "fine"))}

    def close(self):
        if getattr(self, "_h", None):
            load().eb_amr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tag_cells(geom_handle, E, eps=(0.1, 0.8, 0.1, 0.2), keep=None, want_tags=True, stream=None):
    """Refinement tags of one grid (a Geometry's handle or Hierarchy.level_geom(l)).
    Returns (tags uint8 tensor or None, bbox_lo, bbox_hi, n_marked, e_max)."""
    h = geom_handle._h if isinstance(geom_handle, Geometry) else geom_handle
    ep = (C.c_double * 4)(*[float(v) for v in eps])
    klo = khi = None
    if keep is not None:
        klo = (C.c_int * 3)(*[int(v) for v in (list(keep[0]) + [0] * 3)[:3]])
        khi = (C.c_int * 3)(*[int(v) for v in (list(keep[1]) + [1] * 3)[:3]])
    tags = torch.empty(E.shape[-1], dtype=torch.uint8, device=E.device) if want_tags else None
    blo, bhi = (C.c_int * 3)(), (C.c_int * 3)()
    nm, em = C.c_longlong(), C.c_double()
    _check(load().eb_tag_cells(h, _ptr(E.contiguous()), ep, klo, khi, _ptr(tags), blo, bhi, C.byref(nm), C.byref(em),
                               _stream(stream)), "eb_tag_cells")
    return tags, list(blo), list(bhi), nm.value, em.value


def regrid_box(dim, n, cf_lo, cf_hi, bbox_lo, bbox_hi, n_marked, buf=2, block=4):
    """The next finer box from a tag bounding box, or None (host arithmetic in the library)."""
    i3 = lambda v, f: (C.c_int * 3)(*[int(x) for x in (list(v) + [f] * 3)[:3]])  # noqa: E731
    lo, hi, has = (C.c_int * 3)(), (C.c_int * 3)(), C.c_int()
    _check(load().eb_regrid_box(int(dim), i3(n, 1), i3(cf_lo, 0), i3(cf_hi, 0), i3(bbox_lo, 0), i3(bbox_hi, 0),
                                int(n_marked), int(buf), int(block), lo, hi, C.byref(has)), "eb_regrid_box")
    return (list(lo)[:dim], list(hi)[:dim]) if has.value else None


class TGA:
    """Implicit diffusion by TGA steps (Sec. 3.4) on one geometry description
    (owns an eb_tga and the three geometries and solvers it borrows, with
    Helmholtz shifts 0, 1/mu1, 1/mu2 for the step length dt; eps of the
    description is the diffusion coefficient)."""

    def __init__(self, desc: dict, dt: float, *, precision="mixed", tol=1e-10, device="cuda", stream=None):
        self.dt, self.tol = float(dt), float(tol)
        mu = eb_tga_coefficients(self.dt)
        self.mu = mu
        self.handles = []
        for lam in (0.0, 1.0 / mu[0], 1.0 / mu[1]):
            d = dict(desc)
            d["lam"] = (lam, lam)
            g = Geometry(d, device=device)
            self.handles.append(Poisson(g, precision=precision, tol=tol, max_cycles=200))
        self.geom = self.handles[0].geom
        with torch.cuda.device(self.geom.device):
            self._h = eb_tga_create(*(P.geom._h for P in self.handles), *(P._h for P in self.handles), self.dt,
                                    stream)

    def close(self):
        if getattr(self, "_h", None):
            load().eb_tga_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, phi, rho, out=None, stream=None):
        """phi^{n+1} from phi^n and the source rho ([2][n_cells] FP64 on the device)."""
        dev, n = self.geom.device, self.geom.ncell
        phi = _dev(phi, torch.float64, dev).reshape(2, n).contiguous()
        rho = _dev(rho, torch.float64, dev).reshape(2, n).contiguous()
        if out is None:
            out = torch.empty_like(phi)
        infos = eb_tga_step(self._h, phi, rho, out, self.tol, stream)
        return out, infos
