"""Python binding of the C ABI in include/fe.h (ctypes, argument marshalling
only).  Every function keeps the C name; handles are opaque ctypes pointers;
errors raise FeError carrying the fe_status and fe_last_error().  Device
buffers are passed as integer addresses (e.g. torch.Tensor.data_ptr()).

The library must have been built (paper_0704_2344_gb300.build.build()); a
missing library raises instead of falling back to anything else."""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

FE_OK = 0
FE_PENDING = 1
FE_ERR_INVALID_ARG = -1
FE_ERR_MESH = -2
FE_ERR_OOM = -3
FE_ERR_BREAKDOWN = -4
FE_ERR_NOT_CONVERGED = -5
FE_ERR_TIMEOUT = -6
FE_ERR_CUDA = -7
FE_ERR_UNSUPPORTED = -8

FE_VARIANT_S, FE_VARIANT_L, FE_VARIANT_P = 0, 1, 2
FE_PREC_FP64, FE_PREC_MIXED, FE_PREC_DF = 0, 1, 2
FE_BOUNDARY_ABC, FE_BOUNDARY_SYMMETRY, FE_BOUNDARY_ANTISYMMETRY = 0, 1, 2
FE_FORMULATION_H, FE_FORMULATION_E = 0, 1
FE_PRECOND_BLOCK_JACOBI, FE_PRECOND_BICP = 0, 1
FE_RECURRENCE_CG, FE_RECURRENCE_EXPANDED = 0, 1

LIB_PATH = Path(__file__).resolve().parent / "libfe_gb300.so"


class FeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} -> status {status}: {msg}")
        self.status = status


class fe_complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class fe_options(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("variant", C.c_int32), ("abc_sigma", C.c_double),
                ("penalty_s", C.c_double), ("formulation", C.c_int32)]


class fe_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double * 3),
                ("origin", C.c_double * 3), ("material", C.c_void_p), ("material_on_device", C.c_int32),
                ("n_materials", C.c_int32), ("eps_r", C.POINTER(fe_complex)), ("mu_r", C.POINTER(fe_complex)),
                ("boundary", C.c_int32 * 6)]


class fe_mesh_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_elements", "n_active_elements", "n_nodes_total", "n_nodes",
                                          "n_dof", "nnzb", "n_faces_ext", "n_faces_pec", "device_bytes")]


class fe_system_stats(C.Structure):
    _fields_ = [("precision", C.c_int32), ("dict_blocks", C.c_int32)] + [
        (n, C.c_int64) for n in ("n_rows", "nnzb", "rows_general", "rows_diagonal", "blocks_explicit",
                                 "device_bytes")]


class fe_planewave(C.Structure):
    _fields_ = [("k_hat", C.c_double * 3), ("p_hat", C.c_double * 3), ("amplitude", fe_complex)]


class fe_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("reliable", C.c_double),
                ("max_iter", C.c_int32), ("max_outer", C.c_int32), ("rhs_tile", C.c_int32),
                ("max_pass_iter", C.c_int32), ("wait_timeout_us", C.c_int32), ("preconditioner", C.c_int32),
                ("recurrence", C.c_int32)]


class fe_solve_stats(C.Structure):
    _fields_ = [("kernel_ms", C.c_double), ("launches", C.c_int64), ("inner_iters", C.c_int64),
                ("passes", C.c_int64), ("tile_width", C.c_int64), ("grid_ctas", C.c_int64),
                ("tuned", C.c_int64), ("tune_ms", C.c_double)]


class fe_solve_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("outer", C.c_int32),
                ("reserved", C.c_int32), ("rel_residual", C.c_double)]


class fe_serve_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("reliable", C.c_double),
                ("max_iter", C.c_int32), ("max_outer", C.c_int32), ("hbm_budget", C.c_int64),
                ("max_ctas", C.c_int32), ("work_per_cta", C.c_int32), ("max_job_ctas", C.c_int32),
                ("seg_iters", C.c_int32), ("recurrence", C.c_int32)]


class fe_request(C.Structure):
    _fields_ = [("mesh", fe_mesh_desc), ("freq_hz", C.c_double), ("nrhs", C.c_int32),
                ("waves", C.POINTER(fe_planewave))]


class fe_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("nrhs", C.c_int32), ("n_dof", C.c_int64),
                ("x", C.POINTER(fe_complex)), ("node_id", C.POINTER(C.c_int32)),
                ("reports", C.POINTER(fe_solve_report)), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("batch_jobs", C.c_int32), ("batch_ctas", C.c_int32),
                ("message", C.c_char_p)]


class fe_serve_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "failed", "launches", "jobs_launched",
                                         "budget_bytes", "peak_admitted_bytes")] + [("solve_device_s", C.c_double)]


_lib = None
P = C.c_void_p


def load() -> C.CDLL:
    """Loads libfe_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise FileNotFoundError(f"{LIB_PATH} is missing: build it with paper_0704_2344_gb300.build.build()")
    lib = C.CDLL(str(LIB_PATH))
    sig = {
        "fe_options_default": (None, [C.POINTER(fe_options)]),
        "fe_ctx_create": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(fe_options)]),
        "fe_ctx_destroy": (None, [P]),
        "fe_ctx_synchronize": (C.c_int, [P]),
        "fe_mesh_create": (C.c_int, [P, C.POINTER(fe_mesh_desc), C.POINTER(P)]),
        "fe_mesh_info": (C.c_int, [P, C.POINTER(fe_mesh_stats)]),
        "fe_mesh_export_maps": (C.c_int, [P, P, P, P, P, P, P, P]),
        "fe_mesh_destroy": (None, [P]),
        "fe_assemble": (C.c_int, [P, P, C.c_double, C.c_int32, C.POINTER(P)]),
        "fe_system_export": (C.c_int, [P, P, P, P, P]),
        "fe_system_export_df": (C.c_int, [P, P, P]),
        "fe_system_factor_bicp": (C.c_int, [P, P, C.c_int32]),
        "fe_system_export_bicp": (C.c_int, [P, P, P, P]),
        "fe_system_info": (C.c_int, [P, C.POINTER(fe_system_stats)]),
        "fe_system_destroy": (None, [P]),
        "fe_rhs": (C.c_int, [P, P, C.c_int32, C.POINTER(fe_planewave), P, C.c_int32]),
        "fe_spmv": (C.c_int, [P, P, C.c_int32, C.c_int32, P, P]),
        "fe_system_pack_half": (C.c_int, [P, P, P]),
        "fe_spmv_half": (C.c_int, [P, P, C.c_int32, C.c_int32, P, P]),
        "fe_solve_opts_default": (None, [C.POINTER(fe_solve_opts)]),
        "fe_solve_batch": (C.c_int, [P, P, C.c_int32, C.POINTER(fe_planewave), C.POINTER(fe_solve_opts), P,
                                     C.c_int32, C.POINTER(fe_solve_report)]),
        "fe_solve_rhs": (C.c_int, [P, P, C.c_int32, P, C.c_int32, C.POINTER(fe_solve_opts), P, C.c_int32,
                                   C.c_int32, C.POINTER(fe_solve_report)]),
        "fe_last_solve_stats": (C.c_int, [P, C.POINTER(fe_solve_stats)]),
        "fe_solve_rhs_noalloc": (C.c_int, [P, P, C.c_int32, P, P, C.c_int32, C.POINTER(fe_solve_opts),
                                           C.POINTER(fe_solve_report)]),
        "fe_serve_opts_default": (None, [C.POINTER(fe_serve_opts)]),
        "fe_serve_create": (C.c_int, [P, C.POINTER(fe_serve_opts), C.POINTER(P)]),
        "fe_serve_submit": (C.c_int, [P, C.POINTER(fe_request), C.POINTER(C.c_uint64)]),
        "fe_serve_poll": (C.c_int, [P, C.c_uint64, C.POINTER(fe_result)]),
        "fe_serve_wait": (C.c_int, [P, C.c_uint64, C.c_double, C.POINTER(fe_result)]),
        "fe_serve_release": (C.c_int, [P, C.c_uint64]),
        "fe_serve_info": (C.c_int, [P, C.POINTER(fe_serve_stats)]),
        "fe_serve_destroy": (None, [P]),
        "fe_serve_plan": (C.c_int32, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_int32,
                                      C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
        "fe_last_error": (C.c_char_p, []),
        "fe_launch_count": (C.c_int64, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return [n for n in dir(load()) if n.startswith("fe_")]


def _check(status: int, where: str, ok=(FE_OK,)):
    if status not in ok:
        raise FeError(status, where, load().fe_last_error().decode(errors="replace"))
    return status


def fe_last_error() -> str:
    return load().fe_last_error().decode(errors="replace")


def fe_launch_count() -> int:
    return int(load().fe_launch_count())


def fe_last_solve_stats(ctx) -> dict:
    s = fe_solve_stats()
    _check(load().fe_last_solve_stats(ctx, C.byref(s)), "fe_last_solve_stats")
    return {n: (float(getattr(s, n)) if n in ("kernel_ms", "tune_ms") else int(getattr(s, n)))
            for n, _ in fe_solve_stats._fields_}


def _ptr(a) -> int:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


# --------------------------------------------------------------------------
def fe_ctx_create(device: int = 0, stream: int | None = None, variant: int = FE_VARIANT_S,
                  abc_sigma: float = 1.0, penalty_s: float = 1.0, formulation: int = 0):
    lib = load()
    opt = fe_options()
    lib.fe_options_default(C.byref(opt))
    opt.stream = stream
    opt.variant = variant
    opt.abc_sigma = abc_sigma
    opt.penalty_s = penalty_s
    opt.formulation = formulation
    out = P()
    _check(lib.fe_ctx_create(C.byref(out), device, C.byref(opt)), "fe_ctx_create")
    out.device = int(device)
    return out


def fe_ctx_destroy(ctx):
    load().fe_ctx_destroy(ctx)


def fe_ctx_synchronize(ctx):
    _check(load().fe_ctx_synchronize(ctx), "fe_ctx_synchronize")


def fe_mesh_create(ctx, nx, ny, nz, h, origin, material, eps_r, mu_r, material_on_device=False, boundary=None):
    """material: numpy uint8 array (nz, ny, nx) or a device address of nx*ny*nz bytes.
    boundary: fe_boundary per face (-x, +x, -y, +y, -z, +z); None = absorbing box."""
    lib = load()
    d = fe_mesh_desc()
    d.boundary = (C.c_int32 * 6)(*[int(v) for v in (boundary or (0,) * 6)])
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.h = (C.c_double * 3)(*[float(v) for v in h])
    d.origin = (C.c_double * 3)(*[float(v) for v in origin])
    keep = None
    if material_on_device:
        d.material = int(material)
        d.material_on_device = 1
    else:
        keep = np.ascontiguousarray(material, dtype=np.uint8)
        if keep.size != d.nx * d.ny * d.nz:
            raise ValueError("material size does not match the grid")
        d.material = keep.ctypes.data
        d.material_on_device = 0
    eps = np.ascontiguousarray(np.asarray(eps_r, dtype=np.complex128))
    mu = np.ascontiguousarray(np.asarray(mu_r, dtype=np.complex128))
    if eps.shape != mu.shape:
        raise ValueError("eps_r and mu_r differ in length")
    d.n_materials = eps.size
    d.eps_r = eps.ctypes.data_as(C.POINTER(fe_complex))
    d.mu_r = mu.ctypes.data_as(C.POINTER(fe_complex))
    out = P()
    _check(lib.fe_mesh_create(ctx, C.byref(d), C.byref(out)), "fe_mesh_create")
    del keep
    return out


def fe_mesh_create_from(ctx, problem, material_device_ptr: int | None = None):
    """Marshals a workloads.VoxelProblem (or any object with the same fields)."""
    mat = problem.material if material_device_ptr is None else material_device_ptr
    return fe_mesh_create(ctx, problem.nx, problem.ny, problem.nz, problem.h, problem.origin, mat,
                          problem.eps_r, problem.mu_r, material_on_device=material_device_ptr is not None,
                          boundary=tuple(getattr(problem, "boundary", (0,) * 6)))


def fe_mesh_info(mesh) -> dict:
    s = fe_mesh_stats()
    _check(load().fe_mesh_info(mesh, C.byref(s)), "fe_mesh_info")
    return {n: int(getattr(s, n)) for n, _ in fe_mesh_stats._fields_}


def fe_mesh_export_maps(ctx, mesh) -> dict:
    info = fe_mesh_info(mesh)
    out = {
        "node_rank": np.empty(info["n_nodes_total"], np.int32),
        "row_ptr": np.empty(info["n_nodes"] + 1, np.int32),
        "col_idx": np.empty(info["nnzb"], np.int32),
        "elem_slot": np.empty(info["n_elements"] * 64, np.int32),
        "faces_ext": np.empty(info["n_faces_ext"], np.int32),
        "faces_pec": np.empty(info["n_faces_pec"], np.int32),
    }
    _check(load().fe_mesh_export_maps(ctx, mesh, *[out[k].ctypes.data for k in
                                                    ("node_rank", "row_ptr", "col_idx", "elem_slot",
                                                     "faces_ext", "faces_pec")]), "fe_mesh_export_maps")
    out["elem_slot"] = out["elem_slot"].reshape(-1, 8, 8)
    return out


def fe_mesh_destroy(mesh):
    load().fe_mesh_destroy(mesh)


def fe_assemble(ctx, mesh, freq_hz: float, precision: int = FE_PREC_DF):
    out = P()
    _check(load().fe_assemble(ctx, mesh, float(freq_hz), int(precision), C.byref(out)), "fe_assemble")
    return out


def fe_system_export(ctx, system, mesh, c128=True, c64=False, dinv=False) -> dict:
    info = fe_mesh_info(mesh)
    out = {}
    a = np.empty((info["nnzb"], 3, 3), np.complex128) if c128 else None
    b = np.empty((info["nnzb"], 3, 3), np.complex64) if c64 else None
    d = np.empty((info["n_nodes"], 3, 3), np.complex128) if dinv else None
    _check(load().fe_system_export(ctx, system, _ptr(a), _ptr(b), _ptr(d)), "fe_system_export")
    if c128:
        out["c128"] = a
    if c64:
        out["c64"] = b
    if dinv:
        out["dinv"] = d
    return out


def fe_system_info(system) -> dict:
    st = fe_system_stats()
    _check(load().fe_system_info(system, C.byref(st)), "fe_system_info")
    return {n: int(getattr(st, n)) for n, _ in fe_system_stats._fields_}


def fe_system_export_df(ctx, system, mesh) -> np.ndarray:
    """FP32-pair values [nnzb, 3, 3, 4] float32 (re_hi, im_hi, re_lo, im_lo)
    of a system assembled with FE_PREC_DF."""
    info = fe_mesh_info(mesh)
    a = np.empty((info["nnzb"], 3, 3, 4), np.float32)
    _check(load().fe_system_export_df(ctx, system, _ptr(a)), "fe_system_export_df")
    return a


def fe_system_factor_bicp(ctx, system, n_sub: int = 0) -> int:
    """Builds the block incomplete Cholesky factor (n_sub bands; 0 = one per
    CTA of the solve grid) and returns the number of bands."""
    _check(load().fe_system_factor_bicp(ctx, system, int(n_sub)), "fe_system_factor_bicp")
    n = C.c_int32(0)
    _check(load().fe_system_export_bicp(ctx, system, None, C.byref(n)), "fe_system_export_bicp")
    return int(n.value)


def fe_system_export_bicp(ctx, system, mesh):
    """(L [nnzb, 3, 3] complex128 by block slot, number of bands)."""
    info = fe_mesh_info(mesh)
    a = np.empty((info["nnzb"], 3, 3), np.complex128)
    n = C.c_int32(0)
    _check(load().fe_system_export_bicp(ctx, system, _ptr(a), C.byref(n)), "fe_system_export_bicp")
    return a, int(n.value)


def fe_system_destroy(system):
    load().fe_system_destroy(system)


def planewave_array(waves) -> C.Array:
    """waves: workloads.PlaneWaves (k_hat [R,3], p_hat [R,3], amplitude [R])."""
    R = waves.k_hat.shape[0]
    arr = (fe_planewave * R)()
    for r in range(R):
        arr[r].k_hat = (C.c_double * 3)(*waves.k_hat[r])
        arr[r].p_hat = (C.c_double * 3)(*waves.p_hat[r])
        arr[r].amplitude = fe_complex(float(np.real(waves.amplitude[r])), float(np.imag(waves.amplitude[r])))
    return arr


def fe_rhs(ctx, system, waves, n_dof: int, out=None, on_device: bool = False):
    """Returns B [n_dof, R] complex128 (host) unless `out` is a device address."""
    arr = planewave_array(waves)
    R = len(arr)
    if out is None:
        host = np.empty((n_dof, R), np.complex128)
        _check(load().fe_rhs(ctx, system, R, arr, host.ctypes.data, 0), "fe_rhs")
        return host
    _check(load().fe_rhs(ctx, system, R, arr, _ptr(out), 1 if on_device else 0), "fe_rhs")
    return out


def fe_spmv(ctx, system, precision: int, nrhs: int, x, y):
    _check(load().fe_spmv(ctx, system, int(precision), int(nrhs), _ptr(x), _ptr(y)), "fe_spmv")


def fe_system_pack_half(ctx, system) -> int:
    """Builds the half (lower-part) storage of the system; returns the number
    of kept blocks."""
    n = C.c_int64(0)
    _check(load().fe_system_pack_half(ctx, system, C.byref(n)), "fe_system_pack_half")
    return int(n.value)


def fe_spmv_half(ctx, system, precision: int, nrhs: int, x, y):
    _check(load().fe_spmv_half(ctx, system, int(precision), int(nrhs), _ptr(x), _ptr(y)), "fe_spmv_half")


def solve_opts(precision=FE_PREC_DF, tol=1e-8, reliable=1e-4, max_iter=100000, max_outer=200,
               rhs_tile=0, max_pass_iter=None, wait_timeout_us=None,
               preconditioner=FE_PRECOND_BLOCK_JACOBI, recurrence=FE_RECURRENCE_CG) -> fe_solve_opts:
    o = fe_solve_opts()
    load().fe_solve_opts_default(C.byref(o))
    o.precision, o.tol, o.reliable = int(precision), float(tol), float(reliable)
    o.max_iter, o.max_outer, o.rhs_tile = int(max_iter), int(max_outer), int(rhs_tile)
    if max_pass_iter is not None:
        o.max_pass_iter = int(max_pass_iter)
    if wait_timeout_us is not None:
        o.wait_timeout_us = int(wait_timeout_us)
    o.preconditioner = int(preconditioner)
    o.recurrence = int(recurrence)
    return o


def _reports(rep) -> list[dict]:
    return [{"status": r.status, "iterations": r.iterations, "outer": r.outer,
             "rel_residual": r.rel_residual} for r in rep]


_SOLVE_OK = (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN)


def fe_solve_batch(ctx, system, waves, n_dof: int, opts: fe_solve_opts | None = None, x_out=None,
                   x_on_device: bool = False, raise_on_fail: bool = True):
    """Solves A X = B(waves).  x_out: None (a host array is returned), a host
    numpy array [n_dof, R] complex128, or a device address.  Returns
    (status, x, reports)."""
    arr = planewave_array(waves)
    R = len(arr)
    opts = opts or solve_opts()
    rep = (fe_solve_report * R)()
    if x_out is None:
        x_out = np.empty((n_dof, R), np.complex128)
        x_on_device = False
    st = load().fe_solve_batch(ctx, system, R, arr, C.byref(opts), _ptr(x_out), 1 if x_on_device else 0, rep)
    _check(st, "fe_solve_batch", ok=(FE_OK,) if raise_on_fail else _SOLVE_OK)
    return st, x_out, _reports(rep)


def fe_solve_rhs(ctx, system, b, nrhs: int, opts: fe_solve_opts | None = None, x_out=None,
                 b_on_device=False, x_on_device=False, use_x0=False, raise_on_fail=True):
    opts = opts or solve_opts()
    rep = (fe_solve_report * nrhs)()
    if x_out is None:
        x_out = np.zeros((np.asarray(b).shape[0], nrhs), np.complex128)
        x_on_device = False
    if not b_on_device:
        b = np.ascontiguousarray(b, dtype=np.complex128)
    st = load().fe_solve_rhs(ctx, system, int(nrhs), _ptr(b), 1 if b_on_device else 0, C.byref(opts),
                             _ptr(x_out), 1 if x_on_device else 0, 1 if use_x0 else 0, rep)
    _check(st, "fe_solve_rhs", ok=(FE_OK,) if raise_on_fail else _SOLVE_OK)
    return st, x_out, _reports(rep)


def fe_solve_rhs_noalloc(ctx, system, nrhs: int, b_dev, x_dev, opts: fe_solve_opts | None = None,
                         use_x0: bool = False, raise_on_fail: bool = True):
    """Solve with the library's fixed device scratch (no allocation during the
    call); b_dev and x_dev are torch complex128 tensors [n_dof, nrhs],
    contiguous, on the context's CUDA device (the kernel reads and writes them
    in place, so nothing else is accepted)."""
    n_dof = 3 * fe_system_info(system)["n_rows"]
    dev = getattr(ctx, "device", None)
    where = "fe_solve_rhs_noalloc"
    for name, t in (("b_dev", b_dev), ("x_dev", x_dev)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise FeError(FE_ERR_INVALID_ARG, where, f"{name} must be a CUDA tensor")
        if str(t.dtype) != "torch.complex128" or not t.is_contiguous() or tuple(t.shape) != (n_dof, int(nrhs)):
            raise FeError(FE_ERR_INVALID_ARG, where,
                          f"{name} must be a contiguous complex128 tensor of shape ({n_dof}, {int(nrhs)})")
        if dev is not None and t.device.index != dev:
            raise FeError(FE_ERR_INVALID_ARG, where, f"{name} is on cuda:{t.device.index}, the context on cuda:{dev}")
    opts = opts or solve_opts()
    rep = (fe_solve_report * nrhs)()
    st = load().fe_solve_rhs_noalloc(ctx, system, int(nrhs), _ptr(b_dev), _ptr(x_dev), 1 if use_x0 else 0,
                                     C.byref(opts), rep)
    _check(st, "fe_solve_rhs_noalloc", ok=(FE_OK,) if raise_on_fail else _SOLVE_OK)
    return st, _reports(rep)


# --------------------------------------------------------------------------
# Serving
def serve_opts(precision=FE_PREC_DF, tol=1e-8, reliable=1e-4, max_iter=100000, max_outer=200,
               hbm_budget=0, max_ctas=0, work_per_cta=0, max_job_ctas=0, seg_iters=0,
               recurrence=FE_RECURRENCE_EXPANDED) -> fe_serve_opts:
    o = fe_serve_opts()
    load().fe_serve_opts_default(C.byref(o))
    o.precision, o.tol, o.reliable = int(precision), float(tol), float(reliable)
    o.max_iter, o.max_outer, o.hbm_budget = int(max_iter), int(max_outer), int(hbm_budget)
    o.max_ctas = int(max_ctas)
    o.max_job_ctas = int(max_job_ctas)
    if seg_iters:
        o.seg_iters = int(seg_iters)
    if work_per_cta:
        o.work_per_cta = int(work_per_cta)
    o.recurrence = int(recurrence)
    return o


def fe_serve_create(ctx, opts: fe_serve_opts | None = None):
    out = P()
    _check(load().fe_serve_create(ctx, C.byref(opts or serve_opts()), C.byref(out)), "fe_serve_create")
    return out


def fe_serve_submit(server, problem, waves) -> int:
    """Submits a workloads.VoxelProblem with its PlaneWaves; returns the ticket.
    The request is copied, so the arguments may be dropped afterwards."""
    d = fe_mesh_desc()
    d.nx, d.ny, d.nz = int(problem.nx), int(problem.ny), int(problem.nz)
    d.h = (C.c_double * 3)(*[float(v) for v in problem.h])
    d.origin = (C.c_double * 3)(*[float(v) for v in problem.origin])
    mat = np.ascontiguousarray(problem.material, dtype=np.uint8)
    d.material = mat.ctypes.data
    d.material_on_device = 0
    eps = np.ascontiguousarray(np.asarray(problem.eps_r, dtype=np.complex128))
    mu = np.ascontiguousarray(np.asarray(problem.mu_r, dtype=np.complex128))
    d.n_materials = eps.size
    d.eps_r = eps.ctypes.data_as(C.POINTER(fe_complex))
    d.mu_r = mu.ctypes.data_as(C.POINTER(fe_complex))
    d.boundary = (C.c_int32 * 6)(*[int(v) for v in getattr(problem, "boundary", (0,) * 6)])
    arr = planewave_array(waves)
    r = fe_request()
    r.mesh = d
    r.freq_hz = float(problem.freq_hz)
    r.nrhs = len(arr)
    r.waves = C.cast(arr, C.POINTER(fe_planewave))
    t = C.c_uint64()
    _check(load().fe_serve_submit(server, C.byref(r), C.byref(t)), "fe_serve_submit")
    return int(t.value)


def _result_dict(res: fe_result, copy: bool) -> dict:
    out = {"status": int(res.status), "nrhs": int(res.nrhs), "n_dof": int(res.n_dof),
           "t_submit": float(res.t_submit), "t_admit": float(res.t_admit), "t_done": float(res.t_done),
           "batch_jobs": int(res.batch_jobs), "batch_ctas": int(res.batch_ctas),
           "message": (res.message or b"").decode(errors="replace"), "x": None, "node_id": None, "reports": None}
    if copy and res.x:
        n = res.n_dof * res.nrhs
        flat = np.ctypeslib.as_array(C.cast(res.x, C.POINTER(C.c_double)), shape=(2 * n,)).copy()
        out["x"] = flat.view(np.complex128).reshape(res.n_dof, res.nrhs)
    if copy and res.node_id and res.n_dof:
        out["node_id"] = np.ctypeslib.as_array(res.node_id, shape=(res.n_dof // 3,)).copy()
    if res.reports:  # small: always copied
        out["reports"] = _reports([res.reports[i] for i in range(res.nrhs)])
    return out


def fe_serve_poll(server, ticket: int, copy: bool = True):
    """None while pending; else the finished request as a dict (arrays copied)."""
    res = fe_result()
    st = _check(load().fe_serve_poll(server, int(ticket), C.byref(res)), "fe_serve_poll", ok=(FE_OK, FE_PENDING))
    return None if st == FE_PENDING else _result_dict(res, copy)


def fe_serve_wait(server, ticket: int, timeout_s: float = 60.0, copy: bool = True):
    res = fe_result()
    st = _check(load().fe_serve_wait(server, int(ticket), float(timeout_s), C.byref(res)), "fe_serve_wait",
                ok=(FE_OK, FE_PENDING))
    return None if st == FE_PENDING else _result_dict(res, copy)


def fe_serve_release(server, ticket: int):
    return _check(load().fe_serve_release(server, int(ticket)), "fe_serve_release", ok=(FE_OK, FE_PENDING))


def fe_serve_info(server) -> dict:
    s = fe_serve_stats()
    _check(load().fe_serve_info(server, C.byref(s)), "fe_serve_info")
    return {n: (float(getattr(s, n)) if n == "solve_device_s" else int(getattr(s, n)))
            for n, _ in fe_serve_stats._fields_}


def fe_serve_destroy(server):
    load().fe_serve_destroy(server)


def fe_serve_plan(rows, widths, max_ctas: int, work_per_cta: int, max_job_ctas: int = 0) -> tuple[int, np.ndarray]:
    """The server's packing rule (host only): returns (taken, n_cta per request)."""
    r = np.ascontiguousarray(rows, dtype=np.int64)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    out = np.zeros(r.size, np.int32)
    taken = load().fe_serve_plan(int(r.size), r.ctypes.data_as(C.POINTER(C.c_int64)),
                                 w.ctypes.data_as(C.POINTER(C.c_int32)), int(max_ctas), int(max_job_ctas),
                                 int(work_per_cta),
                                 out.ctypes.data_as(C.POINTER(C.c_int32)))
    return int(taken), out
