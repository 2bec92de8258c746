"""Thin Python binding of libmg (include/mg.h, include/mg_kernels.h).

Argument marshalling only: every step of the solver runs in the CUDA library.  Device
arrays are torch CUDA tensors (torch provides device memory and streams), host arrays
are numpy arrays.  If libmg.so has not been built, importing works but every call
raises: there is no CPU fallback.

The C entry points are exposed under their own names (``mg_create``,
``mg_setup_transform``, ``mg_solve``, ``mg_batch_solve``, ``mg_server_start``,
``mg_serve_submit``, ``mg_serve_poll``, ``mg_server_stop``, ``mgk_*``), plus small
convenience classes (``Context``, ``Problem``, ``Server``) that own the handles.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmg.so")

MG_OK, MG_ERR_ARG, MG_ERR_SIZE, MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_MAP_FOLDED = 0, 1, 2, 3, 4, 5
MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, MG_ERR_TIMEOUT, MG_ERR_BUSY, MG_ERR_NOT_FOUND = 6, 7, 8, 9, 10
MG_ERR_NOT_SPD = 11
MG_MEM_HOST, MG_MEM_DEVICE = 0, 1
MG_PREC_FP64, MG_PREC_MIXED = 0, 1
MG_OUTER_VCYCLE, MG_OUTER_FCG, MG_OUTER_SOR = 0, 1, 2
_OUTERS = {"vcycle": MG_OUTER_VCYCLE, "fcg": MG_OUTER_FCG, "sor": MG_OUTER_SOR}
MG_SMOOTH_GS4, MG_SMOOTH_JACOBI, MG_SMOOTH_XLINE = 0, 1, 2
_SMOOTHERS = {"gs4": MG_SMOOTH_GS4, "jacobi": MG_SMOOTH_JACOBI, "xline": MG_SMOOTH_XLINE}
MAP_CODES = {"identity": 0, "sine_warp": 1, "polar": 2, "sinh": 3, "affine": 4, "grid": 5}
MG_HIST_MAX = 256

_DP = C.POINTER(C.c_double)
_FP = C.POINTER(C.c_float)


class mg_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("lx", C.c_double), ("ly", C.c_double), ("periodic_y", C.c_int), ("neumann_y", C.c_int)]


class mg_map_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.c_double * 4), ("xp", C.c_void_p),
                ("yp", C.c_void_p), ("jump_x", C.c_double), ("jump_y", C.c_double)]


class mg_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("outer", C.c_int), ("smoother", C.c_int),
                ("nu1", C.c_int), ("nu2", C.c_int), ("omega_j", C.c_double), ("rtol", C.c_double),
                ("max_iters", C.c_int), ("coarse_max", C.c_int), ("warm_start", C.c_int),
                ("coarse_op", C.c_int)]


class mg_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("levels", C.c_int), ("rel_residual", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("hist", C.c_double * MG_HIST_MAX), ("kernel_launches", C.c_int),
                ("setup_kernel_launches", C.c_int)]

    def history(self):
        return np.array(self.hist[: min(self.iters + 1, MG_HIST_MAX)])


class mgk_op_f64(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("periodic", C.c_int), ("pitch", C.c_int)] + \
               [(n, C.c_void_p) for n in ("cE", "cN", "cNE", "cNW", "diag", "dinv")] + \
               [("five_point", C.c_int)]


class mgk_op_f32(C.Structure):
    _fields_ = mgk_op_f64._fields_


class mg_server_opts(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("queue_capacity", C.c_int), ("mem_budget", C.c_size_t),
                ("host_budget", C.c_size_t)]


class mg_request(C.Structure):
    _fields_ = [("grid", mg_grid_desc), ("map", mg_map_desc), ("eps_phys", C.c_void_p),
                ("rho_phys", C.c_void_p), ("bc", C.c_void_p), ("opts", mg_solve_opts)]


class mg_tune_entry(C.Structure):
    _fields_ = [("precision", C.c_int), ("side", C.c_int), ("ms", C.c_float * 4), ("choice", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("sweeps_per_launch", C.c_int)]


class mg_tune_report(C.Structure):
    _fields_ = [("count", C.c_int), ("entry", mg_tune_entry * 32)]


SMOOTHER_FAMILIES = {1: "colour", 2: "fused", 3: "pipelined", 4: "marching"}


class mg_serve_report(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("failed", C.c_uint64), ("wall_s", C.c_double),
                ("unknowns_per_s", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("mean_batch", C.c_double), ("ticks", C.c_int),
                ("reused", C.c_uint64), ("evicted", C.c_uint64)]


_SIGS = {
    "mg_last_error": ([], C.c_char_p),
    "mg_default_opts": ([C.POINTER(mg_solve_opts)], None),
    "mg_create": ([C.c_int, C.c_size_t, C.POINTER(C.c_void_p)], C.c_int),
    "mg_destroy": ([C.c_void_p], None),
    "mg_set_stream": ([C.c_void_p, C.c_void_p], C.c_int),
    "mg_mem_info": ([C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)], C.c_int),
    "mg_setup_transform": ([C.c_void_p, C.POINTER(mg_grid_desc), C.POINTER(mg_map_desc), C.c_void_p,
                            C.c_int, C.POINTER(mg_solve_opts), C.POINTER(C.c_void_p)], C.c_int),
    "mg_update_transform": ([C.c_void_p, C.POINTER(mg_map_desc), C.c_void_p, C.c_int], C.c_int),
    "mg_map_five_point": ([C.POINTER(mg_map_desc)], C.c_int),
    "mg_problem_five_point": ([C.c_void_p], C.c_int),
    "mg_batch_update_transform": ([C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(mg_map_desc),
                                   C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int)], C.c_int),
    "mg_problem_free": ([C.c_void_p], None),
    "mg_problem_info": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
                        C.c_int),
    "mg_solve": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                  C.POINTER(mg_solve_opts), C.POINTER(mg_solve_stats)], C.c_int),
    "mg_cycle_time": ([C.c_void_p, C.POINTER(mg_solve_opts), C.c_int, C.POINTER(C.c_double)], C.c_int),
    "mg_batch_solve": ([C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                        C.POINTER(mg_solve_opts), C.POINTER(mg_solve_stats)], C.c_int),
    "mg_harmonic_grid": ([C.c_void_p, C.POINTER(mg_grid_desc), C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(mg_solve_stats)], C.c_int),
    "mg_autotune": ([C.c_void_p, C.c_int, C.POINTER(mg_tune_report)], C.c_int),
    "mg_server_start": ([C.c_void_p, C.POINTER(mg_server_opts), C.POINTER(C.c_void_p)], C.c_int),
    "mg_serve_submit": ([C.c_void_p, C.POINTER(mg_request), C.POINTER(C.c_uint64)], C.c_int),
    "mg_serve_poll": ([C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.POINTER(mg_solve_stats)],
                      C.c_int),
    "mg_server_stop": ([C.c_void_p, C.POINTER(mg_serve_report)], C.c_int),
    "mgk_eps_analytic": ([C.c_int, _DP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                          C.c_double, C.c_double, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_eps_grid": ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                      C.c_double, C.c_double, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_assemble": ([C.POINTER(mgk_op_f64), C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                      C.c_void_p, C.c_void_p], C.c_int),
    "mgk_assemble_five": ([C.POINTER(mgk_op_f64), C.POINTER(mgk_op_f32), C.c_double, C.c_double, C.c_void_p,
                           C.c_void_p, C.c_void_p], C.c_int),
    "mgk_rhs": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_galerkin": ([C.POINTER(mgk_op_f64), C.POINTER(mgk_op_f64), C.c_void_p], C.c_int),
    "mgk_coarsen_eps": ([C.POINTER(mgk_op_f64), C.POINTER(mgk_op_f64)] + [C.c_void_p] * 7, C.c_int),
    "mgk_op_to_f32": ([C.POINTER(mgk_op_f64), C.POINTER(mgk_op_f32), C.c_void_p], C.c_int),
    "mgk_smooth_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                        C.c_void_p], C.c_int),
    "mgk_smooth_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                        C.c_void_p], C.c_int),
    "mgk_sor_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p],
                    C.c_int),
    "mgk_sor_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p],
                    C.c_int),
    "mgk_jacobi_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                        C.c_double, C.c_void_p], C.c_int),
    "mgk_residual_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                         C.c_int),
    "mgk_resid_restrict_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                C.c_void_p], C.c_int),
    "mgk_resid_restrict_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                C.c_void_p], C.c_int),
    "mgk_resid_restrict_even_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p], C.c_int),
    "mgk_resid_restrict_even_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p], C.c_int),
    "mgk_prolong_add_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
                            C.c_int),
    "mgk_prolong_add_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
                            C.c_int),
    "mgk_coarse_factor": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_coarse_solve_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p], C.c_int),
    "mgk_coarse_solve_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p], C.c_int),
    "mgk_smooth_fused_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "mgk_smooth_fused_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "mgk_fused_sweeps": ([C.c_int], C.c_int),
    "mgk_smooth_pipe_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                             C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_smooth_pipe_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                             C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_pipe_sweeps": ([C.c_int], C.c_int),
    "mgk_smooth_march_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "mgk_smooth_march_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "mgk_march_sweeps": ([], C.c_int),
    "mgk_march_sweeps_f64": ([], C.c_int),
    "mgk_smooth_variant_info": ([C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)], C.c_int),
    "mgk_smooth_variant_f64": ([C.POINTER(mgk_op_f64), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_smooth_variant_f32": ([C.POINTER(mgk_op_f32), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_line_factor_elems": ([C.c_int, C.c_int, C.c_int], C.c_size_t),
    "mgk_line_factor_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p], C.c_int),
    "mgk_line_factor_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p], C.c_int),
    "mgk_line_rows_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                           C.c_void_p], C.c_int),
    "mgk_line_rows_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                           C.c_void_p], C.c_int),
    "mgk_line_smooth_f64": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                             C.c_int, C.c_void_p], C.c_int),
    "mgk_line_smooth_f32": ([C.POINTER(mgk_op_f32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                             C.c_int, C.c_void_p], C.c_int),
    "mgk_vcycle_line_f64": ([C.c_int, C.POINTER(mgk_op_f64), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                             C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                             C.c_void_p], C.c_int),
    "mgk_vcycle_line_f32": ([C.c_int, C.POINTER(mgk_op_f32), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                             C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                             C.c_void_p], C.c_int),
    "mgk_jacobi_f64_static": ([C.POINTER(mgk_op_f64), C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                               C.c_void_p], C.c_int),
    "mgk_jacobi_f64_static_capacity": ([], C.c_size_t),
    "mgk_server_fail_event_queries": ([C.c_int], None),
    "mgk_fma_rate": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "mgk_fma_rate_flops": ([C.c_int, C.c_int, C.c_int], C.c_double),
    "mgk_vcycle_f64": ([C.c_int, C.POINTER(mgk_op_f64), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                        C.POINTER(C.c_void_p), C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p],
                       C.c_int),
    "mgk_vcycle_f32": ([C.c_int, C.POINTER(mgk_op_f32), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                        C.POINTER(C.c_void_p), C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p],
                       C.c_int),
}

_lib = None


def lib():
    """The loaded libmg.so; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        h = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(h, name)
            f.argtypes = args
            f.restype = res
        _lib = h
    return _lib


def exported_names():
    return list(_SIGS)


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmg status {status}: {msg}")
        self.status = status


def _check(st: int, what: str = ""):
    if st != MG_OK:
        raise MGError(st, (what + ": " if what else "") + lib().mg_last_error().decode())


# ------------------------------------------------------------------ raw names
def mg_last_error() -> str:
    return lib().mg_last_error().decode()


def mg_default_opts() -> mg_solve_opts:
    o = mg_solve_opts()
    lib().mg_default_opts(C.byref(o))
    return o


def mg_create(device: int = 0, mem_budget: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().mg_create(device, mem_budget, C.byref(h)), "mg_create")
    return h.value


def mg_destroy(ctx: int):
    lib().mg_destroy(ctx)


def mg_set_stream(ctx: int, stream_ptr: int):
    _check(lib().mg_set_stream(ctx, stream_ptr), "mg_set_stream")


def mg_mem_info(ctx: int):
    u, b = C.c_size_t(), C.c_size_t()
    _check(lib().mg_mem_info(ctx, C.byref(u), C.byref(b)))
    return u.value, b.value


def _ptr(a) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _mem_kind(*arrays) -> int:
    kinds = set()
    for a in arrays:
        if a is None:
            continue
        if isinstance(a, np.ndarray):
            kinds.add(MG_MEM_HOST)
        else:
            kinds.add(MG_MEM_DEVICE if a.is_cuda else MG_MEM_HOST)
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else MG_MEM_HOST


def _check_array(a, shape, name):
    if a is None:
        return
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(a.shape)} != {tuple(shape)}")
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: need a C-contiguous float64 array")
    else:
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError(f"{name}: need a contiguous float64 tensor")


def grid_desc(grid) -> mg_grid_desc:
    return mg_grid_desc(grid.nx, grid.ny, grid.x0, grid.y0, grid.lx, grid.ly, int(grid.periodic_y),
                        int(getattr(grid, "neumann_y", False)))


def map_desc(mapspec, xp=None, yp=None) -> mg_map_desc:
    m = mg_map_desc()
    m.kind = MAP_CODES[mapspec.kind]
    for k, v in enumerate(list(mapspec.params)[:4]):
        m.params[k] = float(v)
    m.xp = _ptr(xp)
    m.yp = _ptr(yp)
    m.jump_x, m.jump_y = float(mapspec.jump[0]), float(mapspec.jump[1])
    return m


def map_five_point(mapspec) -> bool:
    """Whether the library treats this map's finest operator as a 5-point stencil."""
    m = map_desc(mapspec)
    return bool(lib().mg_map_five_point(C.byref(m)))


def problem_five_point(prob: int) -> bool:
    return bool(lib().mg_problem_five_point(prob))


def mg_setup_transform(ctx: int, grid, mapspec, eps_phys=None, opts: Optional[mg_solve_opts] = None,
                       xp=None, yp=None) -> int:
    """Arrays (xp, yp for a 'grid' map, eps_phys) are numpy (host) or CUDA tensors (device)."""
    if mapspec.kind == "grid" and xp is None:
        xp, yp = np.ascontiguousarray(mapspec.xp), np.ascontiguousarray(mapspec.yp)
    for a, nm in ((xp, "xp"), (yp, "yp"), (eps_phys, "eps_phys")):
        _check_array(a, grid.shape, nm)
    mem = _mem_kind(xp, yp, eps_phys)
    g, m = grid_desc(grid), map_desc(mapspec, xp, yp)
    h = C.c_void_p()
    _check(lib().mg_setup_transform(ctx, C.byref(g), C.byref(m), _ptr(eps_phys), mem,
                                    C.byref(opts) if opts is not None else None, C.byref(h)),
           "mg_setup_transform")
    return h.value


def mg_update_transform(prob: int, grid, mapspec, eps_phys=None, xp=None, yp=None):
    if mapspec.kind == "grid" and xp is None:
        xp, yp = np.ascontiguousarray(mapspec.xp), np.ascontiguousarray(mapspec.yp)
    mem = _mem_kind(xp, yp, eps_phys)
    m = map_desc(mapspec, xp, yp)
    _check(lib().mg_update_transform(prob, C.byref(m), _ptr(eps_phys), mem), "mg_update_transform")


def mg_batch_update_transform(ctx: int, probs: Sequence[int], mapspecs, eps=None, xps=None, yps=None,
                              raise_on_error: bool = True):
    """mg_update_transform for many problems with one synchronisation.  Returns the
    per-instance statuses."""
    n = len(probs)
    xps = xps if xps is not None else [None] * n
    yps = yps if yps is not None else [None] * n
    arrs = []
    maps = (mg_map_desc * max(n, 1))()
    for k, ms in enumerate(mapspecs):
        xp, yp = xps[k], yps[k]
        if ms.kind == "grid" and xp is None:
            xp, yp = np.ascontiguousarray(ms.xp), np.ascontiguousarray(ms.yp)
        maps[k] = map_desc(ms, xp, yp)
        arrs += [xp, yp]
    mem = _mem_kind(*arrs, *([e for e in eps if e is not None] if eps is not None else []))
    P = (C.c_void_p * max(n, 1))(*probs)
    E = (C.c_void_p * max(n, 1))(*[_ptr(e) for e in eps]) if eps is not None else None
    stats = (C.c_int * max(n, 1))()
    st = lib().mg_batch_update_transform(ctx, n, P, maps, E, mem, stats)
    if raise_on_error:
        _check(st, "mg_batch_update_transform")
    return [stats[k] for k in range(n)]


def mg_problem_free(prob: int):
    lib().mg_problem_free(prob)


def mg_problem_info(prob: int):
    L = C.c_int()
    nx = (C.c_int * 24)()
    ny = (C.c_int * 24)()
    _check(lib().mg_problem_info(prob, C.byref(L), nx, ny))
    return [(nx[k], ny[k]) for k in range(L.value)]


def mg_solve(prob: int, rho_phys, bc, phi, opts: Optional[mg_solve_opts] = None,
             allow_not_converged: bool = False) -> mg_solve_stats:
    """rho_phys, bc (nullable), phi: numpy arrays (host) or CUDA tensors (device)."""
    mem = _mem_kind(rho_phys, bc, phi)
    stats = mg_solve_stats()
    st = lib().mg_solve(prob, _ptr(rho_phys), _ptr(bc), _ptr(phi), mem,
                        C.byref(opts) if opts is not None else None, C.byref(stats))
    if st == MG_ERR_NOT_CONVERGED and allow_not_converged:
        return stats
    _check(st, "mg_solve")
    return stats


def mg_cycle_time(prob: int, opts: Optional[mg_solve_opts] = None, reps: int = 10) -> float:
    """Milliseconds per multigrid cycle of a resident problem (see mg.h)."""
    ms = C.c_double()
    _check(lib().mg_cycle_time(prob, C.byref(opts) if opts is not None else None, reps, C.byref(ms)),
           "mg_cycle_time")
    return ms.value


def mg_batch_solve(ctx: int, probs: Sequence[int], rhos, bcs, phis,
                   opts: Optional[mg_solve_opts] = None):
    n = len(probs)
    mem = _mem_kind(*rhos, *phis, *[b for b in (bcs or []) if b is not None])
    P = (C.c_void_p * n)(*probs)
    R = (C.c_void_p * n)(*[_ptr(a) for a in rhos])
    B = (C.c_void_p * n)(*[_ptr(a) for a in bcs]) if bcs is not None else None
    X = (C.c_void_p * n)(*[_ptr(a) for a in phis])
    stats = (mg_solve_stats * max(n, 1))()
    _check(lib().mg_batch_solve(ctx, n, P, R, B, X, mem, C.byref(opts) if opts is not None else None,
                                stats), "mg_batch_solve")
    return list(stats)[:n]


def mg_harmonic_grid(ctx: int, grid, fixed, xp, yp, xp_out, yp_out, rtol: float = 1e-12):
    """Discrete-harmonic x', y' (Sec. 4.2) with Dirichlet data on the outer ring and where
    `fixed` (uint8 node array) is nonzero.  numpy arrays (host) or CUDA tensors (device).
    Returns the two solves' statistics."""
    mem = _mem_kind(xp, yp, xp_out, yp_out)
    for a, nm in ((xp, "xp"), (yp, "yp"), (xp_out, "xp_out"), (yp_out, "yp_out")):
        _check_array(a, grid.shape, nm)
    if tuple(fixed.shape) != tuple(grid.shape):
        raise ValueError("fixed: wrong shape")
    stats = (mg_solve_stats * 2)()
    _check(lib().mg_harmonic_grid(ctx, C.byref(grid_desc(grid)), _ptr(fixed), _ptr(xp), _ptr(yp),
                                  _ptr(xp_out), _ptr(yp_out), mem, rtol, stats), "mg_harmonic_grid")
    return list(stats)


def mg_autotune(ctx: int, max_side: int = 2049, variants: bool = False):
    """Time the smoother families (every variant of each) per level size and make the fastest
    the context's choice.  Returns [(precision, side, {family: best ms}, chosen family)], with
    a fifth element {"tile": (tx, ty), "sweeps": ns} for the chosen variant if variants=True."""
    r = mg_tune_report()
    _check(lib().mg_autotune(ctx, max_side, C.byref(r)), "mg_autotune")
    out = []
    for k in range(r.count):
        e = r.entry[k]
        ms = {SMOOTHER_FAMILIES[f + 1]: float(e.ms[f]) for f in range(4) if e.ms[f] > 0}
        row = ("mixed" if e.precision == MG_PREC_MIXED else "fp64", e.side, ms,
               SMOOTHER_FAMILIES.get(e.choice, "default"))
        if variants:
            row = row + ({"tile": (e.tile_x, e.tile_y), "sweeps": e.sweeps_per_launch},)
        out.append(row)
    return out


def mg_server_start(ctx: int, max_inflight=16, queue_capacity=65536, mem_budget=0, host_budget=0) -> int:
    o = mg_server_opts(max_inflight, queue_capacity, mem_budget, host_budget)
    h = C.c_void_p()
    _check(lib().mg_server_start(ctx, C.byref(o), C.byref(h)), "mg_server_start")
    return h.value


def mg_serve_submit(srv: int, grid, mapspec, rho_phys, bc=None, eps_phys=None,
                    opts: Optional[mg_solve_opts] = None):
    """Host arrays only (copied in at submit).  Returns (status, ticket)."""
    xp = yp = None
    if mapspec.kind == "grid":
        xp, yp = np.ascontiguousarray(mapspec.xp), np.ascontiguousarray(mapspec.yp)
    rq = mg_request()
    rq.grid = grid_desc(grid)
    rq.map = map_desc(mapspec, xp, yp)
    rq.eps_phys = _ptr(eps_phys)
    rq.rho_phys = _ptr(rho_phys)
    rq.bc = _ptr(bc)
    rq.opts = opts if opts is not None else mg_default_opts()
    t = C.c_uint64()
    st = lib().mg_serve_submit(srv, C.byref(rq), C.byref(t))
    return st, t.value


def mg_serve_poll(srv: int, ticket: int, timeout_ms: int, phi_out: Optional[np.ndarray]):
    stats = mg_solve_stats()
    st = lib().mg_serve_poll(srv, ticket, timeout_ms, _ptr(phi_out), C.byref(stats))
    return st, stats


def mg_server_stop(srv: int) -> mg_serve_report:
    r = mg_serve_report()
    _check(lib().mg_server_stop(srv, C.byref(r)), "mg_server_stop")
    return r


# ------------------------------------------------------------------ kernel-level (mgk_*)
def op_struct(arrays, nx, ny, periodic, f32=False, five_point=False):
    """mgk_op_f64/f32 from six pitched CUDA tensors (cE, cN, cNE, cNW, diag, dinv);
    five_point: the NE / NW arrays hold zeros and the kernels skip them."""
    s = (mgk_op_f32 if f32 else mgk_op_f64)()
    s.nx, s.ny, s.periodic, s.pitch = nx, ny, int(periodic), int(arrays[0].shape[-1])
    s.five_point = int(bool(five_point))
    for name, a in zip(("cE", "cN", "cNE", "cNW", "diag", "dinv"), arrays):
        setattr(s, name, a.data_ptr())
    return s


def _stream(stream=None) -> int:
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def smooth_variants(f32: bool, family: int):
    """[(variant, (tile_x, tile_y), sweeps)] of a smoother family (2 fused, 3 pipelined,
    4 marching) in FP32 or FP64."""
    out, v = [], 0
    tx, ty, ns = C.c_int(), C.c_int(), C.c_int()
    while lib().mgk_smooth_variant_info(int(f32), family, v, C.byref(tx), C.byref(ty), C.byref(ns)) == 0:
        out.append((v, (tx.value, ty.value), ns.value))
        v += 1
    return out


def mgk(name: str, *args):
    """Call a kernel-level entry point by name; raises on a non-zero return."""
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        raise MGError(rc, f"{name} returned {rc}")


# ------------------------------------------------------------------ convenience classes
class Context:
    """A library context.  Problems made on it are closed before it is (a problem must not
    outlive its context: its memory belongs to the context's pool)."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        import weakref
        self.h = mg_create(device, mem_budget)
        self._problems = weakref.WeakSet()

    def use_torch_stream(self):
        mg_set_stream(self.h, _stream())

    def mem_info(self):
        return mg_mem_info(self.h)

    def close(self):
        if self.h:
            for p in list(self._problems):
                p.close()
            mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """A resident problem (coefficients + hierarchy) for one instance."""

    def __init__(self, ctx: Context, inst, opts: Optional[mg_solve_opts] = None, device_inputs=False):
        self.ctx, self.inst = ctx, inst
        self.opts = opts if opts is not None else mg_default_opts()
        xp = yp = eps = None
        if inst.map.kind == "grid":
            xp, yp = np.ascontiguousarray(inst.map.xp), np.ascontiguousarray(inst.map.yp)
        if inst.eps_phys is not None:
            eps = np.ascontiguousarray(inst.eps_phys, dtype=np.float64)
        if device_inputs:
            import torch
            xp = None if xp is None else torch.from_numpy(np.array(xp)).cuda()
            yp = None if yp is None else torch.from_numpy(np.array(yp)).cuda()
            eps = None if eps is None else torch.from_numpy(eps).cuda()
        self.h = mg_setup_transform(ctx.h, inst.grid, inst.map, eps, self.opts, xp, yp)
        ctx._problems.add(self)

    def levels(self):
        return mg_problem_info(self.h)

    def solve(self, rho=None, bc=None, phi=None, opts=None, allow_not_converged=False):
        inst = self.inst
        rho = np.ascontiguousarray(inst.rho_phys, dtype=np.float64) if rho is None else rho
        if bc is None and inst.bc is not None:
            bc = np.ascontiguousarray(inst.bc, dtype=np.float64)
            if not isinstance(rho, np.ndarray):
                import torch
                bc = torch.from_numpy(bc).to(rho.device)
        if phi is None:
            phi = np.zeros(inst.grid.shape) if isinstance(rho, np.ndarray) else rho.new_zeros(inst.grid.shape)
        st = mg_solve(self.h, rho, bc, phi, opts if opts is not None else self.opts, allow_not_converged)
        return phi, st

    def close(self):
        if self.h:
            if self.ctx.h:  # a destroyed context has already released the problem
                mg_problem_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_COARSE_OPS = {"galerkin": 0, "rediscretize": 1}


def make_opts(precision="fp64", outer="fcg", rtol=1e-10, max_iters=200, nu1=2, nu2=2,
              smoother="gs4", coarse_max=64, omega_j=0.8, warm_start=False,
              coarse_op="galerkin") -> mg_solve_opts:
    o = mg_default_opts()
    o.precision = MG_PREC_MIXED if precision == "mixed" else MG_PREC_FP64
    if outer not in _OUTERS:
        raise ValueError(f"unknown outer iteration {outer!r} (one of {sorted(_OUTERS)})")
    o.outer = _OUTERS[outer]
    if smoother not in _SMOOTHERS:
        raise ValueError(f"unknown smoother {smoother!r} (one of {sorted(_SMOOTHERS)})")
    o.smoother = _SMOOTHERS[smoother]
    o.rtol, o.max_iters, o.nu1, o.nu2 = rtol, max_iters, nu1, nu2
    o.coarse_max, o.omega_j, o.warm_start = coarse_max, omega_j, int(warm_start)
    if coarse_op not in _COARSE_OPS:
        raise ValueError(f"unknown coarse operator {coarse_op!r} (one of {sorted(_COARSE_OPS)})")
    o.coarse_op = _COARSE_OPS[coarse_op]
    return o
