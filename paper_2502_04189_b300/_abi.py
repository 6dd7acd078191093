"""ctypes declarations of the C ABI in include/fizzy_proj.h (no logic here)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfizzyproj.so")

FIZZY_OK = 0
ERRORS = {-1: "invalid argument", -2: "unsupported size", -3: "out of device memory",
          -4: "CUDA error", -5: "not converged", -6: "device wait timeout"}

# every symbol include/fizzy_proj.h declares
EXPORTED = ("fizzy_proj_plan", "fizzy_proj_workspace_bytes", "fizzy_proj_solve",
            "fizzy_proj_get_stats", "fizzy_proj_solve_host", "fizzy_proj_destroy",
            "fizzy_proj_errstr", "fizzy_proj_last_error", "fizzy_proj_launches_per_solve",
            "fizzy_proj_set_timing", "fizzy_proj_timing", "fizzy_proj_solve_noalloc",
            "fizzy_proj_batch_create", "fizzy_proj_batch_solve", "fizzy_proj_batch_status",
            "fizzy_proj_batch_autotune", "fizzy_proj_batch_info", "fizzy_proj_batch_destroy",
            "fizzy_proj_set_physics", "fizzy_serve_create", "fizzy_serve_admit", "fizzy_serve_stream",
            "fizzy_serve_launch", "fizzy_serve_poll", "fizzy_serve_stats", "fizzy_serve_release",
            "fizzy_serve_info", "fizzy_serve_destroy", "fizzy_proj_solve_host_async",
            "fizzy_proj_host_wait", "fizzy_crop_fill", "fizzy_proj_batch_inject_stall",
            "fizzy_proj_solve_vc", "fizzy_acdi_step", "fizzy_probe_fma_rate",
            "fizzy_poisson_solve")
ERRORS[-7] = "busy"
NOALLOC_MAX_CELLS = 262144
DEFAULT_MAX_REFINE = 4  # FIZZY_DEFAULT_MAX_REFINE


class Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("zf", ctypes.POINTER(ctypes.c_double)),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("div_tol", ctypes.c_double),
                ("flags", ctypes.c_uint), ("periodic_z", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("flux_planes", ctypes.c_int),
                ("x_lines", ctypes.c_int), ("y_cols", ctypes.c_int), ("order", ctypes.c_int),
                ("form", ctypes.c_int), ("chains", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres", ctypes.c_double), ("f_max", ctypes.c_double),
                ("div_max", ctypes.c_double), ("u_rms", ctypes.c_double),
                ("div_metric", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def lib():
    """Load libfizzyproj.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run paper_2502_04189_b300/build.py "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        L.fizzy_proj_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Desc), vp]
        L.fizzy_proj_plan.restype = ctypes.c_int
        L.fizzy_proj_workspace_bytes.argtypes = [ctypes.POINTER(Desc)]
        L.fizzy_proj_workspace_bytes.restype = ctypes.c_size_t
        L.fizzy_proj_solve.argtypes = [vp] + [vp] * 7 + [ctypes.POINTER(Stats), vp]
        L.fizzy_proj_solve.restype = ctypes.c_int
        L.fizzy_proj_solve_vc.argtypes = [vp] + [vp] * 5 + [ctypes.c_int, ctypes.c_double,
                                                             ctypes.POINTER(Stats), vp]
        L.fizzy_proj_solve_vc.restype = ctypes.c_int
        L.fizzy_acdi_step.argtypes = [vp] + [vp] * 4 + [ctypes.c_double] * 3 + [vp, vp, vp]
        L.fizzy_acdi_step.restype = ctypes.c_int
        L.fizzy_proj_solve_host.argtypes = [vp] + [vp] * 7 + [ctypes.POINTER(Stats), vp]
        L.fizzy_proj_solve_host.restype = ctypes.c_int
        L.fizzy_proj_solve_host_async.argtypes = [vp] + [vp] * 10 + [vp]
        L.fizzy_proj_solve_host_async.restype = ctypes.c_int
        L.fizzy_proj_host_wait.argtypes = [vp]
        L.fizzy_proj_host_wait.restype = ctypes.c_int
        L.fizzy_proj_get_stats.argtypes = [vp, ctypes.POINTER(Stats), vp]
        L.fizzy_proj_get_stats.restype = ctypes.c_int
        L.fizzy_proj_destroy.argtypes = [vp]
        L.fizzy_proj_destroy.restype = ctypes.c_int
        L.fizzy_proj_errstr.argtypes = [ctypes.c_int]
        L.fizzy_proj_errstr.restype = ctypes.c_char_p
        L.fizzy_proj_last_error.argtypes = [vp]
        L.fizzy_proj_last_error.restype = ctypes.c_char_p
        L.fizzy_proj_launches_per_solve.argtypes = [vp]
        L.fizzy_proj_launches_per_solve.restype = ctypes.c_int
        L.fizzy_proj_set_timing.argtypes = [vp, ctypes.c_int]
        L.fizzy_proj_set_timing.restype = ctypes.c_int
        L.fizzy_proj_timing.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        L.fizzy_proj_timing.restype = ctypes.c_int
        L.fizzy_proj_solve_noalloc.argtypes = [ctypes.POINTER(Desc)] + [vp] * 7 + [vp]
        L.fizzy_proj_solve_noalloc.restype = ctypes.c_int
        L.fizzy_proj_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                              ctypes.POINTER(vp), ctypes.POINTER(Tuning), vp]
        L.fizzy_proj_batch_create.restype = ctypes.c_int
        L.fizzy_proj_batch_solve.argtypes = [vp, vp]
        L.fizzy_proj_batch_solve.restype = ctypes.c_int
        L.fizzy_proj_batch_status.argtypes = [vp, vp]
        L.fizzy_proj_batch_status.restype = ctypes.c_int
        L.fizzy_proj_batch_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Tuning),
                                                ctypes.POINTER(ctypes.c_double), vp]
        L.fizzy_proj_batch_autotune.restype = ctypes.c_int
        L.fizzy_proj_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]
        L.fizzy_proj_batch_info.restype = ctypes.c_int
        L.fizzy_proj_batch_inject_stall.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
        L.fizzy_proj_batch_inject_stall.restype = ctypes.c_int
        L.fizzy_proj_batch_destroy.argtypes = [vp]
        L.fizzy_proj_batch_destroy.restype = ctypes.c_int
        D = ctypes.c_double
        L.fizzy_proj_set_physics.argtypes = [vp, D, D, D, vp]
        L.fizzy_proj_set_physics.restype = ctypes.c_int
        L.fizzy_serve_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, ctypes.c_int]
        L.fizzy_serve_create.restype = ctypes.c_int
        L.fizzy_serve_admit.argtypes = [vp, ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(vp)]
        L.fizzy_serve_admit.restype = ctypes.c_int
        L.fizzy_serve_stream.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
        L.fizzy_serve_stream.restype = ctypes.c_int
        L.fizzy_serve_launch.argtypes = [vp, ctypes.c_int]
        L.fizzy_serve_launch.restype = ctypes.c_int
        L.fizzy_serve_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.fizzy_serve_poll.restype = ctypes.c_int
        L.fizzy_serve_stats.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Stats)]
        L.fizzy_serve_stats.restype = ctypes.c_int
        L.fizzy_serve_release.argtypes = [vp, ctypes.c_int]
        L.fizzy_serve_release.restype = ctypes.c_int
        L.fizzy_serve_info.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.fizzy_serve_info.restype = ctypes.c_int
        L.fizzy_serve_destroy.argtypes = [vp]
        L.fizzy_serve_destroy.restype = ctypes.c_int
        L.fizzy_crop_fill.argtypes = [ctypes.POINTER(vp)] + [ctypes.c_int] * 3 + [ctypes.POINTER(vp)] + \
            [ctypes.c_int] * 8 + [vp]
        L.fizzy_crop_fill.restype = ctypes.c_int
        L.fizzy_probe_fma_rate.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_double),
                                                                 ctypes.POINTER(ctypes.c_double), vp]
        L.fizzy_probe_fma_rate.restype = ctypes.c_int
        L.fizzy_poisson_solve.argtypes = [vp, vp, vp, ctypes.POINTER(Stats), vp]
        L.fizzy_poisson_solve.restype = ctypes.c_int
        _lib = L
    return _lib
