"""ctypes declarations of the C ABI in include/stokes.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU
fallback for any entry point.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_stokes.so")

STOKES_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NOT_CONVERGED",
          -5: "ERR_BREAKDOWN", -6: "ERR_NAN", -7: "ERR_TIMEOUT", -8: "ERR_INCOMPATIBLE_RHS",
          -9: "ERR_MESH"}

METHOD_SCHUR, METHOD_COUPLED = 0, 1
SCHUR_PREC_LUMPED, SCHUR_PREC_LAPLACE, SCHUR_PREC_MASS = 0, 1, 2
PRECISION_FP64, PRECISION_MIXED = 0, 1

OP = dict(A=0, A3=1, B=2, BT=3, MQ=4, LQ=5, KQ=6, LUMPED_INV=7, VCYCLE_A3=8, VCYCLE_KQ=9,
          SCHUR_PREC=10, SCHUR=11, AGAMMA=12, PROLONG_P2=13, RESTRICT_P2=14, PROLONG_P1=15,
          LOAD=16, A_DF=17, VCYCLE_VEL=18)
MAT = dict(A=0, A3=1, B=2, BT=3, MQ=4, LQ=5, KQ=6, LUMPED=7, AV=8)
KERNEL = dict(SPMM_A3=0, SPMV_A=1, B=2, BT=3, SPMV_P1=4, TRANSFER=5, BLAS1=6, OTHER=7,
              SPMM_A3_COARSE=8, RESIDUAL=9, COARSE_CYCLE=10)


class StokesOptions(C.Structure):
    _fields_ = [
        ("method", C.c_int), ("schur_prec", C.c_int), ("precision", C.c_int),
        ("vcycles", C.c_int), ("cheb_degree", C.c_int), ("mass_steps", C.c_int),
        ("mass_steps_al", C.c_int), ("restart", C.c_int), ("block_lu", C.c_int),
        ("m2_inner_cg", C.c_int), ("inner_tol", C.c_double), ("schur_inner_tol", C.c_double),
        ("eps_pressure", C.c_double), ("max_outer", C.c_int), ("max_inner", C.c_int),
        ("max_refine", C.c_int), ("profile", C.c_int), ("spmv_group", C.c_int),
        ("schur_inner_iters", C.c_int), ("pass_tol", C.c_double), ("format", C.c_int),
        ("graphs", C.c_int), ("vel_prec", C.c_int), ("mass_steps_v", C.c_int),
        ("coarse_kernel", C.c_int), ("pass_schedule", C.c_int),
        ("cheb_low", C.c_double), ("cheb_high", C.c_double), ("sym_batch", C.c_int),
        ("stencil_min_rows", C.c_int),
        ("host_wait", C.c_int),
        ("vcycle_split", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StokesInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters", C.c_int), ("refinements", C.c_int),
                ("status", C.c_int), ("rel_residual", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with paper_2407_01783_gb300.build.build() "
            "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    i64p = C.POINTER(C.c_int64)
    lib.stokes_default_options.argtypes = [C.POINTER(StokesOptions)]
    lib.stokes_default_options.restype = None
    lib.stokes_setup.argtypes = [C.c_int, vp, C.c_double, C.c_double, C.c_double,
                                 C.POINTER(StokesOptions), vp, C.POINTER(vp)]
    lib.stokes_setup.restype = C.c_int
    for name in ("stokes_solve", "stokes_solve_host"):
        fn = getattr(lib, name)
        fn.argtypes = [vp, vp, vp, C.c_double, vp, vp, C.POINTER(StokesInfo)]
        fn.restype = C.c_int
    lib.stokes_solve_multi.argtypes = [vp, C.c_int, vp, vp, C.c_double, vp, vp, C.POINTER(StokesInfo)]
    lib.stokes_solve_multi.restype = C.c_int
    lib.stokes_adjoint.argtypes = [vp, vp, vp, C.c_double, vp, vp, dp, C.POINTER(StokesInfo)]
    lib.stokes_adjoint.restype = C.c_int
    lib.stokes_destroy.argtypes = [vp]
    lib.stokes_destroy.restype = C.c_int
    lib.stokes_status_string.argtypes = [C.c_int]
    lib.stokes_status_string.restype = C.c_char_p
    lib.stokes_last_error.argtypes = []
    lib.stokes_last_error.restype = C.c_char_p
    lib.stokes_apply.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    lib.stokes_apply.restype = C.c_int
    lib.stokes_apply_agamma_noalloc.argtypes = [vp, vp, vp]
    lib.stokes_apply_agamma_noalloc.restype = C.c_int
    lib.stokes_matrix_shape.argtypes = [vp, C.c_int, C.c_int, i64p]
    lib.stokes_matrix_shape.restype = C.c_int
    lib.stokes_matrix_export.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
    lib.stokes_matrix_export.restype = C.c_int
    lib.stokes_sizes.argtypes = [vp, i64p]
    lib.stokes_sizes.restype = C.c_int
    lib.stokes_kernel_stats.argtypes = [vp, C.c_int, i64p, dp, dp]
    lib.stokes_kernel_stats.restype = C.c_int
    lib.stokes_kernel_timing.argtypes = [vp, C.c_int, i64p, dp, dp]
    lib.stokes_kernel_timing.restype = C.c_int
    lib.stokes_kernel_stats_reset.argtypes = [vp]
    lib.stokes_kernel_stats_reset.restype = C.c_int
    lib.stokes_profile_mode.argtypes = [vp, C.c_int]
    lib.stokes_profile_mode.restype = C.c_int
    lib.stokes_setup_phases.argtypes = [vp, dp]
    lib.stokes_setup_phases.restype = C.c_int
    lib.stokes_check_bounded_wait.argtypes = [vp]
    lib.stokes_check_bounded_wait.restype = C.c_int
    _ = ip
    _lib = lib
    return lib


# names declared in include/stokes.h (checked by the CPU test suite)
EXPORTS = ["stokes_default_options", "stokes_setup", "stokes_solve", "stokes_solve_host", "stokes_solve_multi",
           "stokes_adjoint", "stokes_destroy", "stokes_status_string", "stokes_last_error",
           "stokes_apply", "stokes_apply_agamma_noalloc", "stokes_matrix_shape", "stokes_matrix_export", "stokes_sizes",
           "stokes_kernel_stats", "stokes_kernel_timing", "stokes_kernel_stats_reset", "stokes_profile_mode",
           "stokes_setup_phases",
           "stokes_check_bounded_wait"]
SETUP_PHASES = ("assembly", "storage", "coarse", "spectra", "copies", "tuning")
