"""ctypes declarations of the C ABI in include/bddc.h (argument marshalling only).

The shared library is built in-tree by ``paper_1201_5991_gb300.build``.  There is no
fallback: if the library is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbddc_gb300.so")
MAX_LEVELS = 6

OK = 0
ERR_INVALID = -1
ERR_BREAKDOWN = -2
ERR_NOT_CONVERGED = -3
ERR_NAN = -4
ERR_CUDA = -5
ERR_OOM = -6
ERR_TIMEOUT = -7

POISSON = 0
ELASTICITY = 1
STOKES = 2
CORNERS, EDGES, FACES = 1, 2, 4
PREC_FP64, PREC_MIXED = 0, 1
WEIGHTS_STIFFNESS, WEIGHTS_MULTIPLICITY = 0, 1
KRYLOV_AUTO, KRYLOV_PCG, KRYLOV_BICGSTAB, KRYLOV_FGMRES = 0, 1, 2, 3

EXPORTED = [
    "bddc_default_opts", "bddc_analyze", "bddc_setup", "bddc_update_coef", "bddc_solve",
    "bddc_solve_host", "bddc_apply_precond", "bddc_apply_schur", "bddc_grad", "bddc_get_maps",
    "bddc_get_stats", "bddc_sizes", "bddc_free", "bddc_last_error", "bddc_kernel_launches",
    "bddc_reset_profile", "bddc_grad_noalloc", "bddc_batching_ablation", "bddc_get_coarse",
    "bddc_tc_update_check", "bddc_apply_inner_schur",
]
(PROF_TRSV, PROF_FACTOR, PROF_SPMV, PROF_TRMV, PROF_TRSV_IFACE, PROF_COARSE, PROF_TC_UPDATE, PROF_TC_PANEL,
 PROF_CLASSES) = (0, 1, 2, 3, 4, 5, 6, 7, 8)


class Mesh(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nodes_per_elem", C.c_int), ("dofs_per_node", C.c_int), ("physics", C.c_int),
        ("n_nodes", C.c_int64), ("n_elems", C.c_int64),
        ("coords", C.POINTER(C.c_double)), ("conn", C.POINTER(C.c_int32)), ("coef", C.POINTER(C.c_double)),
        ("nu", C.c_double), ("dirichlet", C.POINTER(C.c_uint8)), ("dir_values", C.POINTER(C.c_double)),
    ]


class Partition(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int),
        ("part", C.POINTER(C.c_int32) * (MAX_LEVELS - 1)),
        ("n_parts", C.c_int64 * (MAX_LEVELS - 1)),
    ]


class Opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("weights", C.c_int), ("all_corners", C.c_uint), ("maxit", C.c_int),
        ("refine_steps", C.c_int), ("flexible", C.c_int), ("use_graph", C.c_int), ("verbose", C.c_int),
        ("profile", C.c_int), ("tensor_cores", C.c_int), ("inner_steps", C.c_int), ("inner_tol", C.c_double),
        ("krylov", C.c_int), ("autotune", C.c_int), ("wait_probe", C.c_int), ("inner_operator", C.c_int),
        ("retain_host_memory", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double), ("rhs_norm", C.c_double),
        ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("n_levels", C.c_int),
        ("n_sub", C.c_int64 * MAX_LEVELS), ("n_dof", C.c_int64 * MAX_LEVELS),
        ("n_iface", C.c_int64 * MAX_LEVELS), ("n_coarse", C.c_int64 * MAX_LEVELS),
        ("n_promoted", C.c_int64 * MAX_LEVELS), ("breakdown_level", C.c_int), ("breakdown_sub", C.c_int),
        ("refine_steps", C.c_int), ("inner_steps", C.c_int), ("outer_iterations", C.c_int),
        ("analysis_ms", C.c_double), ("factor_ms", C.c_double),
        ("solve_ms", C.c_double), ("factor_bytes", C.c_int64),
        ("prof_ms", C.c_double * PROF_CLASSES), ("prof_launches", C.c_int64 * PROF_CLASSES),
        ("prof_bytes", C.c_double * PROF_CLASSES), ("prof_flops", C.c_double * PROF_CLASSES),
        ("sweep_ctas", C.c_int * (2 * MAX_LEVELS)), ("sweep_deep", C.c_int * (2 * MAX_LEVELS)),
        ("sweep_order", C.c_int * (2 * MAX_LEVELS)), ("tune_ms", C.c_double), ("prepare_ms", C.c_double),
        ("inner_operator", C.c_int),
    ]


class LevelMaps(C.Structure):
    _fields_ = [
        ("n_dof", C.c_int64), ("n_sub", C.c_int64), ("n_iface", C.c_int64), ("n_coarse", C.c_int64),
        ("n_globs", C.c_int64), ("n_promoted", C.c_int64),
        ("iface_dofs", C.POINTER(C.c_int64)), ("sub_dof_ptr", C.POINTER(C.c_int64)),
        ("sub_dofs", C.POINTER(C.c_int64)), ("sub_nI", C.POINTER(C.c_int64)),
        ("sub_iface", C.POINTER(C.c_int64)), ("sub_wmult", C.POINTER(C.c_double)),
        ("sub_coarse_ptr", C.POINTER(C.c_int64)), ("sub_coarse", C.POINTER(C.c_int64)),
        ("c_ptr", C.POINTER(C.c_int64)), ("c_col", C.POINTER(C.c_int64)), ("c_val", C.POINTER(C.c_double)),
        ("glob_ptr", C.POINTER(C.c_int64)), ("glob_nodes", C.POINTER(C.c_int64)),
        ("glob_kind", C.POINTER(C.c_int32)), ("glob_promoted", C.POINTER(C.c_int32)),
        ("coarse_glob", C.POINTER(C.c_int64)), ("coarse_comp", C.POINTER(C.c_int32)),
    ]


_lib = None


def lib() -> C.CDLL:
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1201_5991_gb300.build`")
    L = C.CDLL(LIB_PATH)
    H = C.c_void_p
    P = C.c_void_p
    L.bddc_default_opts.argtypes = [C.POINTER(Opts)]
    L.bddc_default_opts.restype = None
    L.bddc_analyze.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), C.c_uint, C.POINTER(Opts), C.POINTER(H)]
    L.bddc_setup.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), C.c_uint, C.POINTER(Opts), P, C.POINTER(H)]
    L.bddc_update_coef.argtypes = [H, C.POINTER(C.c_double)]
    L.bddc_solve.argtypes = [H, P, P, C.c_int, C.c_double, C.POINTER(Stats)]
    L.bddc_solve_host.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_double,
                                  C.POINTER(Stats)]
    L.bddc_apply_precond.argtypes = [H, P, P, C.c_int]
    L.bddc_apply_schur.argtypes = [H, P, P, C.c_int]
    L.bddc_apply_inner_schur.argtypes = [H, P, P, C.c_int]
    L.bddc_grad.argtypes = [H, P, P, C.c_int, C.c_double, P, P]
    L.bddc_grad_noalloc.argtypes = [H, P, P, C.c_int, C.c_double, P, P]
    L.bddc_get_maps.argtypes = [H, C.c_int, C.POINTER(LevelMaps)]
    L.bddc_get_coarse.argtypes = [H, C.c_int, C.POINTER(C.c_double), C.c_int64]
    L.bddc_tc_update_check.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_double)]
    L.bddc_get_stats.argtypes = [H, C.POINTER(Stats)]
    L.bddc_sizes.argtypes = [H, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.bddc_free.argtypes = [H]
    L.bddc_free.restype = None
    L.bddc_last_error.argtypes = []
    L.bddc_last_error.restype = C.c_char_p
    L.bddc_kernel_launches.argtypes = []
    L.bddc_kernel_launches.restype = C.c_int64
    L.bddc_reset_profile.argtypes = [H]
    L.bddc_batching_ablation.argtypes = [H, C.POINTER(C.c_double)]
    for name in EXPORTED:
        if name not in ("bddc_default_opts", "bddc_free", "bddc_last_error", "bddc_kernel_launches"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class BddcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bddc error {code}: {msg}")
        self.code = code


def check(code: int, allow=()):
    if code != OK and code not in allow:
        raise BddcError(code, lib().bddc_last_error().decode())
    return code
