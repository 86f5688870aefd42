"""ctypes binding of libcutmg.so (include/cutmg.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels; there is no Python
or CPU fallback.  Loading fails loudly when the library has not been built.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcutmg.so")

CF_OK, CF_EINVAL, CF_ENOMEM, CF_ECUDA, CF_ENOCONV, CF_ETIMEOUT, CF_EUNSUPPORTED = range(7)
CF_LS_SPHERE, CF_LS_PLANE, CF_LS_ELLIPSOID, CF_LS_TORUS, CF_LS_FLOWER, CF_LS_CALLBACK = 0, 1, 2, 3, 4, 5
CF_FP64, CF_MIXED = 0, 1
CF_SMOOTHER_MVS, CF_SMOOTHER_CHEBYSHEV = 0, 1
CF_K_CUT_SOLVE, CF_K_INTERIOR, CF_K_APPLY_BULK, CF_K_APPLY_BND, CF_K_FACE_MOMENTS = 1, 2, 3, 4, 5
CF_VAR_INTERIOR, CF_VAR_CUT, CF_VAR_OPERATOR = 1, 2, 3

EXPORTED = [
    "cf_setup", "cf_destroy", "cf_last_error", "cf_n_levels", "cf_n_dofs", "cf_level_n_dofs",
    "cf_dof_lattice", "cf_dof_coords", "cf_stats", "cf_work_model", "cf_footprint", "cf_problem_footprint", "cf_set_precision", "cf_rhs", "cf_apply",
    "cf_vcycle", "cf_solve", "cf_solve_vcycle", "cf_solve_gmres", "cf_rhs_user", "cf_host_rhs_user", "cf_level_apply", "cf_level_colour_step", "cf_level_smooth",
    "cf_level_restrict", "cf_level_prolongate", "cf_coarse_solve", "cf_setup_host", "cf_host_rhs",
    "cf_host_cell_matrix", "cf_host_patch_counts", "cf_host_interior_update", "cf_host_diagonal", "cf_host_interior_patch", "cf_host_cut_patch",
    "cf_host_coarse_inverse",
    "cf_set_kernel_variant", "cf_set_wait_limit", "cf_launch_count", "cf_profile_start", "cf_profile_start_level", "cf_profile_read", "cf_coarse_solve_noalloc",
    "cf_batch_create", "cf_batch_solve", "cf_batch_launch_count", "cf_batch_destroy",
    "cf_server_create", "cf_server_submit", "cf_server_run", "cf_server_result", "cf_server_stats",
    "cf_server_destroy",
]


class cf_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_cells", ctypes.c_int), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("n_levels", ctypes.c_int)]


# double phi(const double* x, void* user); void grad(const double* x, double* g, void* user)
PHI_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)
GRAD_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class cf_levelset(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("center", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("normal", ctypes.c_double * 3), ("offset", ctypes.c_double),
                ("axes", ctypes.c_double * 3), ("rot", ctypes.c_double * 9), ("major", ctypes.c_double),
                ("lobes", ctypes.c_int), ("amplitude", ctypes.c_double), ("phase", ctypes.c_double),
                ("phi", PHI_FN), ("grad", GRAD_FN), ("user", ctypes.c_void_p)]


class cf_params(ctypes.Structure):
    _fields_ = [("gamma_D", ctypes.c_double), ("gamma_ghost", ctypes.c_double * 4), ("n_c", ctypes.c_int),
                ("quad_q", ctypes.c_int), ("precision", ctypes.c_int), ("smoother", ctypes.c_int),
                ("smoother_degree", ctypes.c_int), ("setup_threads", ctypes.c_int)]


# double f(const double* x, void* user)
DATA_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class cf_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class CutmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cutmg status {status}: {msg}")
        self.status = status


_lib = None


def load():
    """Load the shared library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2508_11608_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.cf_setup.argtypes = [ctypes.POINTER(cf_mesh), ctypes.POINTER(cf_levelset), I,
                             ctypes.POINTER(cf_params), V, ctypes.POINTER(P)]
    lib.cf_setup_host.argtypes = [ctypes.POINTER(cf_mesh), ctypes.POINTER(cf_levelset), I,
                                  ctypes.POINTER(cf_params), ctypes.POINTER(P)]
    lib.cf_destroy.argtypes = [P]
    lib.cf_destroy.restype = None
    lib.cf_last_error.restype = ctypes.c_char_p
    lib.cf_n_levels.argtypes = [P]
    lib.cf_n_dofs.argtypes = [P]
    lib.cf_n_dofs.restype = ctypes.c_int64
    lib.cf_level_n_dofs.argtypes = [P, I]
    lib.cf_level_n_dofs.restype = ctypes.c_int64
    lib.cf_dof_lattice.argtypes = [P, I, P]
    lib.cf_dof_coords.argtypes = [P, I, P]
    lib.cf_stats.argtypes = [P, I, P]
    lib.cf_work_model.argtypes = [P, I, I, I, P]
    lib.cf_footprint.argtypes = [ctypes.POINTER(cf_mesh), ctypes.POINTER(cf_levelset), I,
                                 ctypes.POINTER(cf_params), P]
    lib.cf_problem_footprint.argtypes = [P, P]
    lib.cf_set_precision.argtypes = [P, I]
    lib.cf_set_kernel_variant.argtypes = [P, I, I]
    lib.cf_profile_start_level.argtypes = [P, I, I]
    lib.cf_set_wait_limit.argtypes = [P, ctypes.c_int64]
    lib.cf_rhs.argtypes = [P, P, V]
    lib.cf_apply.argtypes = [P, P, P, V]
    lib.cf_vcycle.argtypes = [P, P, P, V]
    lib.cf_solve.argtypes = [P, P, P, D, I, ctypes.POINTER(cf_info), V]
    lib.cf_solve_vcycle.argtypes = [P, P, P, D, I, ctypes.POINTER(cf_info), V]
    lib.cf_rhs_user.argtypes = [P, DATA_FN, DATA_FN, V, P, V]
    lib.cf_host_rhs_user.argtypes = [P, DATA_FN, DATA_FN, V, P]
    lib.cf_solve_gmres.argtypes = [P, P, P, D, I, I, ctypes.POINTER(cf_info), V]
    lib.cf_level_apply.argtypes = [P, I, I, P, P, V]
    lib.cf_level_colour_step.argtypes = [P, I, I, I, I, P, P, V]
    lib.cf_level_smooth.argtypes = [P, I, I, I, P, P, V]
    lib.cf_level_restrict.argtypes = [P, I, I, P, P, V]
    lib.cf_level_prolongate.argtypes = [P, I, I, P, P, V]
    lib.cf_coarse_solve.argtypes = [P, I, P, P, V]
    lib.cf_host_rhs.argtypes = [P, P]
    lib.cf_host_cell_matrix.argtypes = [P, I, ctypes.c_int64, P]
    lib.cf_host_patch_counts.argtypes = [P, I, P, P]
    lib.cf_host_interior_update.argtypes = [P, I, P]
    lib.cf_host_diagonal.argtypes = [P, I, P]
    lib.cf_host_coarse_inverse.argtypes = [P, P]
    lib.cf_host_interior_patch.argtypes = [P, I, ctypes.c_int64, P]
    lib.cf_host_cut_patch.argtypes = [P, I, ctypes.c_int64, P, P, P, P]
    lib.cf_coarse_solve_noalloc.argtypes = [P, P, P, V]
    lib.cf_batch_create.argtypes = [P, I, ctypes.POINTER(P)]
    lib.cf_batch_solve.argtypes = [P, I, P, P, D, I, P, V]
    lib.cf_batch_launch_count.argtypes = [P]
    lib.cf_batch_launch_count.restype = ctypes.c_int64
    lib.cf_batch_destroy.argtypes = [P]
    lib.cf_batch_destroy.restype = None
    lib.cf_server_create.argtypes = [ctypes.c_size_t, I, I, I, ctypes.POINTER(P)]
    lib.cf_server_submit.argtypes = [P, ctypes.POINTER(cf_mesh), ctypes.POINTER(cf_levelset), I,
                                     ctypes.POINTER(cf_params), D, I, D, ctypes.POINTER(ctypes.c_int64)]
    lib.cf_server_run.argtypes = [P, V]
    lib.cf_server_result.argtypes = [P, ctypes.c_int64, ctypes.POINTER(cf_info), P, P, P]
    lib.cf_server_stats.argtypes = [P, P]
    lib.cf_server_destroy.argtypes = [P]
    lib.cf_server_destroy.restype = None
    lib.cf_launch_count.argtypes = [P]
    lib.cf_launch_count.restype = ctypes.c_int64
    lib.cf_profile_start.argtypes = [P, I]
    lib.cf_profile_read.argtypes = [P, P, P, P, P]
    for name in EXPORTED:
        getattr(lib, name)  # raises AttributeError if the library lacks a symbol
    _lib = lib
    return lib


def check(status):
    if status != CF_OK:
        raise CutmgError(status, load().cf_last_error().decode())


def make_levelset(spec):
    """cf_levelset from a plain dict: {"kind": "sphere", "center", "radius"},
    {"kind": "plane", "normal", "offset"}, {"kind": "ellipsoid", "center",
    "axes", "rot"}, {"kind": "torus", "center", "rot", "major", "minor"},
    {"kind": "flower", "center", "lobes", "phase", "base", "amplitude"},
    {"kind": "callback", "dim", "phi", "grad"} with phi(X) -> values and
    grad(X) -> gradients, vectorised over X of shape (..., dim) (the library
    calls them one point at a time; the returned structure keeps the C
    trampolines alive)."""
    ls = cf_levelset()
    kind = spec["kind"]
    kinds = {"sphere": CF_LS_SPHERE, "plane": CF_LS_PLANE, "ellipsoid": CF_LS_ELLIPSOID,
             "torus": CF_LS_TORUS, "flower": CF_LS_FLOWER, "callback": CF_LS_CALLBACK}
    ls.kind = kinds[kind]
    for k, v in enumerate(spec.get("center", [])):
        ls.center[k] = v
    if kind == "sphere":
        ls.radius = spec["radius"]
    elif kind == "plane":
        for k, v in enumerate(spec["normal"]):
            ls.normal[k] = v
        ls.offset = spec["offset"]
    elif kind == "ellipsoid":
        for k, v in enumerate(spec["axes"]):
            ls.axes[k] = v
        for k, v in enumerate(list(map(float, __import__("numpy").asarray(spec["rot"]).ravel()))):
            ls.rot[k] = v
    elif kind == "torus":
        for k, v in enumerate(list(map(float, __import__("numpy").asarray(spec["rot"]).ravel()))):
            ls.rot[k] = v
        ls.major = spec["major"]
        ls.radius = spec["minor"]
    elif kind == "flower":
        ls.lobes = int(spec["lobes"])
        ls.phase = spec["phase"]
        ls.radius = spec.get("base", 0.6)
        ls.amplitude = spec.get("amplitude", 0.1)
    elif kind == "callback":
        import numpy as np
        d, fphi, fgrad = int(spec["dim"]), spec["phi"], spec["grad"]

        def phi_c(x, user):
            return float(fphi(np.array([x[k] for k in range(d)])))

        def grad_c(x, g, user):
            gv = fgrad(np.array([x[k] for k in range(d)]))
            for k in range(d):
                g[k] = float(gv[k])

        ls.phi, ls.grad = PHI_FN(phi_c), GRAD_FN(grad_c)
        ls._keep = (ls.phi, ls.grad)
    return ls
