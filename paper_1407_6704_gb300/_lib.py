"""ctypes declarations of the C ABI in ``include/pibm.h``.

Argument marshalling only: every step of the method runs in ``libpibm.so``.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libpibm.so")

PIBM_OK = 0
PIBM_EINVAL = -1
PIBM_ENOMEM = -2
PIBM_ECUDA = -3
PIBM_EUNSTABLE = -4
PIBM_EESCAPED = -5
PIBM_ENOTSUP = -6
PIBM_EINTERNAL = -7
PIBM_ETOOBIG = -8
PIBM_ETIMEOUT = -9

PIBM_D2Q9, PIBM_D3Q15, PIBM_D3Q19 = 9, 15, 19
PIBM_WALL, PIBM_PERIODIC = 0, 1
PIBM_IMPLICIT, PIBM_EXPLICIT = 0, 1
PIBM_FP64, PIBM_FP32, PIBM_FP16, PIBM_BF16 = 0, 1, 2, 3
PIBM_INTERP_DELTA, PIBM_INTERP_LAGRANGE4 = 0, 1
PIBM_DEM_LINEAR, PIBM_DEM_HERTZ = 0, 1
PIBM_OVERLAP_AUTO, PIBM_OVERLAP_ON, PIBM_OVERLAP_OFF = 0, 1, 2
PIBM_PARTICLE_FP64, PIBM_PARTICLE_FP32 = 0, 1

FIELD_RHO, FIELD_J, FIELD_POP, FIELD_X, FIELD_U = (1 << k for k in range(5))
NFIELDS = 5

# every symbol include/pibm.h declares
EXPORTS = ["pibm_workspace_bytes", "pibm_create", "pibm_step", "pibm_forces",
           "pibm_read_fields", "pibm_invariants", "pibm_status", "pibm_kernels_per_step",
           "pibm_destroy", "pibm_strerror", "pibm_profile_steps", "pibm_last_error",
           "pibm_fluid_sums_noalloc", "pibm_autotune", "pibm_ensemble_create",
           "pibm_ensemble_step", "pibm_ensemble_status", "pibm_ensemble_destroy",
           "pibm_settling_gradient", "pibm_launch_count", "pibm_ensemble_configure",
           "pibm_ensemble_autotune", "pibm_ensemble_info", "pibm_ensemble_launch_count",
           "pibm_ensemble_inject_skip", "pibm_grid_barrier_test", "pibm_ensemble_set_mode"]

_dp = ctypes.POINTER(ctypes.c_double)


class PibmConfig(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("boundary", ctypes.c_int * 3),
        ("tau", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("delta_width", ctypes.c_int),
        ("coupling", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("deterministic", ctypes.c_int),
        ("dem_kn", ctypes.c_double),
        ("dem_restitution", ctypes.c_double),
        ("n_particles", ctypes.c_int64),
        ("x0", _dp),
        ("u0", _dp),
        ("diameter", _dp),
        ("density_ratio", _dp),
        ("f0", _dp),
        ("interp", ctypes.c_int),
        ("dem_model", ctypes.c_int),
        ("dem_young", ctypes.c_double),
        ("dem_poisson", ctypes.c_double),
        ("wall_young", ctypes.c_double),
        ("wall_poisson", ctypes.c_double),
        ("dem_substeps", ctypes.c_int),
        ("rebin_every", ctypes.c_int),
        ("overlap", ctypes.c_int),
        ("particle_update", ctypes.c_int),
    ]


class PibmError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = load().pibm_strerror(status).decode()
        if status == PIBM_ECUDA:
            msg += " [" + load().pibm_last_error().decode() + "]"
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


_lib = None


def load(path: str = LIB_PATH):
    """Load libpibm.so once; raise if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpibm.so not built at {path}; run paper_1407_6704_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(PibmConfig)
    vp = ctypes.c_void_p
    L.pibm_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.pibm_workspace_bytes.restype = ctypes.c_int
    L.pibm_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    L.pibm_create.restype = ctypes.c_int
    L.pibm_step.argtypes = [vp, ctypes.c_int64]
    L.pibm_step.restype = ctypes.c_int
    L.pibm_forces.argtypes = [vp, vp, vp, ctypes.c_int]
    L.pibm_forces.restype = ctypes.c_int
    L.pibm_read_fields.argtypes = [vp, ctypes.c_uint, ctypes.POINTER(vp), ctypes.c_int]
    L.pibm_read_fields.restype = ctypes.c_int
    L.pibm_invariants.argtypes = [vp, _dp]
    L.pibm_invariants.restype = ctypes.c_int
    L.pibm_status.argtypes = [vp]
    L.pibm_status.restype = ctypes.c_int
    L.pibm_kernels_per_step.argtypes = [vp]
    L.pibm_kernels_per_step.restype = ctypes.c_int
    L.pibm_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.pibm_launch_count.restype = ctypes.c_int
    L.pibm_profile_steps.argtypes = [vp, ctypes.c_int64, _dp]
    L.pibm_profile_steps.restype = ctypes.c_int
    L.pibm_destroy.argtypes = [vp]
    L.pibm_destroy.restype = None
    L.pibm_strerror.argtypes = [ctypes.c_int]
    L.pibm_strerror.restype = ctypes.c_char_p
    L.pibm_fluid_sums_noalloc.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), vp, vp]
    L.pibm_fluid_sums_noalloc.restype = ctypes.c_int
    L.pibm_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.pibm_autotune.restype = ctypes.c_int
    L.pibm_ensemble_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.pibm_ensemble_create.restype = ctypes.c_int
    L.pibm_ensemble_step.argtypes = [vp, ctypes.c_int64]
    L.pibm_ensemble_step.restype = ctypes.c_int
    L.pibm_ensemble_status.argtypes = [vp]
    L.pibm_ensemble_status.restype = ctypes.c_int
    L.pibm_ensemble_destroy.argtypes = [vp]
    L.pibm_ensemble_destroy.restype = None
    ip = ctypes.POINTER(ctypes.c_int)
    L.pibm_ensemble_configure.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.pibm_ensemble_configure.restype = ctypes.c_int
    L.pibm_ensemble_autotune.argtypes = [vp, ctypes.c_int, ip]
    L.pibm_ensemble_autotune.restype = ctypes.c_int
    L.pibm_ensemble_info.argtypes = [vp, ip]
    L.pibm_ensemble_info.restype = ctypes.c_int
    L.pibm_ensemble_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.pibm_ensemble_launch_count.restype = ctypes.c_int
    L.pibm_ensemble_set_mode.argtypes = [vp, ctypes.c_int]
    L.pibm_ensemble_set_mode.restype = ctypes.c_int
    L.pibm_ensemble_inject_skip.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.pibm_ensemble_inject_skip.restype = ctypes.c_int
    L.pibm_grid_barrier_test.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ip]
    L.pibm_grid_barrier_test.restype = ctypes.c_int
    L.pibm_settling_gradient.argtypes = [P, ctypes.c_int64, ctypes.c_int64, vp, _dp, _dp, _dp, _dp]
    L.pibm_settling_gradient.restype = ctypes.c_int
    L.pibm_last_error.argtypes = []
    L.pibm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status, what=""):
    if status != PIBM_OK:
        raise PibmError(status, what)
    return status
