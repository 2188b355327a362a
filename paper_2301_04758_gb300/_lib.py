"""ctypes binding of libvef.so (the C ABI declared in include/vef.h).

Argument marshalling only: every step of the sweep, moments and adjoint runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing; there is no
CPU fallback.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvef.so")
# the bounds-checked build (build(checked=True)); load() takes it when VEF_CHECKED=1
CHECKED_LIB_PATH = os.path.join(_PKG, "libvef_checked.so")

VEF_OK = 0
VEF_ERR_INVALID_ARG = 1
VEF_ERR_CUDA = 2
VEF_ERR_OOM = 3
VEF_ERR_TIMEOUT = 4
VEF_ERR_NOT_CONVERGED = 5
VEF_ERR_NONPOSITIVE_DENOM = 6
VEF_ERR_NOT_IMPLEMENTED = 7
VEF_ERR_BOUNDS = 8

VEF_FP64 = 0
VEF_MIXED = 1
VEF_GROUPS_ITERATIVE = 1
VEF_SWEEP_CLUSTER = 2
VEF_APPLY_SEPARATE = 4
VEF_PIVOT_ALWAYS = 8
VEF_REUSE_FACTORS = 16
VEF_CKPT_FP32 = 32
VEF_STATUS_TIMEOUT = 1
VEF_STATUS_NOT_CONVERGED = 2
VEF_STATUS_NONPOSITIVE = 4
VEF_STATUS_SINGULAR = 8
VEF_STATUS_BOUNDS = 16

# every symbol include/vef.h declares
EXPORTS = ("vef_mesh_create", "vef_mesh_destroy", "vef_mesh_query", "vef_mesh_sync", "vef_sweep",
           "vef_moments", "vef_source_iterate", "vef_adjoint_sweep", "vef_profile",
           "vef_profile_read", "vef_measure_fma_peak", "vef_wait_selftest", "vef_eddington_noalloc",
           "vef_batch_create", "vef_batch_destroy", "vef_batch_sweep", "vef_batch_tune",
           "vef_region_weights", "vef_schedule_host", "vef_mesh_inject_status", "vef_hrt_solve",
           "vef_vef_iterate", "vef_build_checked", "vef_rcp_selftest",
           "vef_status_string", "vef_last_error")

KERNEL_CLASSES = ("geometry", "factor", "sweep", "residual", "source", "moments", "adjoint", "group", "hrt")


class VefOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_passes", ctypes.c_int), ("tile_override", ctypes.c_int),
                ("flags", ctypes.c_int)]


class VefInfo(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("coupled_groups", ctypes.c_longlong), ("lagged_face_points", ctypes.c_longlong),
                ("max_inner_iterations", ctypes.c_int), ("timed_out", ctypes.c_int),
                ("levels", ctypes.c_int), ("pivoted_tasks", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VefHrtInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("multipliers", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VefVefInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("last_change", ctypes.c_double),
                ("hrt_iterations", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VefMeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("mesh_order", ctypes.c_int),
                ("p", ctypes.c_int), ("n", ctypes.c_int), ("nq", ctypes.c_int),
                ("E", ctypes.c_longlong), ("nbf", ctypes.c_longlong)]


class VefKernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double)]


class VefError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {status_name(status)}: {message}")
        self.status = status


_lib = None
P = ctypes.c_void_p
D = ctypes.c_double
I = ctypes.c_int


def _declare(lib):
    lib.vef_mesh_create.argtypes = [I, I, I, I, D, P, ctypes.POINTER(P)]
    lib.vef_mesh_destroy.argtypes = [P]
    lib.vef_mesh_query.argtypes = [P, ctypes.POINTER(VefMeshDesc)]
    lib.vef_mesh_sync.argtypes = [P, P]
    lib.vef_sweep.argtypes = [P, P, P, P, P, I, P, P, P, I, ctypes.POINTER(VefOpts), P,
                              ctypes.POINTER(VefInfo), P]
    lib.vef_moments.argtypes = [P, P, P, P, I, P, P, P, P, P, P, P, P]
    lib.vef_source_iterate.argtypes = [P, P, P, P, P, I, P, P, P, I, I, ctypes.POINTER(VefOpts),
                                       P, P, P, ctypes.POINTER(VefInfo), P]
    lib.vef_adjoint_sweep.argtypes = [P, P, P, P, P, P, I, P, P, P, P, P, ctypes.POINTER(VefOpts),
                                      ctypes.POINTER(VefInfo), P]
    lib.vef_profile.argtypes = [P, I]
    lib.vef_profile_read.argtypes = [P, ctypes.POINTER(VefKernelStat)]
    lib.vef_measure_fma_peak.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
    lib.vef_wait_selftest.argtypes = [I, I, ctypes.c_longlong, P]
    lib.vef_schedule_host.argtypes = [I, I, I, P, P, I, P, P, P, P]
    lib.vef_eddington_noalloc.argtypes = [P, P, P, I, ctypes.c_longlong, I, P, P]
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.vef_batch_create.argtypes = [PP, I, PP, PP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(P)]
    lib.vef_batch_destroy.argtypes = [P]
    lib.vef_batch_sweep.argtypes = [P, PP, PP, PP, PP, PP, PP, ctypes.POINTER(VefOpts),
                                    ctypes.POINTER(VefInfo), P]
    lib.vef_batch_tune.argtypes = [P, P, ctypes.POINTER(ctypes.c_int)]
    lib.vef_region_weights.argtypes = [P, D, D, D, D, P, P]
    lib.vef_mesh_inject_status.argtypes = [P, ctypes.c_uint, P]
    lib.vef_hrt_solve.argtypes = [P, P, P, P, P, P, P, P, P, D, I, P, P, P, ctypes.POINTER(VefHrtInfo), P]
    lib.vef_vef_iterate.argtypes = [P, P, P, P, P, P, P, I, P, I, D, D, I, ctypes.POINTER(VefOpts), P, P, P, P,
                                    ctypes.POINTER(VefVefInfo), P]
    for name in ("vef_mesh_create", "vef_mesh_destroy", "vef_mesh_query", "vef_mesh_sync",
                 "vef_sweep", "vef_moments", "vef_source_iterate", "vef_adjoint_sweep",
                 "vef_profile", "vef_profile_read", "vef_measure_fma_peak", "vef_wait_selftest",
                 "vef_eddington_noalloc", "vef_batch_create", "vef_batch_destroy",
                 "vef_batch_sweep", "vef_batch_tune", "vef_region_weights", "vef_schedule_host",
                 "vef_mesh_inject_status", "vef_hrt_solve", "vef_vef_iterate"):
        getattr(lib, name).restype = I
    lib.vef_status_string.argtypes = [I]
    lib.vef_status_string.restype = ctypes.c_char_p
    lib.vef_last_error.argtypes = []
    lib.vef_last_error.restype = ctypes.c_char_p
    lib.vef_build_checked.argtypes = []
    lib.vef_build_checked.restype = ctypes.c_int
    lib.vef_rcp_selftest.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.vef_rcp_selftest.restype = ctypes.c_int


def load(path=None):
    """Load libvef.so (built by paper_2301_04758_gb300.build.build()), or with VEF_CHECKED=1
    in the environment the bounds-checked libvef_checked.so (build(checked=True))."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or (CHECKED_LIB_PATH if os.environ.get("VEF_CHECKED") == "1" else LIB_PATH)
    if not os.path.exists(p):
        raise RuntimeError(f"libvef.so not found at {p}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    _declare(lib)
    if path is None:
        _lib = lib
    return lib


def status_name(status):
    try:
        return load().vef_status_string(status).decode()
    except Exception:  # library not loadable: still name the code
        return str(status)


def check(status, where):
    if status != VEF_OK:
        raise VefError(status, where, load().vef_last_error().decode())
