"""ctypes binding of the libfrpcpf C ABI (include/fr_pcpf.h).

Argument marshalling only: every step of the FR update runs in the library's
CUDA kernels.  Loading fails loudly if the library has not been built; there
is no CPU fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# FRP_BOUNDS_CHECK=1 selects the bounds-checked build of the same sources
CHECKED = os.environ.get("FRP_BOUNDS_CHECK", "0") == "1"
LIB_PATH = os.path.join(HERE, "libfrpcpf_checked.so" if CHECKED else "libfrpcpf.so")
# fields whose status, read when they were destroyed, showed a fired index
# check (the checked build only)
BOUNDS_FIRED = []

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ENONFINITE, FR_ETIMEOUT, FR_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
FR_EBOUNDS = -7
FR_ADJ_PRECONDITION = 1
FR_QUAD, FR_TRI, FR_HEX = 0, 1, 2
FR_FP64, FR_MIXED = 0, 1
FR_VEL_UNIFORM, FR_VEL_RIDER_KOTHE, FR_VEL_LEVEQUE, FR_VEL_STREAM, FR_VEL_ROTATION = 0, 1, 2, 3, 4
FR_MAX_MODES = 32
FR_IC_CIRCLE, FR_IC_ARRAY = 0, 1
FR_NOALLOC_MAX_BLOCKS = 16384
FR_NOALLOC_MAX_VALUES = FR_NOALLOC_MAX_BLOCKS * 256 * 8

_dp = C.POINTER(C.c_double)


class fr_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("etype", C.c_int32), ("order", C.c_int32), ("reserved", C.c_int32),
                ("n_nodes", C.c_int64), ("nodes", _dp), ("n_elems", C.c_int64),
                ("conn", C.POINTER(C.c_int64)), ("periodic", C.c_int32 * 3), ("period", C.c_double * 3)]


class fr_mesh_info(C.Structure):
    _fields_ = [("dim", C.c_int32), ("etype", C.c_int32), ("order", C.c_int32), ("nu", C.c_int32),
                ("nf", C.c_int32), ("n_faces_per_elem", C.c_int32), ("n_elems", C.c_int64),
                ("n_dof", C.c_int64), ("n_boundary_fpts", C.c_int64), ("h", C.c_double),
                ("volume", C.c_double)]


class fr_velocity(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_modes", C.c_int32), ("T", C.c_double), ("a", C.c_double * 3),
                ("kx", _dp), ("ky", _dp), ("A", _dp), ("B", _dp)]


class fr_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("eps", C.c_double), ("tau", C.c_double), ("tau_psi", C.c_double),
                ("tau_pseudo", C.c_double), ("dt", C.c_double), ("n_precond", C.c_int32),
                ("pseudo_kmax", C.c_int32), ("pseudo_dtau", C.c_double), ("pseudo_tol", C.c_double),
                ("pseudo_fixed", C.c_int32), ("precision", C.c_int32), ("s0", C.c_double),
                ("kappa", C.c_double), ("nu_max", C.c_double), ("delta", C.c_double),
                ("vel", fr_velocity), ("vel_cache", C.c_int32), ("normal", C.c_int32),
                ("wall", C.c_int32), ("variant", C.c_int32)]


class fr_ic(C.Structure):
    _fields_ = [("kind", C.c_int32), ("precondition", C.c_int32), ("centre", C.c_double * 3),
                ("radius", C.c_double), ("beta", C.c_double), ("phi0", _dp)]


class fr_instance(C.Structure):
    _fields_ = [("elem_begin", C.c_int64), ("elem_end", C.c_int64), ("dt", C.c_double), ("eps", C.c_double),
                ("nu_max", C.c_double), ("pseudo_dtau", C.c_double), ("vel", fr_velocity), ("ic", fr_ic)]


class fr_stats(C.Structure):
    _fields_ = [("n_steps", C.c_int64), ("t", C.c_double), ("last_pseudo_iters", C.c_int32),
                ("status", C.c_int32), ("last_pseudo_rms", C.c_double), ("n_preconditions", C.c_int64)]


_vp = C.c_void_p
_SIGS = {
    "fr_mesh_create": (C.c_int, [C.POINTER(fr_mesh_desc), C.POINTER(_vp)]),
    "fr_mesh_info_get": (C.c_int, [_vp, C.POINTER(fr_mesh_info)]),
    "fr_mesh_solution_points": (C.c_int, [_vp, _dp]),
    "fr_mesh_quadrature": (C.c_int, [_vp, _dp]),
    "fr_mesh_destroy": (None, [_vp]),
    "fr_mesh_concat": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "fr_field_init_batch": (C.c_int, [_vp, C.POINTER(fr_params), C.c_int, C.POINTER(fr_instance), C.c_int, _vp,
                                      C.c_size_t, _vp, C.POINTER(_vp)]),
    "fr_field_workspace_bytes": (C.c_int, [_vp, C.POINTER(fr_params), C.POINTER(C.c_size_t)]),
    "fr_field_init": (C.c_int, [_vp, C.POINTER(fr_params), C.POINTER(fr_ic), _vp, C.c_size_t, _vp,
                                C.POINTER(_vp)]),
    "fr_step": (C.c_int, [_vp, C.c_int, _vp]),
    "fr_precondition": (C.c_int, [_vp, _vp]),
    "fr_sync": (C.c_int, [_vp, _vp]),
    "fr_stats_get": (C.c_int, [_vp, _vp, C.POINTER(fr_stats)]),
    "fr_mass_integral": (C.c_int, [_vp, C.c_int, _dp, _vp]),
    "fr_mass_integral_noalloc": (C.c_int, [_vp, _vp, C.c_int64, _dp, _vp]),
    "fr_field_get": (C.c_int, [_vp, C.c_int, _dp, _vp]),
    "fr_field_set": (C.c_int, [_vp, C.c_int, _dp, _vp]),
    "fr_field_get_device": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "fr_field_set_device": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "fr_rhs": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "fr_rhs_pseudo": (C.c_int, [_vp, _vp, _vp]),
    "fr_adjoint_workspace_bytes": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "fr_adjoint_record": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_size_t, _vp]),
    "fr_adjoint_step": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "fr_kernel_variants": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int32)]),
    "fr_probe_hex_apply": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, C.c_int64, _vp, C.c_int64, _vp]),
    "fr_stage": (C.c_int, [_vp, C.c_int, _vp]),
    "fr_halo_row_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "fr_halo_pack": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp]),
    "fr_halo_unpack": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp]),
    "fr_traces": (C.c_int, [_vp, _vp]),
    "fr_pseudo_begin": (C.c_int, [_vp, _vp]),
    "fr_pseudo_stage": (C.c_int, [_vp, C.c_int, _vp]),
    "fr_group_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "fr_group_step": (C.c_int, [_vp, C.c_int, _vp]),
    "fr_group_destroy": (None, [_vp]),
    "fr_profile": (C.c_int, [_vp, C.c_int]),
    "fr_profile_read": (C.c_int, [_vp, _vp, _dp, C.POINTER(C.c_int64)]),
    "fr_profile_kernel": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _dp]),
    "fr_field_destroy": (None, [_vp]),
    "fr_strerror": (C.c_char_p, [C.c_int]),
    "fr_version": (C.c_int, []),
}

_lib = None


def lib():
    """Load libfrpcpf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2006_10967_gb300.build.build"
                               f"(checked={CHECKED})")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FRError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().fr_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def check(code, where):
    if code != FR_OK:
        raise FRError(code, where)
    return code
