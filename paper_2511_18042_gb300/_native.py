"""ctypes binding of the C ABI declared in include/cgflow.h (marshalling only)."""
import ctypes
import os

from .build import LIB

_lib = None


class CgParams(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("minf", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("hybrid_mode", ctypes.c_int),
        ("hybrid_sensor", ctypes.c_int),
        ("hyb_rho", ctypes.c_double),
        ("hyb_p", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("c_beta", ctypes.c_double),
        ("c_kappa", ctypes.c_double),
        ("alpha_f", ctypes.c_double),
        ("sensor_thresh", ctypes.c_double),
        ("mp_eps", ctypes.c_double),
        ("mp_alpha", ctypes.c_double),
        ("filter_on", ctypes.c_int),
        ("omega_window", ctypes.c_int),
        ("inflow", ((ctypes.c_double * 5) * 2) * 3),
        ("viscous", ctypes.c_int),
        ("re", ctypes.c_double),
        ("pr", ctypes.c_double),
        ("suth", ctypes.c_double),
        ("twall", ctypes.c_double),
        ("fma_sweep", ctypes.c_int),
        ("hybrid_buffer", ctypes.c_int),
    ]


_SIGS = {
    "cg_params_default": (None, [ctypes.POINTER(CgParams)]),
    "cg_grid_create_cartesian": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "cg_grid_create_curvilinear": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_void_p)]),
    "cg_grid_destroy": (None, [ctypes.c_void_p]),
    "cg_solver_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(CgParams), ctypes.POINTER(ctypes.c_void_p)]),
    "cg_solver_destroy": (None, [ctypes.c_void_p]),
    "cg_solver_set_inflow_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_double)]),
    "cg_metrics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_rk3_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "cg_rk3_step_dev": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_step_dev": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_step_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_convert_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p]),
    "cg_cfl_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "cg_advance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "cg_advance_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "cg_omega": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_lad_coeffs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "cg_filter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_iface_flux": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "cg_hybrid_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.c_void_p]),
    "cg_sync_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cg_last_bad_index": (ctypes.c_int64, [ctypes.c_void_p]),
    "cg_solver_device_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "cg_last_error": (ctypes.c_char_p, []),
    "cg_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "cg_timing_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "cg_multi_step": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                     ctypes.c_void_p]),
    "cg_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "cg_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cg_batch_destroy": (None, [ctypes.c_void_p]),
    "cg_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "cg_batch_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cg_batch_set_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "cg_batch_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cg_batch_debug_barrier": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "cg_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "cg_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "cg_set_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "cg_timing_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]),
}


def lib(path=None):
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError("cgflow CUDA library not built (%s); run __graft_entry__.build()" % p)
        L = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            if not hasattr(L, name):
                continue
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("cgflow error %d: %s" % (code, msg))
        self.code = code


def check(rc):
    if rc != 0:
        raise CgError(rc, lib().cg_last_error().decode())
    return rc
