"""ctypes binding of libhope.so (include/hope.h): argument marshalling only.

Every function keeps the C name.  A missing or unloadable library raises: there is
no fallback implementation.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhope.so")

HOPE_OK = 0
HOPE_TPP, HOPE_WENO2D, HOPE_WENO1D = 0, 1, 2
HOPE_FP64, HOPE_FP32 = 0, 1
HOPE_SSPRK3, HOPE_WSRK3 = 0, 1
HOPE_STATUS_NONPHYS_PHI, HOPE_STATUS_NAN, HOPE_STATUS_TIMEOUT = 1, 2, 4
HOPE_AUTOTUNE_MAX = 16

EXPORTED = [
    "hope_default_params", "hope_init_grid", "hope_init_ensemble", "hope_destroy", "hope_state_elems",
    "hope_elem_size", "hope_initial_state", "hope_set_state", "hope_get_state", "hope_tendency",
    "hope_step", "hope_step_ssprk3", "hope_step_host", "hope_tendency_vjp", "hope_step_vjp",
    "hope_total_mass", "hope_status", "hope_ghost_nnz", "hope_launches_per_stage", "hope_strerror",
    "hope_last_error_message", "hope_measure_fma_peak", "hope_set_profiling", "hope_kernel_times",
    "hope_total_mass_noalloc", "hope_autotune", "hope_inject_fault", "hope_set_recon_tile", "hope_recon_tile",
    "hope_tape_bytes", "hope_step_record", "hope_step_vjp_tape", "hope_step_ssprk3_vjp",
    "hope_ghost_selfcheck", "hope_set_topography", "hope_topography_tables", "hope_measure_fma_peak_clock",
    "hope_vjp_phase_times", "hope_autotune_candidates",
]


class hope_params(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("gravity", ctypes.c_double), ("omega", ctypes.c_double),
                ("n_gauss", ctypes.c_int), ("precision", ctypes.c_int), ("rk", ctypes.c_int),
                ("ghost_iters", ctypes.c_int), ("weno_eps", ctypes.c_double),
                ("coriolis_tilt", ctypes.c_double)]


class HopeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hope error %d (%s): %s" % (code, _strerror(code), msg))
        self.code = code


_lib = None


def load():
    """Load libhope.so (raises OSError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError("libhope.so is not built (run __graft_entry__.build() or "
                      "python paper_2411_19185_gb300/build.py): %s" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "hope_default_params": (None, [P(hope_params)]),
        "hope_init_grid": (i, [i, i, i, P(hope_params), P(vp)]),
        "hope_init_ensemble": (i, [i, P(i), i, i, P(hope_params), P(vp)]),
        "hope_destroy": (None, [vp]),
        "hope_state_elems": (sz, [vp]),
        "hope_elem_size": (i, [vp]),
        "hope_initial_state": (i, [vp, i, P(d), i, P(d), i, vp, vp]),
        "hope_set_state": (i, [vp, vp, vp]),
        "hope_get_state": (i, [vp, vp, vp]),
        "hope_tendency": (i, [vp, vp, vp, vp]),
        "hope_step": (i, [vp, vp, d, i, vp]),
        "hope_step_ssprk3": (i, [vp, vp, d, vp]),
        "hope_step_host": (i, [vp, vp, vp, d, i, vp]),
        "hope_tendency_vjp": (i, [vp, vp, vp, vp, vp]),
        "hope_step_vjp": (i, [vp, vp, vp, vp, d, vp]),
        "hope_total_mass": (i, [vp, vp, P(d), vp]),
        "hope_status": (i, [vp, P(ctypes.c_uint)]),
        "hope_ghost_nnz": (i, [vp, P(ctypes.c_longlong), P(ctypes.c_longlong)]),
        "hope_launches_per_stage": (i, [vp, P(i)]),
        "hope_strerror": (ctypes.c_char_p, [i]),
        "hope_last_error_message": (ctypes.c_char_p, []),
        "hope_measure_fma_peak": (i, [i, P(d)]),
        "hope_measure_fma_peak_clock": (i, [i, i, P(d), P(d), P(d)]),
        "hope_vjp_phase_times": (i, [vp, P(ctypes.c_float)]),
        "hope_autotune_candidates": (i, [vp]),
        "hope_set_profiling": (i, [vp, i]),
        "hope_total_mass_noalloc": (i, [vp, i, i, P(d), vp]),
        "hope_autotune": (i, [vp, i, P(ctypes.c_float), P(i), P(i), P(i)]),
        "hope_inject_fault": (i, [vp, i]),
        "hope_kernel_times": (i, [vp, P(ctypes.c_float), i, P(i)]),
        "hope_set_recon_tile": (i, [vp, i, i]),
        "hope_recon_tile": (i, [vp, P(i), P(i)]),
        "hope_tape_bytes": (i, [vp, P(sz)]),
        "hope_step_record": (i, [vp, vp, d, vp, vp]),
        "hope_step_vjp_tape": (i, [vp, vp, vp, vp, vp, d, vp]),
        "hope_step_ssprk3_vjp": (i, [vp, vp, vp, vp, d, vp]),
        "hope_ghost_selfcheck": (i, [i, i, i, P(i), P(d), P(d)]),
        "hope_set_topography": (i, [vp, P(d)]),
        "hope_topography_tables": (i, [i, i, d, P(d), P(d), P(d), P(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _strerror(code):
    try:
        return load().hope_strerror(code).decode()
    except OSError:
        return "?"


def check(rc):
    if rc != HOPE_OK:
        raise HopeError(rc, load().hope_last_error_message().decode())
    return rc


def default_params():
    p = hope_params()
    load().hope_default_params(ctypes.byref(p))
    return p
