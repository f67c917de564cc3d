"""ctypes declarations of libapm's C ABI (include/apm.h).  Argument marshalling only."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# APM_LIB selects another build of the library (the bounds-checked one)
LIB_PATH = os.environ.get("APM_LIB") or os.path.join(HERE, "_build", "libapm.so")

c_i32, c_i64, c_dbl, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

APM_OK = 0
STATUS_NAMES = {0: "APM_OK", 1: "APM_E_INVALID", 2: "APM_E_NESTING", 3: "APM_E_NOMEM",
                4: "APM_E_CUDA", 5: "APM_E_OVERFLOW", 6: "APM_E_OUT_OF_BOX", 7: "APM_E_TIMEOUT",
                8: "APM_E_UNSUPPORTED", 9: "APM_E_STATE", 10: "APM_E_BOUNDS"}
APM_FP32, APM_FP64 = 0, 1
APM_BC_ISOLATED, APM_BC_PERIODIC = 0, 1
APM_GRAD_FD2, APM_GRAD_FD4, APM_GRAD_SPECTRAL = 0, 1, 2
GRADIENTS = {"fd2": APM_GRAD_FD2, "fd4": APM_GRAD_FD4, "spectral": APM_GRAD_SPECTRAL}


class ApmConfig(ctypes.Structure):
    _fields_ = [("box", c_dbl), ("a_over_dx", c_dbl), ("refine", c_i32), ("pad_factor", c_dbl),
                ("root_bc", c_i32), ("precision", c_i32), ("mass_frac_bits", c_i32),
                ("root_correction", c_i32), ("device", c_i32), ("gradient", c_i32)]


class ApmGrid(ctypes.Structure):
    _fields_ = [("level", c_i32), ("parent", c_i32), ("start", c_i64 * 3), ("dims", c_i32 * 3)]


class ApmParticles(ctypes.Structure):
    _fields_ = [("n", c_i64), ("x", c_void_p), ("y", c_void_p), ("z", c_void_p),
                ("vx", c_void_p), ("vy", c_void_p), ("vz", c_void_p), ("m", c_void_p)]


class ApmGridInfo(ctypes.Structure):
    _fields_ = [("level", c_i32), ("border", c_i32), ("gmf", c_i32 * 3), ("fft", c_i32 * 3),
                ("phi_short", c_i32 * 3), ("field", c_i32 * 3), ("level_index", c_i32),
                ("delta", c_dbl), ("phi_short_comps", c_i32)]


class ApmFftShapes(ctypes.Structure):
    _fields_ = [("budget", c_i32 * 5), ("threads", c_i32 * 5), ("plan", c_i32 * 5),
                ("max_radix", c_i32), ("packing", c_i32)]


# name -> (restype, argtypes); every function declared in include/apm.h
SIGNATURES = {
    "apm_config_default": (None, [ctypes.POINTER(ApmConfig)]),
    "apm_create": (c_i32, [ctypes.POINTER(ApmConfig), ctypes.POINTER(c_void_p)]),
    "apm_set_hierarchy": (c_i32, [c_void_p, ctypes.POINTER(ApmGrid), c_i32]),
    "apm_validate_hierarchy": (c_i32, [ctypes.POINTER(ApmConfig), ctypes.POINTER(ApmGrid), c_i32]),
    "apm_get_grid_info": (c_i32, [c_void_p, c_i32, ctypes.POINTER(ApmGridInfo)]),
    "apm_num_levels": (c_i32, [c_void_p]),
    "apm_deposit": (c_i32, [c_void_p, c_i32, ctypes.POINTER(ApmParticles), c_dbl,
                            ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                            ctypes.POINTER(c_void_p), c_void_p]),
    "apm_deposit_all": (c_i32, [c_void_p, ctypes.POINTER(ApmParticles), c_dbl, ctypes.POINTER(c_void_p),
                                ctypes.POINTER(c_void_p), c_void_p]),
    "apm_interp_all": (c_i32, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(ApmParticles), c_dbl,
                               c_void_p, c_void_p]),
    "apm_solve_level": (c_i32, [c_void_p, c_i32, ctypes.POINTER(c_void_p),
                                ctypes.POINTER(c_void_p), c_void_p]),
    "apm_accel": (c_i32, [c_void_p, c_i32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                          ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                          ctypes.POINTER(c_void_p), c_void_p]),
    "apm_interp": (c_i32, [c_void_p, c_i32, ctypes.POINTER(c_void_p), ctypes.POINTER(ApmParticles),
                           c_dbl, c_void_p, c_void_p]),
    "apm_autotune_level": (c_i32, [c_void_p, c_i32, ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(c_void_p), c_void_p]),
    "apm_set_grid_batching": (c_i32, [c_void_p, c_i32]),
    "apm_set_deposit_tiles": (c_i32, [c_void_p, c_i32]),
    "apm_reserve_order": (c_i32, [c_void_p, c_i64]),
    "apm_graph_begin": (c_i32, [c_void_p, c_void_p]),
    "apm_graph_end": (c_i32, [c_void_p, c_void_p, ctypes.POINTER(c_i32)]),
    "apm_graph_launch": (c_i32, [c_void_p, c_i32, c_void_p]),
    "apm_graph_destroy": (c_i32, [c_void_p, c_i32]),
    "apm_order_particles": (c_i32, [c_void_p, ctypes.POINTER(ApmParticles), c_dbl, c_void_p]),
    "apm_get_fft_shapes": (c_i32, [c_void_p, c_i32, ctypes.POINTER(ApmFftShapes)]),
    "apm_set_fft_shapes": (c_i32, [c_void_p, c_i32, ctypes.POINTER(ApmFftShapes)]),
    "apm_get_pass_kernels": (c_i32, [c_void_p, c_i32, c_i32, ctypes.POINTER(c_i32), c_i32]),
    "apm_kick_drift": (c_i32, [c_void_p, c_i64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_dbl, c_void_p]),
    "apm_sync_status": (c_i32, [c_void_p, c_void_p]),
    "apm_profile_enable": (c_i32, [c_void_p, c_i32, c_i32]),
    "apm_profile_read": (c_i32, [c_void_p, c_i32, ctypes.POINTER(c_i64), ctypes.POINTER(c_dbl)]),
    "apm_kernel_count": (c_i32, []),
    "apm_kernel_name": (ctypes.c_char_p, [c_i32]),
    "apm_solve_periodic_noalloc": (c_i32, [c_i32, c_dbl, c_dbl, c_i32, c_void_p, c_void_p, c_void_p]),
    "apm_status_string": (ctypes.c_char_p, [c_i32]),
    "apm_destroy": (None, [c_void_p]),
    "apm_version": (ctypes.c_char_p, []),
}

_lib = None


class ApmError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        name = STATUS_NAMES.get(self.code, str(code))
        msg = f"{where}: {name}"
        try:
            msg += f" ({lib().apm_status_string(self.code).decode()})"
        except Exception:  # pragma: no cover
            pass
        super().__init__(msg)


def lib():
    """libapm, loaded once.  Raises if the CUDA library has not been built:
    there is no CPU fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libapm.so not found at {LIB_PATH}: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != APM_OK:
        raise ApmError(code, where)


def ptr_array(ptrs):
    """HOST array of device pointers (None -> NULL entry)."""
    arr = (c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr
