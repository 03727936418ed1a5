"""ctypes binding of include/lbm_pf.h (argument marshalling only).

Every function of the C ABI is exposed under its own name on `lib`.  Loading
fails loudly when the in-tree library has not been built: there is no
fallback implementation.  With LBM_PF_DEBUG=1 in the environment the
bounds-checking build (liblbmpf_debug.so: every computed index checked against
its buffer, failures reported by lbm_sync as LBM_EBOUNDS) is loaded instead.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
DEBUG = os.environ.get("LBM_PF_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "_lib", "liblbmpf_debug.so" if DEBUG else "liblbmpf.so")

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_ENONFINITE = -4
LBM_ETIMEOUT = -5
LBM_EUNSUPPORTED = -6
LBM_EBOUNDS = -7

LBM_COLLISION_BGK = 0
LBM_COLLISION_TRT = 1
LBM_GRAD_CENTRAL = 0
LBM_GRAD_BIASED2 = 1

LBM_D2Q9 = 0
LBM_D3Q19_D3Q7 = 1

LBM_KERNEL_AUTO = 0
LBM_KERNEL_TILED = 1
LBM_KERNEL_TMA = 2

LBM_STORE_FP32 = 0
LBM_STORE_FP16 = 1
LBM_STORE_BF16 = 2

LBM_MODEL_COUPLED = 0
LBM_MODEL_PHASE_FIELD = 1


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32 * 3)]


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
        ("alpha_l", ctypes.c_double), ("alpha_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("M_phi", ctypes.c_double), ("A", ctypes.c_double),
        ("theta_I", ctypes.c_double), ("L", ctypes.c_double),
        ("Cp", ctypes.c_double), ("T_sat", ctypes.c_double),
        ("gravity", ctypes.c_double * 3), ("body_force", ctypes.c_double * 3),
        ("phi_wall", ctypes.c_double * 2), ("T_wall", ctypes.c_double * 2),
        ("normal_eps", ctypes.c_double),
        ("store_ref", ctypes.c_double * 3), ("store_scale", ctypes.c_double * 3),
        ("source_on", ctypes.c_int32), ("visc_interp", ctypes.c_int32),
        ("alpha_interp", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("model", ctypes.c_int32), ("collision", ctypes.c_int32), ("grad_scheme", ctypes.c_int32),
        ("trt_magic", ctypes.c_double * 3), ("mrt_rates", ctypes.c_double * 3),
        ("mrt_rates_g", ctypes.c_double * 4),
    ]


class lbm_fields(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_void_p), ("T", ctypes.c_void_p), ("ux", ctypes.c_void_p),
                ("uy", ctypes.c_void_p), ("uz", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("dtype", ctypes.c_int32)]


H = ctypes.c_void_p
P = ctypes.POINTER

# name -> (restype, argtypes), in header order
SIGNATURES = {
    "lbm_workspace_bytes": (ctypes.c_int, [P(lbm_grid), ctypes.c_int32, P(lbm_params), P(ctypes.c_size_t)]),
    "lbm_create": (ctypes.c_int, [P(lbm_grid), ctypes.c_int32, P(lbm_params), ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_void_p, P(H)]),
    "lbm_set_stream": (ctypes.c_int, [H, ctypes.c_void_p]),
    "lbm_init": (ctypes.c_int, [H, P(lbm_fields)]),
    "lbm_step": (ctypes.c_int, [H, ctypes.c_int32]),
    "lbm_get_fields": (ctypes.c_int, [H, P(lbm_fields)]),
    "lbm_reduce": (ctypes.c_int, [H, P(ctypes.c_double), P(ctypes.c_double)]),
    "lbm_reduce_async": (ctypes.c_int, [H, ctypes.c_void_p]),
    "lbm_state_bytes": (ctypes.c_int, [H, P(ctypes.c_size_t)]),
    "lbm_get_state": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]),
    "lbm_set_state": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]),
    "lbm_stream_map": (ctypes.c_int, [H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_set_kernel": (ctypes.c_int, [H, ctypes.c_int32]),
    "lbm_get_kernel": (ctypes.c_int, [H, P(ctypes.c_int32)]),
    "lbm_steps_done": (ctypes.c_int, [H, P(ctypes.c_int64)]),
    "lbm_last_launches": (ctypes.c_int, [H, P(ctypes.c_int32)]),
    "lbm_sync": (ctypes.c_int, [H]),
    "lbm_field_sums_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_adjoint_bytes": (ctypes.c_int, [H, P(ctypes.c_size_t), P(ctypes.c_size_t)]),
    "lbm_adjoint_terminal": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "lbm_adjoint_step": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_adjoint_steps": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "lbm_adjoint_init": (ctypes.c_int, [H, P(lbm_fields), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "lbm_step_record": (ctypes.c_int, [H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t]),
    "lbm_set_velocity": (ctypes.c_int, [H, P(lbm_fields), ctypes.c_double]),
    "lbm_set_health_check": (ctypes.c_int, [H, ctypes.c_int32, ctypes.c_float]),
    "lbm_set_first_wait_limit": (ctypes.c_int, [ctypes.c_int32]),
    "lbm_columns_bytes": (ctypes.c_int, [H, ctypes.c_int32, P(ctypes.c_size_t)]),
    "lbm_pack_columns": (ctypes.c_int, [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "lbm_unpack_columns": (ctypes.c_int, [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "lbm_destroy": (None, [H]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


class LBMError(RuntimeError):
    def __init__(self, code, call):
        self.code = code
        msg = lib.lbm_strerror(code).decode() if lib is not None else str(code)
        super().__init__(f"{call} failed: {msg} ({code})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2003_06342_b300/build.py` "
            "(or __graft_entry__.build()); there is no non-CUDA implementation")
    lib_ = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib_, name)
        fn.restype = res
        fn.argtypes = args
    return lib_


lib = _load()


def check(code, call):
    if code != LBM_OK:
        raise LBMError(code, call)
