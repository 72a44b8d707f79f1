"""ctypes binding of the C ABI declared in include/sllbm.h (argument marshalling only).

Every step of the method runs in the CUDA library libsllbm.so built in-tree by
``paper_2412_09051_gb300.build``.  Importing this module does not load the
library; ``lib()`` does, and raises if it is missing: there is no CPU fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsllbm.so")
CHECKED_LIB_PATH = os.path.join(HERE, "libsllbm_checked.so")     # bounds-checked debug build

OK = 0
ERRORS = {-1: "SLLBM_ERR_ARG", -2: "SLLBM_ERR_CUDA", -3: "SLLBM_ERR_ARCH", -4: "SLLBM_ERR_NOMEM",
          -5: "SLLBM_ERR_DP_NOT_FOUND", -6: "SLLBM_ERR_UNSTABLE", -7: "SLLBM_ERR_STATE",
          -8: "SLLBM_ERR_UNSUPPORTED"}
MESH = dict(box=0, channel=1, mixing=2, naca=3, explicit=4)
VELSET = dict(D2Q9=0, D2Q19=1, D2Q25=2, D3Q45=3, D3Q125=4, CUSTOM=5)
QMAX_GENERIC = 128
MLP_TENSOR, MLP_SIMT = 0, 1
DEV_TC_TIMEOUT, DEV_BAD_NODE, DEV_BAD_POP, DEV_BAD_REC, DEV_BAD_SMEM, DEV_COPY_TIMEOUT = 1, 2, 4, 8, 16, 32
BUILD_CHECKED = 1
FP64, FP32 = 0, 1
STREAM_AUTO, STREAM_GATHER, STREAM_STRUCTURED, STREAM_STRUCTURED_NODE, STREAM_TILED_REG, STREAM_GATHER_SMEM = \
    0, 1, 2, 3, 4, 5
STREAM_ROW_COPY = 6
STREAM_ROWS_TMEM, STREAM_ROW_SMEM, STREAM_TENSOR, STREAM_ROWS_PAIRS = 7, 8, 9, 10


class Bc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rho", C.c_double), ("u", C.c_double * 3), ("T", C.c_double)]


class MeshDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("p", C.c_int32), ("cells", C.c_int32 * 3),
                ("length", C.c_double * 3), ("stretch", C.c_double), ("central", C.c_int32),
                ("thickness", C.c_double), ("bc", Bc * 2), ("vertices", C.c_void_p * 3)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gamma", C.c_double), ("Pr", C.c_double), ("mu_ref", C.c_double),
                ("T_ref", C.c_double), ("mu_exp", C.c_double), ("precision", C.c_int32),
                ("stream_mode", C.c_int32), ("device", C.c_int32), ("max_newton", C.c_int32),
                ("max_walk", C.c_int32), ("stream", C.c_void_p)]


class VelsetDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("Q", C.c_int32), ("D", C.c_int32), ("reserved", C.c_int32),
                ("xi", C.c_void_p), ("w", C.c_void_p)]


class Control(C.Structure):
    _fields_ = [("target_momentum", C.c_double), ("force0", C.c_double), ("kp", C.c_double), ("ki", C.c_double),
                ("control_every", C.c_int32), ("rescale_every", C.c_int32), ("target_mass", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("Q", C.c_int32), ("dim", C.c_int32), ("p", C.c_int32),
                ("nodes", C.c_int32 * 3), ("cells", C.c_int32 * 3), ("precision", C.c_int32),
                ("stream_mode", C.c_int32), ("state_bytes", C.c_int64), ("table_bytes", C.c_int64),
                ("n_records", C.c_int64), ("n_boundary_records", C.c_int64),
                ("n_isothermal_nodes", C.c_int64), ("step_kernel", C.c_char * 32)]


_P = C.c_void_p
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)     # sllbm_alloc_fn
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)            # sllbm_free_fn
_SIGS = {
    "sllbm_create": (C.c_int, [C.POINTER(MeshDesc), C.c_int32, C.POINTER(Params), C.POINTER(_P)]),
    "sllbm_create_desc": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(VelsetDesc), C.POINTER(Params), C.POINTER(_P)]),
    "sllbm_destroy": (C.c_int, [_P]),
    "sllbm_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, _P]),
    "sllbm_last_error": (C.c_char_p, [_P]),
    "sllbm_info": (C.c_int, [_P, C.POINTER(Info)]),
    "sllbm_node_coords": (C.c_int, [_P, _P, C.c_int32]),
    "sllbm_velocity_set": (C.c_int, [_P, _P, _P, _P]),
    "sllbm_init_state": (C.c_int, [_P, _P, _P, _P, C.c_int32]),
    "sllbm_get_state": (C.c_int, [_P, _P, _P, C.c_int32]),
    "sllbm_set_state": (C.c_int, [_P, _P, _P, C.c_int32]),
    "sllbm_get_state_raw": (C.c_int, [_P, _P, C.c_int32]),
    "sllbm_set_state_raw": (C.c_int, [_P, _P, C.c_int32]),
    "sllbm_get_x_layers": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.c_int32]),
    "sllbm_set_x_layers": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.c_int32]),
    "sllbm_step": (C.c_int, [_P, C.c_int64]),
    "sllbm_step_count": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "sllbm_read_moments": (C.c_int, [_P, _P, _P, _P, C.c_int32]),
    "sllbm_conservation": (C.c_int, [_P, _P]),
    "sllbm_conservation_static": (C.c_int, [_P, _P]),
    "sllbm_set_force": (C.c_int, [_P, _P]),
    "sllbm_rescale_mass": (C.c_int, [_P, C.c_double]),
    "sllbm_step_controlled": (C.c_int, [_P, C.c_int64, C.POINTER(Control), _P]),
    "sllbm_departure_records": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "sllbm_sync": (C.c_int, [_P]),
    "sllbm_stream": (C.c_void_p, [_P]),
    "sllbm_mlp_set": (C.c_int, [_P, _P, _P, _P, C.c_float, C.c_int32]),
    "sllbm_step_features": (C.c_int, [_P, _P, C.c_int32]),
    "sllbm_mlp_path": (C.c_int, [_P, C.c_int32]),
    "sllbm_plane_profiles": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "sllbm_mixing_thickness": (C.c_int, [_P, C.c_double, C.c_double, _P, _P]),
    "sllbm_stats_accumulate": (C.c_int, [_P]),
    "sllbm_stats_reset": (C.c_int, [_P]),
    "sllbm_plane_profiles_mean": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sllbm_plane_cp": (C.c_int, [_P, C.c_int32, C.c_double, C.c_double, _P, _P, _P]),
    "sllbm_device_status": (C.c_int, [_P, _P]),
    "sllbm_build_flags": (C.c_int, []),
    "sllbm_debug_wait_limit": (C.c_int, [_P, C.c_int32]),
    "sllbm_moment_basis": (C.c_int, [_P, _P, _P]),
    "sllbm_train_create": (C.c_int, [_P, _P, C.POINTER(_P)]),
    "sllbm_train_destroy": (C.c_int, [_P]),
    "sllbm_train_last_error": (C.c_char_p, [_P]),
    "sllbm_train_set_data": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, C.c_int32]),
    "sllbm_train_scales": (C.c_int, [_P, _P, _P]),
    "sllbm_train_epoch": (C.c_int, [_P, C.c_int32, C.c_float, _P]),
    "sllbm_train_grads": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P]),
    "sllbm_train_path": (C.c_int, [_P, C.c_int32]),
    "sllbm_train_params": (C.c_int, [_P, _P]),
    "sllbm_train_set_params": (C.c_int, [_P, _P]),
    "sllbm_train_export": (C.c_int, [_P, _P, _P]),
}
EXPORTED = sorted(_SIGS)

_lib = None


def lib(path=None):
    """Load libsllbm.so, or the library at path (the first call decides; raises
    OSError when it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"{p} is missing: build it with `python -m paper_2412_09051_gb300.build` "
                          "(there is no CPU fallback)")
        L = C.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SllbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(rc, ctx=None):
    if rc != OK:
        msg = lib().sllbm_last_error(ctx)
        raise SllbmError(rc, msg.decode() if msg else "")
    return rc


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator
    (sllbm_set_allocator): every buffer a context created while installed
    owns is a torch uint8 tensor on the given device, held here until the
    library releases it.  Keep the object alive while such contexts exist
    (they call back into it).  Argument marshalling only."""

    def __init__(self, device=0):
        self.device = device
        self.blocks = {}
        self._alloc = ALLOC_FN(self._take)
        self._free = FREE_FN(self._give)

    def _take(self, nbytes, user):
        import torch
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=f"cuda:{self.device}")
        self.blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _give(self, ptr, user):
        self.blocks.pop(ptr, None)

    def install(self):
        check(lib().sllbm_set_allocator(self._alloc, self._free, None))
        return self

    def uninstall(self):
        check(lib().sllbm_set_allocator(ALLOC_FN(), FREE_FN(), None))

    def __enter__(self):
        return self.install()

    def __exit__(self, *exc):
        self.uninstall()
