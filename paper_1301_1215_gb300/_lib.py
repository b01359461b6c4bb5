"""ctypes view of libnlinv.so (include/nlinv.h).  Marshals arguments only; every computation runs in the library.

Loading fails loudly when the library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnlinv.so")

OK, EINVAL, ENOMEM, ECUDA, EBREAKDOWN, ETIMEOUT = range(6)
STATUS_NAMES = {OK: "NLINV_OK", EINVAL: "NLINV_EINVAL", ENOMEM: "NLINV_ENOMEM", ECUDA: "NLINV_ECUDA",
                EBREAKDOWN: "NLINV_EBREAKDOWN", ETIMEOUT: "NLINV_ETIMEOUT"}

# Every function that include/nlinv.h declares, with its ctypes signature.
_vp, _int, _dbl, _long = C.c_void_p, C.c_int, C.c_double, C.c_long


class Params(C.Structure):
    """Mirror of nlinv_params."""
    _fields_ = [("n", _int), ("ncoils", _int), ("newton_steps", _int), ("cg_iters", _int),
                ("alpha0", _dbl), ("alpha_q", _dbl), ("alpha_min", _dbl),
                ("sobolev_a", _dbl), ("sobolev_l", _dbl), ("fov", _int), ("use_graph", _int),
                ("tensor_dft", _int)]


class Tuning(C.Structure):
    """Mirror of nlinv_tuning."""
    _fields_ = [("vec_blocks_per_sm", _int), ("pdl", _int), ("ms_per_frame", _dbl), ("split_n1", _int),
                ("col_strip", _int), ("row_blocks_per_sm", _int), ("stage", _int)]


TUNE_TABLE = 16   # entries of the nlinv_autotune table


class FrameDesc(C.Structure):
    """Mirror of nlinv_frame_desc."""
    _fields_ = [("n", _int), ("ncoils", _int), ("y", _vp), ("mask", _vp), ("x_ref", _vp), ("x_inout", _vp),
                ("resid", C.POINTER(_dbl))]


SIGNATURES = {
    "nlinv_supported_size": (_int, [_int]),
    "nlinv_default_params": (_int, [C.POINTER(Params), _int, _int]),
    "nlinv_create": (_int, [C.POINTER(Params), _vp, C.POINTER(_vp)]),
    "nlinv_destroy": (_int, [_vp]),
    "nlinv_forward": (_int, [_vp, _vp, _vp, _vp]),
    "nlinv_derivative": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "nlinv_adjoint": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "nlinv_normal": (_int, [_vp, _vp, _vp, _vp, _dbl, _vp]),
    "nlinv_simulate": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "nlinv_image": (_int, [_vp, _vp, _vp]),
    "nlinv_reconstruct": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "nlinv_reconstruct_checkpoints": (_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nlinv_reconstruct_vjp": (_int, [_vp, _vp, _vp, _vp, _vp, _int, _vp, _vp, _vp]),
    "nlinv_wait": (_int, [_vp, _dbl]),
    "nlinv_profile_cg": (_int, [_vp, _int, C.POINTER(_dbl)]),
    "nlinv_forward_noalloc": (_int, [C.POINTER(Params), _vp, _vp, _vp, _vp]),
    "nlinv_batch_create": (_int, [C.POINTER(Params), _int, C.POINTER(FrameDesc), _vp, C.POINTER(_vp)]),
    "nlinv_reconstruct_batch": (_int, [_vp, _int, C.POINTER(FrameDesc)]),
    "nlinv_batch_launch_count": (_long, [_vp]),
    "nlinv_batch_profile_cg": (_int, [_vp, _int, C.POINTER(_dbl)]),
    "nlinv_batch_destroy": (_int, [_vp]),
    "nlinv_last_launch_count": (_long, [_vp]),
    "nlinv_cg_stops": (_int, [_vp, C.POINTER(_int), _int]),
    "nlinv_gridder_create": (_int, [_int, _int, C.POINTER(_dbl), _vp, C.POINTER(_vp)]),
    "nlinv_grid": (_int, [_vp, _int, _vp, _vp, _vp]),
    "nlinv_gridder_destroy": (_int, [_vp]),
    "nlinv_autotune": (_int, [_vp, _vp, _vp, _vp, _int, C.POINTER(Tuning), C.POINTER(Tuning), _int]),
    "nlinv_set_shapes": (_int, [_vp, C.POINTER(Tuning)]),
    "nlinv_last_error": (C.c_char_p, [_vp]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Loads libnlinv.so once and attaches the signatures; raises if it is missing or incomplete."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnlinv.so not found at {path}: build it first "
                           "(python -m paper_1301_1215_gb300.build, or __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)          # AttributeError if a declared entry point is not exported
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NlinvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, ctx=None) -> None:
    if status != OK:
        msg = load().nlinv_last_error(ctx)
        raise NlinvError(status, msg.decode() if msg else "")
