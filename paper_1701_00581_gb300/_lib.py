"""ctypes binding of ``include/speckle.h`` (argument marshalling only).

Every name here mirrors a C entry point; all computation happens in the CUDA
library.  Loading fails loudly when the library has not been built: there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libspeckle_gb300.so")

SM_OK, SM_PENDING = 0, 1
SM_EINVAL, SM_ENOMEM, SM_EBUSY, SM_ETIMEDOUT, SM_ECUDA, SM_ECANCELED, SM_ENOTFOUND = (
    -1, -2, -3, -4, -5, -6, -7)
SM_FP32, SM_FP16, SM_BF16 = 0, 1, 2
SM_W_BISPEC, SM_W_UNIT, SM_W_SNR = 0, 1, 2
SM_U16, SM_F32 = 0, 1
SM_ACC_PLAIN, SM_ACC_KAHAN = 0, 1
SM_PHASE_FP32, SM_PHASE_FP64, SM_PHASE_FF = 0, 1, 2
SM_EDGE_PAD, SM_EDGE_DROP = 0, 1
SM_MOSAIC_BLEND, SM_MOSAIC_CENTRAL = 0, 1
SM_BATCH_FUSED, SM_BATCH_TILES, SM_BATCH_GRID = 1, 2, 3


class sm_channel(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("N", C.c_int), ("stride", C.c_int), ("R", C.c_int),
                ("fc", C.c_double), ("taper", C.c_int), ("spectra_prec", C.c_int),
                ("phase_weight", C.c_int), ("ck", C.c_double), ("max_frames", C.c_int),
                ("acc_mode", C.c_int), ("phase_prec", C.c_int), ("phase_iters", C.c_int),
                ("edge_mode", C.c_int), ("mosaic_mode", C.c_int), ("photon_gain", C.c_double)]


class sm_plan_info(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("nsx", C.c_int), ("nsy", C.c_int), ("N", C.c_int), ("K", C.c_int),
                ("R", C.c_int), ("box_rows", C.c_int), ("box_cols", C.c_int), ("box_pitch", C.c_int),
                ("hb_rows", C.c_int), ("n_tiles", C.c_int), ("tile_pairs", C.c_int),
                ("n_pairs", C.c_longlong), ("n_rings", C.c_int), ("n_points", C.c_int),
                ("n_U", C.c_int), ("n_V", C.c_int), ("n_cubes", C.c_int)]


class sm_workspace_layout(C.Structure):
    _fields_ = [(n, C.c_size_t) for n in
                ("spec", "flux", "mu", "P", "M", "noise", "A", "B", "z", "rec", "seeing", "stf", "refine",
                 "bytes")]


DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class sm_config(C.Structure):
    _fields_ = [("n_channels", C.c_int), ("ch", C.POINTER(sm_channel)),
                ("hbm_budget_bytes", C.c_size_t), ("max_inflight", C.c_int), ("device", C.c_int),
                ("overlap_kernels", C.c_int), ("dev_alloc", DEV_ALLOC), ("dev_free", DEV_FREE),
                ("alloc_ctx", C.c_void_p)]


class sm_burst(C.Structure):
    _fields_ = [("channel", C.c_int), ("F", C.c_int), ("frames", C.c_void_p), ("frame_type", C.c_int),
                ("frames_on_device", C.c_int), ("stf", C.c_void_p), ("d_over_r0", C.c_void_p),
                ("out", C.c_void_p), ("valid", C.c_void_p)]


class sm_result(C.Structure):
    _fields_ = [("status", C.c_int), ("t_submit_ms", C.c_double), ("t_done_ms", C.c_double),
                ("gpu_ms", C.c_double), ("bytes_admitted", C.c_size_t), ("d_over_r0", C.c_double),
                ("stage_ms", C.c_double * 8)]


class sm_batch_opts(C.Structure):
    _fields_ = [("lookahead", C.c_int), ("ctas_per_sm", C.c_int), ("launch", C.c_int), ("tile_order", C.c_int)]


class sm_batch_io(C.Structure):
    _fields_ = [("frames", C.c_void_p), ("stf", C.c_void_p), ("ws", C.c_void_p),
                ("lay", C.POINTER(sm_workspace_layout)), ("out", C.c_void_p), ("valid", C.c_void_p)]


_P = C.c_void_p
_I = C.c_int
_LAY = C.POINTER(sm_workspace_layout)

# name -> (restype, argtypes), the full public surface of speckle.h
SIGNATURES = {
    "sm_plan_create": (_I, [C.POINTER(sm_channel), _I, C.POINTER(_P)]),
    "sm_plan_destroy": (_I, [_P]),
    "sm_plan_get_info": (_I, [_P, C.POINTER(sm_plan_info)]),
    "sm_plan_subfields": (_I, [_P, _P]),
    "sm_plan_cubes": (_I, [_P, _P]),
    "sm_plan_pair_index": (_I, [_P, C.c_longlong, _P, _P]),
    "sm_workspace_query": (_I, [_P, _I, _I, _LAY]),
    "sm_stage_gain": (_I, [_P, _P, _P, _P, _P]),
    "sm_stage_calibrate": (_I, [_P, _P, _I, _I, _P, _P, _P, _P]),
    "sm_stage_track": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _P]),
    "sm_stage_shift": (_I, [_P, _P, _I, _I, _P, _P, _P]),
    "sm_stage_spectra": (_I, [_P, _P, _I, _I, _I, _I, _P, _LAY, _P]),
    "sm_stage_stats": (_I, [_P, _I, _I, _P, _LAY, _P]),
    "sm_stage_amplitude": (_I, [_P, _I, _P, _P, _LAY, _P]),
    "sm_stage_seeing": (_I, [_P, _I, _I, _I, _P, _LAY, _P]),
    "sm_stage_seeing_stf": (_I, [_P, _P, _LAY, _P]),
    "sm_stage_bispectrum": (_I, [_P, _I, _I, _P, _LAY, _P]),
    "sm_stage_phase": (_I, [_P, _I, _P, _LAY, _P]),
    "sm_stage_inverse": (_I, [_P, _I, _I, _I, _P, _LAY, _P]),
    "sm_stage_mosaic": (_I, [_P, _P, _LAY, _P, _P, _P]),
    "sm_reconstruct": (_I, [_P, _P, _I, _I, _P, _I, _P, _LAY, _P, _P, _P]),
    "sm_reconstruct_noalloc": (_I, [_P, _P, _I, _I, _P, _P, _P, _P]),
    "sm_model_stf": (_I, [C.POINTER(sm_channel), _I, _P, _P]),
    "sm_batch_create": (_I, [_I, C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(sm_batch_opts),
                             C.POINTER(_P)]),
    "sm_batch_get_opts": (_I, [_P, C.POINTER(sm_batch_opts)]),
    "sm_batch_destroy": (_I, [_P]),
    "sm_batch_info": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]),
    "sm_batch_spectra_bispectrum": (_I, [_P, C.POINTER(sm_batch_io), _P]),
    "sm_batch_reconstruct": (_I, [_P, C.POINTER(sm_batch_io), _P]),
    "sm_batch_status": (_I, [_P]),
    "sm_open": (_I, [C.POINTER(sm_config), C.POINTER(_P)]),
    "sm_submit_burst": (_I, [_P, C.POINTER(sm_burst), C.POINTER(C.c_uint64)]),
    "sm_submit_batch": (_I, [_P, _I, C.POINTER(sm_burst), C.POINTER(C.c_uint64)]),
    "sm_poll": (_I, [_P, C.c_uint64, _I, C.POINTER(sm_result)]),
    "sm_close": (_I, [_P]),
    "sm_strerror": (C.c_char_p, [_I]),
    "sm_last_error": (C.c_char_p, []),
}

_lib = None


class SpeckleError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = f"{where}: {lib.sm_strerror(status).decode()} ({status}): {lib.sm_last_error().decode()}"
        super().__init__(msg)
        self.status = status


def load() -> C.CDLL:
    """Load the CUDA library (raises if it is missing; build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_1701_00581_gb300.build` "
                           "(the CUDA library is required; there is no CPU path)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str) -> int:
    if status < 0:
        raise SpeckleError(status, where)
    return status
