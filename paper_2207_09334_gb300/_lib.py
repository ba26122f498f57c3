"""ctypes declarations of the C ABI in include/cronos_ms.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None


class MsParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("g", C.c_float * 3), ("k_c", C.c_float), ("mu", C.c_float),
                ("vel_damping", C.c_float), ("contact_on", C.c_int32), ("integrator", C.c_int32),
                ("strict_stability", C.c_int32), ("reorder", C.c_int32), ("kernel", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class MsAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class MsInfo(C.Structure):
    _fields_ = [("n_masses", C.c_int64), ("n_springs", C.c_int64), ("n_records", C.c_int64),
                ("n_slots", C.c_int64), ("n_back_slots", C.c_int64), ("device_bytes", C.c_int64),
                ("step_count", C.c_int64), ("stability_bound", C.c_double),
                ("max_fwd_degree", C.c_int32), ("max_back_degree", C.c_int32), ("kernel", C.c_int32),
                ("n_tiles", C.c_int32), ("max_tile_local", C.c_int32), ("lattice_guard", C.c_int32)]


class MsbVoxelSpec(C.Structure):
    _fields_ = [("voxel_edge", C.c_float), ("voxel_mass", C.c_float), ("freq", C.c_float),
                ("n_materials", C.c_int32), ("mat_k", C.c_void_p), ("mat_c", C.c_void_p),
                ("mat_amp", C.c_void_p)]


class MsbInfo(C.Structure):
    _fields_ = [("n_robots", C.c_int32), ("n_masses", C.c_int64), ("n_records", C.c_int64),
                ("max_robot_masses", C.c_int32), ("n_block_items", C.c_int32),
                ("n_warp_items", C.c_int32), ("device_bytes", C.c_int64), ("step_count", C.c_int64),
                ("threads", C.c_int32)]


STATUS = {0: "MS_OK", 1: "MS_ERR_ARG", 2: "MS_ERR_OOM", 3: "MS_ERR_CUDA", 4: "MS_ERR_UNSTABLE",
          5: "MS_ERR_NONFINITE", 6: "MS_ERR_TIMEOUT", 7: "MS_ERR_STATE"}


class MsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


VP = C.c_void_p
I32, I64, F32 = C.c_int32, C.c_int64, C.c_float

# name -> (restype, argtypes)
SIGNATURES = {
    "ms_create": (C.c_int, [C.POINTER(MsParams), I32, VP, VP, VP, VP, VP, I64, VP, VP, VP, F32, VP,
                            C.POINTER(MsAllocator), VP, C.POINTER(VP)]),
    "ms_create_materials": (C.c_int, [C.POINTER(MsParams), I32, VP, VP, VP, VP, VP, I64, VP, VP, I32, VP, VP,
                                      VP, VP, C.POINTER(MsAllocator), VP, C.POINTER(VP)]),
    "ms_set_actuation": (C.c_int, [VP, F32, VP, VP]),
    "ms_step": (C.c_int, [VP, I32]),
    "ms_get_state": (C.c_int, [VP, VP, VP, I32]),
    "ms_set_state": (C.c_int, [VP, VP, VP, I32]),
    "ms_sync": (C.c_int, [VP]),
    "ms_set_wait_limit": (C.c_int, [VP, I32]),
    "ms_test_barrier_deficit": (C.c_int, [VP, I32]),
    "ms_get_info": (C.c_int, [VP, C.POINTER(MsInfo)]),
    "ms_energy": (C.c_int, [VP, VP, I32]),
    "ms_trace_set": (C.c_int, [VP, VP, I32, I32]),
    "ms_trace_get": (C.c_int, [VP, VP, VP, I32]),
    "ms_destroy": (C.c_int, [VP]),
    "ms_last_error": (C.c_char_p, []),
    "msb_create": (C.c_int, [C.POINTER(MsParams), C.POINTER(MsbVoxelSpec), I32, VP, VP, VP, VP,
                             C.POINTER(MsAllocator), VP, C.POINTER(VP)]),
    "msb_autotune": (C.c_int, [VP, I32, I32]),
    "msb_set_threads": (C.c_int, [VP, I32]),
    "msb_run": (C.c_int, [VP, I32]),
    "msb_run_loop": (C.c_int, [VP, I32]),
    "msb_com_travel": (C.c_int, [VP, VP, I32]),
    "msb_robot_info": (C.c_int, [VP, I32, C.POINTER(I32), C.POINTER(I64)]),
    "msb_get_state": (C.c_int, [VP, VP, VP]),
    "msb_reset": (C.c_int, [VP]),
    "msb_get_info": (C.c_int, [VP, C.POINTER(MsbInfo)]),
    "msb_destroy": (C.c_int, [VP]),
    "msa_create": (C.c_int, [C.POINTER(MsParams), C.POINTER(MsbVoxelSpec), I32, VP, VP, I32, I32,
                             C.POINTER(MsAllocator), VP, C.POINTER(VP)]),
    "msa_gradients": (C.c_int, [VP, I32, VP, VP, VP, VP, VP, VP, I32]),
    "msa_sizes": (C.c_int, [VP, C.POINTER(I64), C.POINTER(I64)]),
    "msa_set_threads": (C.c_int, [VP, I32]),
    "msa_threads": (I32, [VP]),
    "msa_destroy": (C.c_int, [VP]),
    "mlp_create": (C.c_int, [I32, I32, I32, C.c_uint64, C.POINTER(MsAllocator), VP, C.POINTER(VP)]),
    "mlp_num_params": (I64, [VP]),
    "mlp_set_params": (C.c_int, [VP, VP]),
    "mlp_get_params": (C.c_int, [VP, VP, VP]),
    "mlp_encode": (C.c_int, [VP, VP, I32]),
    "mlp_set_input": (C.c_int, [VP, VP, I32]),
    "mlp_forward": (C.c_int, [VP, I32, VP]),
    "mlp_forward_materials": (C.c_int, [VP, VP, I32, VP]),
    "mlp_backward": (C.c_int, [VP, VP, I32, VP]),
    "mlp_adam": (C.c_int, [VP, F32, F32, F32, F32]),
    "mlp_sync": (C.c_int, [VP]),
    "mlp_destroy": (C.c_int, [VP]),
    "mlp_gemm_bf16": (C.c_int, [VP, VP, VP, I32, I32, I32, VP]),
    "ms_step_csr_noalloc": (C.c_int, [C.POINTER(MsParams), I32, VP, VP, VP, VP, VP, VP, VP, VP, VP, I32, VP, VP,
                                      VP]),
    "ms_version": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the compiled library.  Raises if it is absent: there is no
    fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int):
    if code != 0:
        raise MsError(code, load().ms_last_error().decode())
