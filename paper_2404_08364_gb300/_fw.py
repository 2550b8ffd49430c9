"""ctypes binding of libfw.so (include/fw.h): argument marshalling only.

Every step of the walk runs in the library's CUDA kernels; this module turns
torch tensors into pointers and C structs and raises on a non-zero status.
There is no fallback: if the library is missing or fails to load, importing
the binding raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfw.so")

FW_OK, FW_EINVAL, FW_ENOMEM, FW_ECUDA, FW_EUNSORTED, FW_ETIMEOUT, FW_EBUSY = 0, -1, -2, -3, -4, -5, -6
FW_WEIGHTED, FW_NODE2VEC, FW_METAPATH, FW_PPR = 0, 1, 2, 3
FW_EXACT, FW_FAST = 0, 1
FW_HOST_PTRS, FW_DEVICE_PTRS, FW_BORROW, FW_NO_VALIDATE = 0, 1, 2, 4

ALGOS = {"weighted": FW_WEIGHTED, "deepwalk": FW_WEIGHTED, "node2vec": FW_NODE2VEC,
         "metapath": FW_METAPATH, "ppr": FW_PPR}
MODES = {"exact": FW_EXACT, "fast": FW_FAST}


class FwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fw status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n2v_p", ctypes.c_float), ("n2v_q", ctypes.c_float),
                ("n2v_scale", ctypes.c_int32), ("schema_len", ctypes.c_int32),
                ("schema", ctypes.c_int8 * 16), ("ppr_stop", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("d_warp", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("walks", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("rows_scanned", ctypes.c_uint64),
                ("warp_steps", ctypes.c_uint64), ("block_steps", ctypes.c_uint64),
                ("n2v_tests", ctypes.c_uint64), ("algo_bytes", ctypes.c_uint64),
                ("aux_device_bytes", ctypes.c_uint64), ("last_kernel_ms", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("params", Params), ("starts", ctypes.c_void_p),
                ("n_q", ctypes.c_int64), ("lengths", ctypes.c_void_p), ("max_len", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("q_id0", ctypes.c_int64), ("prev", ctypes.c_void_p),
                ("step0", ctypes.c_void_p), ("paths", ctypes.c_void_p), ("path_len", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("arena_used", ctypes.c_uint64),
                ("arena_capacity", ctypes.c_uint64), ("busy_s", ctypes.c_double)]


# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "fw_load_csr": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P,
                                   ctypes.c_uint32]),
    "fw_free": (None, [_P]),
    "fw_walk": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Params), _P, ctypes.c_int64, _P,
                               ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P, _P]),
    "fw_walk_ex": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Params), _P, ctypes.c_int64, _P,
                                  ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "fw_walk_multi": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.c_int32, _P]),
    "fw_walk_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.c_int32, _P]),
    "fw_walk_batched": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Params), _P, ctypes.c_int64, _P,
                                       ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint64, _P, _P,
                                       ctypes.POINTER(ctypes.c_int64)]),
    "fw_batch_size": (ctypes.c_int64, [ctypes.c_uint64, ctypes.c_int32]),
    "fw_sampler_run": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_uint64, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "fw_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "fw_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "fw_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "fw_stats_reset": (ctypes.c_int, [_P, _P]),
    "fw_sync": (ctypes.c_int, [_P]),
    "fw_graph_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "fw_philox": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "fw_server_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                        ctypes.POINTER(_P)]),
    "fw_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "fw_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]),
    "fw_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "fw_server_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "fw_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "fw_server_destroy": (None, [_P]),
    "fw_capture_multi": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.c_int32, ctypes.POINTER(_P)]),
    "fw_exec_launch": (ctypes.c_int, [_P, _P]),
    "fw_exec_destroy": (None, [_P]),
    "fw_autotune": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_double)]),
    "fw_autotune_clear_cache": (ctypes.c_int, []),
    "fw_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fw_last_error": (ctypes.c_char_p, []),
    "fw_version": (ctypes.c_int, []),
}

_lib = None


def lib(path: str = LIB_PATH):
    """Load libfw.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FwError(FW_ECUDA, f"{path} is missing: build it with paper_2404_08364_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int):
    if rc != FW_OK:
        msg = lib().fw_last_error().decode(errors="replace")
        raise FwError(rc, msg)
    return rc


def make_params(mode="exact", p=1.0, q=1.0, scale=2, schema=(0, 1, 2, 3, 4), ppr_stop=0.2) -> Params:
    c = Params()
    c.mode = MODES.get(mode, mode)
    c.n2v_p, c.n2v_q, c.n2v_scale = float(p), float(q), int(scale)
    if not 0 < len(schema) <= 16:
        raise ValueError("schema length must be in [1, 16]")
    c.schema_len = len(schema)
    for i, s in enumerate(schema):
        c.schema[i] = int(s)
    c.ppr_stop = float(ppr_stop)
    return c
