"""ctypes loader for ``libbm.so``: argument marshalling only.

Every computation happens in the library's CUDA kernels.  If the library is
missing this module raises at import time; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbm.so")
HEADERS = [os.path.join(os.path.dirname(HERE), "include", "bm.h")]

u64, u32, i32, vp, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
P64 = ctypes.POINTER(ctypes.c_uint64)


class bm_query(ctypes.Structure):
    _fields_ = [("ids", vp), ("n", u32), ("kind", u32), ("theta", u32), ("lo", u32), ("hi", u32),
                ("table", vp), ("out_words", vp), ("path", ctypes.c_int32), ("reserved", u32)]


class bm_weighted_query(ctypes.Structure):
    _fields_ = [("ids", vp), ("weights", vp), ("n", u32), ("post_op", u32), ("theta", u64),
                ("post_id", u32), ("reserved", u32), ("out_words", vp)]


class bm_pool_info_t(ctypes.Structure):
    _fields_ = [("r_bits", u64), ("words", u64), ("stride_words", u64), ("capacity", u32),
                ("dense_loaded", u32), ("lists_loaded", u32), ("sm_count", u32),
                ("device_bytes", u64), ("dense_base", vp), ("rle_loaded", u32), ("reserved", u32)]


class bm_dense_config_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("variant", "threads", "stages", "ctas_per_sm",
                                              "adder", "words_per_thread")]


class bm_sparse_config_t(ctypes.Structure):
    _fields_ = [("tile_rows", u32), ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("unroll", ctypes.c_int32)]


class bm_batch_config_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("ctas_per_sm", "adder", "words_per_thread")]


class bm_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", u64), ("max_batch", u32), ("max_inflight", u32), ("max_queue", u32),
                ("batch_window_us", u32), ("slo_us", u32), ("reserved", u32)]


class bm_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", u64), ("completed", u64), ("refused", u64), ("batches", u64),
                ("batched_queries", u64), ("waiting", u32), ("free_slots", u32),
                ("total_slots", u32), ("max_batch_seen", u32), ("last_error", ctypes.c_int32),
                ("cancelled", u64), ("expired", u64)]


# name -> (restype, argtypes)
SIGNATURES = {
    "bm_strerror": (ctypes.c_char_p, [i32]),
    "bm_pool_create": (i32, [i32, u64, u32, u64, ctypes.POINTER(vp)]),
    "bm_pool_destroy": (i32, [vp]),
    "bm_pool_put_dense": (i32, [vp, u32, u32, vp, u64, i32]),
    "bm_pool_put_positions": (i32, [vp, u32, u32, vp, vp, i32]),
    "bm_pool_put_complement_positions": (i32, [vp, u32, u32, vp, vp, i32]),
    "bm_pool_info": (i32, [vp, ctypes.POINTER(bm_pool_info_t)]),
    "bm_pool_put_rle": (i32, [vp, u32, u32]),
    "bm_weighted_threshold": (i32, [vp, ctypes.POINTER(bm_weighted_query), vp, vp]),
    "bm_pool_rle_info": (i32, [vp, u32, P64, P64, P64]),
    "bm_pool_bitmap_cardinality": (i32, [vp, u32, P64]),
    "bm_pool_status": (i32, [vp]),
    "bm_pool_set_dense_config": (i32, [vp, ctypes.POINTER(bm_dense_config_t)]),
    "bm_pool_get_dense_config": (i32, [vp, ctypes.POINTER(bm_dense_config_t)]),
    "bm_pool_set_looped": (i32, [vp, u32]),
    "bm_pool_get_looped": (i32, [vp, ctypes.POINTER(u32)]),
    "bm_pool_get_sparse_config": (i32, [vp, ctypes.POINTER(bm_sparse_config_t)]),
    "bm_pool_get_batch_config": (i32, [vp, ctypes.POINTER(bm_batch_config_t)]),
    "bm_pool_autotune": (i32, [vp, ctypes.c_char_p, ctypes.c_char_p, u64]),
    "bm_threshold_batch": (i32, [vp, vp, u32, vp, vp, vp]),
    "bm_pool_set_batch_config": (i32, [vp, ctypes.POINTER(bm_batch_config_t)]),
    "bm_threshold": (i32, [vp, vp, u32, u32, vp, vp, vp]),
    "bm_symmetric": (i32, [vp, vp, u32, vp, vp, vp, vp]),
    "bm_cardinality": (i32, [vp, u64, vp, vp]),
    "bm_pool_set_sparse_config": (i32, [vp, ctypes.POINTER(bm_sparse_config_t)]),
    "bm_query_run": (i32, [vp, vp, vp, vp, vp]),
    "bm_query_features": (i32, [vp, vp, vp]),
    "bm_pool_set_selector": (i32, [vp, vp, u64, vp, vp, u32]),
    "bm_query_select": (i32, [vp, vp, vp, vp]),
    "bm_mlp_forward": (i32, [vp, u32, u32, u32, vp, u32, vp, vp, vp, vp]),
    "bm_mlp_backward": (i32, [vp, u32, u32, u32, vp, vp, vp, vp, vp, u32, vp, vp, vp, vp]),
    "bm_mlp_adam": (i32, [vp, vp, vp, vp, u64, u32, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, ctypes.c_float, vp]),
    "bm_pool_selftest_wait": (i32, [vp, u32, vp]),
    "bm_server_create": (i32, [vp, ctypes.POINTER(bm_server_config), ctypes.POINTER(vp)]),
    "bm_server_destroy": (i32, [vp]),
    "bm_server_submit": (i32, [vp, vp, ctypes.POINTER(u64)]),
    "bm_server_wait": (i32, [vp, u64, u32]),
    "bm_server_submit_deadline": (i32, [vp, vp, u64, ctypes.POINTER(u64)]),
    "bm_server_cancel": (i32, [vp, u64]),
    "bm_server_result": (i32, [vp, u64, vp, vp, vp, vp, vp]),
    "bm_server_release": (i32, [vp, u64]),
    "bm_server_stats": (i32, [vp, ctypes.POINTER(bm_server_stats_t)]),
    "bm_server_replay": (i32, [vp, vp, u32, vp, vp, vp, vp, vp, vp]),
    "bm_threshold_noalloc": (i32, [vp, u64, u32, u64, vp, u32, u32, vp, vp, vp]),
}


def declared_symbols() -> list[str]:
    """Entry points declared in include/*.h (function prototypes only)."""
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(bm_[a-z0-9_]+)\s*\(", src):
            names.append(m.group(1))
    return sorted(set(names))


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: the CUDA library must be built first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib
