"""ctypes declarations of the C ABI in include/mpt.h.

Argument marshalling only: every step of a transfer runs inside libmpt.so.  The library
is built in-tree (``paper_2604_22228_gb300/libmpt.so``) by ``build.py``; loading fails
loudly when it is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpt.so")

# status codes
MPT_OK, MPT_EINVAL, MPT_ENOMEM, MPT_EAGAIN, MPT_ETIMEDOUT, MPT_ENOTSUP, MPT_ECUDA = range(7)
STATUS_NAMES = {0: "MPT_OK", 1: "MPT_EINVAL", 2: "MPT_ENOMEM", 3: "MPT_EAGAIN", 4: "MPT_ETIMEDOUT",
                5: "MPT_ENOTSUP", 6: "MPT_ECUDA"}
# directions, path kinds, layouts, kernel variants
MPT_D2D, MPT_H2D, MPT_D2H = 0, 1, 2
MPT_PATH_CE, MPT_PATH_SM, MPT_PATH_HS, MPT_PATH_ZC = 1, 2, 4, 8
MPT_LAYOUT_CONTIG, MPT_LAYOUT_INTERLEAVE = 0, 1
MPT_SM_VEC128, MPT_SM_BULK, MPT_SM_TILE8K = 0, 1, 2
MPT_HS_HOST_THREADS = 1
MPT_PLAN_PAGEABLE, MPT_MODE_PAGEABLE = 0x200, 0x10
MPT_PLAN_DUPLEX, MPT_MODE_DUPLEX = 0x400, 0x20
MPT_BATCH_TUNE_TIME, MPT_BATCH_TUNE_P99 = 0, 1
MPT_PLAN_EAGER = 0x100
MPT_MODE_GRAPH, MPT_MODE_EAGER = 0, 1
MPT_PREPARE_GRAPH, MPT_PREPARE_EAGER, MPT_PREPARE_AUTO = 0, 1, 2
MPT_SHARE_ONE = 65536
MPT_MAX_PATHS = 8
MPT_MAX_CHUNKS = 1 << 20
MPT_NOALLOC_MAX_RANGES = 1024
MPT_BULK_CONFIGS = 7


class mpt_path_spec(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("share", C.c_uint32), ("chunk_bytes", C.c_uint64),
                ("ctas", C.c_uint32), ("flags", C.c_uint32)]


class mpt_chunk(C.Structure):
    _fields_ = [("offset", C.c_uint64), ("bytes", C.c_uint64), ("path_index", C.c_uint32),
                ("chunk_index", C.c_uint32)]


class mpt_xfer(C.Structure):
    _fields_ = [("src", C.c_void_p), ("dst", C.c_void_p), ("bytes", C.c_uint64), ("dir", C.c_uint32),
                ("flags", C.c_uint32)]


class mpt_graph_info(C.Structure):
    _fields_ = [("nodes", C.c_uint32), ("memcpy_nodes", C.c_uint32), ("kernel_nodes", C.c_uint32),
                ("memset_nodes", C.c_uint32), ("create_us", C.c_double), ("construct_us", C.c_double),
                ("instantiate_us", C.c_double), ("staging_bytes", C.c_uint64), ("update_us", C.c_double),
                ("rebinds", C.c_uint32), ("mode", C.c_uint32), ("host_nodes", C.c_uint32)]


class mpt_path_model(C.Structure):
    _fields_ = [("alpha_ps", C.c_uint64), ("beta_Bps", C.c_uint64), ("beta2_Bps", C.c_uint64)]


class mpt_model(C.Structure):
    _fields_ = [("launch_ps", C.c_uint64), ("hbm_Bps", C.c_uint64), ("link_h2d_Bps", C.c_uint64),
                ("link_d2h_Bps", C.c_uint64), ("ce", mpt_path_model), ("sm", mpt_path_model),
                ("hs", mpt_path_model), ("zc", mpt_path_model)]


class mpt_batch_tuning(C.Structure):
    _fields_ = [("ctas", C.c_uint32), ("tile_bytes", C.c_uint32), ("dma_lanes", C.c_uint32),
                ("dma_items", C.c_uint32), ("dma_min_bytes", C.c_uint64), ("batch_us", C.c_double),
                ("p99_us", C.c_double), ("candidates", C.c_uint32), ("reserved", C.c_uint32)]


class mpt_serve_config(C.Structure):
    _fields_ = [("staging_budget_bytes", C.c_uint64), ("max_batch", C.c_uint32),
                ("max_inflight_batches", C.c_uint32), ("streams", C.c_uint32), ("batch_ctas", C.c_uint32)]


class mpt_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("arrival_ns", C.c_uint64), ("admit_ns", C.c_uint64),
                ("complete_ns", C.c_uint64), ("bytes", C.c_uint64), ("status", C.c_uint32),
                ("reserved", C.c_uint32)]


class mpt_serve_stats_t(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "batches", "inflight_bytes",
                                          "max_inflight_bytes", "rejected", "max_pending_completions",
                                          "max_turn_ns", "max_waiting", "max_batch_ns", "max_batch_reqs",
                                          "max_batch_bytes", "max_harvest_ns", "max_admit_ns",
                                          "max_launch_ns")]


class mpt_device_info(C.Structure):
    _fields_ = [("name", C.c_char * 96), ("device", C.c_int32), ("sms", C.c_int32), ("copy_engines", C.c_int32),
                ("pageable_access", C.c_int32), ("l2_bytes", C.c_uint64), ("memory_bytes", C.c_uint64)]


H = C.c_void_p  # opaque handles
P = C.POINTER

# name -> (restype, argtypes); the names and order follow include/mpt.h
SIGNATURES = {
    "mpt_version": (C.c_char_p, []),
    "mpt_last_error": (C.c_char_p, []),
    "mpt_ctx_create": (C.c_int, [C.c_int, C.c_char_p, P(H)]),
    "mpt_ctx_destroy": (C.c_int, [H]),
    "mpt_ctx_info": (C.c_int, [H, P(mpt_device_info)]),
    "mpt_ctx_status": (C.c_int, [H, P(C.c_uint32)]),
    "mpt_ctx_set_wait_limit": (C.c_int, [H, C.c_uint64]),
    "mpt_trace_lanes": (C.c_int, [H, C.c_uint32]),
    "mpt_lane_times": (C.c_int, [H, P(C.c_float), C.c_uint32, P(C.c_uint32)]),
    "mpt_plan": (C.c_int, [H, C.c_uint64, C.c_uint32, P(mpt_path_spec), C.c_uint32, C.c_uint32, C.c_uint32,
                          P(H)]),
    "mpt_plan_chunks": (C.c_int, [H, P(mpt_chunk), C.c_size_t, P(C.c_size_t)]),
    "mpt_plan_paths": (C.c_int, [H, P(mpt_path_spec), C.c_uint32, P(C.c_uint32)]),
    "mpt_plan_destroy": (C.c_int, [H]),
    "mpt_capture": (C.c_int, [H, H, C.c_void_p, C.c_void_p, P(H)]),
    "mpt_prepare": (C.c_int, [H, H, C.c_void_p, C.c_void_p, C.c_uint32, P(H)]),
    "mpt_launch": (C.c_int, [H, C.c_void_p]),
    "mpt_graph_get_info": (C.c_int, [H, P(mpt_graph_info)]),
    "mpt_graph_rebind": (C.c_int, [H, H, C.c_void_p, C.c_void_p]),
    "mpt_graph_release": (C.c_int, [H]),
    "mpt_graph_evict": (C.c_int, [H, C.c_void_p, P(C.c_uint32)]),
    "mpt_launch_eager": (C.c_int, [H, H, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mpt_sm_copy": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint32, C.c_void_p]),
    "mpt_hash_device": (C.c_int, [H, C.c_void_p, C.c_uint64, C.c_void_p, P(C.c_uint64)]),
    "mpt_model_time": (C.c_int, [P(mpt_model), C.c_uint32, P(C.c_uint32), P(C.c_uint64), C.c_uint32, C.c_uint64,
                                 P(C.c_uint64)]),
    "mpt_model_optimize": (C.c_int, [P(mpt_model), C.c_uint64, C.c_uint32, P(C.c_uint32), C.c_uint32, C.c_uint32,
                                     P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]),
    "mpt_tune": (C.c_int, [H, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, P(mpt_path_spec), P(C.c_uint32),
                           P(C.c_double)]),
    "mpt_tune_save": (C.c_int, [H, C.c_char_p]),
    "mpt_tune_load": (C.c_int, [H, C.c_char_p]),
    "mpt_tune_get": (C.c_int, [H, C.c_uint32, C.c_uint64, C.c_uint32, P(mpt_path_spec), P(C.c_uint32),
                               P(C.c_double)]),
    "mpt_batch_configure": (C.c_int, [H, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]),
    "mpt_batch_configure_dma": (C.c_int, [H, C.c_uint32, C.c_uint32, C.c_uint64]),
    "mpt_batch_tune": (C.c_int, [H, C.c_void_p, C.c_size_t, C.c_uint32, C.c_uint32, C.c_void_p,
                                 C.POINTER(mpt_batch_tuning)]),
    "mpt_batch_register": (C.c_int, [H, C.c_void_p, C.c_uint64]),
    "mpt_batch_submit": (C.c_int, [H, P(mpt_xfer), C.c_size_t, C.c_void_p, P(H)]),
    "mpt_batch_poll": (C.c_int, [H, P(C.c_size_t), P(C.c_uint8)]),
    "mpt_batch_wait": (C.c_int, [H, C.c_uint64]),
    "mpt_batch_times": (C.c_int, [H, P(C.c_uint64)]),
    "mpt_batch_watch": (C.c_int, [H, C.c_uint64, P(C.c_uint64), C.c_uint64]),
    "mpt_batch_release": (C.c_int, [H]),
    "mpt_copy_each": (C.c_int, [H, P(mpt_xfer), C.c_size_t, P(C.c_void_p), P(C.c_uint64), C.c_uint64]),
    "mpt_now_ns": (C.c_uint64, []),
    "mpt_serve_start": (C.c_int, [H, P(mpt_serve_config), P(H)]),
    "mpt_serve_submit": (C.c_int, [H, P(mpt_xfer), C.c_uint64, C.c_uint64]),
    "mpt_serve_replay": (C.c_int, [H, P(mpt_xfer), P(C.c_uint64), P(C.c_uint64), C.c_size_t, P(C.c_uint64)]),
    "mpt_serve_poll": (C.c_int, [H, P(mpt_completion), C.c_size_t, P(C.c_size_t)]),
    "mpt_serve_stats": (C.c_int, [H, P(mpt_serve_stats_t)]),
    "mpt_serve_reset_stats": (C.c_int, [H]),
    "mpt_serve_stop": (C.c_int, [H]),
    "mpt_demo_jacobi_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint64, C.c_void_p]),
    "mpt_selftest_flag_timeout": (C.c_int, [H, C.c_uint64, P(C.c_uint32)]),
    "mpt_hash_ranges_noalloc": (C.c_int, [P(C.c_void_p), P(C.c_uint64), C.c_uint32, C.c_void_p, P(C.c_uint64)]),
    "mpt_host_alloc": (C.c_int, [H, C.c_uint64, P(C.c_void_p), P(C.c_void_p)]),
    "mpt_host_free": (C.c_int, [H, C.c_void_p]),
    "mpt_host_bandwidth": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, P(C.c_double)]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmpt.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2604_22228_gb300.build` "
                          "(the library has no non-CUDA fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
