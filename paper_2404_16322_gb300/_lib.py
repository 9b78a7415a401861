"""ctypes declarations of every entry point of include/dade.h.

Loads the in-tree ``_build/libdade.so``.  There is no fallback: if the
library is missing, importing this module raises, so the CUDA path is the
only path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdade.so")

c_i32, c_i64, c_u64, c_f64, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
c_vp, c_cp = ctypes.c_void_p, ctypes.c_char_p

STATUS = {0: "DADE_OK", 1: "DADE_EINVAL", 2: "DADE_ENOMEM", 3: "DADE_ECUDA", 4: "DADE_ETIMEOUT",
          5: "DADE_ESTATE", 6: "DADE_ENOTIMPL", 7: "DADE_EIO"}
SLAB = {"f32": 0, "bf16": 1, "fp8": 2}
MODE = {"prune": 0, "full": 1}
ESTIMATOR = {"learned": 0, "res": 1, "pq": 2}
SCAN_KERNEL = {"auto": 0, "cuda": 1, "tensor": 2}


class BuildParams(ctypes.Structure):
    _fields_ = [("nlist", c_i32), ("kmeans_iters", c_i32), ("seed", c_u64), ("dtype", ctypes.c_int),
                ("centroids", c_vp), ("assign", c_vp), ("ids", c_vp)]


class SearchOpts(ctypes.Structure):
    _fields_ = [("mode", c_i32), ("max_K", c_i32), ("max_nprobe", c_i32), ("first_wave", c_i32),
                ("tau_dev", c_vp), ("probe_in_dev", c_vp), ("probe_out_dev", c_vp),
                ("qrot_out_dev", c_vp), ("stats_dev", c_vp), ("status_dev", c_vp),
                ("workspace", c_vp), ("workspace_bytes", c_sz), ("wave_growth_log2", c_i32),
                ("final_test", c_i32), ("estimator", c_i32), ("res_m", ctypes.c_float),
                ("test_steps", c_i32), ("scan_kernel", c_i32), ("candidate_budget_bytes", c_i64),
                ("queries_per_unit", c_i32)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("N", c_i64), ("D", c_i32), ("Dpad", c_i32), ("nlist", c_i32), ("dtype", c_i32),
                ("max_list", c_i64), ("device_bytes", c_i64)]


# name -> (restype, argtypes), in the order of include/dade.h
SIGNATURES = {
    "dade_train_rotation": (ctypes.c_int, [c_vp, c_i64, c_i32, c_i64, c_u64, c_vp, c_vp, c_vp]),
    "dade_random_rotation": (ctypes.c_int, [c_i32, c_u64, c_vp]),
    "dade_pq_train": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_i32, c_u64, c_vp, c_vp]),
    "dade_pq_set": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp]),
    "dade_pq_fit_correction": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_i32, c_f64, c_u64, c_i64, c_vp]),
    "dade_pq_fit_samples": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_f64, c_i32, c_vp]),
    "dade_pq_set_correction": (ctypes.c_int, [c_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "dade_pq_get": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dade_ads_table": (ctypes.c_int, [c_i32, c_i32, c_f64, c_vp, c_vp]),
    "ivf_build": (ctypes.c_int, [c_vp, c_i64, c_i32, c_vp, c_vp, ctypes.POINTER(BuildParams),
                                 ctypes.POINTER(c_vp)]),
    "dade_fit_correction": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_i32, c_i32, c_f64, c_u64, c_i64,
                                           c_vp, c_vp]),
    "dade_fit_collect": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_i32, c_i32, c_u64, c_i64, c_i64,
                                        ctypes.POINTER(c_i64), c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dade_partials_collect": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_i32, c_i64, ctypes.POINTER(c_i64),
                                             c_vp, c_vp, c_vp]),
    "dade_arena_create": (ctypes.c_int, [c_i64, c_i64, ctypes.POINTER(c_vp)]),
    "dade_arena_alloc": (c_i64, [c_vp, c_i64]),
    "dade_arena_free": (ctypes.c_int, [c_vp, c_i64]),
    "dade_arena_used": (c_i64, [c_vp]),
    "dade_arena_largest_free": (c_i64, [c_vp]),
    "dade_arena_destroy": (None, [c_vp]),
    "dade_fit_samples": (ctypes.c_int, [c_vp, c_vp, c_vp, c_i64, c_i32, c_i32, c_f64, c_i32, c_vp, c_vp]),
    "dade_set_correction": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp]),
    "dade_get_correction": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp]),
    "dade_search": (ctypes.c_int, [c_vp, c_vp, c_i64, c_vp, c_vp, c_i32, ctypes.POINTER(SearchOpts),
                                   c_vp, c_vp, c_vp, c_vp]),
    "dade_search_noalloc": (ctypes.c_int, [c_vp, c_vp, c_i64, c_vp, c_vp, c_i32, ctypes.POINTER(SearchOpts),
                                           c_vp, c_vp, c_vp, c_vp]),
    "dade_search_workspace_size": (c_sz, [c_vp, c_i64, c_i32, ctypes.POINTER(SearchOpts)]),
    "dade_search_kernel_count": (ctypes.c_int, [c_vp, c_vp, c_i64, c_vp, c_vp, c_i32, ctypes.POINTER(SearchOpts),
                                                c_vp, c_vp, c_vp, ctypes.POINTER(c_i64)]),
    "dade_index_info_get": (ctypes.c_int, [c_vp, ctypes.POINTER(IndexInfo)]),
    "dade_index_centroids": (ctypes.c_int, [c_vp, c_vp]),
    "dade_index_assignment": (ctypes.c_int, [c_vp, c_vp]),
    "dade_index_list_sizes": (ctypes.c_int, [c_vp, c_vp]),
    "dade_index_stored": (ctypes.c_int, [c_vp, c_i64, c_i64, c_vp]),
    "dade_index_save": (ctypes.c_int, [c_vp, c_cp]),
    "dade_index_load": (ctypes.c_int, [c_cp, ctypes.POINTER(c_vp)]),
    "dade_index_free": (None, [c_vp]),
    "dade_shard_owners": (ctypes.c_int, [c_vp, c_i32, c_i32, c_vp]),
    "dade_index_shard": (ctypes.c_int, [c_vp, c_i32, c_i32, ctypes.POINTER(c_vp)]),
    "dade_merge_topk": (ctypes.c_int, [c_i32, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dade_stage_timing": (ctypes.c_int, [c_i32]),
    "dade_stage_timing_read": (ctypes.c_int, [c_vp, c_vp, c_vp]),
    "dade_last_error": (c_cp, []),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2404_16322_gb300/build.py)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class DadeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
