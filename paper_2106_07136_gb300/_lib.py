"""ctypes declarations of libbdis.so (include/bdis.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_float, c_size_t, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p

BDIS_OK, BDIS_E_INVALID_ARG, BDIS_E_NOMEM, BDIS_E_CUDA, BDIS_E_TIMEOUT, BDIS_E_UNSUPPORTED = range(6)
BDIS_U8, BDIS_F32 = 0, 1
BDIS_FUSION_BDIS, BDIS_FUSION_DIS = 0, 1

# Every symbol include/bdis.h declares.
EXPORTED = [
    "bdis_default_params", "bdis_status_string", "bdis_last_error_string", "bdis_version",
    "bdis_level_dims", "bdis_grid", "bdis_patch_count", "bdis_create", "bdis_reserve",
    "bdis_workspace_bytes", "bdis_destroy", "bdis_match", "bdis_match_host",
    "bdis_match_host_async", "bdis_host_wait",
    "bdis_prepare_level0", "bdis_pyramid_level", "bdis_search_level", "bdis_densify_level",
    "bdis_upsample", "bdis_enable_timing", "bdis_read_timing", "bdis_pack_right",
    "bdis_match_static", "bdis_probe_fp32_tflops", "bdis_set_search_variant",
    "bdis_get_search_variant", "bdis_set_search_tiling", "bdis_get_search_tiling",
    "bdis_set_densify_variant", "bdis_get_densify_variant", "bdis_set_pyramid_variant",
    "bdis_get_pyramid_variant", "bdis_set_net_variant", "bdis_get_net_variant",
    "bdis_plan_create", "bdis_plan_run", "bdis_plan_info",
    "bdis_plan_workspace_bytes", "bdis_plan_destroy", "bdis_match_warm", "bdis_warm_map",
    "bdis_net_weight_count", "bdis_net_create", "bdis_net_forward", "bdis_net_gradient",
    "bdis_net_train_step", "bdis_net_get_weights", "bdis_net_destroy", "bdis_match_seeded",
    "bdis_match_learned", "bdis_select_start", "bdis_host_wait_timeout",
    "bdis_inject_alloc_failures", "bdis_net_status", "bdis_net_inject_timeout",
    "bdis_proposal_level", "bdis_set_launch_overlap", "bdis_get_launch_overlap",
    "bdis_check_status", "bdis_checked_build",
]

BDIS_PLAN_AUTOTUNE = 1
BDIS_PLAN_SCALE_TO_WIDTH = 2

STATIC_SCRATCH_BYTES = 24 << 20  # BDIS_STATIC_SCRATCH_BYTES
ASYNC_SLOTS = 4  # BDIS_ASYNC_SLOTS: bdis_match_host_async calls in flight at once

TIMING_CLASSES = ["prepare_level0", "pyramid_level", "search", "densify", "upsample",
                  "warm_map", "proposal_net", "select_start"]


class BdisParams(ctypes.Structure):
    _fields_ = [
        ("patch_size", c_int), ("overlap", c_float), ("iterations", c_int),
        ("coarsest_scale", c_int), ("finest_scale", c_int), ("sigma_r", c_float),
        ("sigma_s", c_float), ("window_samples", c_int), ("window_step", c_float),
        ("gamma", c_float), ("normalize", c_int), ("fusion", c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BdisImage(ctypes.Structure):
    _fields_ = [
        ("data", c_void_p), ("width", c_int), ("height", c_int), ("pitch_bytes", c_size_t),
        ("image_stride_bytes", c_size_t), ("count", c_int), ("format", c_int),
    ]


class BdisPatchDebug(ctypes.Structure):
    _fields_ = [("u_init", c_void_p), ("posterior", c_void_p), ("energies", c_void_p),
                ("flags", c_void_p), ("n_valid", c_void_p), ("steps", c_void_p)]


class BdisGroup(ctypes.Structure):
    _fields_ = [("left", BdisImage), ("right", BdisImage), ("disparity_out", c_void_p)]


class BdisPlanChoice(ctypes.Structure):
    _fields_ = [("search_columns_per_lane", c_int), ("search_block_threads", c_int),
                ("densify_tile_height", c_int), ("workspace_bytes", c_size_t),
                ("coarsest_scale", c_int), ("search_tiling", c_int)]


class BdisTiming(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8)]


class BdisError(RuntimeError):
    def __init__(self, status, what):
        lib = load()
        msg = lib.bdis_status_string(status).decode()
        detail = lib.bdis_last_error_string().decode()
        super().__init__(f"{what}: {msg}" + (f" ({detail})" if detail else ""))
        self.status = status


_lib = None


def library_path() -> str:
    return os.environ.get("BDIS_LIBRARY") or _build.LIB


def load():
    """Load the in-tree libbdis.so, building it first if it is missing or stale.

    There is no fallback: without the CUDA library nothing here runs."""
    global _lib
    if _lib is not None:
        return _lib
    # BDIS_LIBRARY: a prebuilt library to load instead (the bounds-checked
    # build of the same sources, for tests)
    path = os.environ.get("BDIS_LIBRARY") or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libbdis.so is missing at {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    pp, ip = P(BdisParams), P(BdisImage)
    lib.bdis_default_params.argtypes = [pp]
    lib.bdis_default_params.restype = None
    lib.bdis_status_string.argtypes = [c_int]
    lib.bdis_status_string.restype = ctypes.c_char_p
    lib.bdis_last_error_string.argtypes = []
    lib.bdis_last_error_string.restype = ctypes.c_char_p
    lib.bdis_version.restype = c_int
    lib.bdis_level_dims.argtypes = [c_int, c_int, c_int, P(c_int), P(c_int)]
    lib.bdis_grid.argtypes = [c_int, c_int, c_float, P(c_int), P(c_int)]
    lib.bdis_patch_count.argtypes = [c_int, c_int, pp, P(ctypes.c_int64)]
    lib.bdis_create.argtypes = [P(c_void_p), c_int, c_void_p]
    lib.bdis_reserve.argtypes = [c_void_p, c_int, c_int, c_int, pp]
    lib.bdis_workspace_bytes.argtypes = [c_void_p]
    lib.bdis_workspace_bytes.restype = c_size_t
    lib.bdis_destroy.argtypes = [c_void_p]
    lib.bdis_destroy.restype = None
    lib.bdis_match.argtypes = [c_void_p, ip, ip, pp, c_void_p]
    lib.bdis_match_host.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, pp,
                                    c_void_p]
    lib.bdis_match_host_async.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                          pp, c_void_p, P(ctypes.c_uint64)]
    lib.bdis_host_wait.argtypes = [c_void_p, ctypes.c_uint64]
    lib.bdis_prepare_level0.argtypes = [ip, ip, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.bdis_pyramid_level.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                       c_void_p, c_void_p, c_void_p]
    fp = P(c_float)
    lib.bdis_net_weight_count.restype = c_int
    lib.bdis_proposal_level.argtypes = [c_int]
    lib.bdis_proposal_level.restype = c_int
    lib.bdis_net_create.argtypes = [c_int, c_void_p, P(c_void_p)]
    lib.bdis_net_forward.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                     c_void_p, c_void_p]
    lib.bdis_net_gradient.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                      c_void_p, c_void_p, c_void_p, c_void_p]
    lib.bdis_net_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                        c_void_p, c_float, c_void_p, c_void_p]
    lib.bdis_net_get_weights.argtypes = [c_void_p, c_void_p]
    lib.bdis_net_destroy.argtypes = [c_void_p]
    lib.bdis_net_destroy.restype = None
    del fp
    lib.bdis_match_warm.argtypes = [c_void_p, ip, ip, pp, c_void_p, c_void_p]
    lib.bdis_match_seeded.argtypes = [c_void_p, ip, ip, pp, c_void_p, c_int, c_int, c_void_p]
    lib.bdis_match_learned.argtypes = [c_void_p, c_void_p, ip, ip, pp, c_int, c_void_p]
    lib.bdis_warm_map.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]
    lib.bdis_plan_create.argtypes = [c_int, P(BdisGroup), c_int, pp, c_int, c_void_p,
                                     P(c_void_p)]
    lib.bdis_plan_run.argtypes = [c_void_p, c_void_p]
    lib.bdis_plan_info.argtypes = [c_void_p, c_int, c_int, P(BdisPlanChoice)]
    lib.bdis_plan_workspace_bytes.argtypes = [c_void_p]
    lib.bdis_plan_workspace_bytes.restype = c_size_t
    lib.bdis_plan_destroy.argtypes = [c_void_p]
    lib.bdis_plan_destroy.restype = None
    lib.bdis_set_search_variant.argtypes = [c_int]
    lib.bdis_get_search_variant.restype = c_int
    lib.bdis_set_search_tiling.argtypes = [c_int]
    lib.bdis_set_search_tiling.restype = None
    lib.bdis_get_search_tiling.restype = c_int
    lib.bdis_set_densify_variant.argtypes = [c_int]
    lib.bdis_get_densify_variant.restype = c_int
    lib.bdis_set_pyramid_variant.argtypes = [c_int]
    lib.bdis_set_pyramid_variant.restype = None
    lib.bdis_get_pyramid_variant.restype = c_int
    lib.bdis_set_launch_overlap.argtypes = [c_int]
    lib.bdis_set_launch_overlap.restype = None
    lib.bdis_get_launch_overlap.restype = c_int
    lib.bdis_check_status.argtypes = [P(ctypes.c_uint32)]
    lib.bdis_checked_build.restype = c_int
    lib.bdis_set_net_variant.argtypes = [c_int]
    lib.bdis_set_net_variant.restype = None
    lib.bdis_get_net_variant.restype = c_int
    lib.bdis_probe_fp32_tflops.argtypes = [c_int, P(ctypes.c_double), c_void_p]
    lib.bdis_match_static.argtypes = [ip, ip, pp, c_void_p, c_void_p]
    lib.bdis_pack_right.argtypes = [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]
    lib.bdis_search_level.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                      c_int, c_int, pp, c_void_p, c_void_p,
                                      P(BdisPatchDebug), c_void_p]
    lib.bdis_densify_level.argtypes = [c_int, c_int, c_int, pp, c_void_p, c_void_p, c_void_p,
                                       c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                       c_void_p]
    lib.bdis_upsample.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p,
                                  c_void_p]
    lib.bdis_select_start.argtypes = [c_void_p] * 8 + [ctypes.c_int64, c_void_p]
    lib.bdis_host_wait_timeout.argtypes = [c_void_p, ctypes.c_uint64, ctypes.c_double]
    lib.bdis_inject_alloc_failures.argtypes = [c_int]
    lib.bdis_inject_alloc_failures.restype = None
    lib.bdis_net_status.argtypes = [c_void_p, c_void_p]
    lib.bdis_net_inject_timeout.argtypes = [c_void_p]
    lib.bdis_enable_timing.argtypes = [c_void_p, c_int]
    lib.bdis_read_timing.argtypes = [c_void_p, P(BdisTiming)]
    _lib = lib
    return lib


def check(status: int, what: str):
    if status != BDIS_OK:
        raise BdisError(status, what)
