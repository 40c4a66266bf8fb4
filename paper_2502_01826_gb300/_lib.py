"""ctypes binding of libgsrf.so: the C ABI of include/gsrf.h, name for name.

Argument marshalling only; every step of the render runs in the library's CUDA
kernels.  Loading fails loudly when the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

GSRF_OK, GSRF_ERR_INVALID_ARG, GSRF_ERR_CUDA, GSRF_ERR_CAPACITY = 0, 1, 2, 3
GSRF_ERR_TIMEOUT, GSRF_ERR_NONFINITE, GSRF_ERR_UNSUPPORTED, GSRF_ERR_TOO_LARGE = 4, 5, 6, 7
GSRF_STATIC_SCRATCH_BYTES = 32 << 20
STATUS_NAMES = {0: "GSRF_OK", 1: "GSRF_ERR_INVALID_ARG", 2: "GSRF_ERR_CUDA", 3: "GSRF_ERR_CAPACITY",
                4: "GSRF_ERR_TIMEOUT", 5: "GSRF_ERR_NONFINITE", 6: "GSRF_ERR_UNSUPPORTED",
                7: "GSRF_ERR_TOO_LARGE"}
SIG_COMPLEX_SUM, SIG_RSSI_DB, SIG_POWER_SUM, SIG_SPECTRUM_MAG = 0, 1, 2, 3
VARIANT_RADIANCE_AT_MEAN, VARIANT_NORMALISED_WEIGHT, VARIANT_PAPER_CULLING, VARIANT_PATH_AT_REP = 1, 2, 4, 8
VARIANT_ORDER_T_MID = 16

# every exported symbol of include/gsrf.h
EXPORTS = ["gsrf_workspace_size", "gsrf_workspace_layout", "gsrf_ray_state_bytes", "gsrf_project",
           "gsrf_bin", "gsrf_pair_keys", "gsrf_render_fwd", "gsrf_render_bwd", "gsrf_render", "gsrf_received_signal",
           "gsrf_read_status", "gsrf_render_static", "gsrf_batch_workspace_size", "gsrf_render_batch",
           "gsrf_autotune_workspace_size", "gsrf_autotune", "gsrf_stage_times", "gsrf_version"]
STAGE_PROJECT, STAGE_BIN, STAGE_RENDER_FWD, STAGE_RENDER_BWD, STAGE_BATCH = 0, 1, 2, 3, 4
GSRF_MAX_BATCH_JOBS = 4096
BATCH_JOB_ORDER = 1


class GsrfError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__("%s returned %s" % (fn, STATUS_NAMES.get(code, code)))
        self.code = code


class gsrf_grid(C.Structure):
    _fields_ = [("n_az", C.c_int32), ("n_el", C.c_int32), ("az0_deg", C.c_float), ("daz_deg", C.c_float),
                ("el0_deg", C.c_float), ("del_deg", C.c_float), ("r_rx", C.c_float), ("eps_T", C.c_float),
                ("alpha_max", C.c_float), ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


class gsrf_gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("coeffs", C.c_void_p), ("phase_b", C.c_void_p)]


class gsrf_plan(C.Structure):
    _fields_ = [("n_gauss", C.c_int64), ("n_rx", C.c_int32), ("n_f", C.c_int32), ("f0_hz", C.c_double),
                ("df_hz", C.c_double), ("grid", gsrf_grid), ("pair_capacity", C.c_int64),
                ("ray_block_w", C.c_int32), ("stage", C.c_int32), ("ckpt_every", C.c_int32),
                ("ckpt_slots", C.c_int32), ("variant", C.c_int32), ("fle_degree", C.c_int32)]


class gsrf_layout(C.Structure):
    _fields_ = [("pair_keys", C.c_size_t), ("pair_ids", C.c_size_t), ("rx_pair_base", C.c_size_t),
                ("tile_start", C.c_size_t), ("status", C.c_size_t), ("n_tiles_u", C.c_int32),
                ("n_tiles_v", C.c_int32), ("view", C.c_size_t)]


class gsrf_tune_result(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("ray_block_w", C.c_int32), ("stage", C.c_int32),
                ("project_bin_ms", C.c_float), ("render_ms", C.c_float)]


class gsrf_tune_backward(C.Structure):
    _fields_ = [("ray_state", C.c_void_p), ("grad_rays", C.c_void_p), ("g_means", C.c_void_p),
                ("g_log_scales", C.c_void_p), ("g_quats", C.c_void_p), ("g_opacity_logit", C.c_void_p),
                ("g_coeffs", C.c_void_p), ("g_phase_b", C.c_void_p)]


class gsrf_run_status(C.Structure):
    _fields_ = [("code", C.c_int32), ("first_bad", C.c_int32), ("required_pairs", C.c_int64),
                ("stats", C.c_int64 * 4)]


_lib = None


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = False):
    """Load libgsrf.so.  Raises if it is absent (run __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libgsrf.so not built (%s); call __graft_entry__.build()" % _build.SO)
    L = C.CDLL(_build.SO)
    vp, sz, st = C.c_void_p, C.c_size_t, C.c_int
    P = C.POINTER
    L.gsrf_workspace_size.argtypes = [P(gsrf_plan), P(C.c_size_t)]
    L.gsrf_workspace_layout.argtypes = [P(gsrf_plan), P(gsrf_layout)]
    L.gsrf_ray_state_bytes.argtypes = [P(gsrf_plan)]
    L.gsrf_ray_state_bytes.restype = C.c_size_t
    L.gsrf_project.argtypes = [P(gsrf_plan), P(gsrf_gaussians), vp, vp, vp, sz, vp]
    L.gsrf_bin.argtypes = [P(gsrf_plan), vp, sz, vp]
    L.gsrf_pair_keys.argtypes = [P(gsrf_plan), vp, sz, vp]
    L.gsrf_render_fwd.argtypes = [P(gsrf_plan), P(gsrf_gaussians), vp, sz, vp, vp, vp]
    L.gsrf_render.argtypes = [P(gsrf_plan), P(gsrf_gaussians), vp, vp, vp, sz, vp, vp, vp]
    L.gsrf_render_bwd.argtypes = [P(gsrf_plan), P(gsrf_gaussians), vp, sz, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.gsrf_received_signal.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp]
    L.gsrf_read_status.argtypes = [vp, sz, P(gsrf_run_status), vp]
    L.gsrf_render_static.argtypes = [P(gsrf_plan), P(gsrf_gaussians), vp, vp, vp, P(gsrf_run_status), vp]
    L.gsrf_batch_workspace_size.argtypes = [C.c_int32, P(gsrf_plan), P(C.c_size_t)]
    L.gsrf_render_batch.argtypes = [C.c_int32, P(gsrf_plan), P(vp), P(C.c_size_t), P(vp), vp, sz, vp, C.c_int32, vp]
    L.gsrf_autotune_workspace_size.argtypes = [P(gsrf_plan), P(C.c_size_t)]
    L.gsrf_autotune.argtypes = [P(gsrf_plan), P(gsrf_gaussians), vp, vp, vp, sz, vp, P(gsrf_tune_backward),
                                C.c_int32, P(gsrf_tune_result), C.c_int32, P(C.c_int32), P(gsrf_tune_result), vp]
    L.gsrf_stage_times.argtypes = [vp, P(C.c_float)]
    L.gsrf_version.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("gsrf_ray_state_bytes", "gsrf_version"):
            getattr(L, name).restype = st
    _lib = L
    return L


def check(fn: str, code: int):
    if code != GSRF_OK:
        raise GsrfError(fn, code)


def call(fn: str, *args):
    check(fn, getattr(load(), fn)(*args))
