"""ctypes binding of the C ABI in include/skgemm.h -- argument marshalling only.

Every function here has the same name and arguments as its C counterpart and
returns the raw ``sk_status`` integer.  All computation happens in the CUDA
kernels of ``lib/libskgemm.so``; if that library is missing, importing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

# ----------------------------------------------------------------- enums
SK_OK = 0
SK_ERR_INVALID_ARG = 1
SK_ERR_UNSUPPORTED = 2
SK_ERR_WORKSPACE_TOO_SMALL = 3
SK_ERR_TIMEOUT = 4
SK_ERR_CUDA = 5
SK_ERR_NO_DEVICE = 6

SK_F32, SK_BF16, SK_E4M3 = 0, 1, 2
SK_ROW_MAJOR, SK_COL_MAJOR = 0, 1
SK_MODE_AUTO, SK_MODE_DP, SK_MODE_SK, SK_MODE_HYBRID1, SK_MODE_HYBRID2 = 0, 1, 2, 3, 4
SK_ROLE_WHOLE, SK_ROLE_OWNER, SK_ROLE_PEER, SK_ROLE_DP = 0, 1, 2, 3

MODE_NAMES = {"auto": SK_MODE_AUTO, "dp": SK_MODE_DP, "sk": SK_MODE_SK,
              "hybrid1": SK_MODE_HYBRID1, "hybrid2": SK_MODE_HYBRID2}
ROLE_NAMES = {SK_ROLE_WHOLE: "whole", SK_ROLE_OWNER: "owner", SK_ROLE_PEER: "peer", SK_ROLE_DP: "dp"}


class sk_problem(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
        ("a_type", ctypes.c_int), ("b_type", ctypes.c_int), ("c_type", ctypes.c_int),
        ("a_layout", ctypes.c_int), ("b_layout", ctypes.c_int), ("c_layout", ctypes.c_int),
        ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
        ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
        ("C_in", ctypes.c_void_p), ("C", ctypes.c_void_p),
        ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
        ("scale_a", ctypes.c_void_p), ("scale_b", ctypes.c_void_p),
    ]


class sk_config(ctypes.Structure):
    _fields_ = [
        ("tile_m", ctypes.c_int), ("tile_n", ctypes.c_int), ("stages", ctypes.c_int),
        ("mode", ctypes.c_int), ("num_ctas", ctypes.c_int),
        ("min_iters_per_unit", ctypes.c_int), ("timeout_ns", ctypes.c_uint64),
        ("debug_flags", ctypes.c_int), ("trace", ctypes.c_void_p), ("raster_group", ctypes.c_int),
        ("fixup", ctypes.c_int), ("f32_kernel", ctypes.c_int), ("coverage", ctypes.c_void_p),
    ]

SK_F32_AUTO, SK_F32_FFMA, SK_F32_TF32X3 = 0, 1, 2
F32_KERNEL_NAMES = {"auto": SK_F32_AUTO, "ffma": SK_F32_FFMA, "tf32x3": SK_F32_TF32X3}

SK_FIXUP_OWNER, SK_FIXUP_LAST_ARRIVER, SK_FIXUP_SPLIT, SK_FIXUP_SPLIT_CLUSTER = 0, 1, 2, 3
FIXUP_NAMES = {"owner": SK_FIXUP_OWNER, "last_arriver": SK_FIXUP_LAST_ARRIVER, "split": SK_FIXUP_SPLIT,
               "split_cluster": SK_FIXUP_SPLIT_CLUSTER}

SK_TRACE_ENTRIES = 128
SK_TRACE_BYTES_PER_CTA = SK_TRACE_ENTRIES * 16
TRACE_EVENTS = {1: "start", 2: "mma_begin", 4: "mma_end", 5: "epi_begin",
                6: "epi_flags", 7: "epi_end", 8: "end", 9: "entry", 11: "fix_issue", 12: "fix_first_data",
                13: "fix_last_data", 14: "spill_issued", 15: "spill_visible",
                16: "split_summed"}


class sk_plan_info(ctypes.Structure):
    _fields_ = [
        ("tile_m", ctypes.c_int), ("tile_n", ctypes.c_int), ("tile_k", ctypes.c_int),
        ("stages", ctypes.c_int), ("mode", ctypes.c_int), ("num_ctas", ctypes.c_int),
        ("sk_units", ctypes.c_int),
        ("tiles", ctypes.c_int64), ("sk_tiles", ctypes.c_int64), ("dp_tiles", ctypes.c_int64),
        ("sk_iters", ctypes.c_int64), ("iters_per_unit", ctypes.c_int64),
        ("extra_units", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t),
        ("predicted_us", ctypes.c_double), ("fixup", ctypes.c_int),
        ("coverage_words", ctypes.c_int64),
    ]


class sk_work_item(ctypes.Structure):
    _fields_ = [
        ("problem", ctypes.c_int32), ("tile", ctypes.c_int32),
        ("tile_row", ctypes.c_int32), ("tile_col", ctypes.c_int32),
        ("k0", ctypes.c_int32), ("k1", ctypes.c_int32), ("role", ctypes.c_int32),
        ("peer_first", ctypes.c_int32), ("peer_last", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("global_tile", ctypes.c_int64),
    ]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_st = ctypes.c_int

_SIGNATURES = {
    "sk_workspace_size": (_st, [_P(sk_problem), ctypes.c_int, _P(sk_config), _P(ctypes.c_size_t)]),
    "sk_workspace_init": (_st, [_vp, ctypes.c_size_t, _vp]),
    "sk_gemm": (_st, [_P(sk_problem), _P(sk_config), _vp, ctypes.c_size_t, _vp]),
    "sk_gemm_grouped": (_st, [_P(sk_problem), ctypes.c_int, _P(sk_config), _vp, ctypes.c_size_t, _vp]),
    "sk_gemm_backward": (_st, [_P(sk_problem), _vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp,
                               ctypes.c_int64, _P(sk_config), _vp, ctypes.c_size_t, _vp]),
    "sk_gemm_backward_workspace_size": (_st, [_P(sk_problem), ctypes.c_int, ctypes.c_int, _P(sk_config),
                                              _P(ctypes.c_size_t)]),
    "sk_transpose16": (_st, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp, ctypes.c_int64, _vp]),
    "sk_quantize_e4m3": (_st, [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]),
    "sk_get_status": (_st, [_vp, ctypes.c_size_t, _vp, ctypes.c_int, _P(ctypes.c_int)]),
    "sk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sk_plan_query": (_st, [_P(sk_problem), ctypes.c_int, _P(sk_config), ctypes.c_int, _P(sk_plan_info)]),
    "sk_plan_unit_items": (_st, [_P(sk_problem), ctypes.c_int, _P(sk_config), ctypes.c_int, ctypes.c_int,
                                 _P(sk_work_item), ctypes.c_int, _P(ctypes.c_int)]),
    "sk_gemm_static_ws": (_st, [_P(sk_problem), _P(sk_config), _vp]),
    "sk_static_ws_status": (_st, [_vp, ctypes.c_int, _P(ctypes.c_int)]),
    "sk_last_error": (ctypes.c_char_p, []),
    "sk_version": (ctypes.c_char_p, []),
}

LIB_PATH = _build.LIB_PATH
_lib = None


def load(path: str | None = None):
    """Load libskgemm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libskgemm.so not built ({p}); run __graft_entry__.build()")
    L = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


def declared_symbols():
    return list(_SIGNATURES)


# Same-name thin wrappers ---------------------------------------------------

def sk_workspace_size(problems, count, cfg, bytes_out):
    return load().sk_workspace_size(problems, count, cfg, bytes_out)


def sk_workspace_init(ws, ws_bytes, stream):
    return load().sk_workspace_init(ws, ws_bytes, stream)


def sk_gemm(problem, cfg, ws, ws_bytes, stream):
    return load().sk_gemm(problem, cfg, ws, ws_bytes, stream)


def sk_gemm_grouped(problems, count, cfg, ws, ws_bytes, stream):
    return load().sk_gemm_grouped(problems, count, cfg, ws, ws_bytes, stream)


def sk_gemm_backward(fwd, dC, lddc, dA, ldda, dB, lddb, cfg, ws, ws_bytes, stream):
    return load().sk_gemm_backward(fwd, dC, lddc, dA, ldda, dB, lddb, cfg, ws, ws_bytes, stream)


def sk_gemm_backward_workspace_size(fwd, need_dA, need_dB, cfg, bytes_out):
    return load().sk_gemm_backward_workspace_size(fwd, need_dA, need_dB, cfg, bytes_out)


def sk_transpose16(src, rows, cols, ld_src, dst, ld_dst, stream):
    return load().sk_transpose16(src, rows, cols, ld_src, dst, ld_dst, stream)


def sk_quantize_e4m3(x, n, q, scale_out, amax_work, stream):
    return load().sk_quantize_e4m3(x, n, q, scale_out, amax_work, stream)


def sk_get_status(ws, ws_bytes, stream, clear, out):
    return load().sk_get_status(ws, ws_bytes, stream, clear, out)


def sk_status_string(s) -> str:
    return load().sk_status_string(s).decode()


def sk_plan_query(problems, count, cfg, num_sms, out):
    return load().sk_plan_query(problems, count, cfg, num_sms, out)


def sk_plan_unit_items(problems, count, cfg, num_sms, unit, items, max_items, n_out):
    return load().sk_plan_unit_items(problems, count, cfg, num_sms, unit, items, max_items, n_out)


def sk_gemm_static_ws(problem, cfg, stream):
    return load().sk_gemm_static_ws(problem, cfg, stream)


def sk_static_ws_status(stream, clear, out):
    return load().sk_static_ws_status(stream, clear, out)


def sk_last_error() -> str:
    return load().sk_last_error().decode()


def sk_version() -> str:
    return load().sk_version().decode()


class SkError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        detail = sk_last_error()
        super().__init__(f"{where}: {sk_status_string(status)} ({status})" + (f" [{detail}]" if detail else ""))


def check(status: int, where: str = ""):
    if status != SK_OK:
        raise SkError(status, where)
