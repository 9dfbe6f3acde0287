"""ctypes binding of libmaxent_mh.so (include/maxent_mh.h), argument marshalling only.

The library must be built (``paper_2509_13230_gb300.build``); a missing
library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MH_UBCM = 0
MH_UECM = 1

MH_OK = 0
MH_ERR_ARG = -1
MH_ERR_DOMAIN = -2
MH_ERR_CAPACITY = -3
MH_ERR_WORKSPACE = -4
MH_ERR_OVERFLOW = -5
MH_ERR_DEVICE_TIMEOUT = -6
MH_ERR_CUDA = -7

MH_OUT_COO = 0x01
MH_OUT_CSR = 0x02
MH_BOUND_PAPER = 0x10
MH_INIT_PREV = 0x20
MH_DIRECTED = 0x40
MH_CSR_SYMMETRIC = 0x80
MH_FP64_ONLY = 0x100
MH_TIMING = 0x200
MH_TEST_WAIT_TIMEOUT = 0x400
MH_CHUNG_LU = 0x800

MH_STAT_PROPOSALS = 0
MH_STAT_EDGES = 1
MH_STAT_SEGMENTS = 2
MH_STAT_FALLBACKS = 3
MH_STAT_BOUNDARY = 4
MH_NUM_STATS = 5

# Every symbol include/maxent_mh.h declares.
EXPORTED = (
    "mh_error_string",
    "mh_last_error_detail",
    "mh_last_call_info",
    "mh_workspace_size",
    "mh_sample_ubcm",
    "mh_sample_weighted",
    "mh_sample_range",
    "mh_bf_workspace_size",
    "mh_sample_bf",
    "mh_sample_ubcm_noalloc",
    "mh_segment_table",
    "maxent_expected_fwd",
    "maxent_expected_bwd",
    "maxent_expected_fwd_rows",
    "maxent_expected_bwd_rows",
    "maxent_expected_jacobian_diag",
    "maxent_expected_jacobian_diag_rows",
    "maxent_expected_sym_workspace_size",
    "maxent_expected_fwd_sym",
    "maxent_expected_jacobian_diag_sym",
    "maxent_expected_bwd_sym",
    "maxent_expected_jacobian_diag_sym_f32",
    "maxent_expected_bwd_sym_f32",
    "mh_batch_workspace_size",
    "mh_batch_prepare",
    "mh_sample_batched",
    "mh_bipartite_workspace_size",
    "mh_sample_bipartite",
    "mh_debug_first_level",
)


class MhParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("network_id", ctypes.c_uint32),
        ("sample_begin", ctypes.c_uint32),
        ("num_samples", ctypes.c_uint32),
        ("seg_target", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("walk_ctas_per_sm", ctypes.c_uint32),
        ("max_segments", ctypes.c_int64),
    ]


class MhNetworkDesc(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("network_id", ctypes.c_uint32),
        ("n", ctypes.c_int64),
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("max_segments", ctypes.c_int64),
    ]


def network_descs(entries) -> ctypes.Array:
    """Host array of mh_network_desc from (model, network_id, n, x_ptr, y_ptr[, max_segments]) tuples."""
    arr = (MhNetworkDesc * len(entries))()
    for t, e in enumerate(entries):
        model, network_id, n, x, y = e[:5]
        arr[t] = MhNetworkDesc(int(model), int(network_id), int(n), x, y, int(e[5]) if len(e) > 5 else 0)
    return arr


class MhCallInfo(ctypes.Structure):
    _fields_ = [
        ("kernel_launches", ctypes.c_int64),
        ("walk_launches", ctypes.c_int64),
        ("sample_chunks", ctypes.c_int64),
        ("prepare_ms", ctypes.c_double),
        ("walk_ms", ctypes.c_double),
        ("emit_ms", ctypes.c_double),
        ("total_ms", ctypes.c_double),
    ]


class MhError(RuntimeError):
    def __init__(self, code: int, func: str, detail: str):
        super().__init__(f"{func}: {error_string(code)} ({detail})")
        self.code = code


_LOCK = threading.Lock()
_LIB = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the shared library (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None and path is None:
            return _LIB
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -m paper_2509_13230_gb300.build` "
                               "(there is no fallback implementation)")
        lib = ctypes.CDLL(p)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        P = ctypes.POINTER(MhParams)
        lib.mh_error_string.argtypes = [i32]
        lib.mh_error_string.restype = ctypes.c_char_p
        lib.mh_last_error_detail.argtypes = []
        lib.mh_last_error_detail.restype = ctypes.c_char_p
        lib.mh_last_call_info.argtypes = [ctypes.POINTER(MhCallInfo)]
        lib.mh_last_call_info.restype = i32
        lib.mh_workspace_size.argtypes = [i32, i64, P, i64, ctypes.POINTER(sz)]
        lib.mh_workspace_size.restype = i32
        lib.mh_sample_ubcm.argtypes = [vp, i64, P, vp, sz, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.mh_sample_ubcm.restype = i32
        lib.mh_sample_weighted.argtypes = [vp, vp, i64, P, vp, sz, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.mh_sample_weighted.restype = i32
        lib.mh_sample_range.argtypes = [i32, vp, vp, i64, P, i64, i64, vp, sz, vp, vp, vp, i64, vp, vp, vp]
        lib.mh_sample_range.restype = i32
        lib.mh_bf_workspace_size.argtypes = [i32, i64, P, vp]
        lib.mh_bf_workspace_size.restype = i32
        lib.mh_sample_bf.argtypes = [i32, vp, vp, i64, P, vp, sz, vp, vp, vp, i64, vp, vp, vp]
        lib.mh_sample_bf.restype = i32
        lib.mh_sample_ubcm_noalloc.argtypes = [vp, i64, P, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.mh_sample_ubcm_noalloc.restype = i32
        lib.mh_segment_table.argtypes = [i32, vp, vp, i64, P, vp, sz, vp, vp, vp, vp, vp, i64, vp, vp]
        lib.mh_segment_table.restype = i32
        lib.maxent_expected_fwd.argtypes = [i32, vp, vp, i64, vp, vp, vp]
        lib.maxent_expected_fwd.restype = i32
        lib.maxent_expected_bwd.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp, vp]
        lib.maxent_expected_bwd.restype = i32
        lib.maxent_expected_fwd_rows.argtypes = [i32, vp, vp, i64, i64, i64, vp, vp, vp]
        lib.maxent_expected_fwd_rows.restype = i32
        lib.maxent_expected_bwd_rows.argtypes = [i32, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp]
        lib.maxent_expected_bwd_rows.restype = i32
        lib.maxent_expected_jacobian_diag.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp, vp]
        lib.maxent_expected_jacobian_diag.restype = i32
        lib.maxent_expected_jacobian_diag_rows.argtypes = [i32, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp]
        lib.maxent_expected_jacobian_diag_rows.restype = i32
        lib.maxent_expected_sym_workspace_size.argtypes = [i32, i64, ctypes.POINTER(sz)]
        lib.maxent_expected_sym_workspace_size.restype = i32
        lib.maxent_expected_fwd_sym.argtypes = [i32, vp, vp, i64, vp, vp, vp, sz, vp]
        lib.maxent_expected_fwd_sym.restype = i32
        lib.maxent_expected_jacobian_diag_sym.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp, vp, sz, vp]
        lib.maxent_expected_jacobian_diag_sym.restype = i32
        lib.maxent_expected_bwd_sym.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp, vp, sz, vp]
        lib.maxent_expected_bwd_sym.restype = i32
        lib.maxent_expected_jacobian_diag_sym_f32.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp, vp, sz, vp]
        lib.maxent_expected_jacobian_diag_sym_f32.restype = i32
        lib.maxent_expected_bwd_sym_f32.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp, vp, sz, vp]
        lib.maxent_expected_bwd_sym_f32.restype = i32
        lib.mh_debug_first_level.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
        lib.mh_debug_first_level.restype = i32
        lib.mh_bipartite_workspace_size.argtypes = [i32, i64, i64, P, i64, ctypes.POINTER(sz)]
        lib.mh_bipartite_workspace_size.restype = i32
        lib.mh_sample_bipartite.argtypes = [i32, vp, vp, i64, vp, vp, i64, P, vp, sz, vp, vp, vp, vp, vp, vp, i64,
                                            vp, vp, vp]
        lib.mh_sample_bipartite.restype = i32
        D = ctypes.POINTER(MhNetworkDesc)
        lib.mh_batch_workspace_size.argtypes = [D, i32, P, i64, i64, ctypes.POINTER(sz)]
        lib.mh_batch_workspace_size.restype = i32
        lib.mh_batch_prepare.argtypes = [D, i32, P, vp, sz, vp, vp]
        lib.mh_batch_prepare.restype = i32
        lib.mh_sample_batched.argtypes = [D, i32, P, i64, vp, sz, i64, i64, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.mh_sample_batched.restype = i32
        if path is None:
            _LIB = lib
        return lib


def error_string(code: int) -> str:
    return load().mh_error_string(code).decode()


def last_error_detail() -> str:
    return load().mh_last_error_detail().decode()


def check(code: int, func: str) -> int:
    if code != MH_OK:
        raise MhError(code, func, last_error_detail())
    return code


def make_params(*, seed=0, network_id=0, sample_begin=0, num_samples=1, seg_target=0, flags=MH_OUT_COO,
                max_segments=0, walk_ctas_per_sm=0) -> MhParams:
    return MhParams(int(seed) & 0xFFFFFFFFFFFFFFFF, int(network_id), int(sample_begin), int(num_samples),
                    int(seg_target), int(flags), int(walk_ctas_per_sm), int(max_segments))


# ---- same names as the C ABI ------------------------------------------------------
def mh_last_call_info() -> MhCallInfo:
    info = MhCallInfo()
    check(load().mh_last_call_info(ctypes.byref(info)), "mh_last_call_info")
    return info


def mh_workspace_size(model: int, n: int, params: MhParams, capacity_edges: int) -> int:
    out = ctypes.c_size_t(0)
    check(load().mh_workspace_size(model, n, ctypes.byref(params), capacity_edges, ctypes.byref(out)),
          "mh_workspace_size")
    return out.value


def mh_sample_ubcm(x, n, params, workspace, workspace_bytes, src, dst, csr_offsets, csr_indices, capacity_edges,
                   h_edges_per_sample, h_stats, stream) -> int:
    return load().mh_sample_ubcm(x, n, ctypes.byref(params), workspace, workspace_bytes, src, dst, csr_offsets,
                                 csr_indices, capacity_edges, h_edges_per_sample, h_stats, stream)


def mh_sample_weighted(x, y, n, params, workspace, workspace_bytes, src, dst, w, csr_offsets, csr_indices,
                       csr_weights, capacity_edges, h_edges_per_sample, h_stats, stream) -> int:
    return load().mh_sample_weighted(x, y, n, ctypes.byref(params), workspace, workspace_bytes, src, dst, w,
                                     csr_offsets, csr_indices, csr_weights, capacity_edges, h_edges_per_sample,
                                     h_stats, stream)


def mh_sample_range(model, x, y, n, params, seg_begin, seg_end, workspace, workspace_bytes, src, dst, w,
                    capacity_edges, h_edges_per_sample, h_stats, stream) -> int:
    return load().mh_sample_range(model, x, y, n, ctypes.byref(params), seg_begin, seg_end, workspace,
                                  workspace_bytes, src, dst, w, capacity_edges, h_edges_per_sample, h_stats, stream)


def mh_bf_workspace_size(model, n, params) -> int:
    out = ctypes.c_size_t(0)
    check(load().mh_bf_workspace_size(model, n, ctypes.byref(params), ctypes.byref(out)), "mh_bf_workspace_size")
    return out.value


def mh_sample_bf(model, x, y, n, params, workspace, workspace_bytes, src, dst, w, capacity_edges,
                 h_edges_per_sample, h_stats, stream) -> int:
    return load().mh_sample_bf(model, x, y, n, ctypes.byref(params), workspace, workspace_bytes, src, dst, w,
                               capacity_edges, h_edges_per_sample, h_stats, stream)


def mh_sample_ubcm_noalloc(x, n, params, src, dst, csr_offsets, csr_indices, capacity_edges, h_edges_per_sample,
                           h_stats, stream) -> int:
    return load().mh_sample_ubcm_noalloc(x, n, ctypes.byref(params), src, dst, csr_offsets, csr_indices,
                                         capacity_edges, h_edges_per_sample, h_stats, stream)


def mh_segment_table(model, x, y, n, params, workspace, workspace_bytes, seg_row, seg_k, seg_a, seg_b, perm, cap,
                     h_num_segments, stream) -> int:
    return load().mh_segment_table(model, x, y, n, ctypes.byref(params), workspace, workspace_bytes, seg_row,
                                   seg_k, seg_a, seg_b, perm, cap, h_num_segments, stream)


def maxent_expected_fwd(model, x, y, n, k_out, s_out, stream) -> int:
    return load().maxent_expected_fwd(model, x, y, n, k_out, s_out, stream)


def maxent_expected_bwd(model, x, y, n, g_k, g_s, g_x, g_y, stream) -> int:
    return load().maxent_expected_bwd(model, x, y, n, g_k, g_s, g_x, g_y, stream)


def maxent_expected_fwd_rows(model, x, y, n, row_begin, row_count, k_out, s_out, stream) -> int:
    return load().maxent_expected_fwd_rows(model, x, y, n, row_begin, row_count, k_out, s_out, stream)


def maxent_expected_bwd_rows(model, x, y, n, row_begin, row_count, g_k, g_s, g_x, g_y, stream) -> int:
    return load().maxent_expected_bwd_rows(model, x, y, n, row_begin, row_count, g_k, g_s, g_x, g_y, stream)


def mh_batch_workspace_size(h_nets, n_nets, params, max_wave_items, capacity_edges) -> int:
    out = ctypes.c_size_t(0)
    check(load().mh_batch_workspace_size(h_nets, n_nets, ctypes.byref(params), max_wave_items, capacity_edges,
                                         ctypes.byref(out)), "mh_batch_workspace_size")
    return out.value


def mh_batch_prepare(h_nets, n_nets, params, workspace, workspace_bytes, h_num_segments, stream) -> int:
    return load().mh_batch_prepare(h_nets, n_nets, ctypes.byref(params), workspace, workspace_bytes, h_num_segments,
                                   stream)


def mh_sample_batched(h_nets, n_nets, params, max_wave_items, workspace, workspace_bytes, pair_begin, pair_count,
                      src, dst, w, csr_offsets, csr_indices, csr_weights, capacity_edges, h_edges_per_pair, h_stats,
                      stream) -> int:
    return load().mh_sample_batched(h_nets, n_nets, ctypes.byref(params), max_wave_items, workspace,
                                    workspace_bytes, pair_begin, pair_count, src, dst, w, csr_offsets, csr_indices,
                                    csr_weights, capacity_edges, h_edges_per_pair, h_stats, stream)


def mh_bipartite_workspace_size(model, n_plus, n_minus, params, capacity_edges) -> int:
    out = ctypes.c_size_t(0)
    check(load().mh_bipartite_workspace_size(model, n_plus, n_minus, ctypes.byref(params), capacity_edges,
                                             ctypes.byref(out)), "mh_bipartite_workspace_size")
    return out.value


def mh_sample_bipartite(model, x_plus, y_plus, n_plus, x_minus, y_minus, n_minus, params, workspace, workspace_bytes,
                        src, dst, w, csr_offsets, csr_indices, csr_weights, capacity_edges, h_edges_per_sample,
                        h_stats, stream) -> int:
    return load().mh_sample_bipartite(model, x_plus, y_plus, n_plus, x_minus, y_minus, n_minus, ctypes.byref(params),
                                      workspace, workspace_bytes, src, dst, w, csr_offsets, csr_indices, csr_weights,
                                      capacity_edges, h_edges_per_sample, h_stats, stream)


def maxent_expected_jacobian_diag(model, x, y, n, dk_dx, dk_dy, ds_dx, ds_dy, stream) -> int:
    return load().maxent_expected_jacobian_diag(model, x, y, n, dk_dx, dk_dy, ds_dx, ds_dy, stream)


def maxent_expected_jacobian_diag_rows(model, x, y, n, row_begin, row_count, dk_dx, dk_dy, ds_dx, ds_dy,
                                       stream) -> int:
    return load().maxent_expected_jacobian_diag_rows(model, x, y, n, row_begin, row_count, dk_dx, dk_dy, ds_dx,
                                                     ds_dy, stream)


def mh_debug_first_level(N, z, room, n, E_out, lam_out, fl_out, stream) -> int:
    return load().mh_debug_first_level(N, z, room, n, E_out, lam_out, fl_out, stream)


def maxent_expected_sym_workspace_size(model, n) -> tuple[int, int]:
    out = ctypes.c_size_t(0)
    rc = load().maxent_expected_sym_workspace_size(model, n, ctypes.byref(out))
    return rc, int(out.value)


def maxent_expected_fwd_sym(model, x, y, n, k_out, s_out, ws, ws_bytes, stream) -> int:
    return load().maxent_expected_fwd_sym(model, x, y, n, k_out, s_out, ws, ws_bytes, stream)


def maxent_expected_jacobian_diag_sym(model, x, y, n, dk_dx, dk_dy, ds_dx, ds_dy, ws, ws_bytes, stream) -> int:
    return load().maxent_expected_jacobian_diag_sym(model, x, y, n, dk_dx, dk_dy, ds_dx, ds_dy, ws, ws_bytes, stream)


def maxent_expected_bwd_sym(model, x, y, n, g_k, g_s, g_x, g_y, ws, ws_bytes, stream) -> int:
    return load().maxent_expected_bwd_sym(model, x, y, n, g_k, g_s, g_x, g_y, ws, ws_bytes, stream)


def maxent_expected_jacobian_diag_sym_f32(model, x, y, n, dk_dx, dk_dy, ds_dx, ds_dy, ws, ws_bytes, stream) -> int:
    return load().maxent_expected_jacobian_diag_sym_f32(model, x, y, n, dk_dx, dk_dy, ds_dx, ds_dy, ws, ws_bytes,
                                                        stream)


def maxent_expected_bwd_sym_f32(model, x, y, n, g_k, g_s, g_x, g_y, ws, ws_bytes, stream) -> int:
    return load().maxent_expected_bwd_sym_f32(model, x, y, n, g_k, g_s, g_x, g_y, ws, ws_bytes, stream)
