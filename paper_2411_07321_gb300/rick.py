"""ctypes binding of librick.so -- the C ABI declared in include/rick.h.

Argument marshalling only: every function here forwards to the entry point of
the same name and raises ``RickError`` on a non-zero status.  Pointers are
plain integers (device addresses, e.g. ``tensor.data_ptr()``); streams are
``cudaStream_t`` values as integers (``torch.cuda.current_stream().cuda_stream``).

There is no fallback: if the in-tree librick.so is missing this module raises
on import, naming the build step.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librick.so")

RICK_OK, RICK_EINVAL, RICK_ENOMEM, RICK_ECUDA, RICK_ECUFFT, RICK_ERANGE = 0, -1, -2, -3, -4, -5
RICK_KERNEL_GAUSS, RICK_KERNEL_KB = 0, 1
RICK_PREC_FP32, RICK_PREC_FP32_COMPENSATED = 0, 1
RICK_N_CORRECT, RICK_NORMALIZE, RICK_N_DIVIDE, RICK_PHASE_FP32, RICK_IMAG_PART = 1, 2, 4, 8, 16
RICK_OPT_HERMITIAN_MIRROR, RICK_OPT_DETERMINISTIC = 1, 2
RICK_WAIT_POLLS_DEFAULT = 1 << 24
RICK_WEIGHT_UNIFORM, RICK_WEIGHT_BRIGGS = 1, 2
RICK_MAX_CORR = 4
RICK_GRID_BATCH_MAX = 16
RICK_STREAM_BUFS = 6
(RICK_PROBE_SMEM_RMW, RICK_PROBE_SMEM_ATOMIC_F32, RICK_PROBE_SMEM_ATOMIC_U32,
 RICK_PROBE_SMEM_ATOMIC_U64, RICK_PROBE_FFMA, RICK_PROBE_FFMA2, RICK_PROBE_SHFL,
 RICK_PROBE_F2I) = range(8)


class RickError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn}: {status_string(status)} ({status})")


class rick_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_w", ctypes.c_int32), ("fov", ctypes.c_double),
                ("w_min", ctypes.c_double), ("w_max", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("support", ctypes.c_int32),
                ("kb_beta", ctypes.c_double), ("gauss_sigma", ctypes.c_double),
                ("tile", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("image_n", ctypes.c_int32), ("options", ctypes.c_int32)]


class rick_bin_stats(ctypes.Structure):
    _fields_ = [("n_binned", ctypes.c_int64), ("n_dropped_uv", ctypes.c_int64),
                ("n_dropped_w", ctypes.c_int64), ("sum_weight", ctypes.c_double),
                ("w_min", ctypes.c_double), ("w_max", ctypes.c_double)]


class rick_bin_view(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_size_t), ("perm", ctypes.c_size_t),
                ("rec", ctypes.c_size_t), ("rec_cell", ctypes.c_size_t),
                ("stats", ctypes.c_size_t), ("n_bins", ctypes.c_int64)]


EXPORTS = ["rick_status_string", "rick_plan_create", "rick_plan_destroy", "rick_plan_last_error",
           "rick_plan_launch_count", "rick_plan_set_geometry", "rick_plan_set_kernel",
           "rick_plan_set_image_n", "rick_kb_beta",
           "rick_workspace_bytes", "rick_plan_fft_bytes", "rick_bin_layout", "rick_bin",
           "rick_bin_noalloc", "rick_bin_values", "rick_grid", "rick_grid_accumulate",
           "rick_fft_wplanes", "rick_wcorrect_stack", "rick_wspread", "rick_degrid",
           "rick_stream_bytes", "rick_image_host", "rick_bin_channels",
           "rick_image_host_channels", "rick_density_scratch_bytes", "rick_density_weights",
           "rick_bin_rows", "rick_image_host_rows", "rick_grid_sparse", "rick_fft_wcorrect_bytes",
           "rick_fft_wcorrect", "rick_wspread_fft", "rick_fused_work_bytes",
           "rick_probe_throughput", "rick_plan_set_wait_limit", "rick_plan_set_planes",
           "rick_grid_sparse_batch"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, \
        ctypes.c_size_t
    P = ctypes.POINTER(rick_params)
    L.rick_status_string.restype = ctypes.c_char_p
    L.rick_status_string.argtypes = [i32]
    L.rick_kb_beta.restype = ctypes.c_double
    L.rick_kb_beta.argtypes = [i32, ctypes.c_double]
    for name, args in {
        "rick_plan_create": [P, i64, ctypes.POINTER(vp)],
        "rick_plan_destroy": [vp],
        "rick_plan_last_error": [vp],
        "rick_plan_launch_count": [vp, ctypes.POINTER(ctypes.c_uint64)],
        "rick_plan_set_geometry": [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double],
        "rick_plan_set_kernel": [vp, i32, i32, ctypes.c_double, ctypes.c_double],
        "rick_plan_set_image_n": [vp, i32],
        "rick_workspace_bytes": [P, i64, ctypes.POINTER(sz), ctypes.POINTER(sz)],
        "rick_plan_fft_bytes": [vp, ctypes.POINTER(sz)],
        "rick_bin_layout": [vp, ctypes.POINTER(rick_bin_view)],
        "rick_bin": [vp, i64, vp, vp, vp, vp, sz, vp, vp],
        "rick_bin_noalloc": [vp, i64, vp, vp, vp, vp, sz, vp, vp],
        "rick_bin_values": [vp, vp, vp, vp, vp, vp],
        "rick_grid": [vp, vp, vp, vp],
        "rick_grid_accumulate": [vp, vp, vp, vp],
        "rick_grid_sparse": [vp, vp, vp, vp],
        "rick_grid_sparse_batch": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   i32, vp],
        "rick_fft_wcorrect_bytes": [vp, ctypes.POINTER(sz)],
        "rick_fused_work_bytes": [P, ctypes.POINTER(sz)],
        "rick_fft_wcorrect": [vp, vp, vp, i32, vp, sz, vp, u32, vp],
        "rick_wspread_fft": [vp, vp, vp, vp, sz, vp, u32, vp],
        "rick_stream_bytes": [P, i64, i64, ctypes.POINTER(sz)],
        "rick_image_host": [vp, i64, vp, vp, vp, vp, sz, vp, sz, vp, vp, u32, vp, vp],
        "rick_bin_channels": [vp, i64, i32, vp, vp, vp, vp, vp, sz, vp, vp],
        "rick_bin_rows": [vp, i64, i32, i32, vp, vp, vp, vp, vp, sz, vp, vp],
        "rick_image_host_rows": [vp, i64, i32, i32, vp, vp, vp, vp, vp, sz, vp, sz, vp, vp, u32,
                                 vp, vp],
        "rick_density_scratch_bytes": [P, ctypes.POINTER(sz)],
        "rick_density_weights": [vp, i64, vp, vp, i32, ctypes.c_double, vp, sz, vp, vp],
        "rick_image_host_channels": [vp, i64, i32, vp, vp, vp, vp, vp, sz, vp, sz, vp, vp, u32,
                                     vp, vp],
        "rick_fft_wplanes": [vp, vp, i32, vp],
        "rick_wcorrect_stack": [vp, vp, vp, vp, u32, vp],
        "rick_wspread": [vp, vp, vp, vp, u32, vp],
        "rick_degrid": [vp, vp, vp, vp, vp, vp],
        "rick_probe_throughput": [i32, ctypes.POINTER(ctypes.c_double)],
        "rick_plan_set_wait_limit": [vp, ctypes.c_uint32],
        "rick_plan_set_planes": [vp, i32],
    }.items():
        f = getattr(L, name)
        f.restype = i32
        f.argtypes = args
    return L


_L = _load()


def status_string(s: int) -> str:
    return _L.rick_status_string(int(s)).decode()


def _check(fn: str, s: int) -> None:
    if s != RICK_OK:
        raise RickError(fn, s)


def make_params(n, n_w, fov, kernel=RICK_KERNEL_KB, support=7, w_min=math.nan, w_max=math.nan,
                kb_beta=math.nan, gauss_sigma=math.nan, tile=64,
                precision=RICK_PREC_FP32, image_n=0, options=0) -> rick_params:
    return rick_params(int(n), int(n_w), float(fov), float(w_min), float(w_max), int(kernel),
                       int(support), float(kb_beta), float(gauss_sigma), int(tile),
                       int(precision), int(image_n), int(options))


def rick_plan_create(params: rick_params, max_vis: int) -> int:
    h = ctypes.c_void_p()
    _check("rick_plan_create", _L.rick_plan_create(ctypes.byref(params), int(max_vis),
                                                   ctypes.byref(h)))
    return h.value


def rick_plan_destroy(plan: int) -> None:
    _check("rick_plan_destroy", _L.rick_plan_destroy(plan))


def rick_plan_last_error(plan: int) -> int:
    return int(_L.rick_plan_last_error(plan))


def rick_plan_launch_count(plan: int) -> int:
    c = ctypes.c_uint64()
    _check("rick_plan_launch_count", _L.rick_plan_launch_count(plan, ctypes.byref(c)))
    return c.value


def rick_plan_set_geometry(plan: int, fov: float, w_min: float = math.nan,
                           w_max: float = math.nan) -> None:
    _check("rick_plan_set_geometry", _L.rick_plan_set_geometry(plan, float(fov), float(w_min),
                                                               float(w_max)))


def rick_plan_set_kernel(plan: int, kernel: int, support: int, kb_beta: float = math.nan,
                         gauss_sigma: float = math.nan) -> None:
    _check("rick_plan_set_kernel", _L.rick_plan_set_kernel(plan, int(kernel), int(support),
                                                           float(kb_beta), float(gauss_sigma)))


def rick_plan_set_image_n(plan: int, image_n: int) -> None:
    _check("rick_plan_set_image_n", _L.rick_plan_set_image_n(plan, int(image_n)))


def rick_kb_beta(support: int, alpha: float) -> float:
    return float(_L.rick_kb_beta(int(support), float(alpha)))


def rick_workspace_bytes(params: rick_params, n_vis: int) -> tuple[int, int]:
    b, p = ctypes.c_size_t(), ctypes.c_size_t()
    _check("rick_workspace_bytes", _L.rick_workspace_bytes(ctypes.byref(params), int(n_vis),
                                                           ctypes.byref(b), ctypes.byref(p)))
    return b.value, p.value


def rick_plan_fft_bytes(plan: int) -> int:
    b = ctypes.c_size_t()
    _check("rick_plan_fft_bytes", _L.rick_plan_fft_bytes(plan, ctypes.byref(b)))
    return b.value


def rick_plan_set_planes(plan: int, n_w: int) -> None:
    _check("rick_plan_set_planes", _L.rick_plan_set_planes(plan, int(n_w)))


def rick_plan_set_wait_limit(plan: int, polls: int) -> None:
    _check("rick_plan_set_wait_limit", _L.rick_plan_set_wait_limit(plan, int(polls)))


def rick_probe_throughput(kind: int) -> float:
    """Operations per SM clock of one unit of the current device (RICK_PROBE_*)."""
    v = ctypes.c_double()
    _check("rick_probe_throughput", _L.rick_probe_throughput(int(kind), ctypes.byref(v)))
    return v.value


def rick_bin_layout(plan: int) -> rick_bin_view:
    v = rick_bin_view()
    _check("rick_bin_layout", _L.rick_bin_layout(plan, ctypes.byref(v)))
    return v


def rick_bin(plan, n_vis, uvw, vis, weight, ws, ws_bytes, stats, stream) -> None:
    _check("rick_bin", _L.rick_bin(plan, int(n_vis), uvw, vis, weight or None, ws, int(ws_bytes),
                                   stats or None, stream or None))


def rick_bin_noalloc(plan, n_vis, uvw, vis, weight, ws, ws_bytes, stats, stream) -> None:
    """rick_bin without allocations: temporaries in the library's fixed array
    (n_vis <= 262144, at most 131072 bins)."""
    _check("rick_bin_noalloc", _L.rick_bin_noalloc(plan, int(n_vis), uvw, vis, weight or None, ws,
                                                   int(ws_bytes), stats or None, stream or None))


def rick_bin_channels(plan, n_rows, n_chan, uvw_rows, chan_scale, vis, weight, ws, ws_bytes, stats,
                      stream) -> None:
    """rick_bin for rows of n_chan channels with per-row uvw and per-channel factors."""
    _check("rick_bin_channels", _L.rick_bin_channels(plan, int(n_rows), int(n_chan), uvw_rows,
                                                     chan_scale, vis, weight or None, ws,
                                                     int(ws_bytes), stats or None, stream or None))


def rick_image_host_channels(plan, n_rows, n_chan, uvw_rows_host, chan_scale_host, vis_host,
                             weight_host, ws, ws_bytes, stage, stage_bytes, planes, image, flags,
                             stats, stream) -> None:
    """Streamed imaging of multi-channel rows held in host memory."""
    _check("rick_image_host_channels", _L.rick_image_host_channels(
        plan, int(n_rows), int(n_chan), uvw_rows_host, chan_scale_host, vis_host,
        weight_host or None, ws, int(ws_bytes), stage, int(stage_bytes), planes, image, int(flags),
        stats or None, stream or None))


def rick_bin_rows(plan, n_rows, n_chan, n_corr, uvw_rows, chan_scale, vis, weight, ws, ws_bytes,
                  stats, stream) -> None:
    """rick_bin_channels with n_corr correlations per visibility, folded into one record."""
    _check("rick_bin_rows", _L.rick_bin_rows(plan, int(n_rows), int(n_chan), int(n_corr), uvw_rows,
                                             chan_scale, vis, weight or None, ws, int(ws_bytes),
                                             stats or None, stream or None))


def rick_image_host_rows(plan, n_rows, n_chan, n_corr, uvw_rows_host, chan_scale_host, vis_host,
                         weight_host, ws, ws_bytes, stage, stage_bytes, planes, image, flags,
                         stats, stream) -> None:
    """Streamed imaging of rows of channels with n_corr correlations, in host memory."""
    _check("rick_image_host_rows", _L.rick_image_host_rows(
        plan, int(n_rows), int(n_chan), int(n_corr), uvw_rows_host, chan_scale_host, vis_host,
        weight_host or None, ws, int(ws_bytes), stage, int(stage_bytes), planes, image, int(flags),
        stats or None, stream or None))


def rick_density_scratch_bytes(params: rick_params) -> int:
    b = ctypes.c_size_t()
    _check("rick_density_scratch_bytes", _L.rick_density_scratch_bytes(ctypes.byref(params),
                                                                       ctypes.byref(b)))
    return b.value


def rick_density_weights(plan, n_vis, weight, ws, scheme, robust, scratch, scratch_bytes,
                         weight_out, stream) -> None:
    """Uniform / Briggs imaging weights from the uv-cell density of the last binning."""
    _check("rick_density_weights", _L.rick_density_weights(plan, int(n_vis), weight or None, ws,
                                                           int(scheme), float(robust), scratch,
                                                           int(scratch_bytes), weight_out,
                                                           stream or None))


def rick_bin_values(plan, vis, weight, ws, stats, stream) -> None:
    _check("rick_bin_values", _L.rick_bin_values(plan, vis, weight or None, ws, stats or None,
                                                 stream or None))


def rick_grid(plan, ws, planes, stream) -> None:
    _check("rick_grid", _L.rick_grid(plan, ws, planes, stream or None))


def rick_grid_accumulate(plan, ws, planes, stream) -> None:
    _check("rick_grid_accumulate", _L.rick_grid_accumulate(plan, ws, planes, stream or None))


def rick_grid_sparse(plan, ws, planes, stream) -> None:
    _check("rick_grid_sparse", _L.rick_grid_sparse(plan, ws, planes, stream or None))


def rick_grid_sparse_batch(plans, ws, planes, stream) -> None:
    """One gridding launch for several jobs: plans, ws and planes are equal-length
    sequences of plan handles and device pointers (at most RICK_GRID_BATCH_MAX)."""
    n = len(plans)
    if len(ws) != n or len(planes) != n:
        raise ValueError("plans, ws and planes must have the same length")
    arr = ctypes.c_void_p * max(n, 1)
    _check("rick_grid_sparse_batch",
           _L.rick_grid_sparse_batch(arr(*plans), arr(*ws), arr(*planes), n, stream or None))


def rick_fft_wcorrect_bytes(plan) -> int | None:
    """Work bytes of rick_fft_wcorrect, or None where the plan's n is outside
    the sizes the fused transform covers."""
    b = ctypes.c_size_t()
    s = _L.rick_fft_wcorrect_bytes(plan, ctypes.byref(b))
    if s == RICK_EINVAL:
        return None
    _check("rick_fft_wcorrect_bytes", s)
    return b.value


def rick_fused_work_bytes(params: rick_params) -> int:
    """Work bytes of the fused transform for plans of these parameters (0 where
    it does not cover n); host-only."""
    b = ctypes.c_size_t()
    _check("rick_fused_work_bytes", _L.rick_fused_work_bytes(ctypes.byref(params),
                                                             ctypes.byref(b)))
    return b.value


def rick_fft_wcorrect(plan, planes, ws, sparse, work, work_bytes, image, flags, stream) -> None:
    _check("rick_fft_wcorrect", _L.rick_fft_wcorrect(plan, planes, ws, int(sparse), work,
                                                     int(work_bytes), image, int(flags),
                                                     stream or None))


def rick_wspread_fft(plan, image, ws, work, work_bytes, planes, flags, stream) -> None:
    _check("rick_wspread_fft", _L.rick_wspread_fft(plan, image, ws, work, int(work_bytes), planes,
                                                   int(flags), stream or None))


def rick_stream_bytes(params: rick_params, max_vis: int, n_vis: int) -> int:
    b = ctypes.c_size_t()
    _check("rick_stream_bytes", _L.rick_stream_bytes(ctypes.byref(params), int(max_vis),
                                                     int(n_vis), ctypes.byref(b)))
    return b.value


def rick_image_host(plan, n_vis, uvw_host, vis_host, weight_host, ws, ws_bytes, stage,
                    stage_bytes, planes, image, flags, stats, stream) -> None:
    """Streamed imaging from host arrays (host addresses for the inputs)."""
    _check("rick_image_host", _L.rick_image_host(plan, int(n_vis), uvw_host, vis_host,
                                                 weight_host or None, ws, int(ws_bytes), stage,
                                                 int(stage_bytes), planes, image, int(flags),
                                                 stats or None, stream or None))


def rick_fft_wplanes(plan, planes, direction, stream) -> None:
    _check("rick_fft_wplanes", _L.rick_fft_wplanes(plan, planes, int(direction), stream or None))


def rick_wcorrect_stack(plan, planes, ws, image, flags, stream) -> None:
    _check("rick_wcorrect_stack", _L.rick_wcorrect_stack(plan, planes, ws, image, int(flags),
                                                         stream or None))


def rick_wspread(plan, image, ws, planes, flags, stream) -> None:
    _check("rick_wspread", _L.rick_wspread(plan, image, ws, planes, int(flags), stream or None))


def rick_degrid(plan, ws, planes, weight, vis_out, stream) -> None:
    _check("rick_degrid", _L.rick_degrid(plan, ws, planes, weight or None, vis_out,
                                         stream or None))
