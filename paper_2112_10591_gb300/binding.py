"""Thin Python binding of libebof.so (include/ebof.h), by ctypes.

The functions carry the C names and only marshal arguments: torch tensors
become device pointers, the current torch CUDA stream becomes the
``cuda_stream`` argument, and status codes come back as ints (negative =
error).  Every step of the path runs in the library's CUDA kernels; if the
library is missing, ``load()`` raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

EBOF_OK = 0
EBOF_NO_PREVIOUS = 1
EBOF_ERR_INVALID_ARG = -1
EBOF_ERR_OOM = -2
EBOF_ERR_CUDA = -3
EBOF_ERR_TIMEOUT = -4
EBOF_ERR_DEVICE_BOUNDS = -5
EBOF_ERR_UNSUPPORTED = -6
EBOF_ERR_BUSY = -7
EBOF_QUEUED = 2
EBOF_ERR_CANCELLED = -8


class ebof_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("connectivity", ctypes.c_int32),
        ("n_d", ctypes.c_int32), ("n_f", ctypes.c_int32),
        ("alpha", ctypes.c_float),
        ("levels", ctypes.c_int32), ("patch", ctypes.c_int32),
        ("stride", ctypes.c_int32), ("gn_iters", ctypes.c_int32),
        ("gn_damping", ctypes.c_float),
        ("var_outer", ctypes.c_int32), ("var_sor", ctypes.c_int32),
        ("var_delta", ctypes.c_float), ("var_gamma", ctypes.c_float),
        ("var_alpha", ctypes.c_float), ("sor_omega", ctypes.c_float),
        ("max_batch", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("surface", ctypes.c_int32),
        ("d_sat", ctypes.c_float),
        ("coeff_cw_min_width", ctypes.c_int32),
        ("sor_tma_min_per_sm", ctypes.c_int32),
        ("sor_row_waves", ctypes.c_int32),
        ("var_cluster_max", ctypes.c_int32),
        ("coeff_cw_rows", ctypes.c_int32),
    ]


EBOF_STORAGE_FP32 = 0
EBOF_STORAGE_FP16 = 1
EBOF_SURFACE_EXP, EBOF_SURFACE_LINEAR, EBOF_SURFACE_BOUNDED, EBOF_SURFACE_LOG = 0, 1, 2, 3


class ebof_window_stats(ctypes.Structure):
    _fields_ = [
        ("events", ctypes.c_int64), ("in_window", ctypes.c_int64),
        ("dropped_time", ctypes.c_int64), ("dropped_oob", ctypes.c_int64),
        ("edge_px", ctypes.c_int64), ("levels_used", ctypes.c_int32),
        ("has_flow", ctypes.c_int32),
    ]


class ebof_window_desc(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("t", ctypes.c_void_p),
        ("n_events", ctypes.c_int64), ("t_begin", ctypes.c_int64), ("t_end", ctypes.c_int64),
    ]


class ebof_server_config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("device", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("n_workers", ctypes.c_int32)]


class ebof_completion(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int32), ("status", ctypes.c_int32),
                ("tag", ctypes.c_uint64), ("arrival_ns", ctypes.c_int64),
                ("launch_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("batch", ctypes.c_int32), ("index", ctypes.c_int32)]


class ebof_server_info(ctypes.Structure):
    _fields_ = [("streams_admitted", ctypes.c_int32), ("streams_waiting", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("memory_in_use", ctypes.c_int64),
                ("windows_submitted", ctypes.c_int64), ("windows_completed", ctypes.c_int64),
                ("batches_launched", ctypes.c_int64), ("batches_in_flight", ctypes.c_int32),
                ("max_batch_seen", ctypes.c_int32)]


class EbofError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__("%s: %s (%d)" % (what or "ebof", ebof_status_string(status), status))
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libebof.so; build it first if it is missing and a toolkit exists."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or not _build.up_to_date():
                if not build_if_missing:
                    raise ImportError("libebof.so is not built (%s)" % path)
                _build.build()
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def _declare(L):
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    P = ctypes.POINTER
    L.ebof_default_params.argtypes = [P(ebof_params), i32, i32]
    L.ebof_default_params.restype = None
    L.ebof_alpha_from_dsat.argtypes = [f32]
    L.ebof_alpha_from_dsat.restype = f32
    L.ebof_stream_create.argtypes = [P(ebof_params), ctypes.c_int, P(vp)]
    L.ebof_stream_destroy.argtypes = [vp]
    L.ebof_stream_device_bytes.argtypes = [P(ebof_params)]
    L.ebof_stream_device_bytes.restype = ctypes.c_int64
    L.ebof_stream_reset.argtypes = [vp]
    L.ebof_process_window.argtypes = [vp, vp, vp, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp]
    L.ebof_process_windows.argtypes = [vp, i32, vp, vp, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp]
    L.ebof_process_surface.argtypes = [vp, vp, vp, vp]
    L.ebof_stream_get_pyramid.argtypes = [vp, i32, vp, vp, vp, vp]
    L.ebof_process_window_list.argtypes = [vp, i32, P(ebof_window_desc), P(vp), vp]
    L.ebof_fwl_scratch_bytes.argtypes = [i32, i32]
    L.ebof_fwl_scratch_bytes.restype = ctypes.c_size_t
    L.ebof_fwl.argtypes = [vp, vp, vp, vp, i64, i64, i64, vp, i32, i32, vp, vp, vp]
    L.ebof_now_ns.argtypes = []
    L.ebof_now_ns.restype = i64
    L.ebof_server_default_config.argtypes = [P(ebof_server_config)]
    L.ebof_server_default_config.restype = None
    L.ebof_server_create.argtypes = [P(ebof_server_config), P(vp)]
    L.ebof_server_destroy.argtypes = [vp]
    L.ebof_server_open_stream.argtypes = [vp, P(ebof_params), P(i32)]
    L.ebof_server_close_stream.argtypes = [vp, i32]
    L.ebof_server_submit.argtypes = [vp, i32, P(ebof_window_desc), vp, ctypes.c_uint64, i64]
    L.ebof_server_poll.argtypes = [vp, P(ebof_completion), i32, i32]
    L.ebof_server_drain.argtypes = [vp, i32]
    L.ebof_server_get_info.argtypes = [vp, P(ebof_server_info)]
    L.ebof_process_window_host.argtypes = [vp, vp, vp, vp, i64, i64, i64, vp, vp]
    L.ebof_process_window_host_async.argtypes = [vp, vp, vp, vp, i64, i64, i64, vp, vp]
    L.ebof_process_window_async.argtypes = [vp, vp, vp, vp, vp, i64, i64, i64, vp, vp]
    L.ebof_stream_join.argtypes = [vp, vp]
    L.ebof_stream_sync.argtypes = [vp, P(ebof_window_stats), i32]
    L.ebof_edt.argtypes = [vp, i32, i32, vp, vp, vp, f32, vp]
    L.ebof_edt_static.argtypes = [vp, i32, i32, vp, vp, f32, vp]
    L.ebof_group_create.argtypes = [P(ebof_params), i32, ctypes.c_int, P(vp)]
    L.ebof_group_destroy.argtypes = [vp]
    L.ebof_group_reset.argtypes = [vp]
    L.ebof_group_process.argtypes = [vp, P(ebof_window_desc), vp, vp]
    L.ebof_group_flow.argtypes = [vp, i32]
    L.ebof_group_flow.restype = vp
    L.ebof_group_sync.argtypes = [vp, P(ebof_window_stats), i32]
    L.ebof_multigroup_create.argtypes = [P(vp), i32, P(vp)]
    L.ebof_multigroup_destroy.argtypes = [vp]
    L.ebof_multigroup_process.argtypes = [vp, P(P(ebof_window_desc)), vp]
    L.ebof_multigroup_set_fused.argtypes = [vp, i32]
    L.ebof_stream_set_profiling.argtypes = [vp, i32]
    L.ebof_stream_get_profile.argtypes = [vp, P(ctypes.c_double), P(i64), i32]
    L.ebof_stream_get_profile_level.argtypes = [vp, i32, P(ctypes.c_double), P(i64), i32]
    L.ebof_stage_name.argtypes = [i32]
    L.ebof_stage_name.restype = ctypes.c_char_p
    L.ebof_kernel_launches.argtypes = []
    L.ebof_kernel_launches.restype = ctypes.c_uint64
    L.ebof_status_string.argtypes = [ctypes.c_int]
    L.ebof_status_string.restype = ctypes.c_char_p
    L.ebof_stream_set_wait_limit.argtypes = [vp, i64]
    L.ebof_debug_fail_allocation.argtypes = [i32]
    L.ebof_debug_fail_allocation.restype = None
    for name in ("ebof_stream_create", "ebof_stream_destroy", "ebof_stream_reset",
                 "ebof_process_window", "ebof_process_windows", "ebof_process_surface",
                 "ebof_stream_get_pyramid",
                 "ebof_process_window_host", "ebof_process_window_host_async",
                 "ebof_process_window_async", "ebof_stream_join",
                 "ebof_stream_sync", "ebof_edt",
                 "ebof_stream_set_profiling", "ebof_stream_get_profile", "ebof_edt_static",
                 "ebof_stream_get_profile_level", "ebof_group_create", "ebof_group_destroy",
                 "ebof_group_reset", "ebof_group_process", "ebof_group_sync",
                 "ebof_process_window_list", "ebof_server_create", "ebof_fwl", "ebof_server_destroy",
                 "ebof_server_open_stream", "ebof_server_close_stream", "ebof_server_submit",
                 "ebof_server_poll", "ebof_server_drain", "ebof_server_get_info",
                 "ebof_stream_set_wait_limit", "ebof_multigroup_create",
                 "ebof_multigroup_destroy", "ebof_multigroup_process",
                 "ebof_multigroup_set_fused"):
        getattr(L, name).restype = ctypes.c_int


# ---------------------------------------------------------------- marshalling
def _ptr(t, dtype=None, numel=None, name="tensor", device=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if device is not None and t.device.index != device:
        raise ValueError("%s is on cuda:%d, the stream is on cuda:%d" % (name, t.device.index, device))
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() < numel:
        raise ValueError("%s needs at least %d elements, has %d" % (name, numel, t.numel()))
    return t.data_ptr()


def _hptr(a, dtype, numel=None, name="array"):
    """Host pointer of a contiguous numpy array or CPU tensor."""
    import numpy as np
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                raise ValueError("%s must be in host memory" % name)
            a = a.numpy()
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError("%s must be a C-contiguous %s array" % (name, np.dtype(dtype)))
    if numel is not None and a.size < numel:
        raise ValueError("%s needs at least %d elements" % (name, numel))
    return a.ctypes.data


def _stream_handle(cuda_stream):
    if cuda_stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(cuda_stream, int):
        return cuda_stream
    return cuda_stream.cuda_stream


# ---------------------------------------------------------------- C names
def ebof_default_params(width: int, height: int) -> ebof_params:
    p = ebof_params()
    load().ebof_default_params(ctypes.byref(p), int(width), int(height))
    return p


def ebof_alpha_from_dsat(d_sat: float) -> float:
    return float(load().ebof_alpha_from_dsat(float(d_sat)))


def ebof_status_string(status: int) -> str:
    return load().ebof_status_string(int(status)).decode()


class Stream:
    """Owner of an ``ebof_stream*`` handle (destroyed on close / GC)."""

    def __init__(self, handle: int, params: ebof_params, device: int):
        self.handle = handle
        self.params = params
        self.device = device

    def close(self):
        if self.handle:
            load().ebof_stream_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ebof_stream_create(params: ebof_params, device: int = 0):
    """Returns (status, Stream or None)."""
    h = ctypes.c_void_p()
    st = load().ebof_stream_create(ctypes.byref(params), int(device), ctypes.byref(h))
    if st < 0:
        return st, None
    p = ebof_params()
    ctypes.memmove(ctypes.byref(p), ctypes.byref(params), ctypes.sizeof(p))
    return st, Stream(h.value, p, int(device))


def ebof_stream_device_bytes(params: ebof_params) -> int:
    return int(load().ebof_stream_device_bytes(ctypes.byref(params)))


def ebof_stream_destroy(stream: Stream) -> int:
    stream.close()
    return EBOF_OK


def ebof_stream_reset(stream: Stream) -> int:
    return load().ebof_stream_reset(stream.handle)


def ebof_process_window(stream: Stream, x, y, t, p, t_begin: int, t_end: int, flow,
                        edge=None, edt=None, surface=None, cuda_stream=None) -> int:
    import torch
    W, H, dev = stream.params.width, stream.params.height, stream.device
    n = 0 if x is None else x.numel()
    return load().ebof_process_window(
        stream.handle, _ptr(x, torch.uint16, n, "x", dev), _ptr(y, torch.uint16, n, "y", dev),
        _ptr(t, torch.int64, n, "t", dev), _ptr(p, torch.int8, n, "p", dev), n, int(t_begin),
        int(t_end), _ptr(flow, torch.float32, 2 * W * H, "flow", dev),
        _ptr(edge, torch.uint8, W * H, "edge", dev), _ptr(edt, torch.int32, W * H, "edt", dev),
        _ptr(surface, torch.float32, W * H, "surface", dev), _stream_handle(cuda_stream))


def ebof_process_window_async(stream: Stream, x, y, t, p, t_begin: int, t_end: int, flow,
                              cuda_stream=None) -> int:
    """Pipelined window: returns after enqueueing; the flow is in `flow` (and
    the event tensors may be reused) once ebof_stream_sync returns."""
    import torch
    W, H, dev = stream.params.width, stream.params.height, stream.device
    n = 0 if x is None else x.numel()
    return load().ebof_process_window_async(
        stream.handle, _ptr(x, torch.uint16, n, "x", dev), _ptr(y, torch.uint16, n, "y", dev),
        _ptr(t, torch.int64, n, "t", dev), _ptr(p, torch.int8, n, "p", dev), n, int(t_begin),
        int(t_end), _ptr(flow, torch.float32, 2 * W * H, "flow", dev),
        _stream_handle(cuda_stream))


def ebof_process_windows(stream: Stream, n_windows: int, x, y, t, p, t_begin: int, dt: int,
                         flow, edge=None, edt=None, surface=None, cuda_stream=None) -> int:
    import torch
    W, H, dev = stream.params.width, stream.params.height, stream.device
    n = 0 if x is None else x.numel()
    k = int(n_windows)
    return load().ebof_process_windows(
        stream.handle, k, _ptr(x, torch.uint16, n, "x", dev), _ptr(y, torch.uint16, n, "y", dev),
        _ptr(t, torch.int64, n, "t", dev), _ptr(p, torch.int8, n, "p", dev), n, int(t_begin),
        int(dt), _ptr(flow, torch.float32, k * 2 * W * H, "flow", dev),
        _ptr(edge, torch.uint8, k * W * H, "edge", dev),
        _ptr(edt, torch.int32, k * W * H, "edt", dev),
        _ptr(surface, torch.float32, k * W * H, "surface", dev), _stream_handle(cuda_stream))


def _window_desc(w, device, out=None):
    """(x, y, t, t_begin, t_end) of CUDA tensors and ints -> ebof_window_desc."""
    import torch
    x, y, t, tb, te = w
    n = x.numel()
    d = ebof_window_desc() if out is None else out
    d.x = _ptr(x, torch.uint16, n, "x", device)
    d.y = _ptr(y, torch.uint16, n, "y", device)
    d.t = _ptr(t, torch.int64, n, "t", device)
    d.n_events = n
    d.t_begin = int(tb)
    d.t_end = int(te)
    return d


def ebof_process_window_list(stream: Stream, windows, flows, cuda_stream=None) -> int:
    """windows: n tuples (x, y, t, t_begin, t_end); flows: n CUDA float32
    tensors of [2][H][W] elements each."""
    import torch
    n = len(windows)
    if len(flows) != n:
        raise ValueError("need one flow buffer per window")
    arr = (ebof_window_desc * max(n, 1))()
    dst = (ctypes.c_void_p * max(n, 1))()
    W, H = stream.params.width, stream.params.height
    for k in range(n):
        _window_desc(windows[k], stream.device, arr[k])
        dst[k] = _ptr(flows[k], torch.float32, 2 * W * H, "flow", stream.device)
    return load().ebof_process_window_list(stream.handle, n, arr, dst,
                                           _stream_handle(cuda_stream))


def ebof_process_surface(stream: Stream, surface, flow, cuda_stream=None) -> int:
    import torch
    W, H, dev = stream.params.width, stream.params.height, stream.device
    return load().ebof_process_surface(
        stream.handle, _ptr(surface, torch.float32, W * H, "surface", dev),
        _ptr(flow, torch.float32, 2 * W * H, "flow", dev), _stream_handle(cuda_stream))


def ebof_stream_get_pyramid(stream: Stream, level: int, I=None, Ix=None, Iy=None,
                            cuda_stream=None) -> int:
    """Level `level` of the newest window's pyramid into dense float32 CUDA
    tensors of (H >> level) x (W >> level) elements (any may be None)."""
    import torch
    lv = max(int(level), 0)  # the library refuses a level outside the pyramid
    W, H, dev = stream.params.width >> lv, stream.params.height >> lv, stream.device
    return load().ebof_stream_get_pyramid(
        stream.handle, int(level), _ptr(I, torch.float32, W * H, "I", dev),
        _ptr(Ix, torch.float32, W * H, "Ix", dev), _ptr(Iy, torch.float32, W * H, "Iy", dev),
        _stream_handle(cuda_stream))


def ebof_process_window_host(stream: Stream, x, y, t, t_begin: int, t_end: int, flow,
                             cuda_stream=None) -> int:
    import numpy as np
    W, H = stream.params.width, stream.params.height
    n = len(x)
    return load().ebof_process_window_host(
        stream.handle, _hptr(x, np.uint16, n, "x"), _hptr(y, np.uint16, n, "y"),
        _hptr(t, np.int64, n, "t"), n, int(t_begin), int(t_end),
        _hptr(flow, np.float32, 2 * W * H, "flow"), _stream_handle(cuda_stream))


def ebof_process_window_host_async(stream: Stream, x, y, t, t_begin: int, t_end: int, flow,
                                   cuda_stream=None) -> int:
    """As ebof_process_window_async with host buffers: returns before the
    work completes when every buffer is page-locked (the buffers must then
    stay alive until ebof_stream_sync)."""
    import numpy as np
    W, H = stream.params.width, stream.params.height
    n = len(x)
    return load().ebof_process_window_host_async(
        stream.handle, _hptr(x, np.uint16, n, "x"), _hptr(y, np.uint16, n, "y"),
        _hptr(t, np.int64, n, "t"), n, int(t_begin), int(t_end),
        _hptr(flow, np.float32, 2 * W * H, "flow"), _stream_handle(cuda_stream))


def ebof_stream_join(stream: Stream, cuda_stream=None) -> int:
    """Makes later work on cuda_stream wait for all of the stream's work."""
    return load().ebof_stream_join(stream.handle, _stream_handle(cuda_stream))


def ebof_stream_sync(stream: Stream, n_out: int = 1):
    """Returns (status, [ebof_window_stats] * n_out)."""
    arr = (ebof_window_stats * max(1, n_out))()
    st = load().ebof_stream_sync(stream.handle, arr, int(n_out))
    return st, [arr[i] for i in range(n_out)]


def ebof_edt(edge, width: int, height: int, scratch, edt, surface=None, alpha: float = 1.08,
             cuda_stream=None) -> int:
    import torch
    n = int(width) * int(height)
    return load().ebof_edt(_ptr(edge, torch.uint8, n, "edge"), int(width), int(height),
                           _ptr(scratch, torch.int32, n, "scratch"),
                           _ptr(edt, torch.int32, n, "edt"),
                           _ptr(surface, torch.float32, n, "surface"), float(alpha),
                           _stream_handle(cuda_stream))


def ebof_edt_static(edge, width: int, height: int, edt, surface=None, alpha: float = 1.08,
                    cuda_stream=None) -> int:
    """ebof_edt with the library's static scratch: for callers that cannot
    allocate device memory (width * height <= 2**21)."""
    import torch
    n = int(width) * int(height)
    return load().ebof_edt_static(_ptr(edge, torch.uint8, n, "edge"), int(width), int(height),
                                  _ptr(edt, torch.int32, n, "edt"),
                                  _ptr(surface, torch.float32, n, "surface"), float(alpha),
                                  _stream_handle(cuda_stream))


class Group:
    """Owner of an ``ebof_group*`` handle (n streams of one resolution)."""

    def __init__(self, handle: int, params: ebof_params, n: int, device: int):
        self.handle = handle
        self.params = params
        self.n = n
        self.device = device

    def close(self):
        if self.handle:
            load().ebof_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ebof_group_create(params: ebof_params, n_streams: int, device: int = 0):
    """Returns (status, Group or None)."""
    h = ctypes.c_void_p()
    st = load().ebof_group_create(ctypes.byref(params), int(n_streams), int(device),
                                  ctypes.byref(h))
    if st < 0:
        return st, None
    p = ebof_params()
    ctypes.memmove(ctypes.byref(p), ctypes.byref(params), ctypes.sizeof(p))
    return st, Group(h.value, p, int(n_streams), int(device))


def ebof_group_reset(group: Group) -> int:
    return load().ebof_group_reset(group.handle)


def ebof_group_process(group: Group, windows, flow=None, cuda_stream=None) -> int:
    """windows: n tuples (x, y, t, t_begin, t_end) of CUDA tensors and ints."""
    import torch
    if len(windows) != group.n:
        raise ValueError("need %d windows, got %d" % (group.n, len(windows)))
    arr = (ebof_window_desc * group.n)()
    for k in range(group.n):
        _window_desc(windows[k], group.device, arr[k])
    W, H = group.params.width, group.params.height
    fp = _ptr(flow, torch.float32, group.n * 2 * W * H, "flow", group.device)
    return load().ebof_group_process(group.handle, arr, fp, _stream_handle(cuda_stream))


def ebof_group_flow(group: Group, k: int) -> int:
    """Device address of stream k's flow of the last step ([2][H][W] float32)."""
    return int(load().ebof_group_flow(group.handle, int(k)) or 0)


def ebof_group_sync(group: Group, n_out: int = None):
    n_out = group.n if n_out is None else n_out
    arr = (ebof_window_stats * max(1, n_out))()
    st = load().ebof_group_sync(group.handle, arr, int(n_out))
    return st, [arr[i] for i in range(n_out)]


class MultiGroup:
    """Owner of an ``ebof_multigroup*`` handle: groups of several resolutions
    stepped as one CUDA graph.  Keeps its groups referenced."""

    def __init__(self, handle: int, groups):
        self.handle = handle
        self.groups = list(groups)

    def close(self):
        if self.handle:
            load().ebof_multigroup_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ebof_multigroup_create(groups):
    """Returns (status, MultiGroup or None)."""
    arr = (ctypes.c_void_p * len(groups))(*[g.handle for g in groups])
    h = ctypes.c_void_p()
    st = load().ebof_multigroup_create(arr, len(groups), ctypes.byref(h))
    if st < 0:
        return st, None
    return st, MultiGroup(h.value, groups)


def ebof_multigroup_set_fused(mg: MultiGroup, fused) -> int:
    """0 / False: one launch per stage and group; 1 / True: every stage one
    launch for all groups; 2: the front-end stages fused, the flow levels as
    per-group branches."""
    return load().ebof_multigroup_set_fused(mg.handle, int(fused))


def ebof_multigroup_process(mg: MultiGroup, windows, cuda_stream=None) -> int:
    """windows[i]: groups[i].n tuples (x, y, t, t_begin, t_end) of CUDA tensors
    and ints."""
    if len(windows) != len(mg.groups):
        raise ValueError("need windows for %d groups, got %d" % (len(mg.groups), len(windows)))
    arrs = []
    for g, ws in zip(mg.groups, windows):
        if len(ws) != g.n:
            raise ValueError("need %d windows, got %d" % (g.n, len(ws)))
        a = (ebof_window_desc * g.n)()
        for k in range(g.n):
            _window_desc(ws[k], g.device, a[k])
        arrs.append(a)
    ptrs = (ctypes.POINTER(ebof_window_desc) * len(arrs))(
        *[ctypes.cast(a, ctypes.POINTER(ebof_window_desc)) for a in arrs])
    return load().ebof_multigroup_process(mg.handle, ptrs, _stream_handle(cuda_stream))


EBOF_STAGE_COUNT = 12


def ebof_stream_set_wait_limit(stream: Stream, iterations: int) -> int:
    return load().ebof_stream_set_wait_limit(stream.handle, int(iterations))


def ebof_debug_fail_allocation(n: int) -> None:
    load().ebof_debug_fail_allocation(int(n))


def ebof_stream_set_profiling(stream: Stream, enable: bool) -> int:
    return load().ebof_stream_set_profiling(stream.handle, 1 if enable else 0)


def ebof_stream_get_profile(stream: Stream):
    """Returns (status, {stage name: (ms, launches)})."""
    ms = (ctypes.c_double * EBOF_STAGE_COUNT)()
    ln = (ctypes.c_int64 * EBOF_STAGE_COUNT)()
    st = load().ebof_stream_get_profile(stream.handle, ms, ln, EBOF_STAGE_COUNT)
    return st, {ebof_stage_name(i): (ms[i], ln[i]) for i in range(EBOF_STAGE_COUNT)}


def ebof_stream_get_profile_level(stream: Stream, level: int):
    """Returns (status, {stage name: (ms, launches)}) for one pyramid level."""
    ms = (ctypes.c_double * EBOF_STAGE_COUNT)()
    ln = (ctypes.c_int64 * EBOF_STAGE_COUNT)()
    st = load().ebof_stream_get_profile_level(stream.handle, int(level), ms, ln,
                                              EBOF_STAGE_COUNT)
    return st, {ebof_stage_name(i): (ms[i], ln[i]) for i in range(EBOF_STAGE_COUNT)}


def ebof_stage_name(stage: int) -> str:
    return load().ebof_stage_name(int(stage)).decode()


def ebof_kernel_launches() -> int:
    return int(load().ebof_kernel_launches())


# ---------------------------------------------------------------- FWL
def ebof_fwl_scratch_bytes(width: int, height: int) -> int:
    return int(load().ebof_fwl_scratch_bytes(int(width), int(height)))


def ebof_fwl(x, y, t, p, t_begin: int, t_end: int, flow, width: int, height: int,
             scratch=None, out=None, cuda_stream=None):
    """Flow Warping Loss of one window (§IV-C).  x, y, t, p: CUDA event
    tensors (p int8 polarity or None); flow: CUDA float32 [2][H][W].
    scratch: CUDA uint8 tensor of ebof_fwl_scratch_bytes bytes (allocated
    here if None); out: CUDA float64 tensor of 3 (allocated if None).
    Returns (status, out) with out = [FWL, var(I_comp), var(I_uncomp)]
    written on the stream."""
    import torch
    n = x.numel()
    dev = flow.device.index
    if scratch is None:
        scratch = torch.empty(ebof_fwl_scratch_bytes(width, height), dtype=torch.uint8,
                              device=flow.device)
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=flow.device)
    st = load().ebof_fwl(_ptr(x, torch.uint16, n, "x", dev), _ptr(y, torch.uint16, n, "y", dev),
                         _ptr(t, torch.int64, n, "t", dev),
                         _ptr(p, torch.int8, n, "p", dev) if p is not None else None,
                         n, int(t_begin), int(t_end),
                         _ptr(flow, torch.float32, 2 * width * height, "flow", dev),
                         int(width), int(height),
                         _ptr(scratch, torch.uint8, ebof_fwl_scratch_bytes(width, height),
                              "scratch", dev),
                         _ptr(out, torch.float64, 3, "out", dev), _stream_handle(cuda_stream))
    return st, out


# ---------------------------------------------------------------- serving loop
def ebof_now_ns() -> int:
    return int(load().ebof_now_ns())


def ebof_server_default_config() -> ebof_server_config:
    c = ebof_server_config()
    load().ebof_server_default_config(ctypes.byref(c))
    return c


class Server:
    """Owner of an ``ebof_server*`` handle."""

    def __init__(self, handle: int, config: ebof_server_config):
        self.handle = handle
        self.config = config
        self.params = {}  # stream id -> ebof_params

    def close(self):
        if self.handle:
            load().ebof_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ebof_server_create(config: ebof_server_config = None):
    """Returns (status, Server or None)."""
    c = ebof_server_default_config() if config is None else config
    h = ctypes.c_void_p()
    st = load().ebof_server_create(ctypes.byref(c), ctypes.byref(h))
    if st < 0:
        return st, None
    return st, Server(h.value, c)


def ebof_server_destroy(server: Server) -> int:
    server.close()
    return EBOF_OK


def ebof_server_open_stream(server: Server, params: ebof_params):
    """Returns (status, stream id); status EBOF_QUEUED means waiting for memory."""
    sid = ctypes.c_int32(-1)
    st = load().ebof_server_open_stream(server.handle, ctypes.byref(params), ctypes.byref(sid))
    if st >= 0:
        p = ebof_params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(params), ctypes.sizeof(p))
        server.params[sid.value] = p
    return st, sid.value


def ebof_server_close_stream(server: Server, stream_id: int) -> int:
    return load().ebof_server_close_stream(server.handle, int(stream_id))


def ebof_server_submit(server: Server, stream_id: int, window, flow, tag: int,
                       arrival_ns: int = 0) -> int:
    """window: (x, y, t, t_begin, t_end); flow: CUDA float32 [2][H][W].  The
    tensors must stay alive until the window's completion is polled."""
    import torch
    p = server.params.get(int(stream_id))
    if p is None:
        return EBOF_ERR_INVALID_ARG
    d = _window_desc(window, server.config.device)
    fp = _ptr(flow, torch.float32, 2 * p.width * p.height, "flow", server.config.device)
    return load().ebof_server_submit(server.handle, int(stream_id), ctypes.byref(d), fp,
                                     int(tag), int(arrival_ns))


def ebof_server_poll(server: Server, max_out: int = 256, wait_us: int = 0):
    """Returns a list of ebof_completion (raises EbofError on error)."""
    arr = (ebof_completion * max(1, max_out))()
    n = load().ebof_server_poll(server.handle, arr, int(max_out), int(wait_us))
    check(n, "ebof_server_poll")
    return [arr[i] for i in range(n)]


def ebof_server_drain(server: Server, timeout_ms: int = 60000) -> int:
    return load().ebof_server_drain(server.handle, int(timeout_ms))


def ebof_server_get_info(server: Server) -> ebof_server_info:
    info = ebof_server_info()
    check(load().ebof_server_get_info(server.handle, ctypes.byref(info)), "ebof_server_get_info")
    return info


def check(status: int, what: str = "") -> int:
    """Raise EbofError for a negative status; return it otherwise."""
    if status < 0:
        raise EbofError(status, what)
    return status
