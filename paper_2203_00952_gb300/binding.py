"""ctypes binding of libsrt3d.so (include/srt3d.h). Argument marshalling only.

Every function here has the name of the C entry point it calls. Device
buffers are torch CUDA tensors (torch provides device memory and streams);
host buffers are numpy arrays. Nothing here computes any part of the method:
if the library is missing or no GPU is present the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsrt3d.so")

SRT3D_OK = 0
SRT3D_EINVAL = -1
SRT3D_ENOMEM = -2
SRT3D_ERANGE = -3
SRT3D_ECUDA = -4
SRT3D_EAGAIN = -5
SRT3D_ETIMEDOUT = -6
SRT3D_EBUSY = -7
SRT3D_ENOTFOUND = -8
SRT3D_EOFFSETS = -9

SRT3D_FP32 = 0
SRT3D_FP16_SPLIT = 1
SRT3D_BF16 = 2

SRT3D_INIT_MATCHED = 0
SRT3D_INIT_GIVEN = 1


class srt3d_params(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_uint32),
        ("k_max", ctypes.c_uint32),
        ("radius", ctypes.c_uint32),
        ("init_mode", ctypes.c_int32),
        ("regularize", ctypes.c_int32),
        ("apss_h", ctypes.c_float),
        ("d_max", ctypes.c_float),
        ("depth_scale", ctypes.c_float),
        ("prune_alpha", ctypes.c_float),
        ("smooth_lambda", ctypes.c_float),
        ("min_sep", ctypes.c_float),
        ("weighting", ctypes.c_int32),
        ("birth_every", ctypes.c_uint32),
    ]


def make_params(iters=20, k_max=1, radius=1, init_mode=SRT3D_INIT_MATCHED, regularize=1, apss_h=2.5,
                d_max=24.0, depth_scale=0.125, prune_alpha=0.02, smooth_lambda=0.5, min_sep=12.0, weighting=0,
                birth_every=0):
    return srt3d_params(iters, k_max, radius, init_mode, regularize, apss_h, d_max, depth_scale, prune_alpha,
                        smooth_lambda, min_sep, weighting, birth_every)


class srt3d_frame(ctypes.Structure):
    _fields_ = [
        ("stamps", ctypes.c_void_p),
        ("offsets", ctypes.c_void_p),
        ("num_stamps", ctypes.c_uint64),
        ("rows", ctypes.c_uint32),
        ("cols", ctypes.c_uint32),
        ("T", ctypes.c_uint32),
        ("m", ctypes.c_uint32),
        ("h", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("n", ctypes.c_void_p),
        ("depth", ctypes.c_void_p),
        ("alpha", ctypes.c_void_p),
        ("active", ctypes.c_void_p),
        ("alpha0", ctypes.c_void_p),
    ]


class srt3d_plan_info(ctypes.Structure):
    _fields_ = [
        ("sketch_m", ctypes.c_uint32),
        ("sketch_lanes", ctypes.c_uint32),
        ("init_m", ctypes.c_uint32),
        ("init_grid_spacing", ctypes.c_uint32),
        ("init_grid_points", ctypes.c_uint32),
        ("tile_height", ctypes.c_uint32),
        ("tiles", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("serving_frame_bytes", ctypes.c_uint64),
    ]


class SRT3DError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} ({status})")
        self.status = status


_lib = None
_c = ctypes
_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int

_SIGS = {
    "srt3d_create": (_i32, [_i32, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "srt3d_destroy": (None, [_vp]),
    "srt3d_status_string": (ctypes.c_char_p, [_i32]),
    "srt3d_last_error": (ctypes.c_char_p, [_vp]),
    "srt3d_sync": (_i32, [_vp, _vp]),
    "srt3d_selftest_wait_timeout": (_i32, [_vp, ctypes.c_uint64, _vp]),
    "srt3d_plan": (_i32, [_u32, _u32, _u32, _u32, _u32, _u32, ctypes.c_double, _u32, _u32,
                          ctypes.POINTER(srt3d_plan_info)]),
    "srt3d_hist_from_stream": (_i32, [_vp, _vp, _vp, _u64, _u32, _u32, _vp, _vp]),
    "srt3d_sketch_stream": (_i32, [_vp, _vp, _vp, _u64, _u32, _u32, _u32, _i32, _vp, _vp, _vp]),
    "srt3d_sketch_hist": (_i32, [_vp, _vp, _u32, _u32, _u32, _i32, _vp, _vp, _vp]),
    "srt3d_sketch_stream_tc": (_i32, [_vp, _vp, _vp, ctypes.c_uint64, _u32, _u32, _u32, _i32, _vp, _vp, _vp]),
    "srt3d_sketch_stream_tc_fused": (_i32, [_vp, _vp, _vp, ctypes.c_uint64, _u32, _u32, _u32, _i32, _vp, _vp,
                                             _vp]),
    "srt3d_finalize": (_i32, [_vp, _vp, _vp, _u32, _u32, _vp, _vp]),
    "srt3d_reconstruct": (_i32, [_vp, _vp, _vp, _u32, _u32, _u32, _u32, _vp, ctypes.POINTER(srt3d_params), _vp,
                                 _vp, _vp, _vp, _vp]),
    "srt3d_submit": (_i32, [_vp, _u64, _u32, _u32, _u32, _u32, _vp, ctypes.POINTER(srt3d_params), _vp, _vp, _i32]),
    "srt3d_poll": (_i32, [_vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp]),
}


def lib():
    """Load libsrt3d.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2203_00952_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, status, what):
    if status != SRT3D_OK:
        L = lib()
        name = L.srt3d_status_string(status).decode()
        msg = L.srt3d_last_error(ctx).decode() if ctx else ""
        raise SRT3DError(status, f"{what}: {name}: {msg}")
    return status


def _dev(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return _vp(t.data_ptr())


def _host(a, dtype, name):
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{name} must be a C-contiguous numpy array of {dtype}")
    return _vp(a.ctypes.data)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def srt3d_create(device=0, hbm_budget_bytes=0):
    ctx = _vp()
    L = lib()
    st = L.srt3d_create(int(device), int(hbm_budget_bytes), ctypes.byref(ctx))
    if st != SRT3D_OK:
        raise SRT3DError(st, f"srt3d_create: {L.srt3d_status_string(st).decode()}")
    return ctx


def srt3d_destroy(ctx):
    lib().srt3d_destroy(ctx)


def srt3d_sync(ctx, stream=None, check=True):
    st = lib().srt3d_sync(ctx, _stream(stream))
    return _check(ctx, st, "srt3d_sync") if check else st


def srt3d_hist_from_stream(ctx, stamps, offsets, T, hist, stream=None):
    import torch

    P = offsets.numel() - 1
    st = lib().srt3d_hist_from_stream(ctx, _dev(stamps, torch.int16, "stamps"), _dev(offsets, torch.int32, "offsets"),
                                      stamps.numel(), P, int(T), _dev(hist, torch.int16, "hist"), _stream(stream))
    return _check(ctx, st, "srt3d_hist_from_stream")


def srt3d_sketch_stream(ctx, stamps, offsets, T, m, accumulate, S, n, stream=None):
    import torch

    P = offsets.numel() - 1
    st = lib().srt3d_sketch_stream(ctx, _dev(stamps, torch.int16, "stamps"), _dev(offsets, torch.int32, "offsets"),
                                   stamps.numel(), P, int(T), int(m), int(accumulate), _dev(S, torch.float32, "S"),
                                   _dev(n, torch.int32, "n"), _stream(stream))
    return _check(ctx, st, "srt3d_sketch_stream")


def srt3d_sketch_stream_tc(ctx, stamps, offsets, T, m, precision, S, n, stream=None):
    import torch

    P = offsets.numel() - 1
    st = lib().srt3d_sketch_stream_tc(ctx, _dev(stamps, torch.int16, "stamps"), _dev(offsets, torch.int32, "offsets"),
                                      stamps.numel(), P, int(T), int(m), int(precision), _dev(S, torch.float32, "S"),
                                      _dev(n, torch.int32, "n"), _stream(stream))
    return _check(ctx, st, "srt3d_sketch_stream_tc")


def srt3d_sketch_stream_tc_fused(ctx, stamps, offsets, T, m, precision, S, n, stream=None):
    import torch

    P = offsets.numel() - 1
    st = lib().srt3d_sketch_stream_tc_fused(ctx, _dev(stamps, torch.int16, "stamps"),
                                            _dev(offsets, torch.int32, "offsets"), stamps.numel(), P, int(T), int(m),
                                            int(precision), _dev(S, torch.float32, "S"), _dev(n, torch.int32, "n"),
                                            _stream(stream))
    return _check(ctx, st, "srt3d_sketch_stream_tc_fused")


def srt3d_sketch_hist(ctx, hist, T, m, precision, S, n, stream=None):
    import torch

    P = hist.numel() // int(T)
    st = lib().srt3d_sketch_hist(ctx, _dev(hist, torch.int16, "hist"), P, int(T), int(m), int(precision),
                                 _dev(S, torch.float32, "S"), _dev(n, torch.int32, "n"), _stream(stream))
    return _check(ctx, st, "srt3d_sketch_hist")


def srt3d_finalize(ctx, S, n, m, z, stream=None):
    import torch

    P = n.numel()
    st = lib().srt3d_finalize(ctx, _dev(S, torch.float32, "S"), _dev(n, torch.int32, "n"), P, int(m),
                              _dev(z, torch.float32, "z"), _stream(stream))
    return _check(ctx, st, "srt3d_finalize")


def srt3d_reconstruct(ctx, z, n, rows, cols, T, m, h, params, depth, alpha, active, alpha0, stream=None):
    import torch

    st = lib().srt3d_reconstruct(ctx, _dev(z, torch.float32, "z"), _dev(n, torch.int32, "n"), int(rows), int(cols),
                                 int(T), int(m), _dev(h, torch.float32, "h"), ctypes.byref(params),
                                 _dev(depth, torch.float32, "depth"), _dev(alpha, torch.float32, "alpha"),
                                 _dev(active, torch.uint8, "active"), _dev(alpha0, torch.float32, "alpha0"),
                                 _stream(stream))
    return _check(ctx, st, "srt3d_reconstruct")


SRT3D_LAST_CHUNK, SRT3D_CHUNK_KEEP = 1, 2  # srt3d_submit flags


def srt3d_submit(ctx, frame_id, rows, cols, T, m, h, params, chunk_stamps, chunk_offsets, last_chunk, check=True):
    st = lib().srt3d_submit(ctx, int(frame_id), int(rows), int(cols), int(T), int(m),
                            _host(h, np.float32, "h"), ctypes.byref(params),
                            _host(chunk_stamps, np.uint16, "chunk_stamps"),
                            _host(chunk_offsets, np.uint32, "chunk_offsets"), int(last_chunk))
    return _check(ctx, st, "srt3d_submit") if check else st


def srt3d_poll(ctx, frame_id, timeout_us, depth, alpha, active, alpha0, n=None, check=True):
    st = lib().srt3d_poll(ctx, int(frame_id), int(timeout_us), _host(depth, np.float32, "depth"),
                          _host(alpha, np.float32, "alpha"), _host(active, np.uint8, "active"),
                          _host(alpha0, np.float32, "alpha0"), _host(n, np.uint32, "n"))
    return _check(ctx, st, "srt3d_poll") if check else st


_SIGS.update({
    "srt3d_profile_enable": (_i32, [_vp, _i32]),
    "srt3d_profile_read": (_i32, [_vp, _u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
    "srt3d_kernel_count": (_u32, []),
    "srt3d_kernel_name": (ctypes.c_char_p, [_u32]),
    "srt3d_process_batch": (_i32, [_vp, ctypes.POINTER(srt3d_frame), _u32, ctypes.POINTER(srt3d_params), _vp]),
    "srt3d_reconstruct_noalloc": (_i32, [_vp, _vp, _vp, _u32, _u32, _u32, _u32, _vp, ctypes.POINTER(srt3d_params),
                                         _vp, _vp, _vp, _vp, _vp]),
})


def srt3d_reconstruct_noalloc(ctx, z, n, rows, cols, T, m, h, params, depth, alpha, active, alpha0, stream=None,
                              check=True):
    """Allocation-free reconstruction (see include/srt3d.h)."""
    import torch

    st = lib().srt3d_reconstruct_noalloc(ctx, _dev(z, torch.float32, "z"), _dev(n, torch.int32, "n"), int(rows),
                                         int(cols), int(T), int(m), _dev(h, torch.float32, "h"),
                                         ctypes.byref(params), _dev(depth, torch.float32, "depth"),
                                         _dev(alpha, torch.float32, "alpha"), _dev(active, torch.uint8, "active"),
                                         _dev(alpha0, torch.float32, "alpha0"), _stream(stream))
    return _check(ctx, st, "srt3d_reconstruct_noalloc") if check else st


def srt3d_profile_enable(ctx, enable=True):
    return _check(ctx, lib().srt3d_profile_enable(ctx, int(bool(enable))), "srt3d_profile_enable")


def srt3d_profile_read(ctx, kernel):
    ms = ctypes.c_double()
    cnt = ctypes.c_uint64()
    _check(ctx, lib().srt3d_profile_read(ctx, int(kernel), ctypes.byref(ms), ctypes.byref(cnt)), "srt3d_profile_read")
    return ms.value, cnt.value


def srt3d_kernel_count():
    return int(lib().srt3d_kernel_count())


def srt3d_kernel_name(kernel):
    return lib().srt3d_kernel_name(int(kernel)).decode()


def srt3d_selftest_wait_timeout(ctx, wait_cycles, stream=None, check=True):
    st = lib().srt3d_selftest_wait_timeout(ctx, int(wait_cycles), _stream(stream))
    return _check(ctx, st, "srt3d_selftest_wait_timeout") if check else st


def srt3d_plan(rows, cols, T, m, k_max, radius, mean_photons_per_pixel, num_sms, ctas_per_sm):
    """Launch shapes for a frame (host only, no device needed); raises
    SRT3DError on invalid arguments."""
    info = srt3d_plan_info()
    st = lib().srt3d_plan(int(rows), int(cols), int(T), int(m), int(k_max), int(radius),
                          float(mean_photons_per_pixel), int(num_sms), int(ctas_per_sm), ctypes.byref(info))
    if st != SRT3D_OK:
        raise SRT3DError(st, f"srt3d_plan: status {st}")
    return {name: getattr(info, name) for name, _ in srt3d_plan_info._fields_ if name != "reserved"}


def profile_totals(ctx):
    """{kernel name: (total ms, launches)} for every kernel with launches."""
    out = {}
    for k in range(srt3d_kernel_count()):
        ms, cnt = srt3d_profile_read(ctx, k)
        if cnt:
            out[srt3d_kernel_name(k)] = (ms, cnt)
    return out


def make_frame(stamps, offsets, rows, cols, T, m, h, z, n, depth, alpha, active, alpha0):
    """srt3d_frame from torch CUDA tensors (device pointers)."""
    import torch

    return srt3d_frame(_dev(stamps, torch.int16, "stamps").value if stamps.numel() else None,
                       _dev(offsets, torch.int32, "offsets"), stamps.numel(), int(rows), int(cols), int(T), int(m),
                       _dev(h, torch.float32, "h"), _dev(z, torch.float32, "z"), _dev(n, torch.int32, "n"),
                       _dev(depth, torch.float32, "depth"), _dev(alpha, torch.float32, "alpha"),
                       _dev(active, torch.uint8, "active"), _dev(alpha0, torch.float32, "alpha0"))


def srt3d_process_batch(ctx, frames, params, stream=None):
    arr = (srt3d_frame * len(frames))(*frames)
    st = lib().srt3d_process_batch(ctx, arr, len(frames), ctypes.byref(params), _stream(stream))
    return _check(ctx, st, "srt3d_process_batch")
