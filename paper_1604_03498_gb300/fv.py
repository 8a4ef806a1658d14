"""Thin Python binding of the C ABI in include/fv.h (ctypes).

The functions keep the C names and only marshal arguments: pointers, sizes,
on-device flags and the current CUDA stream of torch. Every step of the
encoder runs in the CUDA library ``_build/libfvgpu.so``; there is no CPU or
PyTorch fallback. If the library cannot be built or loaded, importing this
module raises.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays (host memory).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FV_OK = 0
FV_PENDING = 1
FV_ERR_INVALID = -1
FV_ERR_OOM = -2
FV_ERR_CUDA = -3
FV_ERR_BUSY = -4
FV_ERR_TIMEOUT = -5
FV_ERR_NOTFOUND = -6
FV_ERR_EMPTY = -7
FV_ERR_DEVICE = -8
FV_ERR_UNSUPPORTED = -9

FV_PREC_FP32 = 0
FV_PREC_BF16 = 1
FV_PREC_BF16X2 = 2

_lock = threading.Lock()
_lib = None


class FVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fv status {status}: {msg}")
        self.status = status


class fv_gmm_desc(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("D", ctypes.c_int), ("weights", ctypes.c_void_p),
                ("means", ctypes.c_void_p), ("variances", ctypes.c_void_p)]


class fv_encode_options(ctypes.Structure):
    _fields_ = [("posterior_threshold", ctypes.c_float), ("skip_counts", ctypes.c_void_p)]


class fv_dsift_params(ctypes.Structure):
    _fields_ = [("bin_size", ctypes.c_int), ("stride", ctypes.c_int), ("n_scales", ctypes.c_int),
                ("top_scale", ctypes.c_int)]


class fv_batch_plan_config(ctypes.Structure):
    _fields_ = [("max_frames", ctypes.c_int), ("max_rows", ctypes.c_int64), ("autotune", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p)]


class fv_batch_plan_info(ctypes.Structure):
    _fields_ = [("stat_ctas", ctypes.c_int), ("tuned", ctypes.c_int), ("tuned_ms", ctypes.c_double),
                ("max_rows", ctypes.c_int64), ("max_frames", ctypes.c_int), ("ld_x", ctypes.c_int),
                ("rows_per_tile", ctypes.c_int), ("y_stages", ctypes.c_int), ("candidates", ctypes.c_int),
                ("tiles_per_share", ctypes.c_double)]


class fv_server_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64),
                ("max_batch_descriptors", ctypes.c_int64), ("max_batch_frames", ctypes.c_int),
                ("max_frame_descriptors", ctypes.c_int64), ("batch_window_ns", ctypes.c_int64)]


class fv_result_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("stream_id", ctypes.c_int), ("n", ctypes.c_int64),
                ("latency_ns", ctypes.c_int64), ("queue_ns", ctypes.c_int64), ("batch_frames", ctypes.c_int)]


def lib():
    """Load (building first if needed) the CUDA library. Raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
            P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            L.fv_gmm_load.argtypes = [ctypes.POINTER(fv_gmm_desc), I, ctypes.POINTER(P)]
            L.fv_gmm_load.restype = I
            L.fv_gmm_free.argtypes = [P]
            L.fv_gmm_free.restype = None
            L.fv_gmm_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
            L.fv_gmm_info.restype = I
            L.fv_gmm_constants.argtypes = [P, P, P]
            L.fv_gmm_constants.restype = I
            L.fv_limits.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I)]
            L.fv_limits.restype = I
            L.fv_encode.argtypes = [P, P, I64, I, P, I, P]
            L.fv_encode.restype = I
            L.fv_encode_batch.argtypes = [P, P, P, I, I, P, I, P]
            L.fv_encode_batch.restype = I
            L.fv_encode_batch_opts.argtypes = [P, P, I, I64, P, I, I, P, I, ctypes.POINTER(fv_encode_options), P]
            L.fv_encode_batch_opts.restype = I
            L.fv_encode_batch_bf16.argtypes = [P, P, I64, P, I, P, P]
            L.fv_encode_batch_bf16.restype = I
            L.fv_last_error.argtypes = []
            L.fv_last_error.restype = ctypes.c_char_p
            L.fv_batch_plan_create.argtypes = [P, ctypes.POINTER(fv_batch_plan_config), ctypes.POINTER(P)]
            L.fv_batch_plan_create.restype = I
            L.fv_batch_plan_load_bf16.argtypes = [P, P, I64, I64, P]
            L.fv_batch_plan_load_bf16.restype = I
            L.fv_batch_plan_run.argtypes = [P, P, I, P, I, P]
            L.fv_batch_plan_run.restype = I
            L.fv_batch_plan_run_f32.argtypes = [P, P, P, I, P, I, P]
            L.fv_batch_plan_run_f32.restype = I
            L.fv_batch_plan_get_info.argtypes = [P, ctypes.POINTER(fv_batch_plan_info)]
            L.fv_batch_plan_get_info.restype = I
            L.fv_batch_plan_buffers.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P)]
            L.fv_batch_plan_buffers.restype = I
            L.fv_batch_plan_destroy.argtypes = [P]
            L.fv_batch_plan_destroy.restype = None
            L.fv_server_create.argtypes = [P, ctypes.POINTER(fv_server_config), ctypes.POINTER(P)]
            L.fv_server_create.restype = I
            L.fv_server_submit.argtypes = [P, I, P, I64, ctypes.POINTER(ctypes.c_uint64)]
            L.fv_server_submit.restype = I
            L.fv_server_poll.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(fv_result_info), I64]
            L.fv_server_poll.restype = I
            L.fv_server_stats.argtypes = [P] + [ctypes.POINTER(I64)] * 4
            L.fv_server_stats.restype = I
            L.fv_server_destroy.argtypes = [P]
            L.fv_server_destroy.restype = None
            L.fv_gmm_em_step.argtypes = [P, P, I64, I, ctypes.c_double, P, P, P, I, ctypes.POINTER(ctypes.c_double),
                                         P]
            L.fv_gmm_em_step.restype = I
            L.fv_gmm_fit.argtypes = [ctypes.POINTER(fv_gmm_desc), P, I64, I, I, ctypes.c_double, ctypes.c_double, P, P,
                                     P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_double), P]
            L.fv_gmm_fit.restype = I
            L.fv_pca_load.argtypes = [P, P, I, I, ctypes.POINTER(P)]
            L.fv_pca_load.restype = I
            L.fv_pca_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
            L.fv_pca_info.restype = I
            L.fv_pca_free.argtypes = [P]
            L.fv_pca_free.restype = None
            L.fv_pca_project.argtypes = [P, P, P, I64, P, I, I64, P]
            L.fv_pca_project.restype = I
            L.fv_encode_pca.argtypes = [P, P, P, P, P, I, I, P, I, P]
            L.fv_encode_pca.restype = I
            L.fv_dsift_count.argtypes = [I, I, ctypes.POINTER(fv_dsift_params), ctypes.POINTER(I64)]
            L.fv_dsift_count.restype = I
            L.fv_dsift.argtypes = [P, I, I, I, I, ctypes.POINTER(fv_dsift_params), P, P, P]
            L.fv_dsift.restype = I
            L.fv_encode_images.argtypes = [P, P, P, I, I, I, I, ctypes.POINTER(fv_dsift_params), P, I, P]
            L.fv_encode_images.restype = I
            L.fv_encode_noalloc.argtypes = [P, P, I64, P, P]
            L.fv_encode_noalloc.restype = I
            L.fv_prof_enable.argtypes = [I]
            L.fv_prof_enable.restype = I
            L.fv_prof_collect.argtypes = [P, I, ctypes.POINTER(I)]
            L.fv_prof_collect.restype = I
            L.fv_probe_peaks.argtypes = [P, P, P, P]
            L.fv_probe_peaks.restype = I
            L.fv_launch_count.argtypes = []
            L.fv_launch_count.restype = I64
            _lib = L
    return _lib


def fv_last_error() -> str:
    return lib().fv_last_error().decode()


def _check(st: int, allow=(FV_OK,)) -> int:
    if st not in allow:
        raise FVError(st, fv_last_error())
    return st


def _ptr(a):
    """(pointer, on_device) of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


class Gmm:
    """Owns an fv_gmm handle (freed on close/garbage collection)."""

    def __init__(self, handle, K, D, precision):
        self.handle = handle
        self.K, self.D, self.precision = K, D, precision

    @property
    def fv_len(self):
        return 2 * self.K * self.D

    def close(self):
        if self.handle:
            lib().fv_gmm_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_gmm_load(weights, means, variances, precision: int = FV_PREC_FP32) -> Gmm:
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
    mu = np.ascontiguousarray(np.asarray(means, dtype=np.float32))
    var = np.ascontiguousarray(np.asarray(variances, dtype=np.float32))
    K, D = mu.shape
    desc = fv_gmm_desc(K, D, w.ctypes.data, mu.ctypes.data, var.ctypes.data)
    h = ctypes.c_void_p()
    _check(lib().fv_gmm_load(ctypes.byref(desc), int(precision), ctypes.byref(h)))
    return Gmm(h, K, D, precision)


def fv_gmm_free(g: Gmm) -> None:
    g.close()


def fv_gmm_constants(g: Gmm):
    """C fv_gmm_constants: the FP64 per-component constants (c_direct,
    c_expanded) the loader computed on the device, as two arrays of K."""
    K, _, _ = fv_gmm_info(g)
    cd = np.zeros(K)
    ce = np.zeros(K)
    _check(lib().fv_gmm_constants(g.handle, cd.ctypes.data, ce.ctypes.data))
    return cd, ce


def fv_gmm_info(g: Gmm):
    K, D, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().fv_gmm_info(g.handle, ctypes.byref(K), ctypes.byref(D), ctypes.byref(P)))
    return K.value, D.value, P.value


def fv_limits(precision: int):
    K, D = ctypes.c_int(), ctypes.c_int()
    _check(lib().fv_limits(int(precision), ctypes.byref(K), ctypes.byref(D)))
    return K.value, D.value


def fv_encode(g: Gmm, X, out, stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_encode: X (N x D float32) -> out (2KD float32). Returns the status."""
    xp, xd = _ptr(X)
    op, od = _ptr(out)
    N = int(X.shape[0])
    return _check(lib().fv_encode(g.handle, xp, N, xd, op, od, _stream(stream)), allow)


def fv_encode_batch(g: Gmm, X_packed, offsets, out, stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_encode_batch: offsets is a host int64 array of B+1 entries."""
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    B = offs.size - 1
    xp, xd = _ptr(X_packed)
    op, od = _ptr(out)
    return _check(lib().fv_encode_batch(g.handle, xp, offs.ctypes.data, B, xd, op, od, _stream(stream)), allow)


def fv_encode_batch_bf16(g: Gmm, X_bf16, ld_x: int, offsets, out, stream=None,
                         allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_encode_batch_bf16: X_bf16 is a CUDA tensor of bfloat16 (or int16
    bit patterns) with row pitch ld_x; out a CUDA float32 tensor."""
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    B = offs.size - 1
    xp, _ = _ptr(X_bf16)
    op, _ = _ptr(out)
    return _check(lib().fv_encode_batch_bf16(g.handle, xp, int(ld_x), offs.ctypes.data, B, op, _stream(stream)),
                  allow)


def fv_encode_batch_opts(g: Gmm, X, offsets, out, tau: float = 0.0, skip_counts=None, ld_x: int = 0,
                         stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_encode_batch_opts: X is float32 (host or CUDA) or a CUDA bfloat16
    tensor (row pitch ld_x, default D); tau the posterior threshold (early
    termination); skip_counts an optional CUDA int64 tensor of 2 counters."""
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    xp, xd = _ptr(X)
    op, od = _ptr(out)
    is_bf16 = 0
    try:
        import torch
        is_bf16 = int(isinstance(X, torch.Tensor) and X.dtype == torch.bfloat16)
    except ImportError:
        pass
    opt = fv_encode_options(float(tau), _ptr(skip_counts)[0] if skip_counts is not None else None)
    return _check(lib().fv_encode_batch_opts(g.handle, xp, is_bf16, int(ld_x or g.D), offs.ctypes.data, offs.size - 1,
                                             xd, op, od, ctypes.byref(opt), _stream(stream)), allow)


def fv_encode_noalloc(g: Gmm, X, out, stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_encode_noalloc: like fv_encode (FP32 handle, device tensors only)
    but for callers that must not allocate device memory: the library takes
    its scratch from a fixed array it owns instead of the memory pool."""
    xp, _ = _ptr(X)
    op, _ = _ptr(out)
    return _check(lib().fv_encode_noalloc(g.handle, xp, int(X.shape[0]), op, _stream(stream)), allow)


def fv_gmm_em_step(g: Gmm, X, reg_covar: float = 1e-6, stream=None):
    """C fv_gmm_em_step with host outputs: returns (w, mu, var, mean_loglik)."""
    K, D = g.K, g.D
    xp, xd = _ptr(X)
    w = np.zeros(K, np.float32)
    mu = np.zeros((K, D), np.float32)
    var = np.zeros((K, D), np.float32)
    ll = ctypes.c_double()
    _check(lib().fv_gmm_em_step(g.handle, xp, int(X.shape[0]), xd, float(reg_covar), w.ctypes.data, mu.ctypes.data,
                                var.ctypes.data, 0, ctypes.byref(ll), _stream(stream)))
    return w, mu, var, ll.value


def fv_gmm_fit(w0, mu0, var0, X, max_iter: int = 100, tol: float = 1e-3, reg_covar: float = 1e-6, stream=None):
    """C fv_gmm_fit: returns (w, mu, var, n_iter, mean_loglik)."""
    w0 = np.ascontiguousarray(np.asarray(w0, dtype=np.float32))
    mu0 = np.ascontiguousarray(np.asarray(mu0, dtype=np.float32))
    var0 = np.ascontiguousarray(np.asarray(var0, dtype=np.float32))
    K, D = mu0.shape
    desc = fv_gmm_desc(K, D, w0.ctypes.data, mu0.ctypes.data, var0.ctypes.data)
    xp, xd = _ptr(X)
    w = np.zeros(K, np.float32)
    mu = np.zeros((K, D), np.float32)
    var = np.zeros((K, D), np.float32)
    it = ctypes.c_int()
    ll = ctypes.c_double()
    _check(lib().fv_gmm_fit(ctypes.byref(desc), xp, int(X.shape[0]), xd, int(max_iter), float(tol), float(reg_covar),
                            w.ctypes.data, mu.ctypes.data, var.ctypes.data, ctypes.byref(it), ctypes.byref(ll),
                            _stream(stream)))
    return w, mu, var, it.value, ll.value


class Pca:
    """Owns an fv_pca handle (PCA projection + position append)."""

    def __init__(self, handle, m, Din):
        self.handle = handle
        self.m, self.Din = m, Din

    def close(self):
        if self.handle:
            lib().fv_pca_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_pca_load(basis, mean=None) -> Pca:
    P = np.ascontiguousarray(np.asarray(basis, dtype=np.float32))
    m, Din = P.shape
    mn = None if mean is None else np.ascontiguousarray(np.asarray(mean, dtype=np.float32))
    h = ctypes.c_void_p()
    _check(lib().fv_pca_load(P.ctypes.data, None if mn is None else mn.ctypes.data, m, Din, ctypes.byref(h)))
    return Pca(h, m, Din)


def fv_pca_project(p: Pca, X, xy, Y, y_bf16: bool, ld_y: int = 0, stream=None) -> int:
    """C fv_pca_project (device tensors): Y receives the projected rows."""
    xp, _ = _ptr(X)
    yp, _ = _ptr(Y)
    xyp = _ptr(xy)[0] if xy is not None else None
    return _check(lib().fv_pca_project(p.handle, xp, xyp, int(X.shape[0]), yp, int(bool(y_bf16)), int(ld_y),
                                       _stream(stream)), (FV_OK,))


def fv_encode_pca(g: Gmm, p: Pca, X, xy, offsets, out, stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_encode_pca: X (N x Din) and xy (N x 2 or None) on the same side."""
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    xp, xd = _ptr(X)
    xyp = _ptr(xy)[0] if xy is not None else None
    op, od = _ptr(out)
    return _check(lib().fv_encode_pca(g.handle, p.handle, xp, xyp, offs.ctypes.data, offs.size - 1, xd, op, od,
                                      _stream(stream)), allow)


def _dsift_params(bin_size=4, stride=4, n_scales=8, top_scale=1):
    return fv_dsift_params(int(bin_size), int(stride), int(n_scales), int(top_scale))


def fv_dsift_count(H: int, W: int, **params) -> int:
    n = ctypes.c_int64()
    _check(lib().fv_dsift_count(int(H), int(W), ctypes.byref(_dsift_params(**params)), ctypes.byref(n)))
    return n.value


def fv_dsift(images, desc, xy=None, stream=None, **params) -> int:
    """C fv_dsift: images (B x H x W float32, host or CUDA) -> desc (CUDA,
    B x n x 128) and xy (CUDA, B x n x 2, optional)."""
    B, H, W = (int(v) for v in images.shape)
    ip, idv = _ptr(images)
    dp, _ = _ptr(desc)
    xp = _ptr(xy)[0] if xy is not None else None
    return _check(lib().fv_dsift(ip, B, H, W, idv, ctypes.byref(_dsift_params(**params)), dp, xp, _stream(stream)))


def fv_encode_images(g: Gmm, p: "Pca", images, out, stream=None, allow=(FV_OK,), **params) -> int:
    """C fv_encode_images: images (B x H x W) -> out (B x 2KD)."""
    B, H, W = (int(v) for v in images.shape)
    ip, idv = _ptr(images)
    op, od = _ptr(out)
    return _check(lib().fv_encode_images(g.handle, p.handle, ip, B, H, W, idv, ctypes.byref(_dsift_params(**params)),
                                         op, od, _stream(stream)), allow)


class BatchPlan:
    """Owns an fv_batch_plan (the batched form: one CUDA-graph launch per batch)."""

    def __init__(self, handle, K, D):
        self.handle = handle
        self.K, self.D = K, D

    def close(self):
        if self.handle:
            lib().fv_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_batch_plan_create(g: Gmm, max_frames: int, max_rows: int, autotune: bool = False,
                         tune_cache: str | None = None) -> BatchPlan:
    cfg = fv_batch_plan_config(int(max_frames), int(max_rows), int(bool(autotune)),
                               tune_cache.encode() if tune_cache else None)
    h = ctypes.c_void_p()
    _check(lib().fv_batch_plan_create(g.handle, ctypes.byref(cfg), ctypes.byref(h)))
    return BatchPlan(h, g.K, g.D)


def fv_batch_plan_get_info(p: BatchPlan) -> dict:
    info = fv_batch_plan_info()
    _check(lib().fv_batch_plan_get_info(p.handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in fv_batch_plan_info._fields_}


def fv_batch_plan_load_bf16(p: BatchPlan, X_bf16, ld_x: int, rows: int, stream=None) -> int:
    xp, _ = _ptr(X_bf16)
    return _check(lib().fv_batch_plan_load_bf16(p.handle, xp, int(ld_x), int(rows), _stream(stream)))


def fv_batch_plan_run(p: BatchPlan, offsets, out=None, stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    """C fv_batch_plan_run: encode the batch already in the plan's input buffer;
    out (B x 2KD, host or device) receives a copy of the vectors when given."""
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    op, od = _ptr(out)
    return _check(lib().fv_batch_plan_run(p.handle, offs.ctypes.data, offs.size - 1, op, od, _stream(stream)), allow)


def fv_batch_plan_run_f32(p: BatchPlan, X, offsets, out=None, stream=None, allow=(FV_OK, FV_ERR_EMPTY)) -> int:
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    xp, _ = _ptr(X)
    op, od = _ptr(out)
    return _check(lib().fv_batch_plan_run_f32(p.handle, xp, offs.ctypes.data, offs.size - 1, op, od,
                                              _stream(stream)), allow)


class Server:
    """Owns an fv_server (the serving form: continuous batching)."""

    def __init__(self, handle, K, D):
        self.handle = handle
        self.K, self.D = K, D

    def close(self):
        if self.handle:
            lib().fv_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_server_create(g: Gmm, max_slots: int, hbm_budget_bytes: int, max_batch_descriptors: int,
                     max_batch_frames: int, max_frame_descriptors: int, batch_window_ns: int = 0) -> Server:
    cfg = fv_server_config(int(max_slots), int(hbm_budget_bytes), int(max_batch_descriptors), int(max_batch_frames),
                           int(max_frame_descriptors), int(batch_window_ns))
    h = ctypes.c_void_p()
    _check(lib().fv_server_create(g.handle, ctypes.byref(cfg), ctypes.byref(h)))
    return Server(h, g.K, g.D)


def fv_server_submit(s: Server, stream_id: int, X, allow=(FV_OK,)):
    """C fv_server_submit with host descriptors X (N x D float32).
    Returns (status, ticket)."""
    xp, xd = _ptr(X)
    if xd:
        raise ValueError("fv_server_submit takes host descriptors")
    t = ctypes.c_uint64()
    st = _check(lib().fv_server_submit(s.handle, int(stream_id), xp, int(X.shape[0]), ctypes.byref(t)), allow)
    return st, t.value


def fv_server_poll(s: Server, ticket: int, out=None, timeout_ns: int = -1,
                   allow=(FV_OK, FV_PENDING, FV_ERR_TIMEOUT)):
    """C fv_server_poll; out is a host float32 array of 2KD. Returns (status, info dict)."""
    op, _ = _ptr(out)
    info = fv_result_info()
    st = _check(lib().fv_server_poll(s.handle, ctypes.c_uint64(ticket), op, ctypes.byref(info), int(timeout_ns)), allow)
    return st, {f: getattr(info, f) for f, _ in fv_result_info._fields_}


def fv_server_stats(s: Server) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().fv_server_stats(s.handle, *[ctypes.byref(x) for x in v]))
    return dict(zip(("admitted", "refused", "completed", "batches"), (x.value for x in v)))


class fv_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


def fv_prof_enable(on: bool) -> None:
    _check(lib().fv_prof_enable(int(bool(on))))


def fv_prof_collect() -> dict:
    """{kernel name: (launches, total device ms)} since the last collect."""
    arr = (fv_kernel_stat * 64)()
    n = ctypes.c_int()
    _check(lib().fv_prof_collect(ctypes.cast(arr, ctypes.c_void_p), 64, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, 64))}


def fv_probe_peaks(stream=None) -> dict:
    """C fv_probe_peaks: measured FP32 FMA (scalar, packed f32x2) TFLOP/s and
    ex2 G/s of the current device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().fv_probe_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream(stream)))
    return {"ffma_tflops": a.value, "ffma2_tflops": b.value, "ex2_gops": c.value}


def fv_launch_count() -> int:
    return int(lib().fv_launch_count())
