"""Python binding of the GB300 hybrid multi-noise denoiser (C ABI in libhd.so).

The functions carry the C names (``amf_filter``, ``wiener_filter``,
``hybrid_denoise``, ``hybrid_denoise_batched`` ...) and only marshal
arguments: every stage runs in the CUDA kernels of ``libhd.so``.  Tensors are
``torch`` CUDA tensors (uint8, or uint16 for 9..16-bit images); PyTorch is used
for device memory and streams only.  If the library is missing or cannot be
loaded the import fails loudly; there is no CPU fallback.

Algorithm (Youssef, Mahmoud, El-Horbaty): adaptive median (Algorithm 1,
step 6) followed by a local-statistics Wiener filter (Algorithm 1, step 4d),
and the contrast stretch of step 4e as a separate call.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhd.so")

HD_OK, HD_ERR_ARG, HD_ERR_SMAX, HD_ERR_WINDOW, HD_ERR_DTYPE = 0, 1, 2, 3, 4
HD_ERR_WORKSPACE, HD_ERR_CUDA, HD_ERR_TIMEOUT, HD_ERR_OVERFLOW = 5, 6, 7, 8
HD_U8, HD_U16 = 0, 1
HD_BORDER_SYMMETRIC, HD_BORDER_ZERO = 0, 1
HD_UNRESOLVED_ZMED, HD_UNRESOLVED_KEEP = 0, 1
HD_SMAX_MAX = 15
HD_WIENER_W_MAX = 15

# every symbol include/hybrid_denoise.h declares
EXPORTS = [
    "amf_filter", "wiener_filter", "wiener_workspace_size", "hybrid_denoise", "hybrid_workspace_size",
    "hybrid_min_workspace_size", "hybrid_denoise_host", "hybrid_host_workspace_size", "hybrid_denoise_static", "hybrid_denoise_batched",
    "hybrid_batched_workspace_size", "hd_batch_plan_create", "hd_batch_plan_launch",
    "hd_batch_plan_destroy", "hd_set_tuning", "hd_get_tuning", "hd_set_spin_limit", "hd_get_device_error",
    "hd_status_str", "hd_version", "contrast_stretch", "contrast_workspace_size",
    "hybrid_denoise_strips", "hybrid_strips_workspace_size", "reference_noise_variance",
    "hd_host_pipeline_workspace_size", "hd_host_pipeline_create", "hd_host_pipeline_submit",
    "hd_host_pipeline_wait", "hd_host_pipeline_destroy",
    "hd_batch_pipeline_workspace_size", "hd_batch_pipeline_create", "hd_batch_pipeline_submit",
    "hd_batch_pipeline_wait", "hd_batch_pipeline_destroy",
    "hd_part_halo_rows", "hybrid_part_workspace_size", "hybrid_part_stats", "hybrid_part_apply",
    "wiener_deconv_workspace_size", "wiener_deconvolve",
]


class hd_params(ctypes.Structure):
    _fields_ = [("smax", ctypes.c_int), ("wiener_w", ctypes.c_int), ("noise_var", ctypes.c_double),
                ("border", ctypes.c_int), ("unresolved", ctypes.c_int), ("bits", ctypes.c_int),
                ("wiener_h", ctypes.c_int)]


class hd_image(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("src_pitch", ctypes.c_size_t), ("dst_pitch", ctypes.c_size_t), ("dtype", ctypes.c_int),
                ("p", hd_params), ("noise_var_out", ctypes.c_void_p), ("y_out", ctypes.c_void_p)]


class hd_part(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("src_pitch", ctypes.c_size_t), ("dst", ctypes.c_void_p),
                ("dst_pitch", ctypes.c_size_t), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("buf_row0", ctypes.c_int), ("buf_rows", ctypes.c_int), ("own_row0", ctypes.c_int),
                ("own_rows", ctypes.c_int), ("dtype", ctypes.c_int), ("p", hd_params)]


class hd_tuning(ctypes.Structure):
    _fields_ = [("region_h", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("plane", ctypes.c_int),
                ("small_growth", ctypes.c_int), ("select_lanes", ctypes.c_int), ("batch_lag", ctypes.c_int),
                ("batch_order", ctypes.c_int)]


TUNING_FIELDS = ("region_h", "ctas_per_sm", "plane", "small_growth", "select_lanes", "batch_lag", "batch_order")


class HDError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {hd_status_str(status)} (status {status})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2005_05371_gb300/buildlib.py "
                          "(the denoiser has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    img_p = ctypes.POINTER(hd_image)
    par_p = ctypes.POINTER(hd_params)
    sig = {
        "amf_filter": ([img_p, P], I),
        "wiener_filter": ([img_p, P, S, P], I),
        "wiener_workspace_size": ([I, I, I, par_p, ctypes.POINTER(S)], I),
        "hybrid_denoise": ([img_p, P, S, P], I),
        "hybrid_workspace_size": ([I, I, I, par_p, ctypes.POINTER(S)], I),
        "hybrid_min_workspace_size": ([I, I, I, par_p, ctypes.POINTER(S)], I),
        "hybrid_denoise_host": ([img_p, P, S, P], I),
        "hybrid_host_workspace_size": ([I, I, I, par_p, ctypes.POINTER(S)], I),
        "hybrid_denoise_static": ([img_p, P], I),
        "hybrid_denoise_batched": ([img_p, I, P, S, P], I),
        "hybrid_batched_workspace_size": ([img_p, I, ctypes.POINTER(S)], I),
        "hd_batch_plan_create": ([img_p, I, P, S, ctypes.POINTER(P)], I),
        "hd_batch_plan_launch": ([P, P], I),
        "hd_batch_plan_destroy": ([P], I),
        "hd_set_tuning": ([ctypes.POINTER(hd_tuning)], I),
        "hd_get_tuning": ([ctypes.POINTER(hd_tuning)], I),
        "hd_set_spin_limit": ([ctypes.c_ulonglong], I),
        "hd_get_device_error": ([P], I),
        "contrast_stretch": ([img_p, ctypes.c_double, P, S, P], I),
        "hybrid_denoise_strips": ([img_p, I, P, S, P], I),
        "reference_noise_variance": ([P, S, P, S, I, I, I, P, P, S, P], I),
        "hd_host_pipeline_workspace_size": ([I, I, I, par_p, I, ctypes.POINTER(S)], I),
        "hd_host_pipeline_create": ([I, I, I, par_p, I, P, S, ctypes.POINTER(P)], I),
        "hd_host_pipeline_submit": ([P, P, S, P, S], I),
        "hd_host_pipeline_wait": ([P], I),
        "hd_host_pipeline_destroy": ([P], I),
        "hd_batch_pipeline_workspace_size": ([img_p, I, I, ctypes.POINTER(S)], I),
        "hd_batch_pipeline_create": ([img_p, I, I, P, S, ctypes.POINTER(P)], I),
        "hd_batch_pipeline_submit": ([P, ctypes.POINTER(P), ctypes.POINTER(S), ctypes.POINTER(P),
                                      ctypes.POINTER(S)], I),
        "hd_batch_pipeline_wait": ([P], I),
        "hd_batch_pipeline_destroy": ([P], I),
        "hd_part_halo_rows": ([par_p, ctypes.POINTER(I)], I),
        "wiener_deconv_workspace_size": ([I, I, ctypes.POINTER(S)], I),
        "wiener_deconvolve": ([img_p, P, I, I, ctypes.c_double, P, S, P], I),
        "hybrid_part_workspace_size": ([ctypes.POINTER(hd_part), ctypes.POINTER(S)], I),
        "hybrid_part_stats": ([ctypes.POINTER(hd_part), P, S, P, P], I),
        "hybrid_part_apply": ([ctypes.POINTER(hd_part), P, P, S, P], I),
        "hybrid_strips_workspace_size": ([I, I, I, par_p, I, ctypes.POINTER(S)], I),
        "contrast_workspace_size": ([I, I, I, par_p, ctypes.POINTER(S)], I),
        "hd_status_str": ([I], ctypes.c_char_p),
        "hd_version": ([], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def hd_status_str(status: int) -> str:
    return _lib.hd_status_str(int(status)).decode()


def hd_version() -> int:
    return _lib.hd_version()


def _check(status: int, what: str):
    if status != HD_OK:
        raise HDError(status, what)


# ----------------------------------------------------------------- helpers
@dataclass
class Params:
    """Filter parameters (mirrors hd_params)."""
    smax: int = 11
    wiener_w: int = 5
    noise_var: float = -1.0
    border: int = HD_BORDER_SYMMETRIC
    unresolved: int = HD_UNRESOLVED_ZMED
    bits: int | None = None
    wiener_h: int = 0          # Wiener window rows; 0: square (wiener_w)

    def to_c(self, dtype_code: int) -> hd_params:
        bits = self.bits if self.bits is not None else (8 if dtype_code == HD_U8 else 16)
        return hd_params(int(self.smax), int(self.wiener_w), float(self.noise_var), int(self.border),
                         int(self.unresolved), int(bits), int(self.wiener_h))


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.uint8:
        return HD_U8
    if t.dtype in (torch.uint16, torch.int16):
        return HD_U16
    raise TypeError(f"unsupported tensor dtype {t.dtype}: use uint8 or uint16")


def _pitch(t) -> int:
    if t.dim() != 2:
        raise ValueError("images are 2-D (H, W)")
    if t.stride(1) != 1:
        raise ValueError("image rows must be contiguous")
    return t.stride(0) * t.element_size()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_image(src, dst, params: Params, noise_var_out=None, y_out=None) -> hd_image:
    """hd_image for two CUDA tensors of the same dtype and shape."""
    if src.shape != dst.shape or src.dtype != dst.dtype:
        raise ValueError("src and dst must have the same shape and dtype")
    code = _dtype_code(src)
    H, W = src.shape
    return hd_image(src.data_ptr(), dst.data_ptr(), H, W, _pitch(src), _pitch(dst), code, params.to_c(code),
                    noise_var_out.data_ptr() if noise_var_out is not None else None,
                    y_out.data_ptr() if y_out is not None else None)


def _workspace(nbytes: int, device):
    if nbytes == 0:
        return None
    torch = _torch()
    # over-allocate so the pointer can be rounded up to 256 bytes; the library
    # wants a zero-filled workspace on first use and leaves it zeroed
    buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device=device)
    return buf


def _ws_ptr(buf) -> int | None:
    if buf is None:
        return None
    p = buf.data_ptr()
    return (p + 255) // 256 * 256


def _ws_len(buf) -> int:
    if buf is None:
        return 0
    p = buf.data_ptr()
    return buf.numel() - ((p + 255) // 256 * 256 - p)


# ----------------------------------------------------------------- stages
def amf_filter(src, dst, smax: int = 11, unresolved: int = HD_UNRESOLVED_ZMED, bits: int | None = None,
               stream=None):
    """Adaptive median filter (Algorithm 1, step 6) of ``src`` into ``dst``."""
    img = make_image(src, dst, Params(smax=smax, unresolved=unresolved, bits=bits))
    _check(_lib.amf_filter(ctypes.byref(img), _stream_ptr(stream)), "amf_filter")
    return dst


def hybrid_workspace_size(H: int, W: int, dtype_code: int, params: Params) -> int:
    n = ctypes.c_size_t()
    _check(_lib.hybrid_workspace_size(H, W, dtype_code, ctypes.byref(params.to_c(dtype_code)), ctypes.byref(n)),
           "hybrid_workspace_size")
    return n.value


def hybrid_min_workspace_size(H: int, W: int, dtype_code: int, params: Params) -> int:
    """Least workspace hybrid_denoise accepts (no statistics plane: slower path)."""
    n = ctypes.c_size_t()
    _check(_lib.hybrid_min_workspace_size(H, W, dtype_code, ctypes.byref(params.to_c(dtype_code)),
                                          ctypes.byref(n)), "hybrid_min_workspace_size")
    return n.value


def wiener_workspace_size(H: int, W: int, dtype_code: int, params: Params) -> int:
    n = ctypes.c_size_t()
    _check(_lib.wiener_workspace_size(H, W, dtype_code, ctypes.byref(params.to_c(dtype_code)), ctypes.byref(n)),
           "wiener_workspace_size")
    return n.value


def hybrid_host_workspace_size(H: int, W: int, dtype_code: int, params: Params) -> int:
    n = ctypes.c_size_t()
    _check(_lib.hybrid_host_workspace_size(H, W, dtype_code, ctypes.byref(params.to_c(dtype_code)),
                                           ctypes.byref(n)), "hybrid_host_workspace_size")
    return n.value


def wiener_filter(src, dst, wiener_w: int = 5, noise_var: float = -1.0, border: int = HD_BORDER_SYMMETRIC,
                  bits: int | None = None, workspace=None, noise_var_out=None, y_out=None, stream=None,
                  wiener_h: int = 0):
    """Local-statistics Wiener filter (Algorithm 1, step 4d) of ``src`` into
    ``dst`` over a window of ``wiener_h`` rows (0: square) by ``wiener_w`` columns."""
    p = Params(wiener_w=wiener_w, noise_var=noise_var, border=border, bits=bits, wiener_h=wiener_h)
    img = make_image(src, dst, p, noise_var_out, y_out)
    if workspace is None:
        workspace = _workspace(wiener_workspace_size(img.H, img.W, img.dtype, p), src.device)
    _check(_lib.wiener_filter(ctypes.byref(img), _ws_ptr(workspace), _ws_len(workspace), _stream_ptr(stream)),
           "wiener_filter")
    return dst


def hybrid_strips_workspace_size(H: int, W: int, dtype_code: int, params: Params, parts: int) -> int:
    n = ctypes.c_size_t()
    _check(_lib.hybrid_strips_workspace_size(H, W, dtype_code, ctypes.byref(params.to_c(dtype_code)), int(parts),
                                             ctypes.byref(n)), "hybrid_strips_workspace_size")
    return n.value


def hybrid_denoise_strips(src, dst, parts: int, smax: int = 11, wiener_w: int = 5, noise_var: float = -1.0,
                          border: int = HD_BORDER_SYMMETRIC, unresolved: int = HD_UNRESOLVED_ZMED,
                          bits: int | None = None, workspace=None, noise_var_out=None, y_out=None, stream=None):
    """Hybrid with the listing's partitioned median: ``parts`` row strips
    median-filtered alone, then the Wiener filter of the whole image
    (Algorithm 1, steps 4 and 6)."""
    p = Params(smax, wiener_w, noise_var, border, unresolved, bits)
    img = make_image(src, dst, p, noise_var_out, y_out)
    if workspace is None:
        workspace = _workspace(hybrid_strips_workspace_size(img.H, img.W, img.dtype, p, parts), src.device)
    _check(_lib.hybrid_denoise_strips(ctypes.byref(img), int(parts), _ws_ptr(workspace), _ws_len(workspace),
                                      _stream_ptr(stream)), "hybrid_denoise_strips")
    return dst


HD_REFNOISE_WORKSPACE_BYTES = 256


def reference_noise_variance(f, ref, out=None, workspace=None, stream=None):
    """Noise variance of ``f`` against the clean reference ``ref`` (Algorithm 1,
    step 4d): mean of (f - ref)^2, exact sum, one binary64 division.  Returns a
    one-element float64 CUDA tensor (``out`` if given)."""
    torch = _torch()
    if f.shape != ref.shape or f.dtype != ref.dtype:
        raise ValueError("f and ref must have the same shape and dtype")
    code = _dtype_code(f)
    H, W = f.shape
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=f.device)
    if workspace is None:
        workspace = _workspace(HD_REFNOISE_WORKSPACE_BYTES, f.device)
    _check(_lib.reference_noise_variance(f.data_ptr(), _pitch(f), ref.data_ptr(), _pitch(ref), H, W, code,
                                         out.data_ptr(), _ws_ptr(workspace), _ws_len(workspace),
                                         _stream_ptr(stream)), "reference_noise_variance")
    return out


def contrast_workspace_size(H: int, W: int, dtype_code: int, bits: int | None = None) -> int:
    n = ctypes.c_size_t()
    p = Params(bits=bits).to_c(dtype_code)
    _check(_lib.contrast_workspace_size(H, W, dtype_code, ctypes.byref(p), ctypes.byref(n)),
           "contrast_workspace_size")
    return n.value


def contrast_stretch(src, dst=None, tol: float = 0.01, bits: int | None = None, workspace=None, stream=None):
    """Contrast stretch (Algorithm 1, step 4e) of ``src`` into ``dst`` (in place when ``dst`` is None)."""
    if dst is None:
        dst = src
    img = make_image(src, dst, Params(bits=bits))
    if workspace is None:
        workspace = _workspace(contrast_workspace_size(img.H, img.W, img.dtype, bits), src.device)
    _check(_lib.contrast_stretch(ctypes.byref(img), float(tol), _ws_ptr(workspace), _ws_len(workspace),
                                 _stream_ptr(stream)), "contrast_stretch")
    return dst


def hybrid_denoise(src, dst, smax: int = 11, wiener_w: int = 5, noise_var: float = -1.0,
                   border: int = HD_BORDER_SYMMETRIC, unresolved: int = HD_UNRESOLVED_ZMED,
                   bits: int | None = None, workspace=None, noise_var_out=None, y_out=None, stream=None,
                   wiener_h: int = 0):
    """Hybrid denoise: Wiener(AdaptiveMedian(src)) into ``dst`` (Algorithm 1,
    step 4); the Wiener window is ``wiener_h`` rows (0: square) by ``wiener_w``."""
    p = Params(smax, wiener_w, noise_var, border, unresolved, bits, wiener_h)
    img = make_image(src, dst, p, noise_var_out, y_out)
    if workspace is None:
        workspace = _workspace(hybrid_workspace_size(img.H, img.W, img.dtype, p), src.device)
    _check(_lib.hybrid_denoise(ctypes.byref(img), _ws_ptr(workspace), _ws_len(workspace), _stream_ptr(stream)),
           "hybrid_denoise")
    return dst


def hybrid_denoise_host(src: np.ndarray, dst: np.ndarray, smax: int = 11, wiener_w: int = 5,
                        noise_var: float = -1.0, border: int = HD_BORDER_SYMMETRIC,
                        unresolved: int = HD_UNRESOLVED_ZMED, bits: int | None = None, workspace=None,
                        stream=None):
    """Hybrid denoise of HOST arrays (numpy or pinned CPU tensors): copies in, runs, copies out, waits."""
    def ptr_pitch(a):
        if isinstance(a, np.ndarray):
            if a.ndim != 2 or a.strides[1] != a.itemsize:
                raise ValueError("host image rows must be contiguous")
            return a.ctypes.data, a.strides[0], (HD_U8 if a.dtype == np.uint8 else HD_U16), a.shape
        return a.data_ptr(), _pitch(a), _dtype_code(a), tuple(a.shape)
    sp, spitch, code, shape = ptr_pitch(src)
    dp, dpitch, code2, shape2 = ptr_pitch(dst)
    if code != code2 or shape != shape2:
        raise ValueError("src and dst must have the same shape and dtype")
    p = Params(smax, wiener_w, noise_var, border, unresolved, bits)
    H, W = shape
    img = hd_image(sp, dp, H, W, spitch, dpitch, code, p.to_c(code), None, None)
    if workspace is None:
        workspace = _workspace(hybrid_host_workspace_size(H, W, code, p), "cuda")
    _check(_lib.hybrid_denoise_host(ctypes.byref(img), _ws_ptr(workspace), _ws_len(workspace),
                                    _stream_ptr(stream)), "hybrid_denoise_host")
    return dst


def _host_ptr_pitch(a):
    """(pointer, row pitch, dtype code, shape) of a host image: numpy array or CPU tensor."""
    if isinstance(a, np.ndarray):
        if a.ndim != 2 or a.strides[1] != a.itemsize:
            raise ValueError("host image rows must be contiguous")
        return a.ctypes.data, a.strides[0], (HD_U8 if a.dtype == np.uint8 else HD_U16), a.shape
    return a.data_ptr(), _pitch(a), _dtype_code(a), tuple(a.shape)


class HostPipeline:
    """Host-to-host hybrid of many images of one size (hd_host_pipeline_*):
    the copies of each step overlap the kernels of its neighbours.  ``submit``
    only enqueues; results are valid after ``wait``."""

    def __init__(self, H: int, W: int, dtype_code: int, params: Params, depth: int = 2, device="cuda"):
        self.H, self.W, self.code = H, W, dtype_code
        c = params.to_c(dtype_code)
        n = ctypes.c_size_t()
        _check(_lib.hd_host_pipeline_workspace_size(H, W, dtype_code, ctypes.byref(c), depth, ctypes.byref(n)),
               "hd_host_pipeline_workspace_size")
        self.workspace = _workspace(n.value, device)
        h = ctypes.c_void_p()
        _check(_lib.hd_host_pipeline_create(H, W, dtype_code, ctypes.byref(c), depth, _ws_ptr(self.workspace),
                                            _ws_len(self.workspace), ctypes.byref(h)), "hd_host_pipeline_create")
        self._h = h
        self._pending = []

    def submit(self, src, dst):
        sp, spitch, code, shape = _host_ptr_pitch(src)
        dp, dpitch, code2, shape2 = _host_ptr_pitch(dst)
        if code != self.code or code2 != self.code or tuple(shape) != (self.H, self.W) or tuple(shape2) != (self.H, self.W):
            raise ValueError("images must match the pipeline's size and dtype")
        self._pending.append((src, dst))          # keep the host buffers alive until wait()
        _check(_lib.hd_host_pipeline_submit(self._h, sp, spitch, dp, dpitch), "hd_host_pipeline_submit")

    def wait(self):
        _check(_lib.hd_host_pipeline_wait(self._h), "hd_host_pipeline_wait")
        self._pending.clear()

    def close(self):
        if self._h:
            _lib.hd_host_pipeline_destroy(self._h)
            self._h = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hybrid_denoise_static(src, dst, smax: int = 11, wiener_w: int = 5, noise_var: float = -1.0,
                          border: int = HD_BORDER_SYMMETRIC, unresolved: int = HD_UNRESOLVED_ZMED,
                          bits: int | None = None, noise_var_out=None, y_out=None, stream=None):
    """Hybrid denoise without any device allocation: scratch is a fixed array
    inside the library (for callers that cannot allocate device memory)."""
    p = Params(smax, wiener_w, noise_var, border, unresolved, bits)
    img = make_image(src, dst, p, noise_var_out, y_out)
    _check(_lib.hybrid_denoise_static(ctypes.byref(img), _stream_ptr(stream)), "hybrid_denoise_static")
    return dst


# ----------------------------------------------------------------- batches
def _image_array(items) -> ctypes.Array:
    """items: sequence of (src, dst, Params) or ready hd_image structs."""
    arr = (hd_image * len(items))()
    for i, it in enumerate(items):
        arr[i] = it if isinstance(it, hd_image) else make_image(*it)
    return arr


def hybrid_batched_workspace_size(items) -> int:
    arr = _image_array(items)
    n = ctypes.c_size_t()
    _check(_lib.hybrid_batched_workspace_size(arr, len(arr), ctypes.byref(n)), "hybrid_batched_workspace_size")
    return n.value


def hybrid_denoise_batched(items, workspace=None, stream=None):
    """Hybrid denoise of many images (uneven sizes, own parameters) in one persistent launch."""
    arr = _image_array(items)
    if workspace is None:
        n = ctypes.c_size_t()
        _check(_lib.hybrid_batched_workspace_size(arr, len(arr), ctypes.byref(n)), "hybrid_batched_workspace_size")
        workspace = _workspace(n.value, "cuda")
    _check(_lib.hybrid_denoise_batched(arr, len(arr), _ws_ptr(workspace), _ws_len(workspace),
                                       _stream_ptr(stream)), "hybrid_denoise_batched")
    return workspace


class BatchPlan:
    """hd_batch_plan: a batch fixed once and replayed as a CUDA graph."""

    def __init__(self, items, workspace=None):
        self._arr = _image_array(items)
        if workspace is None:
            n = ctypes.c_size_t()
            _check(_lib.hybrid_batched_workspace_size(self._arr, len(self._arr), ctypes.byref(n)),
                   "hybrid_batched_workspace_size")
            workspace = _workspace(n.value, "cuda")
        self.workspace = workspace
        self._plan = ctypes.c_void_p()
        _check(_lib.hd_batch_plan_create(self._arr, len(self._arr), _ws_ptr(workspace), _ws_len(workspace),
                                         ctypes.byref(self._plan)), "hd_batch_plan_create")

    def launch(self, stream=None):
        _check(_lib.hd_batch_plan_launch(self._plan, _stream_ptr(stream)), "hd_batch_plan_launch")

    def close(self):
        if self._plan:
            _lib.hd_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _shape_image(H: int, W: int, dtype_code: int, params: Params) -> hd_image:
    """hd_image carrying only a size, dtype and parameters (no buffers)."""
    es = 1 if dtype_code == HD_U8 else 2
    return hd_image(None, None, int(H), int(W), W * es, W * es, dtype_code, params.to_c(dtype_code), None, None)


class BatchPipeline:
    """Host-to-host batched hybrid (hd_batch_pipeline_*): the same batch of
    uneven images run step after step from host buffers, each step's copies
    overlapping its neighbours' kernels.  ``shapes`` is a list of
    (H, W, dtype_code, Params).  ``submit`` only enqueues; results are valid
    after ``wait``."""

    def __init__(self, shapes, depth: int = 2, device="cuda"):
        self._arr = (hd_image * len(shapes))()
        for i, (H, W, code, p) in enumerate(shapes):
            self._arr[i] = _shape_image(H, W, code, p)
        self.shapes = [(int(H), int(W), int(code)) for H, W, code, _ in shapes]
        n = ctypes.c_size_t()
        _check(_lib.hd_batch_pipeline_workspace_size(self._arr, len(self._arr), depth, ctypes.byref(n)),
               "hd_batch_pipeline_workspace_size")
        self.workspace = _workspace(n.value, device)
        h = ctypes.c_void_p()
        _check(_lib.hd_batch_pipeline_create(self._arr, len(self._arr), depth, _ws_ptr(self.workspace),
                                             _ws_len(self.workspace), ctypes.byref(h)), "hd_batch_pipeline_create")
        self._h = h
        self._pending = []

    def submit(self, srcs, dsts):
        """srcs / dsts: host images (numpy arrays or pinned CPU tensors), one per batch image."""
        n = len(self.shapes)
        if len(srcs) != n or len(dsts) != n:
            raise ValueError("one source and one destination per batch image")
        sp, spi = (ctypes.c_void_p * n)(), (ctypes.c_size_t * n)()
        dp, dpi = (ctypes.c_void_p * n)(), (ctypes.c_size_t * n)()
        for i, (a, b) in enumerate(zip(srcs, dsts)):
            p0, pitch0, c0, sh0 = _host_ptr_pitch(a)
            p1, pitch1, c1, sh1 = _host_ptr_pitch(b)
            H, W, code = self.shapes[i]
            if c0 != code or c1 != code or tuple(sh0) != (H, W) or tuple(sh1) != (H, W):
                raise ValueError(f"image {i} does not match the pipeline's size and dtype")
            sp[i], spi[i], dp[i], dpi[i] = p0, pitch0, p1, pitch1
        self._pending.append((srcs, dsts))        # keep the host buffers alive until wait()
        _check(_lib.hd_batch_pipeline_submit(self._h, sp, spi, dp, dpi), "hd_batch_pipeline_submit")

    def wait(self):
        _check(_lib.hd_batch_pipeline_wait(self._h), "hd_batch_pipeline_wait")
        self._pending.clear()

    def close(self):
        if self._h:
            _lib.hd_batch_pipeline_destroy(self._h)
            self._h = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- Fourier domain
HD_PSF_MAX = 255


def wiener_deconv_workspace_size(H: int, W: int) -> int:
    n = ctypes.c_size_t()
    _check(_lib.wiener_deconv_workspace_size(int(H), int(W), ctypes.byref(n)), "wiener_deconv_workspace_size")
    return n.value


def wiener_deconvolve(src, dst, psf, nsr: float, bits: int | None = None, workspace=None, y_out=None,
                      stream=None):
    """The Wiener filter in the Fourier domain (Section IV): deconvolution of
    ``src`` by the PSF (a float32 CUDA tensor, kh x kw) with noise-to-signal
    ratio ``nsr``, into ``dst`` (circular boundary)."""
    torch = _torch()
    if psf.dtype != torch.float32 or psf.dim() != 2 or not psf.is_contiguous():
        raise ValueError("psf must be a contiguous 2-D float32 tensor")
    img = make_image(src, dst, Params(bits=bits), None, y_out)
    if workspace is None:
        workspace = _workspace(wiener_deconv_workspace_size(img.H, img.W), src.device)
    _check(_lib.wiener_deconvolve(ctypes.byref(img), psf.data_ptr(), int(psf.shape[0]), int(psf.shape[1]),
                                  float(nsr), _ws_ptr(workspace), _ws_len(workspace), _stream_ptr(stream)),
           "wiener_deconvolve")
    return dst


# ----------------------------------------------------------------- image parts
def part_halo_rows(params: Params, dtype_code: int = HD_U8) -> int:
    """Rows of halo a part needs above and below its own rows: smax/2 + w/2."""
    n = ctypes.c_int()
    _check(_lib.hd_part_halo_rows(ctypes.byref(params.to_c(dtype_code)), ctypes.byref(n)), "hd_part_halo_rows")
    return n.value


def make_part(buf, dst, H: int, W: int, buf_row0: int, own_row0: int, own_rows: int, params: Params) -> hd_part:
    """hd_part for a buffer of rows [buf_row0, buf_row0 + len(buf)) of an H x W
    image and the part's own rows [own_row0, own_row0 + own_rows) (dst: their
    output, or None for the statistics call)."""
    code = _dtype_code(buf)
    return hd_part(buf.data_ptr(), _pitch(buf), dst.data_ptr() if dst is not None else None,
                   _pitch(dst) if dst is not None else 0, int(H), int(W), int(buf_row0), int(buf.shape[0]),
                   int(own_row0), int(own_rows), code, params.to_c(code))


def hybrid_part_workspace_size(part: hd_part) -> int:
    n = ctypes.c_size_t()
    _check(_lib.hybrid_part_workspace_size(ctypes.byref(part), ctypes.byref(n)), "hybrid_part_workspace_size")
    return n.value


def hybrid_part_stats(part: hd_part, workspace, sums_out, stream=None):
    """Median and local statistics of a part's own rows; its four sums into
    ``sums_out`` (a 4-element int64 CUDA tensor)."""
    _check(_lib.hybrid_part_stats(ctypes.byref(part), _ws_ptr(workspace), _ws_len(workspace), sums_out.data_ptr(),
                                  _stream_ptr(stream)), "hybrid_part_stats")
    return sums_out


def hybrid_part_apply(part: hd_part, sums, workspace, stream=None):
    """Wiener output of a part's own rows, with the sums of all parts."""
    _check(_lib.hybrid_part_apply(ctypes.byref(part), sums.data_ptr(), _ws_ptr(workspace), _ws_len(workspace),
                                  _stream_ptr(stream)), "hybrid_part_apply")


# ----------------------------------------------------------------- tuning / errors
def hd_set_tuning(region_h: int = 32, ctas_per_sm: int = 0, plane: int = 0, small_growth: int = 0,
                  select_lanes: int = 0, batch_lag: int = 0, batch_order: int = 0):
    """Work-item shape and scheduling knobs (see hd_tuning in the header):
    rows per work item (multiple of 8 in [16, 128]), CTAs per SM (0 = all that
    fit), statistics plane (0 = when there is room, its Wiener pass read from
    L2 or staged by the working set; 1 = never; 2 = staged; 3 = from L2), one-warp growth
    cut-over (0 = 32, -1 = never), lanes per median selection (0, 1, 2, 4, 8),
    batch Wiener lag in grids (0 = 6) and batch order (0 = the caller's, 1 = largest first)."""
    t = hd_tuning(region_h, ctas_per_sm, plane, small_growth, select_lanes, batch_lag, batch_order)
    _check(_lib.hd_set_tuning(ctypes.byref(t)), "hd_set_tuning")


def hd_get_tuning() -> tuple:
    """The current knobs, in the order hd_set_tuning takes them."""
    t = hd_tuning()
    _check(_lib.hd_get_tuning(ctypes.byref(t)), "hd_get_tuning")
    return tuple(getattr(t, f) for f in TUNING_FIELDS)


def hd_set_spin_limit(polls: int = 0):
    """Polls before a device-side wait gives up (0 restores the default of about 2 s)."""
    _check(_lib.hd_set_spin_limit(int(polls)), "hd_set_spin_limit")


def hd_get_device_error(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device error status."""
    return _lib.hd_get_device_error(_stream_ptr(stream))
