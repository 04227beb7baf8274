"""Thin ctypes binding of libradon (include/radon.h): argument marshalling only.

Every transform runs in the library's CUDA kernels; there is no CPU path.  Functions carry
the C names.  Device arrays are torch CUDA tensors (float32, contiguous) and the CUDA stream
defaults to torch's current stream on the tensor's device.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_c_int = ctypes.c_int
_c_void_p = ctypes.c_void_p


class radon_plan_info(ctypes.Structure):
    _fields_ = [
        ("N", _c_int), ("n_angles", _c_int), ("n_det", _c_int), ("interp_order", _c_int),
        ("n_partitions", _c_int), ("N_rho", _c_int), ("n_theta_half", _c_int), ("n_theta", _c_int),
        ("r", _c_int), ("n_quad", _c_int), ("n_filter", _c_int), ("column_group", _c_int),
        ("beta", ctypes.c_double), ("a_R", ctypes.c_double), ("a_r", ctypes.c_double), ("L", ctypes.c_double),
        ("d_phi", ctypes.c_double), ("d_rho", ctypes.c_double), ("d_s", ctypes.c_double),
        ("d_theta", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
    ]


RADON_OK = 0
RADON_FILTER_RAMP = 0
RADON_FILTER_SHEPP_LOGAN = 1
RADON_FILTER_COSINE = 2

EXPORTED = (
    "radon_plan_create", "radon_plan_destroy", "radon_plan_get_info", "radon_forward",
    "radon_backproject", "radon_fbp", "radon_forward_host", "radon_backproject_host",
    "radon_geometry", "radon_kernel_quadrant", "radon_status_string", "radon_profile_enable",
    "radon_profile_read", "radon_forward_static_scratch", "radon_plan_reserve_batch",
    "radon_forward_batch", "radon_backproject_batch", "radon_plan_set_column_group",
    "radon_plan_kernel_launches", "radon_transpose", "radon_transpose_batch", "radon_forward_multi",
    "radon_backproject_multi",
)

RADON_NUM_STAGES = 18
STAGE_NAMES = (
    "prefilter_image", "rows_fwd", "columns_fwd", "rows_inv_fwd", "gather_sino",
    "prefilter_sino", "rows_bp", "columns_bp", "rows_inv_bp", "gather_image", "sino_filter",
    "sample_fwd", "scatter_sino_t", "rows_t", "columns_t", "rows_inv_t", "scatter_image_t", "prefilter_t",
)
TRANSPOSE_STAGES = STAGE_NAMES[12:]

_lib = None


class RadonError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {radon_status_string(status)} (status {status})")


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libradon.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libradon.so not found at {path}; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.radon_plan_create.argtypes = [P(_c_void_p), _c_int, _c_int, _c_int, _c_int, _c_int]
    lib.radon_plan_destroy.argtypes = [_c_void_p]
    lib.radon_plan_destroy.restype = None
    lib.radon_plan_get_info.argtypes = [_c_void_p, P(radon_plan_info)]
    for name in ("radon_forward", "radon_backproject", "radon_forward_host", "radon_backproject_host",
                 "radon_forward_static_scratch", "radon_transpose"):
        getattr(lib, name).argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p]
    lib.radon_fbp.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_int, _c_void_p]
    lib.radon_geometry.argtypes = [_c_int, _c_int, _c_int, _c_int, _c_int, P(radon_plan_info)]
    lib.radon_kernel_quadrant.argtypes = [_c_int, _c_int, _c_int, _c_int, _c_int, P(ctypes.c_double)]
    lib.radon_plan_reserve_batch.argtypes = [_c_void_p, _c_int]
    lib.radon_plan_set_column_group.argtypes = [_c_void_p, _c_int]
    lib.radon_plan_kernel_launches.argtypes = [_c_void_p, _c_int, P(_c_int)]
    for name in ("radon_forward_batch", "radon_backproject_batch", "radon_transpose_batch"):
        getattr(lib, name).argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_int, _c_void_p]
    for name in ("radon_forward_multi", "radon_backproject_multi"):
        getattr(lib, name).argtypes = [P(_c_void_p), P(_c_void_p), P(_c_void_p), _c_int, _c_void_p]
    lib.radon_profile_enable.argtypes = [_c_void_p, _c_int]
    lib.radon_profile_read.argtypes = [_c_void_p, P(ctypes.c_double), P(_c_int)]
    lib.radon_status_string.argtypes = [_c_int]
    lib.radon_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("radon_plan_destroy", "radon_status_string"):
            getattr(lib, name).restype = _c_int
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != RADON_OK:
        raise RadonError(status, what)


def radon_status_string(status: int) -> str:
    return load().radon_status_string(int(status)).decode()


def _info_dict(info: radon_plan_info) -> dict:
    return {name: getattr(info, name) for name, _ in info._fields_}


def radon_geometry(N: int, n_angles: int, n_det: int, interp_order: int = 3, n_partitions: int = 3) -> dict:
    info = radon_plan_info()
    _check(load().radon_geometry(N, n_angles, n_det, interp_order, n_partitions, ctypes.byref(info)), "radon_geometry")
    return _info_dict(info)


def radon_kernel_quadrant(N: int, n_angles: int, n_det: int, n_partitions: int, which: int) -> np.ndarray:
    g = radon_geometry(N, n_angles, n_det, 3, n_partitions)
    nkt, nkr = g["n_theta"] // 2 + 1, g["N_rho"] // 2 + 1
    out = np.zeros(2 * nkt * nkr, dtype=np.float64)
    _check(load().radon_kernel_quadrant(N, n_angles, n_det, n_partitions, which,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "radon_kernel_quadrant")
    return (out[0::2] + 1j * out[1::2]).reshape(nkt, nkr)


class RadonPlan:
    """Owns a radon_plan handle (destroyed with the object)."""

    def __init__(self, handle: int, info: dict):
        self.handle = handle
        self.info = info
        self.max_batch = 1  # slices one batched call may take (radon_plan_reserve_batch)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.radon_plan_destroy(h)

    @property
    def image_shape(self):
        return (self.info["N"], self.info["N"])

    @property
    def sino_shape(self):
        return (self.info["n_angles"], self.info["n_det"])


def radon_plan_create(N: int, n_angles: int, n_det: int, interp_order: int = 3, n_partitions: int = 3) -> RadonPlan:
    lib = load()
    h = _c_void_p()
    _check(lib.radon_plan_create(ctypes.byref(h), N, n_angles, n_det, interp_order, n_partitions), "radon_plan_create")
    info = radon_plan_info()
    _check(lib.radon_plan_get_info(h, ctypes.byref(info)), "radon_plan_get_info")
    return RadonPlan(h.value, _info_dict(info))


def radon_plan_destroy(plan: RadonPlan):
    h, plan.handle = plan.handle, None
    if h:
        load().radon_plan_destroy(h)


def radon_plan_get_info(plan: RadonPlan) -> dict:
    info = radon_plan_info()
    _check(load().radon_plan_get_info(plan.handle, ctypes.byref(info)), "radon_plan_get_info")
    return _info_dict(info)


def _dev(t, shape, name):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _stream(stream, tensor):
    import torch

    if stream is None:
        return torch.cuda.current_stream(tensor.device).cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def radon_forward(plan: RadonPlan, image, sino, stream=None):
    _check(load().radon_forward(plan.handle, _dev(image, plan.image_shape, "image"),
                                _dev(sino, plan.sino_shape, "sino"), _stream(stream, image)), "radon_forward")
    return sino


def radon_forward_static_scratch(plan: RadonPlan, image, sino, stream=None):
    """radon_forward with the intermediates in the library's static device array (no allocation)."""
    _check(load().radon_forward_static_scratch(plan.handle, _dev(image, plan.image_shape, "image"),
                                               _dev(sino, plan.sino_shape, "sino"), _stream(stream, image)),
           "radon_forward_static_scratch")
    return sino


def radon_backproject(plan: RadonPlan, sino, image, stream=None):
    _check(load().radon_backproject(plan.handle, _dev(sino, plan.sino_shape, "sino"),
                                    _dev(image, plan.image_shape, "image"), _stream(stream, sino)), "radon_backproject")
    return image


def radon_transpose(plan: RadonPlan, sino, image, stream=None):
    """R^T, the exact transpose of radon_forward's discrete map (not R#)."""
    _check(load().radon_transpose(plan.handle, _dev(sino, plan.sino_shape, "sino"),
                                  _dev(image, plan.image_shape, "image"), _stream(stream, sino)), "radon_transpose")
    return image


def radon_fbp(plan: RadonPlan, sino, image, filter: int = RADON_FILTER_RAMP, stream=None):
    _check(load().radon_fbp(plan.handle, _dev(sino, plan.sino_shape, "sino"), _dev(image, plan.image_shape, "image"),
                            int(filter), _stream(stream, sino)), "radon_fbp")
    return image


def _host(a, shape, name):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous or a.shape != tuple(shape):
            raise TypeError(f"{name} must be a C-contiguous float32 array of shape {tuple(shape)}")
        return a.ctypes.data
    import torch

    if not (isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 host tensor or array")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")
    return a.data_ptr()


def radon_forward_host(plan: RadonPlan, h_image, h_sino, stream=None):
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load().radon_forward_host(plan.handle, _host(h_image, plan.image_shape, "image"),
                                     _host(h_sino, plan.sino_shape, "sino"), s), "radon_forward_host")
    return h_sino


def radon_backproject_host(plan: RadonPlan, h_sino, h_image, stream=None):
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load().radon_backproject_host(plan.handle, _host(h_sino, plan.sino_shape, "sino"),
                                         _host(h_image, plan.image_shape, "image"), s), "radon_backproject_host")
    return h_image


def radon_profile_enable(plan: RadonPlan, enable: bool = True):
    _check(load().radon_profile_enable(plan.handle, int(bool(enable))), "radon_profile_enable")


def radon_profile_read(plan: RadonPlan):
    """Per-stage (total ms, launches) accumulated since the last read, keyed by stage name."""
    ms = (ctypes.c_double * RADON_NUM_STAGES)()
    n = (_c_int * RADON_NUM_STAGES)()
    _check(load().radon_profile_read(plan.handle, ms, n), "radon_profile_read")
    return {STAGE_NAMES[i]: (ms[i], n[i]) for i in range(RADON_NUM_STAGES)}


def radon_plan_kernel_launches(plan: RadonPlan, op: str) -> int:
    """Kernels one call of op ("forward", "backproject", "fbp" or "transpose") launches."""
    n = _c_int()
    code = {"forward": 0, "backproject": 1, "fbp": 2, "transpose": 3}[op]
    _check(load().radon_plan_kernel_launches(plan.handle, code, ctypes.byref(n)), "radon_plan_kernel_launches")
    return n.value


def radon_plan_reserve_batch(plan: RadonPlan, max_batch: int):
    _check(load().radon_plan_reserve_batch(plan.handle, int(max_batch)), "radon_plan_reserve_batch")
    plan.info = radon_plan_get_info(plan)
    plan.max_batch = max(plan.max_batch, int(max_batch))


def radon_plan_set_column_group(plan: RadonPlan, group: int):
    _check(load().radon_plan_set_column_group(plan.handle, int(group)), "radon_plan_set_column_group")
    plan.info = radon_plan_get_info(plan)


def radon_forward_batch(plan: RadonPlan, images, sinos, stream=None):
    """images [B, N, N] -> sinos [B, n_angles, n_det] (contiguous float32 CUDA tensors)."""
    b = images.shape[0]
    _check(load().radon_forward_batch(plan.handle, _dev(images, (b,) + plan.image_shape, "images"),
                                      _dev(sinos, (b,) + plan.sino_shape, "sinos"), b, _stream(stream, images)),
           "radon_forward_batch")
    return sinos


def radon_backproject_batch(plan: RadonPlan, sinos, images, stream=None):
    """sinos [B, n_angles, n_det] -> images [B, N, N] (contiguous float32 CUDA tensors)."""
    b = sinos.shape[0]
    _check(load().radon_backproject_batch(plan.handle, _dev(sinos, (b,) + plan.sino_shape, "sinos"),
                                          _dev(images, (b,) + plan.image_shape, "images"), b, _stream(stream, sinos)),
           "radon_backproject_batch")
    return images


def _multi(name: str, plans, ins, outs, in_shape, out_shape, stream):
    n = len(plans)
    if len(ins) != n or len(outs) != n:
        raise ValueError(f"{name}: plans, inputs and outputs differ in length")
    arr_p = (ctypes.c_void_p * n)(*[pl.handle for pl in plans])
    arr_i = (ctypes.c_void_p * n)(*[_dev(t, in_shape(pl), "input") for pl, t in zip(plans, ins)])
    arr_o = (ctypes.c_void_p * n)(*[_dev(t, out_shape(pl), "output") for pl, t in zip(plans, outs)])
    st = _stream(stream, ins[0]) if n else None
    _check(getattr(load(), name)(arr_p, arr_i, arr_o, n, st), name)
    return outs


def radon_forward_multi(plans, images, sinos, stream=None):
    """Slice i: images[i] -> sinos[i] with plans[i] (plans may differ in size), one stream."""
    return _multi("radon_forward_multi", plans, images, sinos, lambda pl: pl.image_shape, lambda pl: pl.sino_shape,
                  stream)


def radon_backproject_multi(plans, sinos, images, stream=None):
    """Slice i: sinos[i] -> images[i] with plans[i] (plans may differ in size), one stream."""
    return _multi("radon_backproject_multi", plans, sinos, images, lambda pl: pl.sino_shape,
                  lambda pl: pl.image_shape, stream)


def radon_transpose_batch(plan: RadonPlan, sinos, images, stream=None):
    """sinos [B, n_angles, n_det] -> images [B, N, N]: R^T of each slice."""
    b = sinos.shape[0]
    _check(load().radon_transpose_batch(plan.handle, _dev(sinos, (b,) + plan.sino_shape, "sinos"),
                                        _dev(images, (b,) + plan.image_shape, "images"), b, _stream(stream, sinos)),
           "radon_transpose_batch")
    return images
