"""Thin ctypes binding of libdic (include/dic.h): the same calls under the same
names, with argument marshalling only. Every step of the correlation runs in the
library's CUDA kernels; there is no Python or CPU fallback, and loading fails
loudly if the compiled library is missing."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdic.so")

DIC_OK, DIC_EINVAL, DIC_ENOMEM, DIC_ECUDA, DIC_ETIMEOUT, DIC_ENOSEED, DIC_ESTATE = 0, -1, -2, -3, -4, -5, -6
DIC_U8, DIC_U16, DIC_BF16, DIC_F32, DIC_F64 = range(5)
DIC_RIGID, DIC_AFFINE, DIC_QUADRATIC = range(3)
DIC_BSPLINE3, DIC_BICUBIC = 0, 1
INTERPS = {"bspline3": DIC_BSPLINE3, "bicubic": DIC_BICUBIC}
DIC_FP64, DIC_MIXED, DIC_MIXED_FP64_SOLVE = 0, 1, 2
PRECISIONS = {"fp64": DIC_FP64, "mixed": DIC_MIXED, "mixed_fp64_solve": DIC_MIXED_FP64_SOLVE}
DIC_COST_ZNSSD, DIC_COST_NSSD, DIC_COST_SSD = 0, 1, 2
COSTS = {"znssd": DIC_COST_ZNSSD, "nssd": DIC_COST_NSSD, "ssd": DIC_COST_SSD}
DIC_OPT_GAUSS_NEWTON, DIC_OPT_LEVENBERG_MARQUARDT = 0, 1
OPTIMIZERS = {"gn": DIC_OPT_GAUSS_NEWTON, "lm": DIC_OPT_LEVENBERG_MARQUARDT}
DIC_INIT_SEARCH, DIC_INIT_FFT = 0, 1
INITS = {"search": DIC_INIT_SEARCH, "fft": DIC_INIT_FFT}
(PT_OK, PT_NOT_IN_ROI, PT_NOT_REACHED, PT_OUT_OF_BOUNDS, PT_MAX_ITER, PT_LOW_ZNCC, PT_SINGULAR,
 PT_FLAT) = range(8)
SHAPES = {"rigid": DIC_RIGID, "affine": DIC_AFFINE, "quadratic": DIC_QUADRATIC}
DIC_STRAIN_BILINEAR, DIC_STRAIN_BIQUADRATIC = 0, 1
DIC_GREEN_LAGRANGE, DIC_HENCKY, DIC_EULER_ALMANSI, DIC_BIOT_RIGHT, DIC_BIOT_LEFT = range(5)
STRAIN_BASES = {"bilinear": DIC_STRAIN_BILINEAR, "biquadratic": DIC_STRAIN_BIQUADRATIC}
STRAIN_MEASURES = {"green_lagrange": DIC_GREEN_LAGRANGE, "hencky": DIC_HENCKY,
                   "euler_almansi": DIC_EULER_ALMANSI, "biot_right": DIC_BIOT_RIGHT, "biot_left": DIC_BIOT_LEFT}
STRAIN_FIELDS = ("dudx", "dudy", "dvdx", "dvdy", "exx", "eyy", "exy", "valid")
N_PARAMS = {DIC_RIGID: 2, DIC_AFFINE: 6, DIC_QUADRATIC: 12}

# every function declared in include/dic.h
EXPORTS = ("dic_default_params", "dic_create", "dic_set_params", "dic_get_params",
           "dic_set_reference", "dic_set_deformed", "dic_correlate", "dic_get_results",
           "dic_get_coefficients", "dic_get_timing", "dic_destroy", "dic_last_error",
           "dic_correlate_static", "dic_correlate_sequence", "dic_set_subsets",
           "dic_estimate_device_bytes", "dic_estimate_regrid_bytes", "dic_get_device_bytes",
           "dic_strain_field", "dic_fft_default_params", "dic_fft_field", "dic_get_fft_results",
           "dic_fftcc_windows", "dic_mad_filter", "dic_update_reference", "dic_get_total_results",
           "dic_test_expire_tile_waits")


class DicImage(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("row_stride_bytes", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("on_device", ctypes.c_int32)]


class DicParams(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("search_radius", ctypes.c_int32),
                ("conv_threshold", ctypes.c_double), ("zncc_min", ctypes.c_double),
                ("precision", ctypes.c_int32), ("nan_unconverged", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("cost", ctypes.c_int32),
                ("optimizer", ctypes.c_int32), ("init", ctypes.c_int32),
                ("max_displacement", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mad_tau", ctypes.c_double), ("mad_eps", ctypes.c_double)]


class DicTotalResults(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("n_params", ctypes.c_int32), ("n_updates", ctypes.c_int32),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class DicFftParams(ctypes.Structure):
    _fields_ = [("max_displacement", ctypes.c_int32), ("subpixel", ctypes.c_int32),
                ("mad_tau", ctypes.c_double), ("mad_eps", ctypes.c_double)]


class DicFftResults(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("window", ctypes.c_int32 * 16),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("peak", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("replaced", ctypes.c_void_p)]


class DicResults(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("n_params", ctypes.c_int32), ("n_waves", ctypes.c_int32),
                ("n_accepted", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("p", ctypes.c_void_p), ("zncc", ctypes.c_void_p),
                ("iters", ctypes.c_void_p), ("converged", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("wave", ctypes.c_void_p)]


class DicTiming(ctypes.Structure):
    _fields_ = [("prefilter_ms", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("waves_ms", ctypes.c_double), ("icgn_kernel_ms", ctypes.c_double),
                ("seed_kernel_ms", ctypes.c_double), ("n_wave_launches", ctypes.c_int32),
                ("n_waves", ctypes.c_int32), ("n_points_attempted", ctypes.c_int64),
                ("sum_sample_passes", ctypes.c_int64)]


class DicStaticOutputs(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("zncc", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("converged", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("wave", ctypes.c_void_p), ("n_accepted", ctypes.c_void_p)]


class DicStrainOutputs(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in STRAIN_FIELDS]


class DicError(RuntimeError):
    def __init__(self, code, message):
        super().__init__("libdic error %d: %s" % (code, message))
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """The compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libdic.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.dic_default_params.argtypes = []
    lib.dic_default_params.restype = DicParams
    lib.dic_create.argtypes = [P(DicImage), P(DicImage), P(DicImage), ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_int32, P(vp)]
    lib.dic_create.restype = ctypes.c_int
    lib.dic_set_params.argtypes = [vp, P(DicParams)]
    lib.dic_set_params.restype = ctypes.c_int
    lib.dic_get_params.argtypes = [vp, P(DicParams)]
    lib.dic_get_params.restype = ctypes.c_int
    lib.dic_set_reference.argtypes = [vp, P(DicImage)]
    lib.dic_set_reference.restype = ctypes.c_int
    lib.dic_set_deformed.argtypes = [vp, P(DicImage)]
    lib.dic_set_deformed.restype = ctypes.c_int
    lib.dic_correlate.argtypes = [vp, P(ctypes.c_int32), ctypes.c_int32, vp]
    lib.dic_correlate.restype = ctypes.c_int
    lib.dic_correlate_sequence.argtypes = [vp, vp]
    lib.dic_correlate_sequence.restype = ctypes.c_int
    lib.dic_get_results.argtypes = [vp, P(DicResults), ctypes.c_int32]
    lib.dic_get_results.restype = ctypes.c_int
    lib.dic_get_coefficients.argtypes = [vp, ctypes.c_int32, P(vp), P(ctypes.c_int64),
                                         P(ctypes.c_int32)]
    lib.dic_get_coefficients.restype = ctypes.c_int
    lib.dic_get_timing.argtypes = [vp, P(DicTiming)]
    lib.dic_get_timing.restype = ctypes.c_int
    lib.dic_destroy.argtypes = [vp]
    lib.dic_destroy.restype = None
    lib.dic_last_error.argtypes = []
    lib.dic_last_error.restype = ctypes.c_char_p
    lib.dic_test_expire_tile_waits.argtypes = [ctypes.c_int32]
    lib.dic_test_expire_tile_waits.restype = ctypes.c_int
    lib.dic_correlate_static.argtypes = [P(DicImage), P(DicImage), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, P(DicParams), P(ctypes.c_int32), ctypes.c_int32,
                                         P(DicStaticOutputs), vp, ctypes.c_char_p, ctypes.c_int32]
    lib.dic_correlate_static.restype = ctypes.c_int
    lib.dic_set_subsets.argtypes = [vp, P(DicImage), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.dic_set_subsets.restype = ctypes.c_int
    lib.dic_estimate_device_bytes.argtypes = [P(DicImage), P(DicImage), ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, P(DicParams), ctypes.c_int32,
                                              P(ctypes.c_int64)]
    lib.dic_estimate_device_bytes.restype = ctypes.c_int
    lib.dic_estimate_regrid_bytes.argtypes = [vp, P(DicImage), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, P(DicParams), ctypes.c_int32, P(ctypes.c_int64)]
    lib.dic_estimate_regrid_bytes.restype = ctypes.c_int
    lib.dic_strain_field.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, P(DicStrainOutputs), vp]
    lib.dic_strain_field.restype = ctypes.c_int
    lib.dic_get_device_bytes.argtypes = [vp, P(ctypes.c_int64)]
    lib.dic_update_reference.argtypes = [vp, vp]
    lib.dic_update_reference.restype = ctypes.c_int
    lib.dic_get_total_results.argtypes = [vp, P(DicTotalResults), vp]
    lib.dic_get_total_results.restype = ctypes.c_int
    lib.dic_fft_default_params.argtypes = []
    lib.dic_fft_default_params.restype = DicFftParams
    lib.dic_fft_field.argtypes = [vp, P(DicFftParams), vp]
    lib.dic_fft_field.restype = ctypes.c_int
    lib.dic_get_fft_results.argtypes = [vp, P(DicFftResults)]
    lib.dic_get_fft_results.restype = ctypes.c_int
    lib.dic_fftcc_windows.argtypes = [vp, ctypes.c_int32, ctypes.c_int64, vp, ctypes.c_int32, vp, vp, vp, vp]
    lib.dic_fftcc_windows.restype = ctypes.c_int
    lib.dic_mad_filter.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                   vp, vp, vp, vp]
    lib.dic_mad_filter.restype = ctypes.c_int
    lib.dic_get_device_bytes.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc):
    if rc != DIC_OK:
        raise DicError(rc, load().dic_last_error().decode(errors="replace"))


_NP_DTYPES = {np.dtype(np.uint8): DIC_U8, np.dtype(np.uint16): DIC_U16,
              np.dtype(np.float32): DIC_F32, np.dtype(np.float64): DIC_F64}


def make_image(arr, bf16: bool = False) -> tuple:
    """dic_image for a 2-D numpy array (host, copied by the library) or a 2-D CUDA
    tensor (device, borrowed). torch.int16 / uint16 tensors are read as DIC_U16,
    torch.bfloat16 as DIC_BF16. Returns (image, keep-alive object)."""
    if isinstance(arr, np.ndarray):
        if arr.ndim != 2:
            raise ValueError("images are 2-D")
        a = arr if arr.strides[1] == arr.itemsize else np.ascontiguousarray(arr)
        dt = _NP_DTYPES.get(a.dtype)
        if dt is None:
            raise ValueError("unsupported image dtype %s" % a.dtype)
        return DicImage(a.ctypes.data, a.shape[1], a.shape[0], a.strides[0], dt, 0), a
    import torch

    t = arr
    if t.dim() != 2 or not t.is_cuda or t.stride(1) != 1:
        raise ValueError("device images are 2-D CUDA tensors with contiguous rows")
    dt = image_dtype_code(t)
    return DicImage(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0) * t.element_size(), dt, 1), t


def dic_default_params() -> DicParams:
    return load().dic_default_params()


def dic_create(ref, deformed, roi, subset_size, subset_step, shape_fn, interp=DIC_BSPLINE3):
    lib = load()
    ri, rk = make_image(ref)
    di, dk = make_image(deformed)
    mi, mask = _roi_image(roi)
    h = ctypes.c_void_p()
    _check(lib.dic_create(ctypes.byref(ri), ctypes.byref(di), ctypes.byref(mi) if mask is not None else None,
                          subset_size, subset_step, shape_fn, interp, ctypes.byref(h)))
    return h, (rk, dk)


def _roi_image(roi):
    if roi is None:
        return None, None
    if isinstance(roi, np.ndarray):
        roi = np.ascontiguousarray(roi.astype(np.uint8))
    return make_image(roi)


def dic_set_subsets(h, roi, subset_size, subset_step, shape_fn):
    mi, keep = _roi_image(roi)
    _check(load().dic_set_subsets(h, ctypes.byref(mi) if mi is not None else None, subset_size, subset_step,
                                  shape_fn))


def image_desc(width, height, dtype, on_device) -> DicImage:
    """A dic_image that describes an image without data (for dic_estimate_device_bytes)."""
    return DicImage(None, width, height, 0, dtype, 1 if on_device else 0)


def image_dtype_code(arr) -> int:
    """The dic_dtype of a numpy array or CUDA tensor, as make_image reads it."""
    if isinstance(arr, np.ndarray):
        dt = _NP_DTYPES.get(arr.dtype)
        if dt is None:
            raise ValueError("unsupported image dtype %s" % arr.dtype)
        return dt
    import torch

    kinds = {torch.uint8: DIC_U8, torch.int16: DIC_U16, torch.bfloat16: DIC_BF16,
             torch.float32: DIC_F32, torch.float64: DIC_F64}
    if hasattr(torch, "uint16"):
        kinds[torch.uint16] = DIC_U16
    if arr.dtype not in kinds:
        raise ValueError("unsupported tensor dtype %s" % arr.dtype)
    return kinds[arr.dtype]


def dic_estimate_device_bytes(ref: DicImage, deformed: DicImage, has_roi, subset_size, subset_step, shape_fn,
                              prm: DicParams, n_seeds) -> int:
    out = ctypes.c_int64(0)
    _check(load().dic_estimate_device_bytes(ctypes.byref(ref), ctypes.byref(deformed), 1 if has_roi else 0,
                                            subset_size, subset_step, shape_fn, ctypes.byref(prm), n_seeds,
                                            ctypes.byref(out)))
    return out.value


def dic_estimate_regrid_bytes(h, deformed: DicImage, has_roi, subset_size, subset_step, shape_fn,
                              prm: DicParams, n_seeds) -> int:
    out = ctypes.c_int64(0)
    _check(load().dic_estimate_regrid_bytes(h, ctypes.byref(deformed), 1 if has_roi else 0, subset_size,
                                            subset_step, shape_fn, ctypes.byref(prm), n_seeds, ctypes.byref(out)))
    return out.value


def dic_get_device_bytes(h) -> int:
    out = ctypes.c_int64(0)
    _check(load().dic_get_device_bytes(h, ctypes.byref(out)))
    return out.value


def dic_set_params(h, params: DicParams):
    _check(load().dic_set_params(h, ctypes.byref(params)))


def dic_get_params(h) -> DicParams:
    p = DicParams()
    _check(load().dic_get_params(h, ctypes.byref(p)))
    return p


def dic_set_reference(h, ref):
    im, keep = make_image(ref)
    _check(load().dic_set_reference(h, ctypes.byref(im)))
    return keep


def dic_set_deformed(h, deformed):
    im, keep = make_image(deformed)
    _check(load().dic_set_deformed(h, ctypes.byref(im)))
    return keep


def dic_correlate(h, seeds, stream_ptr: int = 0):
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).reshape(-1, 2))
    _check(load().dic_correlate(h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), s.shape[0],
                                ctypes.c_void_p(stream_ptr)))


def dic_correlate_sequence(h, stream_ptr: int = 0):
    _check(load().dic_correlate_sequence(h, ctypes.c_void_p(stream_ptr)))


def _host_array(ptr, count, dtype, copy=True):
    if count == 0:
        return np.zeros(0, dtype)
    buf = (ctypes.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr)
    a = np.frombuffer(buf, dtype=dtype, count=count)
    return a.copy() if copy else a


class _DeviceArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=shape, typestr=typestr, data=(ptr, False),
                                             version=3, strides=None)


def dic_get_results(h, on_device: bool = False, copy: bool = True) -> dict:
    """Per-point arrays in grid order: numpy arrays (host) or zero-copy CUDA tensors
    viewing the handle's buffers (device; valid until the next correlate/destroy).
    Host arrays are copies, or with copy=False views of the handle's pinned host
    buffers (valid until the next dic_get_results, correlate or destroy)."""
    r = DicResults()
    _check(load().dic_get_results(h, ctypes.byref(r), 1 if on_device else 0))
    n, npar = r.n_points, r.n_params
    spec = [("x", np.int32, (n,)), ("y", np.int32, (n,)), ("u", np.float64, (n,)),
            ("v", np.float64, (n,)), ("p", np.float64, (n, npar)), ("zncc", np.float32, (n,)),
            ("iters", np.int32, (n,)), ("converged", np.uint8, (n,)), ("status", np.uint8, (n,)),
            ("wave", np.int32, (n,))]
    out = dict(n_points=n, nx=r.nx, ny=r.ny, n_params=npar, n_waves=r.n_waves,
               n_accepted=r.n_accepted)
    if on_device:
        import torch

        for name, dt, shape in spec:
            out[name] = torch.as_tensor(_DeviceArray(getattr(r, name), shape, np.dtype(dt).str),
                                        device="cuda")
    else:
        for name, dt, shape in spec:
            out[name] = _host_array(getattr(r, name), int(np.prod(shape)), dt, copy).reshape(shape)
    return out


def dic_get_coefficients(h, which: int):
    """The coefficient plane as a zero-copy CUDA tensor view [height, ld]."""
    import torch

    ptr = ctypes.c_void_p()
    ld = ctypes.c_int64()
    es = ctypes.c_int32()
    _check(load().dic_get_coefficients(h, which, ctypes.byref(ptr), ctypes.byref(ld), ctypes.byref(es)))
    return ptr.value, ld.value, es.value


def dic_get_timing(h) -> dict:
    t = DicTiming()
    _check(load().dic_get_timing(h, ctypes.byref(t)))
    return {name: getattr(t, name) for name, _ in DicTiming._fields_}


def dic_destroy(h):
    if h is not None and h.value:
        load().dic_destroy(h)


def dic_test_expire_tile_waits(on: bool):
    """Test hook: tile-load waits of later wave launches give up at once (True) or
    run normally (False)."""
    _check(load().dic_test_expire_tile_waits(1 if on else 0))


def dic_last_error() -> str:
    return load().dic_last_error().decode(errors="replace")


def _device_output(t, name: str, dtype, count: int):
    """Raises DicError unless t is a contiguous CUDA tensor of the current device with
    the given dtype and at least count elements: the C side receives only the raw
    pointer and writes count elements through it."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise DicError(DIC_EINVAL, "output %s is not a tensor" % name)
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise DicError(DIC_EINVAL, "output %s must be a CUDA tensor of the current device" % name)
    if t.dtype != dtype:
        raise DicError(DIC_EINVAL, "output %s has dtype %s, %s is needed" % (name, t.dtype, dtype))
    if not t.is_contiguous():
        raise DicError(DIC_EINVAL, "output %s must be contiguous" % name)
    if t.numel() < count:
        raise DicError(DIC_EINVAL, "output %s holds %d elements, %d are needed" % (name, t.numel(), count))


def grid_size(width: int, height: int, subset_size: int, subset_step: int) -> tuple:
    """(nx, ny) of the subset grid: centres r + k step, n = (side - 1 - 2r) // step + 1."""
    r = (subset_size - 1) // 2
    return (width - 1 - 2 * r) // subset_step + 1, (height - 1 - 2 * r) // subset_step + 1


def dic_correlate_static(ref, deformed, subset_size, subset_step, shape_fn, prm: DicParams, seeds,
                         out: dict, stream_ptr: int = 0) -> int:
    """Allocation-free correlation into caller-owned CUDA tensors ``out`` (keys u, v,
    p, zncc, iters, converged, status, wave); returns the accepted-point count. Every
    output is checked against the grid size before the call."""
    import torch

    ri, rk = make_image(ref)
    di, dk = make_image(deformed)
    if 3 <= subset_size <= min(ri.width, ri.height) and subset_step >= 1 and shape_fn in N_PARAMS:
        nx, ny = grid_size(ri.width, ri.height, subset_size, subset_step)
        n = max(nx, 0) * max(ny, 0)
        for name, dt, cnt in (("u", torch.float64, n), ("v", torch.float64, n),
                              ("p", torch.float64, n * N_PARAMS[shape_fn]), ("zncc", torch.float32, n),
                              ("iters", torch.int32, n), ("converged", torch.uint8, n),
                              ("status", torch.uint8, n), ("wave", torch.int32, n)):
            _device_output(out.get(name), name, dt, cnt)
    else:
        # the library refuses these arguments before touching any output
        for name in ("u", "v", "p", "zncc", "iters", "converged", "status", "wave"):
            if not isinstance(out.get(name), torch.Tensor):
                raise DicError(DIC_EINVAL, "output %s is not a tensor" % name)
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).reshape(-1, 2))
    acc = ctypes.c_int64(0)
    o = DicStaticOutputs(*[out[k].data_ptr() for k in ("u", "v", "p", "zncc", "iters", "converged",
                                                         "status", "wave")],
                         ctypes.cast(ctypes.byref(acc), ctypes.c_void_p))
    err = ctypes.create_string_buffer(512)
    rc = load().dic_correlate_static(ctypes.byref(ri), ctypes.byref(di), subset_size, subset_step, shape_fn,
                                     ctypes.byref(prm), s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     s.shape[0], ctypes.byref(o), ctypes.c_void_p(stream_ptr), err, 512)
    if rc != DIC_OK:
        raise DicError(rc, err.value.decode(errors="replace"))
    return acc.value


def dic_strain_field(u, v, status, nx, ny, subset_step, window, basis, measure, out: dict, stream_ptr: int = 0):
    """Sec. 2.3 strain on device arrays: u, v (float64), status (uint8) CUDA tensors of
    nx * ny points; out maps STRAIN_FIELDS to CUDA tensors (float32, valid uint8)."""
    import torch

    basis = STRAIN_BASES[basis] if isinstance(basis, str) else basis
    measure = STRAIN_MEASURES[measure] if isinstance(measure, str) else measure
    n = max(int(nx), 0) * max(int(ny), 0)
    _device_output(u, "u", torch.float64, n)
    _device_output(v, "v", torch.float64, n)
    _device_output(status, "status", torch.uint8, n)
    for k in STRAIN_FIELDS:
        _device_output(out.get(k), k, torch.uint8 if k == "valid" else torch.float32, n)
    o = DicStrainOutputs(*[out[k].data_ptr() for k in STRAIN_FIELDS])
    _check(load().dic_strain_field(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                   ctypes.c_void_p(status.data_ptr()), nx, ny, subset_step, window, basis, measure,
                                   ctypes.byref(o), ctypes.c_void_p(stream_ptr)))


def dic_update_reference(h, stream_ptr: int = 0):
    """The current deformed image becomes the reference (incremental updating)."""
    _check(load().dic_update_reference(h, ctypes.c_void_p(stream_ptr)))


def dic_get_total_results(h, on_device: bool = False, stream_ptr: int = 0) -> dict:
    """Total warps from the first reference to the last frame: u, v, p, status (CUDA
    tensors viewing the handle's arrays, or numpy copies)."""
    import torch

    r = DicTotalResults()
    _check(load().dic_get_total_results(h, ctypes.byref(r), ctypes.c_void_p(stream_ptr)))
    n, npar = r.n_points, r.n_params
    out = dict(n_points=n, nx=r.nx, ny=r.ny, n_params=npar, n_updates=r.n_updates)
    for name, dt, shape in (("u", np.float64, (n,)), ("v", np.float64, (n,)), ("p", np.float64, (n, npar)),
                            ("status", np.uint8, (n,))):
        t = torch.as_tensor(_DeviceArray(getattr(r, name), shape, np.dtype(dt).str), device="cuda")
        out[name] = t if on_device else t.cpu().numpy()
    return out


def dic_fft_default_params() -> DicFftParams:
    return load().dic_fft_default_params()


def fft_params(**kw) -> DicFftParams:
    p = dic_fft_default_params()
    for k, v in kw.items():
        if k not in {name for name, _ in DicFftParams._fields_}:
            raise TypeError("unknown FFT parameter %r" % k)
        setattr(p, k, v)
    return p


def dic_fft_field(h, fp: DicFftParams, stream_ptr: int = 0):
    """The multi-window FFT initialiser over the handle's grid (Sec. 2.2)."""
    _check(load().dic_fft_field(h, ctypes.byref(fp), ctypes.c_void_p(stream_ptr)))


def dic_get_fft_results(h) -> dict:
    """Zero-copy CUDA tensors of the last initialiser run: u, v, peak (float32),
    status, replaced (uint8); plus nx, ny and the window sizes of its levels."""
    import torch

    r = DicFftResults()
    _check(load().dic_get_fft_results(h, ctypes.byref(r)))
    n = r.n_points
    out = dict(n_points=n, nx=r.nx, ny=r.ny, windows=[r.window[i] for i in range(r.n_levels)])
    for name, dt in (("u", np.float32), ("v", np.float32), ("peak", np.float32), ("status", np.uint8),
                     ("replaced", np.uint8)):
        out[name] = torch.as_tensor(_DeviceArray(getattr(r, name), (n,), np.dtype(dt).str), device="cuda")
    return out


def dic_fftcc_windows(h, window: int, origins, subpixel: bool, u, v, peak, stream_ptr: int = 0):
    """Eq. 1 over explicit windows: origins an int32 CUDA tensor [n, 4] of (x0, y0,
    gx0, gy0); u, v, peak float32 CUDA tensors [n]."""
    import torch

    n = int(origins.shape[0])
    _device_output(origins, "origins", torch.int32, 4 * n)
    for name, t in (("u", u), ("v", v), ("peak", peak)):
        _device_output(t, name, torch.float32, n)
    _check(load().dic_fftcc_windows(h, window, n, ctypes.c_void_p(origins.data_ptr()), 1 if subpixel else 0,
                                    ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                    ctypes.c_void_p(peak.data_ptr()), ctypes.c_void_p(stream_ptr)))


def dic_mad_filter(u, v, valid, nx: int, ny: int, tau: float, eps: float, u_out, v_out, replaced=None,
                   stream_ptr: int = 0):
    """The initialiser's MAD rule on float32 CUDA tensors of nx * ny values."""
    import torch

    n = max(int(nx), 0) * max(int(ny), 0)
    for name, t, dt in (("u", u, torch.float32), ("v", v, torch.float32), ("u_out", u_out, torch.float32),
                        ("v_out", v_out, torch.float32), ("valid", valid, torch.uint8),
                        ("replaced", replaced, torch.uint8)):
        if t is not None or name in ("u", "v", "u_out", "v_out"):
            _device_output(t, name, dt, n)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().dic_mad_filter(ptr(u), ptr(v), ptr(valid), nx, ny, tau, eps, ptr(u_out), ptr(v_out),
                                 ptr(replaced), ctypes.c_void_p(stream_ptr)))


def strain_outputs(n: int, device="cuda") -> dict:
    """Output tensors for dic_strain_field over n points."""
    import torch

    out = {k: torch.empty(n, dtype=torch.float32, device=device) for k in STRAIN_FIELDS[:-1]}
    out["valid"] = torch.empty(n, dtype=torch.uint8, device=device)
    return out


def _apply(p: DicParams, kw: dict) -> DicParams:
    fields = {name for name, _ in DicParams._fields_}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError("unknown parameter %r" % k)
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "cost" and isinstance(v, str):
            v = COSTS[v]
        if k == "optimizer" and isinstance(v, str):
            v = OPTIMIZERS[v]
        if k == "init" and isinstance(v, str):
            v = INITS[v]
        setattr(p, k, v)
    return p


def params(**kw) -> DicParams:
    """Default parameters with the given fields replaced (precision, cost and optimizer
    may be strings: "fp64"/"mixed", "znssd"/"nssd"/"ssd", "gn"/"lm")."""
    return _apply(dic_default_params(), kw)


class Correlation:
    """One reference/deformed pair on one handle (convenience over the calls above)."""

    def __init__(self, ref, deformed, roi=None, subset_size=21, subset_step=5, shape="affine",
                 interp="bspline3", **param_kw):
        self.shape = SHAPES[shape] if isinstance(shape, str) else shape
        self.step = subset_step
        interp = INTERPS[interp] if isinstance(interp, str) else interp
        self.h, self._keep = dic_create(ref, deformed, roi, subset_size, subset_step, self.shape, interp)
        if param_kw:
            dic_set_params(self.h, params(**param_kw))

    def set_params(self, **kw):
        dic_set_params(self.h, _apply(dic_get_params(self.h), kw))

    def set_reference(self, ref):
        self._keep = (dic_set_reference(self.h, ref), self._keep[1])

    def set_deformed(self, deformed):
        self._keep = (self._keep[0], dic_set_deformed(self.h, deformed))

    def set_subsets(self, subset_size, subset_step, shape, roi=None):
        """Re-grid for other subset settings; the reference stays resident."""
        shape = SHAPES[shape] if isinstance(shape, str) else shape
        dic_set_subsets(self.h, roi, subset_size, subset_step, shape)
        self.shape = shape
        self.step = subset_step

    def device_bytes(self) -> int:
        return dic_get_device_bytes(self.h)

    def run(self, seeds, stream_ptr: int = 0):
        dic_correlate(self.h, seeds, stream_ptr)
        return self

    def run_next(self, stream_ptr: int = 0):
        """Next frame: the current deformed image, started from the last result."""
        dic_correlate_sequence(self.h, stream_ptr)
        return self

    def results(self, on_device=False, copy=True):
        return dic_get_results(self.h, on_device, copy)

    def timing(self):
        return dic_get_timing(self.h)

    def update_reference(self, stream_ptr: int = 0):
        """Incremental updating: the current deformed image becomes the reference."""
        dic_update_reference(self.h, stream_ptr)
        return self

    def totals(self, on_device=False, stream_ptr: int = 0) -> dict:
        """Total warps from the first reference to the last correlated frame."""
        return dic_get_total_results(self.h, on_device, stream_ptr)

    def fft_field(self, max_displacement=32, subpixel=True, mad_tau=3.0, mad_eps=0.5, stream_ptr: int = 0) -> dict:
        """The multi-window FFT initialiser alone (the paper's MULTIWINDOW method)."""
        dic_fft_field(self.h, fft_params(max_displacement=max_displacement, subpixel=1 if subpixel else 0,
                                         mad_tau=mad_tau, mad_eps=mad_eps), stream_ptr)
        return dic_get_fft_results(self.h)

    def strain(self, window=9, basis="biquadratic", measure="green_lagrange", stream_ptr: int = 0) -> dict:
        """Sec. 2.3 strain of the last correlation: CUDA tensors per STRAIN_FIELDS."""
        r = self.results(on_device=True)
        out = strain_outputs(r["n_points"])
        dic_strain_field(r["u"], r["v"], r["status"], r["nx"], r["ny"], self.step, window, basis, measure, out,
                         stream_ptr)
        return out

    def close(self):
        if self.h is not None:
            dic_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
