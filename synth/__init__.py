"""Seeded synthetic speckle image pairs with a known displacement field.

Input generation only: this package holds none of the correlation method's
arithmetic. Both the FP64 oracle and the CUDA library consume its images.

The host renderer (``libsynth_host.so``, gcc) and the device renderer
(``libsynth_gpu.so``, nvcc) compile the same header, ``csrc/speckle.h``, with
floating-point contraction off, so a window rendered on either side holds the
same doubles up to rare last-ulp differences between libm and CUDA's exp/log/cos.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
HOST_LIB = os.path.join(_HERE, "libsynth_host.so")
GPU_LIB = os.path.join(_HERE, "libsynth_gpu.so")
_lock = threading.Lock()


class _Speckle(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("density", ctypes.c_double),
                ("sigma_lo", ctypes.c_double), ("sigma_hi", ctypes.c_double),
                ("amp_lo", ctypes.c_double), ("amp_hi", ctypes.c_double),
                ("cutoff", ctypes.c_double), ("cell", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("u0", ctypes.c_double), ("v0", ctypes.c_double),
                ("exx", ctypes.c_double), ("exy", ctypes.c_double),
                ("eyx", ctypes.c_double), ("eyy", ctypes.c_double),
                ("jump", ctypes.c_double), ("amp", ctypes.c_double),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("width", ctypes.c_double),
                ("uxx", ctypes.c_double), ("uxy", ctypes.c_double), ("uyy", ctypes.c_double),
                ("vxx", ctypes.c_double), ("vxy", ctypes.c_double), ("vyy", ctypes.c_double)]


class _Intensity(ctypes.Structure):
    _fields_ = [("gray_max", ctypes.c_double), ("noise", ctypes.c_double),
                ("noise_seed", ctypes.c_uint64)]


FIELD_IDENTITY, FIELD_AFFINE, FIELD_SINE_V, FIELD_QUADRATIC = 0, 1, 2, 3
GRAY_MAX = {"u8": 255.0, "u16": 65535.0}
_OUT_KIND = {"u8": 0, "u16": 1, "f32": 2, "f64": 3}


def _mix64(z: int) -> int:
    m = (1 << 64) - 1
    z &= m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


@dataclass(frozen=True)
class Speckle:
    """Gaussian-dot speckle: dots per px^2, sigma and amplitude ranges."""
    seed: int
    density: float
    sigma: tuple = (1.5, 3.0)
    amplitude: tuple = (0.2, 1.0)
    cell: int = 16
    cutoff_sigmas: float = 6.0

    def _c(self) -> _Speckle:
        return _Speckle(self.seed & ((1 << 64) - 1), self.density, self.sigma[0], self.sigma[1],
                        self.amplitude[0], self.amplitude[1], self.cutoff_sigmas * self.sigma[1],
                        self.cell, 0)


@dataclass(frozen=True)
class Field:
    """Displacement field u(X) (x = X + u(X)).

    kind FIELD_AFFINE: u = u0 + exx X' + exy Y', v = v0 + eyx X' + eyy Y' about
    (cx, cy), plus an optional slip of ``jump`` px along (1,1)/sqrt(2) where Y' > X'.
    kind FIELD_SINE_V: u = 0, v = amp sin(2 pi Y / T(X)), T rising linearly from
    t0 at X = 0 to t1 at X = width - 1.
    kind FIELD_QUADRATIC: the affine terms plus uxx X'^2 + uxy X'Y' + uyy Y'^2 in u
    and vxx X'^2 + vxy X'Y' + vyy Y'^2 in v.
    """
    kind: int = FIELD_IDENTITY
    cx: float = 0.0
    cy: float = 0.0
    u0: float = 0.0
    v0: float = 0.0
    exx: float = 0.0
    exy: float = 0.0
    eyx: float = 0.0
    eyy: float = 0.0
    jump: float = 0.0
    amp: float = 0.0
    t0: float = 1.0
    t1: float = 1.0
    width: float = 2.0
    uxx: float = 0.0
    uxy: float = 0.0
    uyy: float = 0.0
    vxx: float = 0.0
    vxy: float = 0.0
    vyy: float = 0.0

    def _c(self) -> _Field:
        return _Field(self.kind, 0, self.cx, self.cy, self.u0, self.v0, self.exx, self.exy,
                      self.eyx, self.eyy, self.jump, self.amp, self.t0, self.t1, self.width,
                      self.uxx, self.uxy, self.uyy, self.vxx, self.vxy, self.vyy)


IDENTITY = Field()


def affine_field(W, H, u0=0.0, v0=0.0, exx=0.0, exy=0.0, eyx=0.0, eyy=0.0, jump=0.0) -> Field:
    """Affine field about the image centre ((W-1)/2, (H-1)/2)."""
    return Field(FIELD_AFFINE, (W - 1) / 2.0, (H - 1) / 2.0, u0, v0, exx, exy, eyx, eyy, jump)


def quadratic_field(W, H, u0=0.0, v0=0.0, exx=0.0, exy=0.0, eyx=0.0, eyy=0.0, uxx=0.0, uxy=0.0,
                    uyy=0.0, vxx=0.0, vxy=0.0, vyy=0.0) -> Field:
    """Quadratic field about the image centre."""
    return Field(FIELD_QUADRATIC, (W - 1) / 2.0, (H - 1) / 2.0, u0, v0, exx, exy, eyx, eyy,
                 uxx=uxx, uxy=uxy, uyy=uyy, vxx=vxx, vxy=vxy, vyy=vyy)


def sine_field(W, amp, t0, t1) -> Field:
    return Field(FIELD_SINE_V, amp=amp, t0=t0, t1=t1, width=float(W))


def _build(cmd, out):
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.run(cmd + ["-o", tmp], check=True, cwd=_CSRC)
    os.replace(tmp, out)


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(os.path.join(_CSRC, s)) > t for s in srcs)


def build_host(force=False) -> str:
    with _lock:
        if force or _stale(HOST_LIB, ["speckle_cpu.c", "speckle.h"]):
            _build(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "speckle_cpu.c", "-lm"], HOST_LIB)
    return HOST_LIB


def build_gpu(force=False) -> str:
    with _lock:
        if force or _stale(GPU_LIB, ["speckle_gpu.cu", "speckle.h"]):
            _build(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false",
                    "-Xcompiler", "-fPIC", "-shared", "speckle_gpu.cu"], GPU_LIB)
    return GPU_LIB


_host = None
_gpu = None


def _host_lib():
    global _host
    if _host is None:
        lib = ctypes.CDLL(build_host())
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        for name in ("syn_render_window", "syn_render_window_direct"):
            fn = getattr(lib, name)
            fn.argtypes = [P(_Speckle), P(_Field), P(_Intensity), ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, d]
            fn.restype = ctypes.c_int
        for name in ("syn_displacement_at", "syn_inverse_map_at"):
            fn = getattr(lib, name)
            fn.argtypes = [P(_Field), d, d, ctypes.c_int64, d, d]
            fn.restype = None
        _host = lib
    return _host


def _gpu_lib():
    global _gpu
    if _gpu is None:
        lib = ctypes.CDLL(build_gpu())
        P = ctypes.POINTER
        lib.syn_render_gpu.argtypes = [P(_Speckle), P(_Field), P(_Intensity), ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p]
        lib.syn_render_gpu.restype = ctypes.c_int
        _gpu = lib
    return _gpu


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass(frozen=True)
class ImageSpec:
    """One image of a pair: which field deforms the pattern, gray range and noise."""
    speckle: Speckle
    field: Field = IDENTITY
    gray_max: float = 255.0
    noise: float = 0.0
    noise_tag: int = 0

    def _intensity(self) -> _Intensity:
        ns = _mix64(self.speckle.seed ^ (0xD1B54A32D192ED03 + self.noise_tag))
        return _Intensity(self.gray_max, self.noise, ns)


def render_window(spec: ImageSpec, width: int, x0: int, y0: int, w: int, h: int,
                  direct: bool = False) -> np.ndarray:
    """Pixels [x0, x0+w) x [y0, y0+h) of a ``width``-wide image, as float64 before
    quantisation (noise included)."""
    out = np.empty((h, w), dtype=np.float64)
    lib = _host_lib()
    fn = lib.syn_render_window_direct if direct else lib.syn_render_window
    sp, fd, it = spec.speckle._c(), spec.field._c(), spec._intensity()
    rc = fn(ctypes.byref(sp), ctypes.byref(fd), ctypes.byref(it), width, x0, y0, w, h, _dptr(out))
    if rc != 0:
        raise MemoryError("speckle render failed")
    return out


def quantise(values: np.ndarray, dtype: str, gray_max: float) -> np.ndarray:
    """Round half to even and clip to [0, G]; float dtypes are returned as they are."""
    if dtype in ("f32", "f64"):
        return values.astype(np.float32 if dtype == "f32" else np.float64)
    q = np.clip(np.rint(values), 0.0, gray_max)
    return q.astype(np.uint8 if dtype == "u8" else np.uint16)


def render(spec: ImageSpec, width: int, height: int, dtype: str = "u8") -> np.ndarray:
    """Whole image on the host."""
    return quantise(render_window(spec, width, 0, 0, width, height), dtype, spec.gray_max)


def render_crop(spec: ImageSpec, width: int, height: int, x0: int, y0: int, w: int, h: int,
                dtype: str = "u8") -> np.ndarray:
    """Crop of an image (clipped to the image) on the host; returns (crop, (x0, y0))."""
    xa, ya = max(0, x0), max(0, y0)
    xb, yb = min(width, x0 + w), min(height, y0 + h)
    vals = render_window(spec, width, xa, ya, xb - xa, yb - ya)
    return quantise(vals, dtype, spec.gray_max), (xa, ya)


def render_gpu(spec: ImageSpec, out, stream_ptr: int = 0) -> None:
    """Render into a 2-D CUDA tensor ``out`` (uint8, uint16 via int16 storage,
    float32 or float64) on the device; the tensor's shape gives H x W."""
    import torch

    kinds = {torch.uint8: "u8", torch.int16: "u16", torch.float32: "f32", torch.float64: "f64"}
    if hasattr(torch, "uint16"):
        kinds[torch.uint16] = "u16"
    kind = kinds[out.dtype]
    H, W = out.shape
    if out.stride(1) != 1:
        raise ValueError("rows must be contiguous")
    sp, fd, it = spec.speckle._c(), spec.field._c(), spec._intensity()
    rc = _gpu_lib().syn_render_gpu(ctypes.byref(sp), ctypes.byref(fd), ctypes.byref(it), W, H,
                                   _OUT_KIND[kind], ctypes.c_void_p(out.data_ptr()),
                                   out.stride(0) * out.element_size(), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError("device speckle render failed (%d)" % rc)


def displacement(fld: Field, X, Y):
    """Truth u(X), v(X) at reference-frame points."""
    X = np.ascontiguousarray(X, dtype=np.float64).ravel()
    Y = np.ascontiguousarray(Y, dtype=np.float64).ravel()
    u = np.empty_like(X)
    v = np.empty_like(X)
    f = fld._c()
    _host_lib().syn_displacement_at(ctypes.byref(f), _dptr(X), _dptr(Y), X.size, _dptr(u), _dptr(v))
    return u, v


def inverse_map(fld: Field, x, y):
    """Reference-frame coordinates X = phi^-1(x) of deformed-image points."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    X = np.empty_like(x)
    Y = np.empty_like(x)
    f = fld._c()
    _host_lib().syn_inverse_map_at(ctypes.byref(f), _dptr(x), _dptr(y), x.size, _dptr(X), _dptr(Y))
    return X, Y
