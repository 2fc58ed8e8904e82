"""The C-ABI library loads on a machine without a GPU and exports exactly the
calls that include/dic.h declares; host-side argument checks answer before any
CUDA call. No compute call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_12941_gb300 import binding, build

    build.build()
    return binding.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "dic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(dic_[a-z_]+)\s*\(", text))


def test_header_and_binding_agree():
    from paper_2601_12941_gb300 import binding

    assert _declared() == set(binding.EXPORTS)


def test_library_exports_every_declared_call(lib):
    so = os.path.join(ROOT, "paper_2601_12941_gb300", "libdic.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dic_\w+)", out))
    assert _declared() <= exported
    for name in _declared():
        assert hasattr(lib, name)


def test_default_params_are_the_papers(lib):
    from paper_2601_12941_gb300 import binding

    p = binding.dic_default_params()
    assert (p.max_iter, p.conv_threshold, p.zncc_min) == (40, 0.01, 0.70)
    assert p.precision == binding.DIC_MIXED and p.nan_unconverged == 0
    # ZNSSD (Eq. 4) is the paper's default cost; undamped Gauss-Newton the default optimiser
    assert p.cost == binding.DIC_COST_ZNSSD and p.optimizer == binding.DIC_OPT_GAUSS_NEWTON


def test_invalid_arguments_fail_before_any_device_work(lib):
    from paper_2601_12941_gb300 import binding as B

    img = np.zeros((64, 64), np.uint8)
    ri, _ = B.make_image(img)
    h = ctypes.c_void_p()
    # even subset size, zero step, unknown shape, mismatched sizes, NULL image
    assert lib.dic_create(ctypes.byref(ri), ctypes.byref(ri), None, 20, 5, 1, 0, ctypes.byref(h)) == B.DIC_EINVAL
    assert b"odd" in lib.dic_last_error()
    assert lib.dic_create(ctypes.byref(ri), ctypes.byref(ri), None, 21, 0, 1, 0, ctypes.byref(h)) == B.DIC_EINVAL
    assert lib.dic_create(ctypes.byref(ri), ctypes.byref(ri), None, 21, 5, 7, 0, ctypes.byref(h)) == B.DIC_EINVAL
    small, _ = B.make_image(np.zeros((32, 40), np.uint8))
    assert lib.dic_create(ctypes.byref(ri), ctypes.byref(small), None, 21, 5, 1, 0, ctypes.byref(h)) == B.DIC_EINVAL
    assert lib.dic_create(None, ctypes.byref(ri), None, 21, 5, 1, 0, ctypes.byref(h)) == B.DIC_EINVAL
    assert lib.dic_create(ctypes.byref(ri), ctypes.byref(ri), None, 63, 5, 1, 0, ctypes.byref(h)) == B.DIC_EINVAL
    # unknown interpolant (DIC_BSPLINE3 = 0 and DIC_BICUBIC = 1 exist)
    assert lib.dic_create(ctypes.byref(ri), ctypes.byref(ri), None, 21, 5, 1, 2, ctypes.byref(h)) == B.DIC_EINVAL
    assert b"interpolation" in lib.dic_last_error()
    assert h.value is None
    # parameter validation on a NULL handle
    p = B.dic_default_params()
    assert lib.dic_set_params(None, ctypes.byref(p)) == B.DIC_EINVAL
    assert lib.dic_correlate(None, None, 0, None) == B.DIC_EINVAL
    # strain: arguments are checked before anything is launched (the pointers below
    # are never dereferenced)
    fake = ctypes.c_void_p(16)
    out = B.DicStrainOutputs(*([16] * len(B.STRAIN_FIELDS)))
    assert lib.dic_strain_field(None, fake, fake, 10, 10, 5, 9, 1, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    assert lib.dic_strain_field(fake, fake, fake, 10, 10, 5, 8, 1, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    assert b"odd" in lib.dic_last_error()
    assert lib.dic_strain_field(fake, fake, fake, 10, 10, 5, 33, 1, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    assert lib.dic_strain_field(fake, fake, fake, 10, 10, 0, 9, 1, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    assert lib.dic_strain_field(fake, fake, fake, 0, 10, 5, 9, 1, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    assert lib.dic_strain_field(fake, fake, fake, 10, 10, 5, 9, 2, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    assert lib.dic_strain_field(fake, fake, fake, 10, 10, 5, 9, 1, 5, ctypes.byref(out), None) == B.DIC_EINVAL
    out.exy = None
    assert lib.dic_strain_field(fake, fake, fake, 10, 10, 5, 9, 1, 0, ctypes.byref(out), None) == B.DIC_EINVAL
    # estimates and re-grids on NULL
    assert lib.dic_set_subsets(None, None, 21, 5, 1) == B.DIC_EINVAL
    assert lib.dic_get_device_bytes(None, None) == B.DIC_EINVAL
    nb = ctypes.c_int64(0)
    assert lib.dic_estimate_device_bytes(ctypes.byref(ri), ctypes.byref(ri), 0, 20, 5, 1, ctypes.byref(p), 1,
                                         ctypes.byref(nb)) == B.DIC_EINVAL
    assert lib.dic_estimate_device_bytes(ctypes.byref(ri), ctypes.byref(ri), 0, 21, 5, 1, ctypes.byref(p), 1,
                                         ctypes.byref(nb)) == B.DIC_OK
    assert nb.value > 2 * 64 * 64 * 4      # at least the two FP32 coefficient planes
    # FFT seeds: their buffers are counted, and the parameters are validated
    pf = B.params(init="fft", max_displacement=40)
    nf = ctypes.c_int64(0)
    assert lib.dic_estimate_device_bytes(ctypes.byref(ri), ctypes.byref(ri), 0, 21, 5, 1, ctypes.byref(pf), 1,
                                         ctypes.byref(nf)) == B.DIC_OK
    assert nf.value > nb.value
    # the mixed path with FP64 solves: estimated like the mixed path (FP32 planes);
    # Gauss-Newton with ZNSSD only
    p2 = B.params(precision="mixed_fp64_solve")
    n2 = ctypes.c_int64(0)
    assert lib.dic_estimate_device_bytes(ctypes.byref(ri), ctypes.byref(ri), 0, 21, 5, 1, ctypes.byref(p2), 1,
                                         ctypes.byref(n2)) == B.DIC_OK
    assert n2.value == nb.value
    for bad in (dict(init=2), dict(init="fft", max_displacement=4096), dict(init="fft", max_displacement=-1),
                dict(mad_eps=-1.0), dict(precision=3), dict(precision="mixed_fp64_solve", cost="nssd"),
                dict(precision="mixed_fp64_solve", optimizer="lm")):
        pb = B.params(**bad)
        assert lib.dic_estimate_device_bytes(ctypes.byref(ri), ctypes.byref(ri), 0, 21, 5, 1, ctypes.byref(pb), 1,
                                             ctypes.byref(nf)) == B.DIC_EINVAL, bad


def test_next_row_calls_check_their_arguments_first(lib):
    from paper_2601_12941_gb300 import binding as B

    fake = ctypes.c_void_p(16)
    fp = B.dic_fft_default_params()
    assert (fp.max_displacement, fp.subpixel, fp.mad_tau, fp.mad_eps) == (32, 1, 3.0, 0.5)
    assert lib.dic_fft_field(None, ctypes.byref(fp), None) == B.DIC_EINVAL
    assert lib.dic_get_fft_results(None, ctypes.byref(B.DicFftResults())) == B.DIC_EINVAL
    assert lib.dic_fftcc_windows(None, 31, 1, fake, 0, fake, fake, fake, None) == B.DIC_EINVAL
    assert lib.dic_update_reference(None, None) == B.DIC_EINVAL
    assert lib.dic_get_total_results(None, ctypes.byref(B.DicTotalResults()), None) == B.DIC_EINVAL
    # the MAD rule: sizes, NULL arrays and in-place calls are refused before any launch;
    # an empty field is a no-op
    assert lib.dic_mad_filter(fake, fake, None, -1, 4, 3.0, 0.5, fake, fake, None, None) == B.DIC_EINVAL
    assert lib.dic_mad_filter(fake, fake, None, 0, 4, 3.0, 0.5, fake, fake, None, None) == B.DIC_OK
    assert lib.dic_mad_filter(None, fake, None, 3, 4, 3.0, 0.5, ctypes.c_void_p(32), ctypes.c_void_p(48), None,
                              None) == B.DIC_EINVAL
    assert lib.dic_mad_filter(fake, ctypes.c_void_p(32), None, 3, 4, 3.0, 0.5, fake, ctypes.c_void_p(48), None,
                              None) == B.DIC_EINVAL
    assert b"in-place" in lib.dic_last_error()
    assert lib.dic_mad_filter(fake, ctypes.c_void_p(32), None, 3, 4, 3.0, -0.5, ctypes.c_void_p(48),
                              ctypes.c_void_p(64), None, None) == B.DIC_EINVAL


def test_loading_fails_loudly_without_the_library(tmp_path):
    from paper_2601_12941_gb300 import binding

    with pytest.raises(ImportError):
        binding._lib_saved = binding._lib
        try:
            binding._lib = None
            binding.load(str(tmp_path / "missing.so"))
        finally:
            binding._lib = binding._lib_saved


def test_pointer_entry_points_refuse_outputs_they_cannot_write(lib):
    """The calls that take raw device pointers (the allocation-free correlation,
    strain, FFT windows, MAD) cannot check what a pointer holds, so the binding
    refuses host tensors, wrong dtypes and short buffers before the call."""
    import torch

    from paper_2601_12941_gb300 import binding as B

    ref = np.zeros((64, 64), np.uint8)
    n = 1
    out = dict(u=torch.zeros(n, dtype=torch.float64), v=torch.zeros(n, dtype=torch.float64),
               p=torch.zeros(n * 6, dtype=torch.float64), zncc=torch.zeros(n, dtype=torch.float32),
               iters=torch.zeros(n, dtype=torch.int32), converged=torch.zeros(n, dtype=torch.uint8),
               status=torch.zeros(n, dtype=torch.uint8), wave=torch.zeros(n, dtype=torch.int32))
    with pytest.raises(B.DicError) as e:
        B.dic_correlate_static(ref, ref, 21, 40, B.DIC_AFFINE, B.params(), [(32, 32)], out)
    assert e.value.code == B.DIC_EINVAL and "CUDA" in str(e.value)
    with pytest.raises(B.DicError):
        B.dic_strain_field(torch.zeros(4, dtype=torch.float64), torch.zeros(4, dtype=torch.float64),
                           torch.zeros(4, dtype=torch.uint8), 2, 2, 5, 3, "bilinear", "green_lagrange",
                           {k: torch.zeros(4) for k in B.STRAIN_FIELDS})
    with pytest.raises(B.DicError):
        B.dic_mad_filter(torch.zeros(4), torch.zeros(4), None, 2, 2, 3.0, 0.5, torch.zeros(4), torch.zeros(4))
    assert B.grid_size(256, 256, 21, 5) == (48, 48)
    assert B.grid_size(32768, 32768, 41, 10) == (3273, 3273)
