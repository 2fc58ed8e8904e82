"""Pins of the oracle's bicubic interpolant (reading R14: Keys' cubic convolution,
a = -1/2, on the gray levels) to closed forms other than its own formula: the
kernel's printed values, the four-point midpoint rule, exact reproduction of
quadratics but not of cubics (the order of accuracy that fixes a = -1/2), central
differences at the pixels, and IC-GN recovering integer shifts and a known
affine field. CPU only."""
import numpy as np
import pytest

import synth
from oracle import dic_oracle as O
from synth import workloads as wl

RNG = np.random.default_rng(1981)


def _plane(img):
    return O.Plane(img, interp=O.BICUBIC)


def test_kernel_values_and_partition_of_unity():
    # K(0) = 1, K(+-1) = K(+-2) = 0 (interpolating), K(1/2) = 9/16, K(3/2) = -1/16
    assert O.keys(np.array([0.0, 1.0, -1.0, 2.0, -2.0, 2.5])).tolist() == [1.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    assert O.keys(0.5) == 9 / 16 and O.keys(-1.5) == -1 / 16
    t = RNG.uniform(0, 1, 100)
    w = sum(O.keys(t - k) for k in (-1, 0, 1, 2))
    assert np.abs(w - 1.0).max() < 1e-14


def test_midpoint_is_the_four_point_rule():
    img = RNG.uniform(0, 255, size=(20, 24))
    plane = _plane(img)
    y = np.repeat(np.arange(1, 17), 20)
    x = np.tile(np.arange(1, 21), 16) + 0.5
    val, valid = O.interpolate(plane, x, y)
    assert valid.all()
    i = np.floor(x).astype(int)
    want = (-img[y, i - 1] + 9 * img[y, i] + 9 * img[y, i + 1] - img[y, i + 2]) / 16
    assert np.abs(val - want).max() < 1e-12


def test_quadratics_are_reproduced_and_cubics_are_not():
    yy, xx = np.mgrid[0:30, 0:34].astype(np.float64)
    x = RNG.uniform(1, 31.999, 400)
    y = RNG.uniform(1, 27.999, 400)
    quad = lambda X, Y: 3.0 + 0.7 * X - 1.1 * Y + 0.05 * X * X - 0.02 * X * Y + 0.03 * Y * Y + 1e-3 * X * X * Y * Y
    val, valid = O.interpolate(_plane(quad(xx, yy)), x, y)
    assert valid.all()
    assert np.abs(val - quad(x, y)).max() < 1e-9
    cub = lambda X, Y: 0.1 * X ** 3
    val, _ = O.interpolate(_plane(cub(xx, yy)), x, y)
    assert np.abs(val - cub(x, y)).max() > 1e-3        # third-order accurate, not exact


def test_other_a_breaks_quadratic_reproduction():
    # the planted mistake a = -3/4 (another common choice) is caught by the pin above
    xx = np.arange(12, dtype=np.float64)
    f = 0.05 * xx * xx
    t = 0.3
    val = sum(f[5 + k] * O.keys(t - k, a=-0.75) for k in (-1, 0, 1, 2))
    assert abs(val - 0.05 * 5.3 ** 2) > 1e-3
    val = sum(f[5 + k] * O.keys(t - k) for k in (-1, 0, 1, 2))
    assert abs(val - 0.05 * 5.3 ** 2) < 1e-13


def test_gradient_is_the_central_difference_and_mirrored_at_the_border():
    img = RNG.uniform(0, 255, size=(15, 18))
    xs = np.array([0, 1, 9, 17, 4, 4])
    ys = np.array([3, 7, 0, 5, 14, 8])
    fx, fy = O.gradient_at_pixels(_plane(img), xs, ys)
    pad = np.pad(img, 1, mode="reflect")          # whole-sample mirror: I[-1] = I[1]
    want_x = (pad[ys + 1, xs + 2] - pad[ys + 1, xs]) / 2
    want_y = (pad[ys + 2, xs + 1] - pad[ys, xs + 1]) / 2
    assert np.abs(fx - want_x).max() < 1e-12 and np.abs(fy - want_y).max() < 1e-12
    assert fx[0] == 0.0 and fx[3] == 0.0 and fy[2] == 0.0 and fy[4] == 0.0


def test_integer_shift_is_recovered_exactly():
    sp = synth.Speckle(seed=7, density=0.03, sigma=(1.5, 3.0), cell=16)
    big = synth.render(synth.ImageSpec(sp, gray_max=255.0), 110, 110, "u8")
    ref = big[5:105, 5:105]
    dfm = big[5 + 2:105 + 2, 5 - 3:105 - 3]          # the pattern moves by (+3, -2)
    refp, defp = _plane(ref), _plane(dfm)
    for shape in (O.RIGID, O.AFFINE, O.QUADRATIC):
        res = O.icgn(refp, defp, 50, 50, 21, shape, [3.0, -2.0], dict(conv_threshold=1e-8))
        want = np.zeros(O.N_PARAMS[shape])
        want[:2] = (3.0, -2.0)
        assert res["status"] == O.OK
        assert np.abs(res["p"] - want).max() < 1e-10
        assert abs(res["zncc"] - 1.0) < 1e-12


def test_affine_field_is_recovered_and_correlate_uses_the_interpolant():
    w = wl.affine_256_u8()
    ref = synth.render(w.ref, 256, 256, "f64")
    dfm = synth.render(w.deformed, 256, 256, "f64")
    refp, defp = _plane(ref), _plane(dfm)
    for (xc, yc) in [(60, 70), (128, 128), (190, 60)]:
        u, v = synth.displacement(w.field, np.array([float(xc)]), np.array([float(yc)]))
        res = O.icgn(refp, defp, xc, yc, 21, O.AFFINE, [round(u[0]), round(v[0])],
                     dict(conv_threshold=1e-8, max_iter=100))
        assert res["status"] == O.OK
        # Keys' kernel has a larger interpolation bias than the spline's (up to about
        # 1e-2 px on fine speckle)
        assert max(abs(res["p"][0] - u[0]), abs(res["p"][1] - v[0])) < 1e-2
        assert np.abs(res["p"][2:6] - np.array([1e-3, 2e-4, 2e-4, -5e-4])).max() < 3e-4
    # the whole-image path builds bicubic planes when asked, and the two interpolants
    # give different (both close) answers
    seeds = [(128, 128)]
    a = O.correlate(ref, dfm, None, 21, 40, O.AFFINE, seeds, dict(interp=O.BICUBIC, conv_threshold=1e-6))
    b = O.correlate(ref, dfm, None, 21, 40, O.AFFINE, seeds, dict(conv_threshold=1e-6))
    ok = (a["status"] == O.OK) & (b["status"] == O.OK)
    assert ok.sum() >= 20
    d = np.abs(a["u"][ok] - b["u"][ok])
    assert 0 < d.max() < 2e-2


def test_unknown_interpolant_is_rejected():
    with pytest.raises(ValueError):
        O.Plane(np.zeros((8, 8)), interp="lanczos")
