"""Pins of the multi-window FFT initialiser's oracle (Eq. 1, Sec. 2.2; readings F1-F8)
to things other than itself: the paper's own window-size example, a DFT written
from its definition, exact recovery of circular and non-circular integer shifts
(a planted conj on the wrong factor flips the sign and fails), the Gaussian
vertex of exact Gaussian samples, bilinear reproduction of linear fields, the
median/MAD rule on hand-built neighbourhoods, and large displacements that the
integer ZNCC search cannot reach. CPU only."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import dic_oracle as O
from oracle import fft_oracle as F

RNG = np.random.default_rng(1993)


def _speckle(W, H, seed=11, fld=synth.IDENTITY, dtype="f64", noise=0.0):
    sp = synth.Speckle(seed=seed, density=0.03, sigma=(1.5, 3.0), cell=16)
    return synth.render(synth.ImageSpec(sp, field=fld, gray_max=250.0, noise=noise, noise_tag=2 if fld is not
                                        synth.IDENTITY else 1), W, H, dtype)


def test_window_sizes_follow_the_papers_example():
    with open(os.path.join(os.path.dirname(__file__), "golden", "fft_window_sizes.json")) as fh:
        g = json.load(fh)
    ex = g["example"]                  # Sec. 2.2's worked example
    assert F.window_sizes(ex["max_displacement"], ex["subset_size"], 5000, 5000) == ex["windows"]
    sem = g["sem_study"]               # Sec. 4: the SEM study's settings on a 32768 px image
    assert F.window_sizes(sem["max_displacement"], sem["subset_size"], 32768, 32768) == \
        [2048, 1024, 512, 256, 128, 64, 32, 31]
    # windows larger than the image are dropped; no displacement: the subset alone
    assert F.window_sizes(800, 17, 300, 600) == [256, 128, 64, 32, 17]
    assert F.window_sizes(0, 21, 256, 256) == [21]
    assert F.window_sizes(1024, 21, 4096, 4096)[0] == 2048            # strictly above D


def _dft2(a):
    """2-D DFT from its definition, sum_x a[x] exp(-2 pi i k.x / L)."""
    L = a.shape[0]
    k = np.arange(L)
    Wm = np.exp(-2j * np.pi * np.outer(k, k) / L)
    return Wm @ a @ Wm.T


@pytest.mark.parametrize("L", [4, 5, 8, 21])
def test_eq1_is_the_circular_zncc_computed_by_brute_force(L):
    f = RNG.uniform(0, 255, (L, L))
    g = RNG.uniform(0, 255, (L, L))
    fb, gb = f - f.mean(), g - g.mean()
    want = np.empty((L, L))
    for sy in range(L):
        for sx in range(L):
            # R(s) = sum_x fbar(x) gbar(x - s), indices modulo L
            want[sy, sx] = np.sum(fb * np.roll(gb, shift=(sy, sx), axis=(0, 1)))
    want /= np.sqrt(np.sum(fb * fb) * np.sum(gb * gb))
    assert np.abs(F.fftcc(f, g) - want).max() < 1e-12
    # and through a DFT written from its definition
    Fd, Gd = _dft2(fb), _dft2(gb)
    R = np.real(np.conj(_dft2(np.conj(Fd * np.conj(Gd))))) / (L * L)  # inverse DFT via the forward one
    assert np.abs(R / np.sqrt(np.sum(fb * fb) * np.sum(gb * gb)) - want).max() < 1e-12


@pytest.mark.parametrize("L", [21, 31, 32, 64])
def test_eq1_matches_scipys_wrapped_spatial_correlation(L):
    # scipy's spatial correlation with periodic boundaries, its kernel origin at the
    # centre (hence the roll by -floor(L/2)), on the mean-removed windows
    from scipy import ndimage

    f = RNG.uniform(0, 255, (L, L))
    g = RNG.uniform(0, 255, (L, L))
    fb, gb = f - f.mean(), g - g.mean()
    c = np.roll(ndimage.correlate(fb, gb, mode="wrap"), (-(L // 2), -(L // 2)), (0, 1))
    assert np.abs(F.fftcc(f, g) - c / np.sqrt(np.sum(fb * fb) * np.sum(gb * gb))).max() < 1e-12


def test_eq1_is_invariant_to_gain_and_offset_and_zero_on_flat_windows():
    f = RNG.uniform(0, 255, (16, 16))
    g = RNG.uniform(0, 255, (16, 16))
    assert np.abs(F.fftcc(3.0 * f + 40.0, 0.5 * g - 7.0) - F.fftcc(f, g)).max() < 1e-12
    assert not F.fftcc(np.full((16, 16), 9.0), g).any()
    # exactly zero for any size and either window (no transform noise gets through)
    h = RNG.uniform(0, 255, (31, 31))
    assert not F.fftcc(np.full((31, 31), 9.0), h).any() and not F.fftcc(h, np.full((31, 31), 0.3)).any()
    assert F.peak(F.fftcc(h, np.full((31, 31), 0.3)))[:2] == (0.0, 0.0)


@pytest.mark.parametrize("L,d", [(32, (5, -7)), (32, (-16, 15)), (64, (0, 0)), (21, (10, -10)), (21, (-3, 4))])
def test_circular_shift_gives_a_delta_at_minus_the_shift(L, d):
    f = RNG.uniform(0, 255, (L, L))
    g = np.roll(f, shift=(d[1], d[0]), axis=(0, 1))                   # g(x) = f(x - d)
    R = F.fftcc(f, g)
    dx, dy, pk = F.peak(R)
    assert (dx, dy) == d
    assert abs(pk - 1.0) < 1e-12                                      # a perfect match there
    others = np.delete(R.ravel(), int(np.argmax(R)))
    assert others.max() < 0.5


def test_a_conj_on_the_wrong_factor_is_caught(monkeypatch):
    f = RNG.uniform(0, 255, (32, 32))
    g = np.roll(f, shift=(3, 6), axis=(0, 1))
    real = F.fftcc

    def swapped(a, b):
        return real(b, a)

    monkeypatch.setattr(F, "fftcc", swapped)
    dx, dy, _ = F.peak(F.fftcc(f, g))
    assert (dx, dy) == (-6, -3)


def test_non_circular_integer_shift_of_a_window():
    big = _speckle(300, 300)
    ref = big[40:260, 40:260]
    for (du, dv) in [(7, -4), (-13, 9), (0, 0), (15, 15)]:
        dfm = big[40 - dv:260 - dv, 40 - du:260 - du]                  # content moves by (du, dv)
        u, v, pk, org = F.window_level(ref, dfm, 64, [(70, 80)], [(0, 0)])
        assert (u[0], v[0]) == (du, dv)
        assert pk[0] > 0.3
        # with the guess right the residual shift is zero and the windows coincide
        u2, v2, pk2, org2 = F.window_level(ref, dfm, 64, [(70, 80)], [(du, dv)])
        assert (u2[0], v2[0]) == (du, dv) and tuple(org2[0]) == (70 + du, 80 + dv)
        assert pk2[0] > 0.99


def test_deformed_window_is_clamped_into_the_image():
    big = _speckle(200, 200)
    ref = big[20:180, 20:180]
    dfm = big[20 + 3:180 + 3, 20 - 5:180 - 5]                          # moves by (+5, -3)
    u, v, _, org = F.window_level(ref, dfm, 32, [(120, 2)], [(30, -9)])
    assert tuple(org[0]) == (128, 0)                                   # clamped to W - L and 0
    assert (u[0], v[0]) == (5, -3)


def test_gaussian_vertex_of_exact_gaussian_samples():
    for x0, s in [(0.3, 1.2), (-0.45, 0.8), (0.0, 2.0)]:
        g = [math.exp(-((k - x0) ** 2) / (2 * s * s)) for k in (-1, 0, 1)]
        assert abs(F.gauss3(*g) - x0) < 1e-12
    assert F.gauss3(-0.1, 1.0, 0.5) == 0.0 and F.gauss3(0.5, 0.2, 0.5) == 0.0


def test_subpixel_estimate_of_a_smooth_shift():
    W = H = 160
    fld = synth.affine_field(W, H, u0=2.3, v0=-1.6)
    ref = _speckle(W, H)
    dfm = _speckle(W, H, fld=fld)
    u, v, _, _ = F.window_level(ref, dfm, 41, [(60, 60)], [(2, -2)], subpixel=True)
    ui, vi, _, _ = F.window_level(ref, dfm, 41, [(60, 60)], [(2, -2)], subpixel=False)
    assert abs(u[0] - 2.3) < 0.2 and abs(v[0] + 1.6) < 0.2
    assert abs(u[0] - 2.3) < abs(ui[0] - 2.3) and abs(v[0] + 1.6) < abs(vi[0] + 1.6)


def test_bilinear_reproduces_linear_fields_and_holds_beyond_the_centres():
    ny, nx, L = 5, 7, 64
    j, i = np.mgrid[0:ny, 0:nx]
    cx, cy = i * L + L / 2, j * L + L / 2
    field = 3.0 + 0.25 * cx - 0.125 * cy
    x = RNG.uniform(L / 2, (nx - 1) * L + L / 2, 200)
    y = RNG.uniform(L / 2, (ny - 1) * L + L / 2, 200)
    assert np.abs(F.bilinear(field, L / 2, L, x, y) - (3.0 + 0.25 * x - 0.125 * y)).max() < 1e-12
    assert F.bilinear(field, L / 2, L, np.array([0.0]), np.array([0.0]))[0] == field[0, 0]
    assert F.bilinear(field, L / 2, L, np.array([1e4]), np.array([1e4]))[0] == field[-1, -1]
    one = np.array([[4.0]])
    assert F.bilinear(one, 32.0, 64.0, np.array([500.0]), np.array([-3.0]))[0] == 4.0
    assert F.round_half_up(np.array([0.5, -0.5, 1.49, -1.5]).tolist()).tolist() == [1.0, 0.0, 1.0, -1.0]


def test_mad_rule_on_hand_built_neighbourhoods():
    u = np.array([[1.0, 1.0, 2.0], [1.0, 9.0, 1.0], [2.0, 1.0, 1.0]])
    v = np.zeros((3, 3))
    valid = np.ones((3, 3), bool)
    fu, fv, rep = F.mad_filter(u, v, valid)
    # centre: median 1, MAD 0, |9 - 1| = 8 > 3 (0 + 0.5): replaced by the median
    assert rep[1, 1] and fu[1, 1] == 1.0
    # corner (0, 0): values 1, 1, 1, 9, median 1, MAD 0: 1 stays
    assert not rep[0, 0]
    # a ramp of one pixel per window is not an outlier anywhere
    ramp = np.add.outer(np.arange(5.0), np.arange(6.0))
    fu2, _, rep2 = F.mad_filter(ramp, np.zeros_like(ramp), np.ones_like(ramp, bool))
    assert not rep2.any() and np.array_equal(fu2, ramp)
    # even counts take the mean of the middle two; switched off with tau <= 0
    u3 = np.array([[0.0, 10.0], [1.0, 2.0]])
    fu3, _, rep3 = F.mad_filter(u3, np.zeros((2, 2)), np.ones((2, 2), bool))
    assert rep3[0, 1] and fu3[0, 1] == 1.5
    _, _, rep4 = F.mad_filter(u3, np.zeros((2, 2)), np.ones((2, 2), bool), tau=0.0)
    assert not rep4.any()
    # invalid windows neither count nor get a value
    valid5 = np.ones((3, 3), bool)
    valid5[1, 1] = False
    fu5, _, rep5 = F.mad_filter(u, v, valid5)
    assert not rep5.any() and fu5[1, 1] == 9.0


def _shifted_pair(seed, du, dv, N, patch=None):
    big = _speckle(N + 150, N + 150, seed=seed)
    o = 70
    ref = big[o:o + N, o:o + N].copy()
    dfm = big[o - dv:o + N - dv, o - du:o + N - du].copy()         # content moves by (du, dv)
    if patch is not None:
        x0, y0, w = patch
        dfm[y0:y0 + w, x0:x0 + w] = np.random.default_rng(1).uniform(0, 250, (w, w))
    return ref, dfm


def _interior_errors(out, du, dv, S, step, N, border, key="u"):
    lv = out["levels"][-1]
    r = (S - 1) // 2
    X, Y = np.meshgrid(np.arange(lv["nx"]) * step + r, np.arange(lv["ny"]) * step + r)
    inside = (X >= border) & (X < N - border) & (Y >= border) & (Y < N - border)
    su, sv = ("u", "v") if key == "u" else ("raw_u", "raw_v")
    e = np.maximum(np.abs(lv[su] - du), np.abs(lv[sv] - dv))
    return e[inside]


def test_multiwindow_recovers_a_large_rigid_shift_inside_a_border():
    # the shift (37 px) is beyond the reach of the radius-8 integer search; near the
    # image edges the displaced content leaves the image (the paper's SEM study
    # excludes a border for that reason), so the check keeps 100 px off the edges
    N, du, dv = 512, 37, -23
    ref, dfm = _shifted_pair(3, du, dv, N)
    out = F.multiwindow(ref, dfm, None, 21, 8, 80, subpixel=False)
    assert [lv["L"] for lv in out["levels"]] == [128, 64, 32, 21]
    e = _interior_errors(out, du, dv, 21, 8, N, 100)
    assert e.max() <= 1.0 and (e == 0).mean() > 0.97
    # the coarsest level (64 px of overlap at least) resolves the whole shift
    lv0 = out["levels"][0]
    inner = lv0["raw_u"][1:-1, 1:-1], lv0["raw_v"][1:-1, 1:-1]
    assert (inner[0] == du).all() and (inner[1] == dv).all()


def test_mad_removal_cuts_the_errors_of_a_corrupted_patch():
    N, du, dv = 384, 12, 9
    ref, dfm = _shifted_pair(5, du, dv, N, patch=(180, 180, 30))
    out = F.multiwindow(ref, dfm, None, 21, 8, 60, subpixel=False)
    raw = _interior_errors(out, du, dv, 21, 8, N, 60, key="raw")
    filt = _interior_errors(out, du, dv, 21, 8, N, 60)
    assert (raw > 2).sum() >= 3 and (filt > 2).sum() < (raw > 2).sum()
    assert out["replaced"].any()
    off = F.multiwindow(ref, dfm, None, 21, 8, 60, subpixel=False, tau=0.0)
    assert not off["replaced"].any()
    assert np.array_equal(off["levels"][-1]["u"], off["levels"][-1]["raw_u"])


def test_fft_seeds_reach_what_the_integer_search_cannot():
    W = H = 256
    fld = synth.affine_field(W, H, u0=37.4, v0=-21.7, exx=1e-3, eyy=-5e-4)
    ref = _speckle(W, H, seed=9, dtype="u8", noise=1.0)
    dfm = _speckle(W, H, seed=9, fld=fld, dtype="u8", noise=1.0)
    seeds = [(128, 128)]
    prm = dict(conv_threshold=1e-6, init="fft", max_displacement=100)
    a = O.correlate(ref, dfm, None, 21, 16, O.AFFINE, seeds, prm)
    ok = a["status"] == O.OK
    assert ok.sum() > 0.5 * len(ok)
    u, v = synth.displacement(fld, a["x"][ok].astype(float), a["y"][ok].astype(float))
    assert np.abs(a["u"][ok] - u).max() < 5e-2 and np.abs(a["v"][ok] - v).max() < 5e-2
    # the default integer search (radius 8) finds no usable start for the seed
    b = O.correlate(ref, dfm, None, 21, 16, O.AFFINE, seeds, dict(conv_threshold=1e-6))
    assert (b["status"] == O.OK).sum() == 0


def test_roi_points_only_and_subpixel_field_near_the_truth():
    # only in-ROI grid points get a last-level value; with the Gaussian fit the field
    # of a smooth sub-pixel translation lies within a fraction of a pixel of the truth
    W = H = 256
    fld = synth.affine_field(W, H, u0=6.3, v0=-4.6)
    ref = _speckle(W, H, seed=21)
    dfm = _speckle(W, H, seed=21, fld=fld)
    roi = np.zeros((H, W), np.uint8)
    roi[30:220, 40:200] = 1
    out = F.multiwindow(ref, dfm, roi, 21, 8, 30, subpixel=True)
    inroi = O.roi_points(roi, W, H, 21, 8).ravel()
    assert np.array_equal(out["status"] == O.OK, inroi)
    assert not out["u"][~inroi].any() and not out["peak"][~inroi].any()
    ok = inroi & (out["peak"] > 0.5)
    assert ok.sum() > 0.8 * inroi.sum()
    eu, ev = np.median(np.abs(out["u"][ok] - 6.3)), np.median(np.abs(out["v"][ok] + 4.6))
    assert eu < 0.35 and ev < 0.35          # the three-point fit locks towards integers a little
    # without the fit the same field is integer-valued, and further from the truth
    out_i = F.multiwindow(ref, dfm, roi, 21, 8, 30, subpixel=False)
    assert np.array_equal(out_i["u"][inroi], np.round(out_i["u"][inroi]))
    assert np.median(np.abs(out_i["u"][ok] - 6.3)) > eu and np.median(np.abs(out_i["v"][ok] + 4.6)) > ev


def test_mad_rule_matches_scipy_filters_on_interior_points():
    from scipy import ndimage

    u = RNG.integers(-3, 4, (30, 40)).astype(float)
    v = RNG.normal(0.0, 1.0, (30, 40))
    u[RNG.random(u.shape) < 0.05] += 25.0
    fu, fv, rep = F.mad_filter(u, v, np.ones(u.shape, bool))
    mad = lambda w: np.median(np.abs(w - np.median(w)))
    for c, f in ((u, fu), (v, fv)):
        med = ndimage.median_filter(c, size=3, mode="nearest")
        dev = ndimage.generic_filter(c, mad, size=3, mode="nearest")
        out = np.abs(c - med) > 3.0 * (1.4826 * dev + 0.5)
        inner = (slice(1, -1), slice(1, -1))
        # outliers in either component take both medians
        assert np.all(rep[inner] >= out[inner])
        assert np.array_equal(f[inner][rep[inner]], med[inner][rep[inner]])
    bu = np.abs(u - ndimage.median_filter(u, 3, mode="nearest")) > 3.0 * (
        1.4826 * ndimage.generic_filter(u, mad, size=3, mode="nearest") + 0.5)
    bv = np.abs(v - ndimage.median_filter(v, 3, mode="nearest")) > 3.0 * (
        1.4826 * ndimage.generic_filter(v, mad, size=3, mode="nearest") + 0.5)
    assert np.array_equal(rep[1:-1, 1:-1], (bu | bv)[1:-1, 1:-1])


def test_bilinear_matches_scipys_regular_grid_interpolator_inside():
    from scipy.interpolate import RegularGridInterpolator

    ny, nx, L = 6, 9, 32
    field = RNG.normal(0.0, 3.0, (ny, nx))
    cx = np.arange(nx) * L + L / 2
    cy = np.arange(ny) * L + L / 2
    interp = RegularGridInterpolator((cy, cx), field)
    x = RNG.uniform(cx[0], cx[-1], 300)
    y = RNG.uniform(cy[0], cy[-1], 300)
    assert np.abs(F.bilinear(field, L / 2, L, x, y) - interp(np.stack([y, x], 1))).max() < 1e-12
