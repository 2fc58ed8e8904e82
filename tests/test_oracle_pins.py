"""Pins of the FP64 oracle to things other than itself: library routines that
compute the same quantity (scipy's spline filter and spline sampling, numpy's
correlation coefficient and linear solves, scipy's graph BFS), closed forms
(cubic reproduction, integer shifts, known affine and quadratic fields), the
paper's stated defaults, invariances of the ZNSSD cost (Eq. 4), and brute-force
minimisation on tiny subsets. CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage, optimize
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle
import synth
from oracle import dic_oracle as O
from synth import workloads as wl

RNG = np.random.default_rng(20260112)


def _speckle_pair(W, H, fld, seed=7, dtype="f64", noise=0.0):
    sp = synth.Speckle(seed=seed, density=0.03, sigma=(1.5, 3.0), cell=16)
    ref = synth.ImageSpec(sp, gray_max=255.0, noise=noise, noise_tag=1)
    dfm = synth.ImageSpec(sp, field=fld, gray_max=255.0, noise=noise, noise_tag=2)
    return synth.render(ref, W, H, dtype), synth.render(dfm, W, H, dtype)


# ------------------------------------------------------------------ interpolant (Sec. 2.2)
def test_prefilter_matches_scipy_mirror_spline_filter():
    img = RNG.uniform(0, 255, size=(37, 53))
    c = O.bspline_coefficients(img)
    ref = ndimage.spline_filter(img, order=3, mode="mirror", output=np.float64)
    assert np.abs(c - ref).max() < 1e-9 * np.abs(ref).max()


def test_prefilter_rows_satisfy_the_tridiagonal_system():
    line = RNG.uniform(-5, 5, size=(3, 11))
    c = O._solve_mirror_tridiagonal(line)
    lhs = np.empty_like(c)
    lhs[:, 1:-1] = (c[:, :-2] + 4 * c[:, 1:-1] + c[:, 2:]) / 6
    lhs[:, 0] = (4 * c[:, 0] + 2 * c[:, 1]) / 6
    lhs[:, -1] = (2 * c[:, -2] + 4 * c[:, -1]) / 6
    assert np.abs(lhs - line).max() < 1e-12


def test_interpolate_matches_scipy_map_coordinates():
    img = RNG.uniform(0, 255, size=(40, 50))
    plane = O.Plane(img)
    x = RNG.uniform(1, 47.999, size=500)
    y = RNG.uniform(1, 37.999, size=500)
    val, valid = O.interpolate(plane, x, y)
    assert valid.all()
    ref = ndimage.map_coordinates(img, [y, x], order=3, mode="mirror")
    assert np.abs(val - ref).max() < 1e-9


def test_interpolate_reproduces_data_at_integer_pixels():
    img = RNG.uniform(0, 255, size=(20, 24))
    plane = O.Plane(img)
    yy, xx = np.mgrid[1:17, 1:21]
    val, valid = O.interpolate(plane, xx.ravel().astype(float), yy.ravel().astype(float))
    assert valid.all()
    assert np.abs(val - img[1:17, 1:21].ravel()).max() < 1e-10


def test_bounds_rule():
    plane = O.Plane(np.zeros((10, 12)))
    _, valid = O.interpolate(plane, np.array([0.999, 1.0, 9.999, 10.0, 5.0, 5.0]),
                             np.array([5.0, 5.0, 5.0, 5.0, 0.5, 7.9]))
    assert valid.tolist() == [False, True, True, False, False, True]


def test_cubic_polynomials_are_reproduced():
    H, W = 128, 128
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    a = RNG.uniform(-1, 1, size=(4, 4)) / np.array([[1, 64, 64 ** 2, 64 ** 3]]).T / np.array(
        [[1, 64, 64 ** 2, 64 ** 3]])

    def f(x, y):
        return sum(a[i, j] * x ** i * y ** j for i in range(4) for j in range(4))

    plane = O.Plane(f(xx, yy))
    x = RNG.uniform(32, W - 33, size=400)
    y = RNG.uniform(32, H - 33, size=400)
    val, valid = O.interpolate(plane, x, y)
    exact = f(x, y)
    assert valid.all()
    assert np.abs(val - exact).max() <= 1e-9 * np.abs(exact).max()
    # the derivative at integer pixels is the polynomial's derivative
    xi = RNG.integers(32, W - 33, size=100)
    yi = RNG.integers(32, H - 33, size=100)
    fx, fy = O.gradient_at_pixels(plane, xi, yi)
    dfx = sum(i * a[i, j] * xi.astype(float) ** (i - 1) * yi.astype(float) ** j
              for i in range(1, 4) for j in range(4))
    dfy = sum(j * a[i, j] * xi.astype(float) ** i * yi.astype(float) ** (j - 1)
              for i in range(4) for j in range(1, 4))
    scale = np.abs(exact).max() / 64
    assert np.abs(fx - dfx).max() < 1e-9 * scale
    assert np.abs(fy - dfy).max() < 1e-9 * scale


def test_gradient_matches_finite_differences_of_scipy_spline():
    img = RNG.uniform(0, 255, size=(30, 30))
    plane = O.Plane(img)
    xi = RNG.integers(3, 26, size=50)
    yi = RNG.integers(3, 26, size=50)
    fx, fy = O.gradient_at_pixels(plane, xi, yi)
    h = 1e-5

    def ms(x, y):
        return ndimage.map_coordinates(img, [y, x], order=3, mode="mirror")

    x = xi.astype(float)
    y = yi.astype(float)
    gx = (ms(x + h, y) - ms(x - h, y)) / (2 * h)
    gy = (ms(x, y + h) - ms(x, y - h)) / (2 * h)
    assert np.abs(fx - gx).max() < 1e-5
    assert np.abs(fy - gy).max() < 1e-5


def test_gradient_is_zero_across_the_mirror_border():
    img = RNG.uniform(0, 255, size=(12, 12))
    fx, fy = O.gradient_at_pixels(O.Plane(img), np.array([0, 11, 5]), np.array([5, 5, 0]))
    assert abs(fx[0]) < 1e-12 and abs(fx[1]) < 1e-12 and abs(fy[2]) < 1e-12


# ------------------------------------------------------------------ cost (Eq. 4)
def test_zncc_equals_one_minus_half_znssd_and_numpy_corrcoef():
    f = RNG.normal(size=200)
    g = 0.7 * f + 0.3 * RNG.normal(size=200) + 5.0
    fbar, gbar = f - f.mean(), g - g.mean()
    C = np.sum(fbar * gbar) / math.sqrt(np.sum(fbar ** 2) * np.sum(gbar ** 2))
    assert abs(C - np.corrcoef(f, g)[0, 1]) < 1e-12
    assert abs((1 - O.znssd(fbar, gbar) / 2) - C) < 1e-12


# ------------------------------------------------------------------ shape functions (Eq. 5)
def test_warp_follows_eq5_term_by_term():
    p = RNG.normal(size=12)
    x, y = 3.0, -2.0
    wx, wy = O.warp(p, np.array([x]), np.array([y]))
    ex = p[0] + (1 + p[2]) * x + p[3] * y + p[6] * x * x + p[7] * x * y + p[8] * y * y
    ey = p[1] + p[4] * x + (1 + p[5]) * y + p[9] * x * x + p[10] * x * y + p[11] * y * y
    assert abs(wx[0] - ex) < 1e-12 and abs(wy[0] - ey) < 1e-12
    # nesting: affine and rigid use the leading parameters only
    wx6, wy6 = O.warp(p[:6], np.array([x]), np.array([y]))
    assert abs(wx6[0] - (p[0] + (1 + p[2]) * x + p[3] * y)) < 1e-12
    wx2, _ = O.warp(p[:2], np.array([x]), np.array([y]))
    assert abs(wx2[0] - (p[0] + x)) < 1e-12


def test_affine_update_is_the_composition_of_maps():
    dx, dy = O.local_coordinates(9)
    p = np.array([1.3, -0.4, 0.02, -0.01, 0.015, -0.03])
    dp = np.array([0.05, 0.02, 0.001, 0.002, -0.001, 0.0015])
    q = O.compose_inverse(p, dp, dx, dy)
    # W(W^-1(x; dp); p) == W(x; q) at arbitrary points
    pts = RNG.uniform(-4, 4, size=(2, 20))
    inv = np.linalg.solve(np.array([[1 + dp[2], dp[3]], [dp[4], 1 + dp[5]]]),
                          pts - dp[:2, None])
    a = O.warp(p, inv[0], inv[1])
    b = O.warp(q, pts[0], pts[1])
    assert np.abs(np.array(a) - np.array(b)).max() < 1e-12
    # the quadratic refit, given affine maps, reproduces the same update exactly
    q12 = O.compose_inverse(np.r_[p, np.zeros(6)], np.r_[dp, np.zeros(6)], dx, dy)
    assert np.abs(q12[:6] - q).max() < 1e-12 and np.abs(q12[6:]).max() < 1e-12
    # rigid: translations compose by subtraction
    assert np.allclose(O.compose_inverse(p[:2], dp[:2], dx, dy), p[:2] - dp[:2])


def test_quadratic_update_fits_the_composed_map():
    dx, dy = O.local_coordinates(15)
    p = np.r_[0.5, -0.3, 1e-3, 2e-3, -1e-3, 5e-4, 1e-5, -2e-5, 1e-5, 2e-5, 1e-5, -1e-5]
    dp = np.r_[0.01, -0.02, 1e-4, -2e-4, 1e-4, 1e-4, 1e-6, 2e-6, -1e-6, 1e-6, -2e-6, 1e-6]
    q = O.compose_inverse(p, dp, dx, dy)
    u, v = O._invert_warp_pointwise(dp, dx, dy)
    zx, zy = O.warp(p, u, v)
    wx, wy = O.warp(q, dx, dy)
    # the composed map is quartic; the refit misses it by products of the small terms
    assert np.abs(zx - wx).max() < 1e-6 and np.abs(zy - wy).max() < 1e-6
    # dp = 0 leaves p unchanged
    assert np.abs(O.compose_inverse(p, np.zeros(12), dx, dy) - p).max() < 1e-14


def test_transfer_re_expands_the_same_map():
    p = RNG.normal(size=12) * np.r_[1, 1, [1e-2] * 4, [1e-4] * 6]
    q = O.transfer_warp(p, 5.0, -5.0)
    d = RNG.uniform(-6, 6, size=(2, 10))
    a = O.warp(p, d[0] + 5.0, d[1] - 5.0)
    b = O.warp(q, d[0], d[1])
    assert np.abs((a[0] - 5.0) - b[0]).max() < 1e-12 and np.abs((a[1] + 5.0) - b[1]).max() < 1e-12


# ------------------------------------------------------------------ JtJ
def test_hessian_is_gauss_newton_hessian_of_the_warped_reference():
    img, _ = _speckle_pair(64, 64, synth.IDENTITY)
    plane = O.Plane(img)
    xc, yc, S, n = 32, 31, 11, 6
    rs = O.ReferenceSubset(plane, xc, yc, S, n)
    assert np.allclose(rs.H, rs.H.T) and np.linalg.eigvalsh(rs.H).min() > 0
    # J_ij = d f(W(x_i; dp)) / d dp_j at dp = 0, by central differences of scipy's spline
    h = 1e-6
    J = np.empty((S * S, n))
    for jdx in range(n):
        e = np.zeros(n)
        e[jdx] = h
        xp, yp = O.warp(e, rs.dx, rs.dy)
        xm, ym = O.warp(-e, rs.dx, rs.dy)
        fp = ndimage.map_coordinates(img, [yc + yp, xc + xp], order=3, mode="mirror")
        fm = ndimage.map_coordinates(img, [yc + ym, xc + xm], order=3, mode="mirror")
        J[:, jdx] = (fp - fm) / (2 * h)
    Hfd = J.T @ J
    assert np.abs(Hfd - rs.H).max() < 1e-4 * np.abs(rs.H).max()


def test_lu_matches_numpy_solve_and_flags_singular():
    A = RNG.normal(size=(12, 12))
    A = A @ A.T + 12 * np.eye(12)
    b = RNG.normal(size=12)
    LU, piv, sing = O.lu_partial_pivot(A)
    assert not sing
    assert np.abs(O.lu_solve(LU, piv, b) - np.linalg.solve(A, b)).max() < 1e-10
    B = A.copy()
    B[:, 3] = B[:, 2]
    B[3, :] = B[2, :]
    assert O.lu_partial_pivot(B)[2]


# ------------------------------------------------------------------ grid, seeds, defaults
def test_grid_counts_of_the_paper_workloads():
    def count(W, H, S, s):
        xs, ys = O.grid(W, H, S, s)
        return len(xs), len(ys)

    assert count(256, 256, 21, 5) == (48, 48)
    assert count(2048, 2048, 31, 2) == (1009, 1009)
    assert count(32768, 32768, 41, 10) == (3273, 3273)
    assert count(4096, 3000, 21, 10) == (408, 298)
    xs, _ = O.grid(256, 256, 21, 5)
    assert xs[0] == 10 and xs[-1] == 245


def test_seed_snapping_ties_go_to_the_lower_index():
    assert O.snap_seed(127.5, 127.5, 256, 256, 21, 5) == (23, 23)   # 125 and 130 tie
    assert O.snap_seed(128, 127, 256, 256, 21, 5) == (24, 23)
    assert O.snap_seed(-50, 1e6, 256, 256, 21, 5) == (0, 47)


def test_paper_defaults():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_defaults.json")) as fh:
        d = json.load(fh)
    assert O.DEFAULT_PARAMS["max_iter"] == d["max_iter"]
    assert O.DEFAULT_PARAMS["conv_threshold"] == d["conv_threshold"]
    assert O.DEFAULT_PARAMS["zncc_min"] == d["zncc_min"]
    assert len(O._neighbours(5 * 10 + 5, 10, 10)) == d["neighbours"]


def test_seed_search_scores_are_numpy_corrcoef_and_argmax_is_brute_force():
    ref, dfm = _speckle_pair(96, 96, synth.affine_field(96, 96, u0=3.0, v0=-2.0), dtype="u8")
    xc, yc, S, R = 48, 47, 15, 5
    du, dv, C = O.seed_search(ref, dfm, xc, yc, S, R)
    r = S // 2
    f = ref[yc - r:yc + r + 1, xc - r:xc + r + 1].ravel().astype(float)
    scores = {}
    for v in range(-R, R + 1):
        for u in range(-R, R + 1):
            g = dfm[yc + v - r:yc + v + r + 1, xc + u - r:xc + u + r + 1].ravel().astype(float)
            scores[(u, v)] = np.corrcoef(f, g)[0, 1]
    best = max(scores, key=lambda k: scores[k])
    assert (du, dv) == best == (3, -2)
    assert abs(C - scores[best]) < 1e-12


# ------------------------------------------------------------------ IC-GN
def test_integer_shift_is_recovered_exactly():
    big, _ = _speckle_pair(110, 110, synth.IDENTITY, dtype="u8")
    ref = big[5:105, 5:105]
    dfm = big[5 + 2:105 + 2, 5 - 3:105 - 3]
    # dfm[y, x] = big[y + 7, x + 2] = ref[y + 2, x - 3]: the pattern moves by (+3, -2)
    refp, defp = O.Plane(ref), O.Plane(dfm)
    found = O.seed_search(ref, dfm, 50, 50, 21, 6)
    assert found[:2] == (3, -2) and abs(found[2] - 1.0) < 1e-12
    for shape in (O.RIGID, O.AFFINE, O.QUADRATIC):
        res = O.icgn(refp, defp, 50, 50, 21, shape, [3.0, -2.0], dict(conv_threshold=1e-8))
        n = O.N_PARAMS[shape]
        want = np.zeros(n)
        want[:2] = (3.0, -2.0)
        assert res["status"] == O.OK
        assert np.abs(res["p"] - want).max() < 1e-10
        assert abs(res["zncc"] - 1.0) < 1e-12
        assert res["iters"] <= 2


def _point_truth_affine(fld, x, y):
    u, v = synth.displacement(fld, np.array([float(x)]), np.array([float(y)]))
    return u[0], v[0]


def test_affine_field_is_recovered_from_an_unquantised_render():
    w = wl.affine_256_u8()
    ref = synth.render(w.ref, 256, 256, "f64")
    dfm = synth.render(w.deformed, 256, 256, "f64")
    refp, defp = O.Plane(ref), O.Plane(dfm)
    errs = []
    for (xc, yc) in [(60, 70), (128, 128), (190, 60), (100, 200)]:
        u, v = _point_truth_affine(w.field, xc, yc)
        res = O.icgn(refp, defp, xc, yc, 21, O.AFFINE, [round(u), round(v)],
                     dict(conv_threshold=1e-8, max_iter=100))
        assert res["status"] == O.OK
        p = res["p"]
        errs.append(max(abs(p[0] - u), abs(p[1] - v)))
        strain = np.abs(p[2:6] - np.array([1e-3, 2e-4, 2e-4, -5e-4])).max()
        assert strain < 3e-4, strain
    assert max(errs) < 2e-3, errs


def test_quadratic_field_is_recovered_with_the_12_parameter_shape_function():
    W = H = 160
    q = dict(uxx=2e-5, uxy=-1.5e-5, uyy=1e-5, vxx=-1e-5, vxy=2e-5, vyy=1.5e-5)
    fld = synth.quadratic_field(W, H, u0=1.7, v0=-0.8, exx=2e-3, exy=-1e-3, eyx=1e-3,
                                eyy=-1.5e-3, **q)
    ref, dfm = _speckle_pair(W, H, fld, seed=11)
    refp, defp = O.Plane(ref), O.Plane(dfm)
    cx = cy = (W - 1) / 2.0
    for (xc, yc) in [(70, 80), (95, 60)]:
        X, Y = xc - cx, yc - cy
        # local expansion of the field about the centre: Eq. 5 with no 1/2 factor
        truth = np.array([
            1.7 + 2e-3 * X - 1e-3 * Y + q["uxx"] * X * X + q["uxy"] * X * Y + q["uyy"] * Y * Y,
            -0.8 + 1e-3 * X - 1.5e-3 * Y + q["vxx"] * X * X + q["vxy"] * X * Y + q["vyy"] * Y * Y,
            2e-3 + 2 * q["uxx"] * X + q["uxy"] * Y, -1e-3 + q["uxy"] * X + 2 * q["uyy"] * Y,
            1e-3 + 2 * q["vxx"] * X + q["vxy"] * Y, -1.5e-3 + q["vxy"] * X + 2 * q["vyy"] * Y,
            q["uxx"], q["uxy"], q["uyy"], q["vxx"], q["vxy"], q["vyy"]])
        res = O.icgn(refp, defp, xc, yc, 31, O.QUADRATIC, [2.0, -1.0],
                     dict(conv_threshold=1e-8, max_iter=100))
        assert res["status"] == O.OK
        p = res["p"]
        assert np.abs(p[:2] - truth[:2]).max() < 2e-3
        assert np.abs(p[2:6] - truth[2:6]).max() < 3e-4
        assert np.abs(p[6:] - truth[6:]).max() < 3e-5
        # an affine fit of the same subset cannot follow the curvature as well
        ra = O.icgn(refp, defp, xc, yc, 31, O.AFFINE, [2.0, -1.0],
                    dict(conv_threshold=1e-8, max_iter=100))
        assert ra["zncc"] < res["zncc"]


def test_znssd_invariance_to_gain_and_offset():
    ref, dfm = _speckle_pair(96, 96, synth.affine_field(96, 96, u0=1.3, v0=0.6, exx=2e-3))
    refp = O.Plane(ref)
    a = O.icgn(refp, O.Plane(dfm), 48, 48, 17, O.AFFINE, [1, 1], dict(conv_threshold=1e-10))
    b = O.icgn(refp, O.Plane(2.7 * dfm + 31.0), 48, 48, 17, O.AFFINE, [1, 1],
               dict(conv_threshold=1e-10))
    assert a["status"] == b["status"] == O.OK
    assert np.abs(a["p"] - b["p"]).max() < 1e-10
    assert abs(a["zncc"] - b["zncc"]) < 1e-12


def _independent_stationarity(img_ref, img_def, xc, yc, S, p):
    """min over dp of || fbar + J dp - (df/dg) gbar(p) ||, with J, f, g from scipy alone."""
    n = len(p)
    r = S // 2
    dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
    dx = dx.ravel().astype(float)
    dy = dy.ravel().astype(float)
    f = img_ref[yc + dy.astype(int), xc + dx.astype(int)]
    fbar = f - f.mean()
    h = 1e-6
    J = np.empty((S * S, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        xp, yp = O.warp(e, dx, dy)
        xm, ym = O.warp(-e, dx, dy)
        J[:, j] = (ndimage.map_coordinates(img_ref, [yc + yp, xc + xp], order=3, mode="mirror")
                   - ndimage.map_coordinates(img_ref, [yc + ym, xc + xm], order=3,
                                             mode="mirror")) / (2 * h)
    wx, wy = O.warp(p, dx, dy)
    g = ndimage.map_coordinates(img_def, [yc + wy, xc + wx], order=3, mode="mirror")
    gbar = g - g.mean()
    e = fbar - math.sqrt(np.sum(fbar ** 2) / np.sum(gbar ** 2)) * gbar
    return np.linalg.lstsq(J, -e, rcond=None)[0]


@pytest.mark.parametrize("shape,S", [(O.RIGID, 9), (O.AFFINE, 11)])
def test_tiny_subsets_agree_with_brute_force_minimisation(shape, S):
    fld = synth.affine_field(64, 64, u0=0.4, v0=-0.3, exx=4e-3, exy=-2e-3, eyx=1e-3, eyy=3e-3)
    ref, dfm = _speckle_pair(64, 64, fld, seed=3)
    xc, yc = 31, 33
    res = O.icgn(O.Plane(ref), O.Plane(dfm), xc, yc, S, shape, [0, 0],
                 dict(conv_threshold=1e-12, max_iter=200))
    assert res["status"] == O.OK
    p = res["p"]
    # 1) the IC stationarity condition holds with every ingredient from scipy
    assert np.abs(_independent_stationarity(ref, dfm, xc, yc, S, p)).max() < 1e-6
    # 2) a dense grid then Nelder-Mead on the forward ZNSSD (Eq. 4) lands next to p
    r = S // 2
    dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
    dx = dx.ravel().astype(float)
    dy = dy.ravel().astype(float)
    f = ref[yc + dy.astype(int), xc + dx.astype(int)]
    fbar = f - f.mean()

    def cost(q):
        wx, wy = O.warp(q, dx, dy)
        g = ndimage.map_coordinates(dfm, [yc + wy, xc + wx], order=3, mode="mirror")
        return O.znssd(fbar, g - g.mean())

    n = O.N_PARAMS[shape]
    grid_uv = [(u, v) for u in np.linspace(-1, 1, 21) for v in np.linspace(-1, 1, 21)]
    u0, v0 = min(grid_uv, key=lambda uv: cost(np.r_[uv, np.zeros(n - 2)]))
    sol = optimize.minimize(cost, np.r_[u0, v0, np.zeros(n - 2)], method="Nelder-Mead",
                            options=dict(xatol=1e-10, fatol=1e-16, maxiter=40000, maxfev=40000))
    # the forward-additive minimum and the IC root differ at second order in the
    # residual (interpolation error, model mismatch): a few 1e-5 px on these renders
    assert np.abs(sol.x[:2] - p[:2]).max() < 1e-4
    assert sol.fun <= cost(p) + 1e-9


# ------------------------------------------------------------------ cost functions (Eq. 2-4)
def test_costs_have_exactly_the_invariances_of_eq2_to_eq4():
    """An integer shift of the pattern under an intensity change g = a f + c: ZNSSD
    (Eq. 4) recovers it for any a, c; NSSD (Eq. 3) for c = 0 only; SSD (Eq. 2) only
    without a change. A cost that subtracts a mean it should not, or omits a
    normalisation, fails one of these."""
    big, _ = _speckle_pair(110, 110, synth.IDENTITY, dtype="f64")
    ref = big[5:105, 5:105]
    shifted = big[5 + 2:105 + 2, 5 - 3:105 - 3]      # pattern moved by (+3, -2)
    refp = O.Plane(ref)
    want = np.array([3.0, -2.0, 0, 0, 0, 0])
    prm = dict(conv_threshold=1e-10, max_iter=100)

    def err(cost, a, c):
        res = O.icgn(refp, O.Plane(a * shifted + c), 50, 50, 21, O.AFFINE, [3.2, -1.8], dict(prm, cost=cost))
        assert res["status"] in (O.OK, O.LOW_ZNCC), (cost, a, c, res["status"])
        return np.abs(res["p"] - want).max()

    for cost in (O.ZNSSD, O.NSSD, O.SSD):
        assert err(cost, 1.0, 0.0) < 1e-9, cost
    assert err(O.ZNSSD, 1.7, 25.0) < 1e-9
    assert err(O.NSSD, 1.7, 0.0) < 1e-9
    assert err(O.NSSD, 1.0, 25.0) > 1e-4
    assert err(O.SSD, 1.7, 0.0) > 1e-4


def _stationarity(img_ref, img_def, xc, yc, S, p, cost):
    """min over dp of || e + J dp || with e the residual of the cost and J, f, g from scipy alone."""
    n = len(p)
    r = S // 2
    dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
    dx = dx.ravel().astype(float)
    dy = dy.ravel().astype(float)
    f = img_ref[yc + dy.astype(int), xc + dx.astype(int)]
    h = 1e-6
    J = np.empty((S * S, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        xp, yp = O.warp(e, dx, dy)
        xm, ym = O.warp(-e, dx, dy)
        J[:, j] = (ndimage.map_coordinates(img_ref, [yc + yp, xc + xp], order=3, mode="mirror")
                   - ndimage.map_coordinates(img_ref, [yc + ym, xc + xm], order=3,
                                             mode="mirror")) / (2 * h)
    wx, wy = O.warp(p, dx, dy)
    g = ndimage.map_coordinates(img_def, [yc + wy, xc + wx], order=3, mode="mirror")
    if cost == O.NSSD:
        e = f - math.sqrt(np.sum(f ** 2) / np.sum(g ** 2)) * g
    else:
        e = f - g
    return np.linalg.lstsq(J, -e, rcond=None)[0]


@pytest.mark.parametrize("cost", [O.NSSD, O.SSD])
def test_nssd_and_ssd_roots_are_stationary_points_computed_independently(cost):
    fld = synth.affine_field(64, 64, u0=0.4, v0=-0.3, exx=4e-3, exy=-2e-3, eyx=1e-3, eyy=3e-3)
    ref, dfm = _speckle_pair(64, 64, fld, seed=3)
    res = O.icgn(O.Plane(ref), O.Plane(dfm), 31, 33, 11, O.AFFINE, [0, 0],
                 dict(conv_threshold=1e-12, max_iter=200, cost=cost))
    assert res["status"] == O.OK
    assert np.abs(_stationarity(ref, dfm, 31, 33, 11, res["p"], cost)).max() < 1e-6


# ------------------------------------------------------------------ Levenberg-Marquardt (Sec. 2.2)
def test_levenberg_marquardt_reaches_the_gauss_newton_root(monkeypatch):
    fld = synth.affine_field(64, 64, u0=0.4, v0=-0.3, exx=4e-3, exy=-2e-3, eyx=1e-3, eyy=3e-3)
    ref, dfm = _speckle_pair(64, 64, fld, seed=3)
    refp, defp = O.Plane(ref), O.Plane(dfm)
    prm = dict(conv_threshold=1e-12, max_iter=200)
    gn = O.icgn(refp, defp, 31, 33, 11, O.AFFINE, [0, 0], prm)
    lm = O.icgn(refp, defp, 31, 33, 11, O.AFFINE, [0, 0], dict(prm, optimizer=O.LEVENBERG_MARQUARDT))
    assert gn["status"] == lm["status"] == O.OK
    assert np.abs(gn["p"] - lm["p"]).max() < 1e-9
    # the LM root is a stationary point of Eq. 4 by an independent computation
    assert np.abs(_independent_stationarity(ref, dfm, 31, 33, 11, lm["p"])).max() < 1e-6
    # without damping (lambda0 = 0, factor 1) and with every trial improving, LM is
    # Gauss-Newton step for step
    monkeypatch.setattr(O, "LM_LAMBDA0", 0.0)
    monkeypatch.setattr(O, "LM_FACTOR", 1.0)
    prm2 = dict(conv_threshold=1e-3, max_iter=3)
    a = O.icgn(refp, defp, 31, 33, 11, O.AFFINE, [0.3, -0.2], prm2)
    b = O.icgn(refp, defp, 31, 33, 11, O.AFFINE, [0.3, -0.2], dict(prm2, optimizer=O.LEVENBERG_MARQUARDT))
    assert np.abs(a["p"] - b["p"]).max() < 1e-12 and a["iters"] == b["iters"]


def test_levenberg_marquardt_matches_gauss_newton_on_every_point_of_a_correlation():
    # the convergence test is Gauss-Newton's, so every accepted point lands on the same root
    fld = synth.affine_field(120, 110, u0=1.2, v0=-0.7, exx=1.5e-3, exy=4e-4, eyx=4e-4, eyy=-8e-4)
    ref, dfm = _speckle_pair(120, 110, fld, seed=9, noise=1.0)
    prm = dict(conv_threshold=1e-8, max_iter=100, search_radius=4)
    gn = oracle.correlate(ref, dfm, None, 17, 6, O.AFFINE, [(60, 55)], prm)
    lm = oracle.correlate(ref, dfm, None, 17, 6, O.AFFINE, [(60, 55)], dict(prm, optimizer=O.LEVENBERG_MARQUARDT))
    both = (gn["status"] == O.OK) & (lm["status"] == O.OK)
    assert both.sum() > 0.85 * len(gn["status"])    # the rest leave the image near its edges, in both
    assert np.array_equal(gn["status"] == O.OK, lm["status"] == O.OK)
    assert np.abs(gn["p"][both] - lm["p"][both]).max() < 1e-7


def test_levenberg_marquardt_recovers_from_a_poor_start():
    fld = synth.affine_field(96, 96, u0=1.3, v0=0.6, exx=2e-3)
    ref, dfm = _speckle_pair(96, 96, fld)
    refp, defp = O.Plane(ref), O.Plane(dfm)
    prm = dict(conv_threshold=1e-10, max_iter=100, optimizer=O.LEVENBERG_MARQUARDT)
    near = O.icgn(refp, defp, 48, 48, 21, O.AFFINE, [1.3, 0.6], prm)
    far = O.icgn(refp, defp, 48, 48, 21, O.AFFINE, [2.4, -0.3], prm)
    assert near["status"] == far["status"] == O.OK
    assert np.abs(near["p"] - far["p"]).max() < 1e-8


def test_flat_and_singular_subsets():
    flat = np.full((40, 40), 100.0)
    res = O.icgn(O.Plane(flat), O.Plane(flat), 20, 20, 11, O.AFFINE, [0, 0])
    assert res["status"] == O.FLAT_SUBSET
    stripes = np.tile(100 + 50 * np.sin(np.arange(40) / 2.0), (40, 1))   # no y texture
    res = O.icgn(O.Plane(stripes), O.Plane(stripes), 20, 20, 11, O.AFFINE, [0, 0])
    assert res["status"] == O.SINGULAR_H


def test_out_of_bounds_is_reported():
    ref, dfm = _speckle_pair(64, 64, synth.affine_field(64, 64, u0=0.3))
    res = O.icgn(O.Plane(ref), O.Plane(dfm), 10, 32, 21, O.AFFINE, [-0.5, 0])
    assert res["status"] == O.OUT_OF_BOUNDS


# ------------------------------------------------------------------ propagation (Sec. 2.4)
def test_propagation_waves_are_bfs_distances_over_accepted_points():
    W = H = 120
    fld = synth.affine_field(W, H, u0=1.2, v0=-0.6, exx=1e-3, eyy=-1e-3)
    ref, dfm = _speckle_pair(W, H, fld, seed=5, dtype="u8")
    roi = np.ones((H, W), bool)
    roi[50:70, 20:45] = False        # a hole the front must go around
    roi[:, 100:] = False
    S, step = 11, 6
    res = O.correlate(ref, dfm, roi, S, step, O.AFFINE, [(60, 30)], dict(search_radius=3))
    nx, ny = res["nx"], res["ny"]
    st, wave = res["status"], res["wave"]
    inroi = O.roi_points(roi, W, H, S, step).ravel()
    assert (st[~inroi] == O.NOT_IN_ROI).all()
    seed = int(np.flatnonzero(wave == 0)[0])
    # BFS over the grid graph, leaving only from accepted points, into in-ROI points
    rows, cols = [], []
    for q in range(nx * ny):
        if st[q] == O.OK:
            for nb in O._neighbours(q, nx, ny):
                if inroi[nb]:
                    rows.append(q)
                    cols.append(nb)
    G = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nx * ny, nx * ny))
    dist = shortest_path(G, unweighted=True, indices=[seed])[0]
    attempted = wave >= 0
    assert np.array_equal(np.isfinite(dist), attempted)
    assert np.array_equal(dist[attempted].astype(int), wave[attempted])
    assert (st[inroi & ~attempted] == O.NOT_REACHED).all()
    assert (st == O.OK).sum() > 0.8 * inroi.sum()
    # every accepted non-seed point has an accepted neighbour one wave earlier
    for q in np.flatnonzero((st == O.OK) & (wave > 0)):
        assert any(st[nb] == O.OK and wave[nb] == wave[q] - 1 for nb in O._neighbours(q, nx, ny))


def test_nan_flag_blanks_rejected_points_only():
    w = wl.affine_256_u8()
    ref = synth.render(w.ref, 96, 96, "u8")
    dfm = synth.render(w.deformed, 96, 96, "u8")
    res = O.correlate(ref, dfm, None, 21, 8, O.AFFINE, [(48, 48)],
                      dict(search_radius=4, nan_unconverged=True))
    ok = res["status"] == O.OK
    assert ok.any() and (~ok).any()
    assert np.isfinite(res["u"][ok]).all() and np.isnan(res["u"][~ok]).all()


# ------------------------------------------------------------------ the pins catch planted mistakes
def test_pins_catch_a_planted_sign_error(monkeypatch):
    """A wrong sign in the steepest-descent images (a plausible slip) must break the
    affine recovery check above: plant it in the oracle and re-run the check."""
    orig = O.warp_jacobian_p

    def bad(dx, dy, n):
        jx, jy = orig(dx, dy, n)
        jx = jx.copy()
        jx[:, 3] = -jx[:, 3]
        return jx, jy

    monkeypatch.setattr(O, "warp_jacobian_p", bad)
    with pytest.raises(AssertionError):
        test_affine_field_is_recovered_from_an_unquantised_render()


def test_pins_catch_a_planted_transposed_update(monkeypatch):
    """Composing the update the wrong way round (p o dp instead of p o dp^-1)."""
    def bad(p, dp, dx, dy):
        M = O._affine_matrix(p) @ O._affine_matrix(dp)
        return np.array([M[0, 2], M[1, 2], M[0, 0] - 1.0, M[0, 1], M[1, 0], M[1, 1] - 1.0])

    monkeypatch.setattr(O, "compose_inverse", bad)
    with pytest.raises(AssertionError):
        test_affine_field_is_recovered_from_an_unquantised_render()


def test_final_coefficient_is_taken_at_the_warp_of_reading_8():
    # Gauss-Newton: the coefficient of the last iteration's pass (the warp before the
    # final update); Levenberg-Marquardt: one more pass at the final p. Both checked
    # against numpy's correlation coefficient of independently sampled subsets.
    w = wl.affine_256_u8()
    ref = synth.render(w.ref, 256, 256, "f64")
    dfm = synth.render(w.deformed, 256, 256, "f64")
    refp, defp = O.Plane(ref), O.Plane(dfm)
    xc, yc, S = 120, 130, 21
    dx, dy = O.local_coordinates(S)
    f = ref[yc + dy.astype(int), xc + dx.astype(int)]
    start = [2.0, -2.0, 0.0, 0.0, 0.0, 0.0]

    def coefficient(p):
        wx, wy = O.warp(np.asarray(p, float), dx, dy)
        g, valid = O.interpolate(defp, xc + wx, yc + wy)
        assert valid.all()
        return np.corrcoef(f, g)[0, 1]

    # one Gauss-Newton iteration: the coefficient is the start warp's, p is updated
    one = O.icgn(refp, defp, xc, yc, S, O.AFFINE, start, dict(max_iter=1, conv_threshold=1e-12))
    assert one["iters"] == 1 and np.abs(one["p"] - np.array(start)).max() > 0.1
    assert abs(one["zncc"] - coefficient(start)) < 1e-12
    # converged: the coefficient of the last pass, within the threshold of the final p's
    full = O.icgn(refp, defp, xc, yc, S, O.AFFINE, start, dict(conv_threshold=1e-3, max_iter=100))
    assert full["converged"] and full["status"] == O.OK
    assert abs(full["zncc"] - coefficient(full["p"])) < 1e-5
    lm = O.icgn(refp, defp, xc, yc, S, O.AFFINE, start, dict(conv_threshold=1e-3, max_iter=100, optimizer="lm"))
    assert lm["converged"] and abs(lm["zncc"] - coefficient(lm["p"])) < 1e-14


# --------------------------------------------------------------------------- ROI rule
# Sec. 2.1 gives the region of interest as a boolean mask; the rule read from it is
# that a grid point is in the ROI when every pixel of its S x S reference subset is
# in the mask. The expected flags below are worked out by hand from that rule (they
# are not computed by the oracle).

def _mask(W, H, value=True):
    return np.full((H, W), value, dtype=bool)


def test_roi_rule_one_hole_pixel_removes_exactly_the_subsets_that_cover_it():
    # 12 x 12, S = 5 (r = 2), step 1: centres 2..9 on both axes (8 x 8 points). A hole
    # at (x, y) = (5, 5) lies in the subsets with centres 3..7 on both axes.
    m = _mask(12, 12)
    m[5, 5] = False
    got = O.roi_points(m, 12, 12, 5, 1)
    want = np.ones((8, 8), bool)
    want[1:6, 1:6] = False            # centres 3..7 are indices 1..5
    assert got.shape == (8, 8)
    assert np.array_equal(got, want)
    assert got.sum() == 39
    # the hole at each corner of a subset: centre (7, 7) has it at its top-left
    # corner, (3, 3) at its bottom-right, (7, 3) at its bottom-left, (3, 7) at its
    # top-right; one step further out the subset misses it
    for xc, yc in ((7, 7), (3, 3), (7, 3), (3, 7)):
        assert not got[yc - 2, xc - 2], (xc, yc)
    for xc, yc in ((8, 7), (2, 3), (7, 8), (3, 2)):
        assert got[yc - 2, xc - 2], (xc, yc)


def test_roi_rule_mask_edge_exactly_at_the_subset_edge():
    # mask true for x <= 7 only: centre xc is in when xc + r <= 7, i.e. xc <= 5 (r = 2)
    m = _mask(12, 12)
    m[:, 8:] = False
    got = O.roi_points(m, 12, 12, 5, 1)
    want = np.zeros((8, 8), bool)
    want[:, :4] = True                # centres 2, 3, 4, 5
    assert np.array_equal(got, want)
    # the same edge along y: true for y >= 4 only, so yc - r >= 4, yc >= 6
    m = _mask(12, 12)
    m[:4, :] = False
    got = O.roi_points(m, 12, 12, 5, 1)
    want = np.zeros((8, 8), bool)
    want[4:, :] = True                # centres 6, 7, 8, 9
    assert np.array_equal(got, want)


def test_roi_rule_narrow_regions():
    # a one-pixel-wide ROI holds no subset of side 3 or more
    m = _mask(12, 12, False)
    m[:, 6] = True
    assert not O.roi_points(m, 12, 12, 3, 1).any()
    assert not O.roi_points(m, 12, 12, 5, 1).any()
    # a band exactly S wide (columns 3..7, S = 5) holds one column of centres, xc = 5
    m = _mask(12, 12, False)
    m[:, 3:8] = True
    got = O.roi_points(m, 12, 12, 5, 1)
    want = np.zeros((8, 8), bool)
    want[:, 3] = True
    assert np.array_equal(got, want)


def test_roi_rule_with_a_step():
    # 10 x 10, S = 3 (r = 1), step 3: centres 1, 4, 7 per axis; subsets cover
    # columns (and rows) 0..2, 3..5 and 6..8. A hole at (4, 4) lies in the subset of
    # centre (4, 4) only; so does a hole at (x, y) = (3, 5).
    m = _mask(10, 10)
    m[4, 4] = False
    got = O.roi_points(m, 10, 10, 3, 3)
    want = np.ones((3, 3), bool)
    want[1, 1] = False
    assert np.array_equal(got, want)
    m = _mask(10, 10)
    m[5, 3] = False                   # row y = 5, column x = 3
    assert np.array_equal(O.roi_points(m, 10, 10, 3, 3), want)
    # a hole at (2, 0) lies in the subset of centre (1, 1) only
    m = _mask(10, 10)
    m[0, 2] = False
    want = np.ones((3, 3), bool)
    want[0, 0] = False
    assert np.array_equal(O.roi_points(m, 10, 10, 3, 3), want)
    # row 9 and column 9 lie in no subset: a hole there removes nothing
    m = _mask(10, 10)
    m[9, :] = False
    m[:, 9] = False
    assert O.roi_points(m, 10, 10, 3, 3).all()


def test_out_of_bounds_test_applies_to_the_warp_of_the_last_pass():
    # R8: Gauss-Newton takes the coefficient, the in-bounds test and the
    # flatness test from the sampling pass of its last iteration, whose warp is the one
    # before the final update. A point whose last pass lies inside the sampling bounds
    # is accepted even when the final update carries its subset outside them.
    W, H = 64, 40
    rng = np.random.default_rng(3)
    base = ndimage.gaussian_filter(rng.random((H, W + 8)), 1.5) * 200.0
    ref = np.ascontiguousarray(base[:, 4:4 + W])
    dfm = np.ascontiguousarray(base[:, 1:1 + W])        # the content moves 3 px to +x
    refp, defp = O.Plane(ref), O.Plane(dfm)
    S, r = 11, 5
    xc, yc = W - 2 - r - 1, 20                          # at p = 0 the last column is x = W - 3
    prm = dict(max_iter=1, conv_threshold=10.0, zncc_min=-1.0)
    res = O.icgn(refp, defp, xc, yc, S, O.AFFINE, [0.0] * 6, prm)
    assert res["iters"] == 1 and res["converged"] and res["status"] == O.OK
    assert res["p"][0] > 1.0                            # the update moved the subset right
    dx, dy = O.local_coordinates(S)
    wx, wy = O.warp(res["p"], dx, dy)
    _, valid = O.interpolate(defp, xc + wx, yc + wy)
    assert not valid.all()                              # the final warp leaves the bounds
    _, valid0 = O.interpolate(defp, xc + dx, yc + dy)
    assert valid0.all()                                 # the pass that decided was inside
