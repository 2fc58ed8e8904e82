"""FP64 CPU oracle for local-subset 2D DIC: ZNSSD cost, rigid / affine / quadratic
shape functions, cubic B-spline (or Keys bicubic) interpolation,
inverse-compositional Gauss-Newton (IC-GN) per subset, integer ZNCC seed search
and reliability-guided propagation in deterministic waves.

TEST INFRASTRUCTURE. This module is the plain, slow, obviously correct reference
that the CUDA library is checked against. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and it shares
no code, table or constant with the library.

Paper: Hirst et al., "Pyvale: a fast, scalable, open-source 2D DIC engine capable
of handling gigapixel images" (arXiv 2601.12941). What each part follows:

  * Eq. 4, Sec. 2.2   ZNSSD cost; the correlation coefficient reported is
                      ZNCC = 1 - ZNSSD / 2.
  * Eq. 5, Sec. 2.2   shape functions xi(x, y; p), nested rigid (p0..p1), affine
                      (p0..p5) and quadratic (p0..p11), no 1/2 on the quadratic terms.
  * Sec. 2.2          a bicubic B-spline gives gray levels at sub-pixel positions.
  * Sec. 2.2          per-subset non-linear optimisation of p; the paper names
                      Levenberg-Marquardt and leaves the details to the literature.
                      This oracle runs the undamped inverse-compositional
                      Gauss-Newton form (Pan, Li & Tong 2013).
  * Sec. 4            defaults: 40 iterations, threshold 0.01, "precision" 0.70.
  * Sec. 2.4, Fig. 3  reliability-guided propagation from a seed to its four
                      nearest neighbours, ranked by correlation coefficient.

Readings taken where the paper is silent (all of them, in one place):

  R1  Interpolant: interpolating cubic B-spline. Coefficients c solve
      (c[k-1] + 4 c[k] + c[k+1]) / 6 = I[k] along rows then columns, whole-sample
      mirror boundary c[-1] = c[1], c[N] = c[N-2].
  R2  Sampling bounds: a sample at (x, y) is valid iff 1 <= x < W-2 and
      1 <= y < H-2; any invalid sample makes the subset out-of-bounds.
  R3  Grid: r = (S-1)/2, centres r + k*step, n = floor((W-1-2r)/step) + 1 per axis,
      point index q = j * nx + i. A point is in the ROI iff every pixel of its
      S x S reference subset is in the mask.
  R4  Local coordinates (dx, dy) in [-r, r]^2 about the subset centre. f is the
      reference gray level; grad f is the exact derivative of the reference spline
      at the integer pixel, with the mirror extension of R1 at the image border.
  R5  Singular H: a pivot of Gaussian elimination with partial pivoting at or below
      1e-12 * max|diag(H)|. Flat subset: RMS of f - f_m (or g - g_m) at or below
      1e-6 * max(|mean|, 1).
  R6  Quadratic update: W(.; p) o W(.; dp)^-1 is not quadratic; the oracle inverts
      W(.; dp) at every subset pixel by Newton's method, applies W(.; p) and refits
      the 12 parameters by least squares over the subset pixels.
  R7  Convergence: ||dp||_s = sqrt(dp0^2 + dp1^2 + r^2 sum dp2..5^2 + r^4 sum dp6..11^2)
      below the threshold; iters counts applied updates.
  R8  "Precision 0.70" is the ZNCC acceptance cut-off; "threshold 0.01" is the
      ||dp||_s threshold. Accepted iff converged, ZNCC >= cut-off and in bounds. The
      paper does not say at which warp the coefficient is taken. Gauss-Newton takes
      it, with the in-bounds and flatness tests, from the sampling pass of the last
      iteration (the warp the final, sub-threshold update was computed at); the
      reported p includes that update. Levenberg-Marquardt (R13) takes it with one
      more sampling pass at the final p.
  R9  Seed search: integer offsets |du|, |dv| <= R whose whole deformed subset is
      inside the image, scored by ZNCC from exact integer sums (float images: FP64
      sums) as C = (N Sfg - Sf Sg) / sqrt((N Sff - Sf^2)(N Sgg - Sg^2)); the best is
      the larger C, then smaller |du|+|dv|, then smaller dv, then smaller du.
  R10 Propagation in waves: wave 0 is the seeds (snapped to the nearest grid point,
      ties to the lower index); wave k+1 is every in-ROI, never-attempted
      4-neighbour of a point accepted in wave k. Each point is attempted once, from
      the warp of its accepted neighbour (earlier waves) with the highest ZNCC
      (ties to the lower index), re-expanded about the new centre.
  R11 Sequences (one reference, many deformed images, Sec. 2.1): frame k starts
      every point accepted in frame k-1 from its frame k-1 warp, all in wave 0;
      the remaining points are reached by propagation as in R10.
  R12 Cost functions (Eq. 2-4): ZNSSD (the default), NSSD and SSD. The IC-GN
      step solves H dp = -b with b = sum SD_i e_i and
        ZNSSD  e_i = fbar_i - (df / dg) gbar_i,   df = ||fbar||, dg = ||gbar||,
        NSSD   e_i = f_i - (||f|| / ||g||) g_i,
        SSD    e_i = f_i - g_i,
      the Gauss-Newton step of each cost in the inverse-compositional form (H =
      sum SD_i^T SD_i for all three). Whatever the cost, the reported coefficient
      and the acceptance test stay the ZNCC at the final p (R8).
  R13 Levenberg-Marquardt (Sec. 2.2 names the method and leaves its details to the
      literature; optimizer "lm"): every iteration samples the trial warp p_k and
      evaluates the cost C_k (Eq. 2-4) and the undamped Gauss-Newton step
      s_k = ||-H^-1 b(p_k)||_s (R7) there. The trial is kept when it is the first,
      lowers the cost (C_k < C_best) or shortens that step (s_k < s_best): the
      inverse-compositional root and the minimum of the cost differ at second order,
      so near convergence the cost alone can refuse every step towards the root.
      Keeping divides lambda by 10 (p_best, b_best, C_best, s_best become the
      trial's), refusing multiplies it by 10; lambda starts at 1e-3. The point has
      converged when s_best is below the threshold; the undamped step is then
      applied (p_best o dp^-1), so the stopping rule, and the root, are those of
      Gauss-Newton. Otherwise the damped step solves (H + lambda diag(H)) dp =
      -b_best and the next trial is p_best o dp^-1. iters counts the trials.
  R14 Bicubic interpolation (interp "bicubic"; Sec. 2.2 names the bicubic B-spline
      as the default, the library's create call takes the interpolant as an
      argument): Keys' cubic convolution kernel with a = -1/2,
        K(s) = (a+2)|s|^3 - (a+3)|s|^2 + 1         on |s| <= 1,
        K(s) = a|s|^3 - 5a|s|^2 + 8a|s| - 4a       on 1 < |s| < 2,  0 beyond,
      applied to the gray levels themselves (no prefilter: K interpolates), with the
      same support {-1, 0, 1, 2}, sampling bounds (R2) and mirror boundary (R1) as
      the spline. grad f at a pixel is the derivative of that interpolant there,
      which is the central difference (f[k+1] - f[k-1]) / 2.
  R15 Seeds from the multi-window FFT initialiser (init "fft"; Sec. 2.2): the
      seeds start from its estimate instead of the integer search of R9, as stated
      in reading F8 of fft_oracle, which holds the initialiser's own readings.
"""
from __future__ import annotations

import math

import numpy as np

RIGID, AFFINE, QUADRATIC = "rigid", "affine", "quadratic"
N_PARAMS = {RIGID: 2, AFFINE: 6, QUADRATIC: 12}

OK, NOT_IN_ROI, NOT_REACHED, OUT_OF_BOUNDS, MAX_ITER, LOW_ZNCC, SINGULAR_H, FLAT_SUBSET = range(8)

# Sec. 4: 40 iterations, convergence threshold 0.01, precision 0.70 (reading R8)
ZNSSD, NSSD, SSD = "znssd", "nssd", "ssd"
GAUSS_NEWTON, LEVENBERG_MARQUARDT = "gn", "lm"
LM_LAMBDA0, LM_FACTOR = 1e-3, 10.0
BSPLINE3, BICUBIC = "bspline3", "bicubic"
KEYS_A = -0.5
DEFAULT_PARAMS = dict(max_iter=40, conv_threshold=0.01, zncc_min=0.70, search_radius=8,
                      nan_unconverged=False, cost=ZNSSD, optimizer=GAUSS_NEWTON, interp=BSPLINE3,
                      init="search", max_displacement=32, mad_tau=3.0, mad_eps=0.5)


# --------------------------------------------------------------------------- R1
def _solve_mirror_tridiagonal(rhs: np.ndarray) -> np.ndarray:
    """Solve (c[k-1] + 4c[k] + c[k+1]) / 6 = rhs[k] along the last axis, with
    c[-1] = c[1] and c[N] = c[N-2], by forward elimination and back substitution
    (Thomas algorithm). Rows 0 and N-1 read (4c0 + 2c1)/6 and (2c[N-2] + 4c[N-1])/6."""
    N = rhs.shape[-1]
    if N < 2:
        raise ValueError("a line needs at least 2 samples")
    sub = np.ones(N)
    sup = np.ones(N)
    diag = np.full(N, 4.0)
    sup[0] = 2.0
    sub[N - 1] = 2.0
    r = 6.0 * np.moveaxis(np.asarray(rhs, dtype=np.float64), -1, 0).copy()
    cp = np.empty(N)
    cp[0] = sup[0] / diag[0]
    r[0] = r[0] / diag[0]
    for k in range(1, N):
        m = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / m if k < N - 1 else 0.0
        r[k] = (r[k] - sub[k] * r[k - 1]) / m
    for k in range(N - 2, -1, -1):
        r[k] = r[k] - cp[k] * r[k + 1]
    return np.moveaxis(r, 0, -1)


def bspline_coefficients(image: np.ndarray) -> np.ndarray:
    """Interpolating cubic B-spline coefficients (Sec. 2.2, reading R1): rows, then columns."""
    img = np.asarray(image, dtype=np.float64)
    c = _solve_mirror_tridiagonal(img)            # along x (last axis)
    c = _solve_mirror_tridiagonal(c.T).T          # along y
    return c


# --------------------------------------------------------------------------- R2
def beta3(s):
    """Centred cubic B-spline: 2/3 - s^2 + |s|^3/2 on |s| <= 1, (2-|s|)^3/6 on 1 < |s| < 2."""
    a = np.abs(np.asarray(s, dtype=np.float64))
    return np.where(a <= 1.0, 2.0 / 3.0 - a * a + 0.5 * a ** 3,
                    np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))


def beta3_prime(s):
    """Derivative of beta3."""
    s = np.asarray(s, dtype=np.float64)
    a = np.abs(s)
    d = np.where(a <= 1.0, -2.0 * a + 1.5 * a * a, np.where(a < 2.0, -0.5 * (2.0 - a) ** 2, 0.0))
    return np.sign(s) * d


def keys(s, a=KEYS_A):
    """Keys' cubic convolution kernel (reading R14)."""
    s = np.abs(np.asarray(s, dtype=np.float64))
    return np.where(s <= 1.0, (a + 2.0) * s ** 3 - (a + 3.0) * s * s + 1.0,
                    np.where(s < 2.0, a * s ** 3 - 5.0 * a * s * s + 8.0 * a * s - 4.0 * a, 0.0))


def keys_prime(s, a=KEYS_A):
    """Derivative of keys."""
    s = np.asarray(s, dtype=np.float64)
    m = np.abs(s)
    d = np.where(m <= 1.0, 3.0 * (a + 2.0) * m * m - 2.0 * (a + 3.0) * m,
                 np.where(m < 2.0, 3.0 * a * m * m - 10.0 * a * m + 8.0 * a, 0.0))
    return np.sign(s) * d


_KERNELS = {BSPLINE3: (beta3, beta3_prime), BICUBIC: (keys, keys_prime)}


class Plane:
    """Gray levels and interpolation coefficients of an image, or of a crop of it
    whose top-left pixel is (x0, y0) in a width x height image. Spline coefficients
    (R1) carry the mirror boundary at a crop's own edges; where a crop edge is not an
    image edge, points must stay far from it (the influence decays as
    0.268^distance). The bicubic interpolant (R14) uses the gray levels as its
    coefficients."""

    def __init__(self, gray, x0=0, y0=0, width=None, height=None, interp=BSPLINE3):
        self.gray = np.asarray(gray)
        if interp not in _KERNELS:
            raise ValueError("unknown interpolant %r" % (interp,))
        self.interp = interp
        self.kernel, self.kernel_prime = _KERNELS[interp]
        self.c = bspline_coefficients(self.gray) if interp == BSPLINE3 else self.gray.astype(np.float64)
        self.x0, self.y0 = int(x0), int(y0)
        self.h, self.w = self.gray.shape
        self.W = int(width) if width is not None else self.w
        self.H = int(height) if height is not None else self.h

    def gray_at(self, xs, ys):
        return self.gray[np.asarray(ys) - self.y0, np.asarray(xs) - self.x0]


class CropMiss(RuntimeError):
    """A sample needs coefficients outside the crop that the oracle was given."""


def interpolate(plane: Plane, x, y):
    """Interpolated value at (x, y) (image coordinates) and the validity mask of
    reading R2. value = sum over l, k in {-1, 0, 1, 2} of c[j+l, i+k] K(tx-k) K(ty-l),
    K = beta3 on spline coefficients (R1) or Keys' kernel on gray levels (R14)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    valid = (x >= 1.0) & (x < plane.W - 2) & (y >= 1.0) & (y < plane.H - 2)
    i = np.floor(x).astype(np.int64)
    j = np.floor(y).astype(np.int64)
    tx = x - i
    ty = y - j
    li = i - plane.x0
    lj = j - plane.y0
    if valid.any():
        vi, vj = li[valid], lj[valid]
        if vi.min() < 1 or vj.min() < 1 or vi.max() > plane.w - 3 or vj.max() > plane.h - 3:
            raise CropMiss("sample outside the crop")
    li = np.clip(li, 1, plane.w - 3)
    lj = np.clip(lj, 1, plane.h - 3)
    out = np.zeros_like(x)
    K = plane.kernel
    for l in range(-1, 3):
        wy = K(ty - l)
        for k in range(-1, 3):
            out += plane.c[lj + l, li + k] * K(tx - k) * wy
    return out, valid


def gradient_at_pixels(plane: Plane, xs, ys):
    """Exact derivatives of the interpolant at integer pixels (readings R4, R14):
    fx = sum_{l,k} c[y+l, x+k] K'(-k) K(-l), fy likewise; coefficients beyond the
    image border are mirrored (c[-1] = c[1], c[N] = c[N-2])."""
    xs = np.asarray(xs, dtype=np.int64)
    ys = np.asarray(ys, dtype=np.int64)

    def mirror(a, n):
        a = np.where(a < 0, -a, a)
        return np.where(a > n - 1, 2 * (n - 1) - a, a)

    fx = np.zeros(xs.shape)
    fy = np.zeros(xs.shape)
    for l in (-1, 0, 1):
        for k in (-1, 0, 1):
            gx = mirror(xs + k, plane.W) - plane.x0
            gy = mirror(ys + l, plane.H) - plane.y0
            if gx.min() < 0 or gy.min() < 0 or gx.max() >= plane.w or gy.max() >= plane.h:
                raise CropMiss("gradient stencil outside the crop")
            cv = plane.c[gy, gx]
            fx += cv * plane.kernel_prime(-k) * plane.kernel(-l)
            fy += cv * plane.kernel(-k) * plane.kernel_prime(-l)
    return fx, fy


# --------------------------------------------------------------------------- R3
def grid(width: int, height: int, subset_size: int, subset_step: int):
    """Subset centres along x and y (reading R3)."""
    r = (subset_size - 1) // 2
    nx = (width - 1 - 2 * r) // subset_step + 1
    ny = (height - 1 - 2 * r) // subset_step + 1
    if nx <= 0 or ny <= 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return r + subset_step * np.arange(nx), r + subset_step * np.arange(ny)


def roi_points(roi, width, height, subset_size, subset_step):
    """In-ROI flag per grid point, shape (ny, nx): the whole S x S subset is in the mask."""
    xs, ys = grid(width, height, subset_size, subset_step)
    if roi is None:
        return np.ones((len(ys), len(xs)), dtype=bool)
    m = np.asarray(roi).astype(bool)
    r = (subset_size - 1) // 2
    out = np.zeros((len(ys), len(xs)), dtype=bool)
    for j, yc in enumerate(ys):
        for i, xc in enumerate(xs):
            out[j, i] = m[yc - r:yc + r + 1, xc - r:xc + r + 1].all()
    return out


def snap_seed(sx, sy, width, height, subset_size, subset_step):
    """Nearest grid point to a seed pixel, ties to the lower index; returns (i, j)."""
    xs, ys = grid(width, height, subset_size, subset_step)
    i = int(np.argmin(np.abs(xs - sx)))   # argmin keeps the first (lower) of equal distances
    j = int(np.argmin(np.abs(ys - sy)))
    return i, j


# --------------------------------------------------------------------------- R4, Eq. 5
def local_coordinates(subset_size: int):
    """(dx, dy) of the subset pixels, row-major (dy outer, dx inner)."""
    r = (subset_size - 1) // 2
    dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
    return dx.ravel().astype(np.float64), dy.ravel().astype(np.float64)


def warp(p, dx, dy):
    """xi(x, y; p) of Eq. 5 in local coordinates: returns (xi_x, xi_y) = (dx, dy) mapped."""
    p = np.asarray(p, dtype=np.float64)
    n = p.size
    xx = dx + p[0]
    yy = dy + p[1]
    if n >= 6:
        xx = xx + p[2] * dx + p[3] * dy
        yy = yy + p[4] * dx + p[5] * dy
    if n >= 12:
        xx = xx + p[6] * dx * dx + p[7] * dx * dy + p[8] * dy * dy
        yy = yy + p[9] * dx * dx + p[10] * dx * dy + p[11] * dy * dy
    return xx, yy


def warp_jacobian_p(dx, dy, n):
    """d xi / d p at p = 0 (Eq. 5): rows for xi_x and xi_y, one column per parameter."""
    z = np.zeros_like(dx)
    o = np.ones_like(dx)
    jx = [o, z, dx, dy, z, z, dx * dx, dx * dy, dy * dy, z, z, z][:n]
    jy = [z, o, z, z, dx, dy, z, z, z, dx * dx, dx * dy, dy * dy][:n]
    return np.stack(jx, axis=1), np.stack(jy, axis=1)


def steepest_descent_images(fx, fy, dx, dy, n):
    """SD_i = grad f_i . d xi / d p, an (N, n) matrix."""
    jx, jy = warp_jacobian_p(dx, dy, n)
    return fx[:, None] * jx + fy[:, None] * jy


def lu_partial_pivot(H):
    """Gaussian elimination with partial pivoting; singular per reading R5."""
    A = np.array(H, dtype=np.float64)
    n = A.shape[0]
    piv = np.arange(n)
    tol = 1e-12 * np.max(np.abs(np.diag(A))) if n else 0.0
    for k in range(n):
        m = k + int(np.argmax(np.abs(A[k:, k])))
        if abs(A[m, k]) <= tol:
            return A, piv, True
        if m != k:
            A[[k, m]] = A[[m, k]]
            piv[[k, m]] = piv[[m, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv, False


def lu_solve(LU, piv, b):
    n = LU.shape[0]
    y = np.asarray(b, dtype=np.float64)[piv].copy()
    for i in range(n):
        y[i] -= LU[i, :i] @ y[:i]
    for i in range(n - 1, -1, -1):
        y[i] = (y[i] - LU[i, i + 1:] @ y[i + 1:]) / LU[i, i]
    return y


def _affine_matrix(p):
    return np.array([[1.0 + p[2], p[3], p[0]], [p[4], 1.0 + p[5], p[1]], [0.0, 0.0, 1.0]])


def _invert_warp_pointwise(dp, x, y, tol=1e-13, max_steps=60):
    """y solving W(y; dp) = x at every point, by Newton's method (reading R6)."""
    u, v = x - dp[0], y - dp[1]
    for _ in range(max_steps):
        wx, wy = warp(dp, u, v)
        rx, ry = wx - x, wy - y
        if max(np.abs(rx).max(), np.abs(ry).max()) < tol:
            break
        a = 1.0 + dp[2] + 2.0 * dp[6] * u + dp[7] * v
        b = dp[3] + dp[7] * u + 2.0 * dp[8] * v
        c = dp[4] + 2.0 * dp[9] * u + dp[10] * v
        d = 1.0 + dp[5] + dp[10] * u + 2.0 * dp[11] * v
        det = a * d - b * c
        u = u - (d * rx - b * ry) / det
        v = v - (-c * rx + a * ry) / det
    return u, v


def compose_inverse(p, dp, dx, dy):
    """Inverse-compositional update p <- p o dp^-1, i.e. W(W^-1(x; dp); p).
    Rigid: p - dp. Affine: M(p) M(dp)^-1 with M the 3x3 homogeneous matrix.
    Quadratic: reading R6 (pointwise Newton inverse, then least-squares refit)."""
    p = np.asarray(p, dtype=np.float64)
    dp = np.asarray(dp, dtype=np.float64)
    n = p.size
    if n == 2:
        return p - dp
    if n == 6:
        M = _affine_matrix(p) @ np.linalg.inv(_affine_matrix(dp))
        return np.array([M[0, 2], M[1, 2], M[0, 0] - 1.0, M[0, 1], M[1, 0], M[1, 1] - 1.0])
    u, v = _invert_warp_pointwise(dp, dx, dy)
    zx, zy = warp(p, u, v)
    A = np.stack([np.ones_like(dx), dx, dy, dx * dx, dx * dy, dy * dy], axis=1)
    cx = np.linalg.lstsq(A, zx - dx, rcond=None)[0]
    cy = np.linalg.lstsq(A, zy - dy, rcond=None)[0]
    return np.array([cx[0], cy[0], cx[1], cx[2], cy[1], cy[2],
                     cx[3], cx[4], cx[5], cy[3], cy[4], cy[5]])


def update_norm(dp, r):
    """||dp||_s of reading R7."""
    dp = np.asarray(dp, dtype=np.float64)
    s = dp[0] ** 2 + dp[1] ** 2
    if dp.size >= 6:
        s += r * r * np.sum(dp[2:6] ** 2)
    if dp.size >= 12:
        s += r ** 4 * np.sum(dp[6:12] ** 2)
    return math.sqrt(s)


def transfer_warp(p, ddx, ddy):
    """Warp of a neighbour re-expanded about a centre offset (ddx, ddy) from it
    (reading R10): displacement at the offset, first derivatives there, quadratic
    terms kept."""
    p = np.asarray(p, dtype=np.float64)
    q = p.copy()
    n = p.size
    if n >= 6:
        q[0] = p[0] + p[2] * ddx + p[3] * ddy
        q[1] = p[1] + p[4] * ddx + p[5] * ddy
    if n >= 12:
        q[0] += p[6] * ddx * ddx + p[7] * ddx * ddy + p[8] * ddy * ddy
        q[1] += p[9] * ddx * ddx + p[10] * ddx * ddy + p[11] * ddy * ddy
        q[2] = p[2] + 2.0 * p[6] * ddx + p[7] * ddy
        q[3] = p[3] + p[7] * ddx + 2.0 * p[8] * ddy
        q[4] = p[4] + 2.0 * p[9] * ddx + p[10] * ddy
        q[5] = p[5] + p[10] * ddx + 2.0 * p[11] * ddy
    return q


def _flat(delta, mean, count):
    return delta / math.sqrt(count) <= 1e-6 * max(abs(mean), 1.0)


class ReferenceSubset:
    """Everything IC-GN needs from the reference subset (reading R4, Eq. 4)."""

    def __init__(self, ref: Plane, xc, yc, subset_size, n):
        self.dx, self.dy = local_coordinates(subset_size)
        self.r = (subset_size - 1) // 2
        xi = xc + self.dx.astype(np.int64)
        yi = yc + self.dy.astype(np.int64)
        f = ref.gray_at(xi, yi).astype(np.float64)
        self.f = f
        self.norm_f = math.sqrt(np.sum(f * f))
        self.f_m = f.mean()
        self.fbar = f - self.f_m
        self.delta_f = math.sqrt(np.sum(self.fbar ** 2))
        self.flat = _flat(self.delta_f, self.f_m, f.size)
        fx, fy = gradient_at_pixels(ref, xi, yi)
        self.SD = steepest_descent_images(fx, fy, self.dx, self.dy, n)
        self.H = self.SD.T @ self.SD
        self.LU, self.piv, self.singular = lu_partial_pivot(self.H)


def residual(rs: ReferenceSubset, g, gbar, delta_g, cost):
    """e_i of reading R12 for the cost (Eq. 2-4)."""
    if cost == ZNSSD:
        return rs.fbar - (rs.delta_f / delta_g) * gbar
    if cost == NSSD:
        return rs.f - (rs.norm_f / math.sqrt(np.sum(g * g))) * g
    if cost == SSD:
        return rs.f - g
    raise ValueError("unknown cost %r" % cost)


def cost_value(rs: ReferenceSubset, g, cost):
    """Eq. 2 (SSD), Eq. 3 (NSSD) or Eq. 4 (ZNSSD) of the samples g."""
    if cost == ZNSSD:
        gbar = g - g.mean()
        return znssd(rs.fbar, gbar)
    if cost == NSSD:
        return float(np.sum((rs.f / rs.norm_f - g / math.sqrt(np.sum(g * g))) ** 2))
    if cost == SSD:
        return float(np.sum((rs.f - g) ** 2))
    raise ValueError("unknown cost %r" % cost)


def icgn(ref: Plane, dfm: Plane, xc, yc, subset_size, shape, p_init, params=None, ref_subset=None):
    """IC-GN for one subset from p_init; returns p, zncc, iters, converged, status."""
    prm = dict(DEFAULT_PARAMS)
    if params:
        prm.update(params)
    n = N_PARAMS[shape]
    rs = ref_subset or ReferenceSubset(ref, xc, yc, subset_size, n)
    p = np.zeros(n)
    p[:len(p_init)] = np.asarray(p_init, dtype=np.float64)[:n]
    out = dict(p=p, zncc=float("nan"), iters=0, converged=False, status=MAX_ITER)
    if rs.flat:
        out["status"] = FLAT_SUBSET
        return out
    if rs.singular:
        out["status"] = SINGULAR_H
        return out
    ratio_status = None
    lm = prm["optimizer"] == LEVENBERG_MARQUARDT
    lam, c_best, s_best, p_best, b_best = LM_LAMBDA0, None, None, None, None
    for _ in range(int(prm["max_iter"])):
        wx, wy = warp(p, rs.dx, rs.dy)
        g, valid = interpolate(dfm, xc + wx, yc + wy)
        if not valid.all():
            ratio_status = OUT_OF_BOUNDS
            break
        g_m = g.mean()
        gbar = g - g_m
        delta_g = math.sqrt(np.sum(gbar ** 2))
        if _flat(delta_g, g_m, g.size):
            ratio_status = FLAT_SUBSET
            break
        e = residual(rs, g, gbar, delta_g, prm["cost"])
        b = rs.SD.T @ e
        if lm:
            c = cost_value(rs, g, prm["cost"])
            s_k = update_norm(-lu_solve(rs.LU, rs.piv, b), rs.r)
            if c_best is None or c < c_best or s_k < s_best:
                c_best, s_best, p_best, b_best = c, s_k, p.copy(), b
                lam /= LM_FACTOR
            else:
                lam *= LM_FACTOR
            dp = -lu_solve(rs.LU, rs.piv, b_best)         # undamped: the convergence test
            if update_norm(dp, rs.r) >= prm["conv_threshold"]:
                Hd = rs.H + lam * np.diag(np.diag(rs.H))
                LU, piv, _ = lu_partial_pivot(Hd)
                dp = -lu_solve(LU, piv, b_best)
                p = compose_inverse(p_best, dp, rs.dx, rs.dy)
                out["iters"] += 1
                continue
            p = compose_inverse(p_best, dp, rs.dx, rs.dy)
        else:
            dp = -lu_solve(rs.LU, rs.piv, b)
            p = compose_inverse(p, dp, rs.dx, rs.dy)
        out["iters"] += 1
        if update_norm(dp, rs.r) < prm["conv_threshold"]:
            out["converged"] = True
            break
    out["p"] = p
    if ratio_status is not None:
        out["status"] = ratio_status
        return out
    if lm:
        # R8: Levenberg-Marquardt samples once more at the final p
        wx, wy = warp(p, rs.dx, rs.dy)
        g, valid = interpolate(dfm, xc + wx, yc + wy)
        if not valid.all():
            out["status"] = OUT_OF_BOUNDS
            return out
        g_m = g.mean()
        gbar = g - g_m
        delta_g = math.sqrt(np.sum(gbar ** 2))
        if _flat(delta_g, g_m, g.size):
            out["status"] = FLAT_SUBSET
            return out
    # R8: Gauss-Newton keeps gbar and delta_g of its last iteration's pass (already
    # tested in bounds and not flat inside the loop)
    out["zncc"] = float(np.sum(rs.fbar * gbar) / (rs.delta_f * delta_g))
    if not out["converged"]:
        out["status"] = MAX_ITER
    elif out["zncc"] < prm["zncc_min"]:
        out["status"] = LOW_ZNCC
    else:
        out["status"] = OK
    return out


def znssd(fbar, gbar):
    """Eq. 4."""
    return float(np.sum((fbar / np.sqrt(np.sum(fbar ** 2)) - gbar / np.sqrt(np.sum(gbar ** 2))) ** 2))


# --------------------------------------------------------------------------- R9
def seed_search(ref_gray, def_gray, xc, yc, subset_size, radius, ref_off=(0, 0),
                def_off=(0, 0), width=None, height=None):
    """Integer-offset ZNCC search (reading R9); returns (du, dv, C) or None."""
    r = (subset_size - 1) // 2
    N = subset_size * subset_size
    integer = np.issubdtype(np.asarray(ref_gray).dtype, np.integer)
    acc = np.int64 if integer else np.float64
    W = width if width is not None else def_gray.shape[1] + def_off[0]
    H = height if height is not None else def_gray.shape[0] + def_off[1]
    f = np.asarray(ref_gray)[yc - r - ref_off[1]:yc + r + 1 - ref_off[1],
                             xc - r - ref_off[0]:xc + r + 1 - ref_off[0]].astype(acc)
    Sf = f.sum()
    Sff = (f * f).sum()
    Df = (int(N) * int(Sff) - int(Sf) * int(Sf)) if integer else N * Sff - Sf * Sf
    if Df == 0:
        return None
    best = None
    for dv in range(-radius, radius + 1):
        for du in range(-radius, radius + 1):
            x0, y0 = xc + du - r, yc + dv - r
            if x0 < 0 or y0 < 0 or x0 + subset_size > W or y0 + subset_size > H:
                continue
            g = np.asarray(def_gray)[y0 - def_off[1]:y0 - def_off[1] + subset_size,
                                     x0 - def_off[0]:x0 - def_off[0] + subset_size].astype(acc)
            Sg = g.sum()
            Sgg = (g * g).sum()
            Sfg = (f * g).sum()
            if integer:
                Dg = int(N) * int(Sgg) - int(Sg) * int(Sg)
                num = int(N) * int(Sfg) - int(Sf) * int(Sg)
            else:
                Dg = N * Sgg - Sg * Sg
                num = N * Sfg - Sf * Sg
            if Dg == 0:
                continue
            C = float(num) / math.sqrt(float(Df) * float(Dg))
            key = (C, -(abs(du) + abs(dv)), -dv, -du)
            if best is None or key > best[0]:
                best = (key, du, dv, C)
    if best is None:
        return None
    return best[1], best[2], best[3]


# --------------------------------------------------------------------------- R10
def correlate(ref, deformed, roi, subset_size, subset_step, shape, seeds, params=None,
              progress=None):
    """Whole-image correlation by waves (reading R10). Returns a dict of per-point
    arrays in grid order (q = j * nx + i): x, y, u, v, p, zncc, iters, converged,
    status, wave; plus nx, ny."""
    return _propagate(ref, deformed, roi, subset_size, subset_step, shape, params, progress,
                      seeds=seeds)


def correlate_sequence(ref, deformed, roi, subset_size, subset_step, shape, previous, params=None,
                       progress=None):
    """One frame of a sequence against the same reference (Sec. 2.1: one result per
    deformed image). Reading R11: wave 0 is every point accepted in the previous
    frame's result `previous`, each starting from its previous warp; the other
    points are reached by propagation exactly as in correlate()."""
    starts = {int(q): np.asarray(previous["p"][q], dtype=np.float64)
              for q in np.flatnonzero(np.asarray(previous["status"]) == OK)}
    return _propagate(ref, deformed, roi, subset_size, subset_step, shape, params, progress,
                      starts=starts)


def _propagate(ref, deformed, roi, subset_size, subset_step, shape, params, progress, seeds=None,
               starts=None):
    prm = dict(DEFAULT_PARAMS)
    if params:
        prm.update(params)
    ref = np.asarray(ref)
    deformed = np.asarray(deformed)
    H, W = ref.shape
    n = N_PARAMS[shape]
    xs, ys = grid(W, H, subset_size, subset_step)
    nx, ny = len(xs), len(ys)
    npts = nx * ny
    inroi = roi_points(roi, W, H, subset_size, subset_step).ravel()
    refp = Plane(ref, interp=prm["interp"])
    defp = Plane(deformed, interp=prm["interp"])
    P = np.zeros((npts, n))
    zncc = np.full(npts, np.nan)
    iters = np.zeros(npts, np.int32)
    conv = np.zeros(npts, bool)
    status = np.where(inroi, NOT_REACHED, NOT_IN_ROI).astype(np.int32)
    wave = np.full(npts, -1, np.int32)
    px = np.tile(xs, ny)
    py = np.repeat(ys, nx)

    fft_field = None
    if seeds is not None and prm["init"] == "fft":
        # reading F8 of the FFT initialiser's oracle: the seeds start from its estimate
        from .fft_oracle import multiwindow, round_half_up
        fft_field = multiwindow(ref, deformed, roi, subset_size, subset_step, int(prm["max_displacement"]),
                                False, prm["mad_tau"], prm["mad_eps"])
    elif prm["init"] not in ("search", "fft"):
        raise ValueError("unknown init %r" % (prm["init"],))
    current = []
    if seeds is not None:
        for (sx, sy) in seeds:
            i, j = snap_seed(sx, sy, W, H, subset_size, subset_step)
            q = j * nx + i
            if inroi[q] and wave[q] < 0:
                wave[q] = 0
                current.append(q)
    else:
        for q in sorted(starts):
            if inroi[q]:
                wave[q] = 0
                current.append(q)
    k = 0
    while current:
        for q in current:
            xc, yc = int(px[q]), int(py[q])
            if k == 0 and fft_field is not None:
                p0 = np.zeros(n)
                p0[0] = round_half_up(fft_field["u"][q])
                p0[1] = round_half_up(fft_field["v"][q])
            elif k == 0 and seeds is not None:
                found = seed_search(ref, deformed, xc, yc, subset_size, int(prm["search_radius"]))
                if found is None:
                    status[q] = OUT_OF_BOUNDS
                    continue
                p0 = np.zeros(n)
                p0[0], p0[1] = found[0], found[1]
            elif k == 0:
                p0 = starts[q]
            else:
                best = None
                for nb in _neighbours(q, nx, ny):
                    if 0 <= wave[nb] < k and status[nb] == OK:
                        key = (zncc[nb], -nb)
                        if best is None or key > best[0]:
                            best = (key, nb)
                nb = best[1]
                p0 = transfer_warp(P[nb], float(px[q] - px[nb]), float(py[q] - py[nb]))
            res = icgn(refp, defp, xc, yc, subset_size, shape, p0, prm)
            P[q] = res["p"]
            zncc[q] = res["zncc"]
            iters[q] = res["iters"]
            conv[q] = res["converged"]
            status[q] = res["status"]
        nxt = set()
        for q in current:
            if status[q] != OK:
                continue
            for nb in _neighbours(q, nx, ny):
                if inroi[nb] and wave[nb] < 0:
                    nxt.add(nb)
        current = sorted(nxt)
        for q in current:
            wave[q] = k + 1
        k += 1
        if progress:
            progress(k, len(current))
    if prm["nan_unconverged"]:
        P[status != OK] = np.nan
    return dict(x=px, y=py, u=P[:, 0].copy(), v=P[:, 1].copy(), p=P, zncc=zncc, iters=iters,
                converged=conv, status=status, wave=wave, nx=nx, ny=ny)


def _neighbours(q, nx, ny):
    """4-neighbours of grid point q: left, right, up, down."""
    i, j = q % nx, q // nx
    out = []
    if i > 0:
        out.append(q - 1)
    if i < nx - 1:
        out.append(q + 1)
    if j > 0:
        out.append(q - nx)
    if j < ny - 1:
        out.append(q + nx)
    return out
