"""FP64 CPU oracle of the multi-window FFT initialiser: normalised FFT
cross-correlation (Eq. 1) over windows that halve from above the largest expected
displacement down to the subset size (Sec. 2.2), the estimate of each coarser level
guiding the next, median-absolute-deviation outlier removal at every level (Sec. 4,
SEM study) and the Gaussian peak fit of the FFT-only method (Sec. 2.2).

TEST INFRASTRUCTURE. This module is the plain, slow, obviously correct reference
that the CUDA library is checked against. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and it shares
no code, table or constant with the library.

Readings taken where the paper is silent (all of them, in one place):

  F1 Window sizes: L0 is the smallest power of two above the expected maximum
     displacement D (2^n > D); the size halves while it stays above the subset size
     S; sizes larger than min(W, H) are dropped; the last level uses S itself.
     D = 800, S = 17 gives 1024, 512, 256, 128, 64, 32, 17 (the paper's example).
  F2 A power-of-two level tiles the image: window (i, j) covers x in [iL, iL + L),
     y in [jL, jL + L) for i < W // L, j < H // L, with centre (iL + L/2, jL + L/2).
     The last level's windows are the subsets of the correlation grid (reading R3):
     S x S about every in-ROI grid point.
  F3 The guess of a window is (0, 0) on the first level; on later levels it is the
     previous level's (filtered) field interpolated bilinearly between the four
     nearest window centres (held constant beyond the outermost centres), rounded
     to the nearest integer, halves up. The deformed window is the reference window
     moved by the guess, clamped into the image.
  F4 Eq. 1, "normalised FFT cross-correlation": |F{f}| and |F{g}| are read as the
     norms of the transforms of the mean-removed windows, so that R is the
     zero-normalised circular cross-correlation
        R(s) = IDFT( F conj(G) )(s) / (||f - f_m|| ||g - g_m||),
     F and G the L x L DFTs of the mean-removed windows, the inverse carrying 1/L^2
     (by Parseval the denominator is ||F|| ||G|| / L^2). R is 1 at the
     shift of a circularly shifted copy, and unchanged by gain and offset of either
     window; a flat window (all its values equal) gives R = 0. (Dividing each frequency by its own |F| |G|,
     phase correlation, fails on smooth speckle inside hard-edged windows: the
     frequencies without speckle content carry the windows' edge leakage, which
     aligns at zero shift. Nor would its delta-like peak suit the Gaussian peak
     fit that the paper pairs with this correlation.) No taper or padding.
  F5 The peak is the largest R, ties to the lowest row-major index (ky, kx). With
     F conj(G) in Eq. 1, R peaks at minus the shift of the deformed window's
     content: d = wrap(-k), wrap(m) = ((m + floor(L/2)) mod L) - floor(L/2), so a
     level resolves shifts in [-floor(L/2), ceil(L/2) - 1]. The window's
     displacement is (deformed origin - reference origin) + d.
  F6 Sub-pixel (last level, when asked): per axis, the three-point Gaussian through
     the peak and its two circular neighbours along that axis,
        delta = (ln R[-1] - ln R[+1]) / (2 (ln R[-1] - 2 ln R[0] + ln R[+1])),
     delta = 0 when one of the three is not positive or the denominator is not
     negative; the displacement becomes d - delta.
  F7 MAD outlier removal after every level: for each window with a value, over the
     values of its 3 x 3 neighbourhood of windows (itself included, clipped at the
     grid edges), per component c in (u, v): med = median, mad = median |c - med|;
     the window is an outlier when |c - med| > tau (1.4826 mad + eps) for u or v
     (tau = 3, eps = 0.5 px); an outlier takes (med_u, med_v). Every test reads the
     unfiltered values; tau <= 0 switches the removal off.
  F8 Seeding the correlation (MULTIWINDOW_RG): a seed starts from the last-level
     estimate (without sub-pixel fit) at its grid point, rounded to the nearest
     integer, halves up, in place of the integer ZNCC search (reading R9). The
     propagation is unchanged (reading R10).
"""
from __future__ import annotations

import math

import numpy as np

from .dic_oracle import NOT_IN_ROI, OK, grid, roi_points

MAD_TAU, MAD_EPS, MAD_SCALE = 3.0, 0.5, 1.4826


def window_sizes(max_displacement: int, subset_size: int, width: int, height: int):
    """Reading F1."""
    L = 1
    while L <= max_displacement:
        L *= 2
    out = []
    while L > subset_size:
        if L <= min(width, height):
            out.append(L)
        L //= 2
    out.append(subset_size)
    return out


def fftcc(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Eq. 1 as reading F4 takes it: the zero-normalised circular cross-correlation
    of two L x L windows, computed through their DFTs."""
    fb = np.asarray(f, dtype=np.float64)
    gb = np.asarray(g, dtype=np.float64)
    if (fb == fb.flat[0]).all() or (gb == gb.flat[0]).all():
        return np.zeros(fb.shape)              # a flat (constant) window: R = 0
    fb = fb - fb.mean()
    gb = gb - gb.mean()
    den = math.sqrt(np.sum(fb * fb)) * math.sqrt(np.sum(gb * gb))
    F = np.fft.fft2(fb)
    G = np.fft.fft2(gb)
    return np.real(np.fft.ifft2(F * np.conj(G))) / den


def wrap(m: int, L: int) -> int:
    h = L // 2
    return ((m + h) % L) - h


def gauss3(rm: float, r0: float, rp: float) -> float:
    """Reading F6: vertex offset of the Gaussian through three samples."""
    if rm <= 0 or r0 <= 0 or rp <= 0:
        return 0.0
    lm, l0, lp = math.log(rm), math.log(r0), math.log(rp)
    den = 2.0 * (lm - 2.0 * l0 + lp)
    if not den < 0:
        return 0.0
    return (lm - lp) / den


def peak(R: np.ndarray, subpixel: bool = False):
    """Reading F5 (and F6): shift (dx, dy) of the deformed window's content and the
    peak value."""
    L = R.shape[0]
    k = int(np.argmax(R))                      # first maximum in row-major order
    ky, kx = divmod(k, R.shape[1])
    dx, dy = float(wrap(-kx, L)), float(wrap(-ky, L))
    if subpixel:
        dx -= gauss3(R[ky, (kx - 1) % L], R[ky, kx], R[ky, (kx + 1) % L])
        dy -= gauss3(R[(ky - 1) % L, kx], R[ky, kx], R[(ky + 1) % L, kx])
    return dx, dy, float(R[ky, kx])


def round_half_up(v):
    return np.floor(np.asarray(v, dtype=np.float64) + 0.5)


def bilinear(field: np.ndarray, c0: float, step: float, x, y):
    """Reading F3: field[j, i] sits at (c0 + i step, c0 + j step); bilinear between
    the four nearest centres, constant beyond the outermost ones."""
    ny, nx = field.shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    tx = np.clip((x - c0) / step, 0.0, nx - 1)
    ty = np.clip((y - c0) / step, 0.0, ny - 1)
    i0 = np.minimum(np.floor(tx).astype(np.int64), max(nx - 2, 0))
    j0 = np.minimum(np.floor(ty).astype(np.int64), max(ny - 2, 0))
    i1 = np.minimum(i0 + 1, nx - 1)
    j1 = np.minimum(j0 + 1, ny - 1)
    fx = tx - i0
    fy = ty - j0
    top = (1.0 - fx) * field[j0, i0] + fx * field[j0, i1]
    bot = (1.0 - fx) * field[j1, i0] + fx * field[j1, i1]
    return (1.0 - fy) * top + fy * bot


def mad_filter(u: np.ndarray, v: np.ndarray, valid: np.ndarray, tau=MAD_TAU, eps=MAD_EPS):
    """Reading F7 on a (ny, nx) field; returns filtered u, v and the replaced mask."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ny, nx = u.shape
    uo, vo = u.copy(), v.copy()
    rep = np.zeros((ny, nx), bool)
    if tau <= 0:
        return uo, vo, rep
    for j in range(ny):
        for i in range(nx):
            if not valid[j, i]:
                continue
            sl = (slice(max(j - 1, 0), j + 2), slice(max(i - 1, 0), i + 2))
            m = valid[sl]
            nu, nv = u[sl][m], v[sl][m]
            mu, mv = np.median(nu), np.median(nv)
            du, dv = np.median(np.abs(nu - mu)), np.median(np.abs(nv - mv))
            if (abs(u[j, i] - mu) > tau * (MAD_SCALE * du + eps) or
                    abs(v[j, i] - mv) > tau * (MAD_SCALE * dv + eps)):
                uo[j, i], vo[j, i] = mu, mv
                rep[j, i] = True
    return uo, vo, rep


def _gray(img):
    return np.asarray(img, dtype=np.float64)


def window_level(ref, deformed, L, origins, guesses, subpixel=False):
    """One level over explicit windows (readings F3-F6): origins[k] = (x0, y0) of the
    reference window, guesses[k] = integer (gu, gv). Returns per-window arrays
    u, v, peak, and the deformed origins used."""
    ref = _gray(ref)
    deformed = _gray(deformed)
    H, W = ref.shape
    n = len(origins)
    u = np.zeros(n)
    v = np.zeros(n)
    pk = np.zeros(n)
    dorg = np.zeros((n, 2), np.int64)
    for k in range(n):
        x0, y0 = int(origins[k][0]), int(origins[k][1])
        gx0 = min(max(x0 + int(guesses[k][0]), 0), W - L)
        gy0 = min(max(y0 + int(guesses[k][1]), 0), H - L)
        R = fftcc(ref[y0:y0 + L, x0:x0 + L], deformed[gy0:gy0 + L, gx0:gx0 + L])
        dx, dy, p = peak(R, subpixel)
        u[k] = (gx0 - x0) + dx
        v[k] = (gy0 - y0) + dy
        pk[k] = p
        dorg[k] = (gx0, gy0)
    return u, v, pk, dorg


def multiwindow(ref, deformed, roi, subset_size, subset_step, max_displacement, subpixel=False,
                tau=MAD_TAU, eps=MAD_EPS):
    """The whole initialiser (readings F1-F7). Returns a dict with the last level's
    u, v, peak, status and replaced flags in grid order (q = j * nx + i), nx, ny,
    and `levels`: per level L, nx, ny, guess_u, guess_v, raw_u, raw_v, peak, u, v,
    replaced, valid (arrays over that level's window grid)."""
    ref = _gray(ref)
    deformed = _gray(deformed)
    H, W = ref.shape
    S = subset_size
    r = (S - 1) // 2
    sizes = window_sizes(max_displacement, S, W, H)
    levels = []
    prev = None                                # (u, v, c0, step) of the previous level
    for li, L in enumerate(sizes):
        last = li == len(sizes) - 1
        if not last:
            nx, ny = W // L, H // L
            cx = np.arange(nx) * L + L // 2
            cy = np.arange(ny) * L + L // 2
            valid = np.ones((ny, nx), bool)
            ox = np.arange(nx) * L
            oy = np.arange(ny) * L
        else:
            xs, ys = grid(W, H, S, subset_step)
            nx, ny = len(xs), len(ys)
            cx, cy = xs, ys
            valid = roi_points(roi, W, H, S, subset_step)
            ox, oy = xs - r, ys - r
        CX, CY = np.meshgrid(cx, cy)
        if prev is None:
            gu = np.zeros((ny, nx))
            gv = np.zeros((ny, nx))
        else:
            pu, pv, c0, st = prev
            gu = round_half_up(bilinear(pu, c0, st, CX, CY))
            gv = round_half_up(bilinear(pv, c0, st, CX, CY))
        OX, OY = np.meshgrid(ox, oy)
        sel = np.flatnonzero(valid.ravel())
        origins = np.stack([OX.ravel()[sel], OY.ravel()[sel]], 1)
        guesses = np.stack([gu.ravel()[sel], gv.ravel()[sel]], 1)
        uu, vv, pk, _ = window_level(ref, deformed, L, origins, guesses, subpixel and last)
        raw_u = np.zeros(ny * nx)
        raw_v = np.zeros(ny * nx)
        peak_a = np.zeros(ny * nx)
        raw_u[sel], raw_v[sel], peak_a[sel] = uu, vv, pk
        raw_u = raw_u.reshape(ny, nx)
        raw_v = raw_v.reshape(ny, nx)
        fu, fv, rep = mad_filter(raw_u, raw_v, valid, tau, eps)
        levels.append(dict(L=L, nx=nx, ny=ny, guess_u=gu, guess_v=gv, raw_u=raw_u, raw_v=raw_v,
                           peak=peak_a.reshape(ny, nx), u=fu, v=fv, replaced=rep, valid=valid))
        if not last:
            prev = (fu, fv, float(L // 2), float(L))
    lv = levels[-1]
    status = np.where(lv["valid"].ravel(), OK, NOT_IN_ROI).astype(np.int32)
    return dict(u=lv["u"].ravel(), v=lv["v"].ravel(), peak=lv["peak"].ravel(), status=status,
                replaced=lv["replaced"].ravel(), nx=lv["nx"], ny=lv["ny"], levels=levels)
