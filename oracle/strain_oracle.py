"""FP64 CPU oracle for strain post-processing (Sec. 2.3 of Hirst et al., "Pyvale",
arXiv 2601.12941): the displacement gradient of a windowed least-squares fit of the
correlated displacement field, the deformation gradient and five strain measures.

TEST INFRASTRUCTURE. Like ``dic_oracle``, only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; it shares nothing with the library.

What each part follows:

  * Eq. 6        F = I + grad u, u = (u_x, u_y).
  * Eq. 7        VSG = (N - 1) s + w for an N x N window of grid points at step s
                 with subsets of size w.
  * Eq. 8, 9     u(x, y) = P(x, y) c over the window by linear least squares, with
                 P = [1, x, y] ("bilinear") or
                 P = [1, x, y, x^2, y^2, x^2 y, x y^2, x^2 y^2] ("biquadratic").
  * Sec. 2.3     strain measures: Green-Lagrange (F^T F - I) / 2, Hencky
                 ln sqrt(F^T F), Euler-Almansi (I - (F F^T)^-1) / 2, Biot right
                 sqrt(F^T F) - I, Biot left sqrt(F F^T) - I.

Readings taken where the paper is silent:

  S1  The window is centred on its grid point; x and y are pixel offsets from the
      centre ((i - i_c) s, (j - j_c) s). grad u is the derivative of the fit at the
      centre: the coefficients of x and y (every other basis term has zero
      derivative there).
  S2  A window uses its grid points that lie inside the grid and were accepted
      (status 0); the centre itself must be accepted. The fit needs at least as many
      points as basis terms, and the normal matrix in grid units (x / s, y / s),
      scaled to unit diagonal, must have every pivot of its LDL^T factorisation
      (no exchanges) above 1e-5; otherwise the point has no strain (NaN).
  S3  The bases are taken as printed: neither contains the xy term.
  S4  Square roots and logarithms of the symmetric positive definite C = F^T F and
      B = F F^T are taken through their eigen decompositions.
"""
from __future__ import annotations

import numpy as np

BILINEAR, BIQUADRATIC = "bilinear", "biquadratic"
GREEN_LAGRANGE, HENCKY, EULER_ALMANSI, BIOT_RIGHT, BIOT_LEFT = (
    "green_lagrange", "hencky", "euler_almansi", "biot_right", "biot_left")
MEASURES = (GREEN_LAGRANGE, HENCKY, EULER_ALMANSI, BIOT_RIGHT, BIOT_LEFT)
MIN_SCALED_PIVOT = 1e-5


def vsg(window: int, step: int, subset_size: int) -> int:
    """Eq. 7: virtual strain gauge size in pixels."""
    return (window - 1) * step + subset_size


def basis(x, y, kind: str) -> np.ndarray:
    """Eq. 9: rows P(x, y) for the points (x, y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    one = np.ones_like(x)
    if kind == BILINEAR:
        return np.stack([one, x, y], axis=-1)
    if kind == BIQUADRATIC:
        return np.stack([one, x, y, x * x, y * y, x * x * y, x * y * y, x * x * y * y], axis=-1)
    raise ValueError("unknown basis %r" % kind)


def well_posed(P_grid: np.ndarray) -> bool:
    """Reading S2: enough points, and every pivot of the LDL^T factorisation of the
    unit-diagonal normal matrix above MIN_SCALED_PIVOT."""
    n, k = P_grid.shape
    if n < k:
        return False
    M = P_grid.T @ P_grid
    d = np.sqrt(np.diag(M))
    if np.any(d <= 0.0):
        return False
    A = M / np.outer(d, d)
    for j in range(k):          # Gaussian elimination without exchanges
        piv = A[j, j]
        if not piv > MIN_SCALED_PIVOT:
            return False
        A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:]) / piv
    return True


def displacement_gradient(u, v, status, nx: int, ny: int, step: int, window: int, kind: str):
    """grad u at every grid point (point order q = j nx + i) by Eq. 8-9 and readings
    S1-S3. Returns (dudx, dudy, dvdx, dvdy, valid); points without a fit are NaN."""
    u = np.asarray(u, dtype=np.float64).reshape(ny, nx)
    v = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    ok = (np.asarray(status).reshape(ny, nx) == 0)
    h = (window - 1) // 2
    out = np.full((4, ny, nx), np.nan)
    valid = np.zeros((ny, nx), dtype=bool)
    for jc in range(ny):
        for ic in range(nx):
            if not ok[jc, ic]:
                continue
            j0, j1 = max(jc - h, 0), min(jc + h, ny - 1)
            i0, i1 = max(ic - h, 0), min(ic + h, nx - 1)
            jj, ii = np.mgrid[j0:j1 + 1, i0:i1 + 1]
            m = ok[j0:j1 + 1, i0:i1 + 1]
            gi = (ii[m] - ic).astype(np.float64)
            gj = (jj[m] - jc).astype(np.float64)
            if not well_posed(basis(gi, gj, kind)):
                continue
            P = basis(gi * step, gj * step, kind)
            cu = np.linalg.lstsq(P, u[j0:j1 + 1, i0:i1 + 1][m], rcond=None)[0]
            cv = np.linalg.lstsq(P, v[j0:j1 + 1, i0:i1 + 1][m], rcond=None)[0]
            out[:, jc, ic] = (cu[1], cu[2], cv[1], cv[2])
            valid[jc, ic] = True
    return out[0].ravel(), out[1].ravel(), out[2].ravel(), out[3].ravel(), valid.ravel()


def _spd_function(C: np.ndarray, f) -> np.ndarray:
    """f(C) for a symmetric positive definite C via its eigen decomposition (S4)."""
    lam, Q = np.linalg.eigh(C)
    return (Q * f(lam)) @ Q.T


def strain_tensor(F: np.ndarray, measure: str) -> np.ndarray:
    """Sec. 2.3: the 2 x 2 strain tensor of the deformation gradient F."""
    F = np.asarray(F, dtype=np.float64)
    I = np.eye(2)
    if measure == GREEN_LAGRANGE:
        return 0.5 * (F.T @ F - I)
    if measure == HENCKY:
        return _spd_function(F.T @ F, lambda lam: np.log(np.sqrt(lam)))
    if measure == EULER_ALMANSI:
        return 0.5 * (I - np.linalg.inv(F @ F.T))
    if measure == BIOT_RIGHT:
        return _spd_function(F.T @ F, np.sqrt) - I
    if measure == BIOT_LEFT:
        return _spd_function(F @ F.T, np.sqrt) - I
    raise ValueError("unknown measure %r" % measure)


def strain_field(u, v, status, nx: int, ny: int, step: int, window: int, kind: str, measure: str):
    """Displacement gradient and strain (exx, eyy, exy) at every grid point."""
    dudx, dudy, dvdx, dvdy, valid = displacement_gradient(u, v, status, nx, ny, step, window, kind)
    e = np.full((3, nx * ny), np.nan)
    for q in np.flatnonzero(valid):
        F = np.array([[1.0 + dudx[q], dudy[q]], [dvdx[q], 1.0 + dvdy[q]]])    # Eq. 6
        E = strain_tensor(F, measure)
        e[:, q] = (E[0, 0], E[1, 1], E[0, 1])
    return dict(dudx=dudx, dudy=dudy, dvdx=dvdx, dvdy=dvdy, exx=e[0], eyy=e[1], exy=e[2], valid=valid)
