"""Pins of the strain oracle (Sec. 2.3) against closed forms, identities and library
matrix functions, chosen so that a plausible mistake (a dropped step factor, a
swapped axis, a missing transpose, a wrong measure) fails one of them."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import strain_oracle as SO


def _grid(nx, ny, step):
    j, i = np.mgrid[0:ny, 0:nx]
    return (i * step).astype(np.float64), (j * step).astype(np.float64)


@pytest.mark.parametrize("kind", [SO.BILINEAR, SO.BIQUADRATIC])
def test_linear_field_gives_its_gradient_everywhere(kind):
    nx, ny, step = 23, 17, 7
    X, Y = _grid(nx, ny, step)
    u = 3.25 + 2e-3 * X - 1.5e-3 * Y
    v = -0.5 + 4e-4 * X + 2.5e-3 * Y
    r = SO.strain_field(u.ravel(), v.ravel(), np.zeros(nx * ny, np.uint8), nx, ny, step, 5, kind,
                        SO.GREEN_LAGRANGE)
    assert r["valid"].all()          # edge windows are clipped, still well posed
    for key, want in (("dudx", 2e-3), ("dudy", -1.5e-3), ("dvdx", 4e-4), ("dvdy", 2.5e-3)):
        assert np.max(np.abs(r[key] - want)) < 1e-13, key


def test_biquadratic_fit_is_exact_on_its_basis_and_blind_to_xy_on_full_windows():
    nx, ny, step, N = 21, 21, 3, 7
    X, Y = _grid(nx, ny, step)
    # terms of the printed basis (about any centre they stay in the basis or drop
    # in order), plus an xy term that the basis lacks
    u = 1e-3 * X + 2e-4 * Y + 3e-6 * X * X - 2e-6 * Y * Y + 4e-7 * X * X * Y + 5e-6 * X * Y
    v = -2e-3 * Y + 1e-6 * X * Y * Y
    r = SO.strain_field(u.ravel(), v.ravel(), np.zeros(nx * ny, np.uint8), nx, ny, step, N, SO.BIQUADRATIC,
                        SO.GREEN_LAGRANGE)
    h = (N - 1) // 2
    interior = np.zeros((ny, nx), bool)
    interior[h:ny - h, h:nx - h] = True
    interior = interior.ravel()
    Xc, Yc = X.ravel(), Y.ravel()
    # the exact gradient at the centre (the xy term is orthogonal to the basis on a
    # symmetric window, so its derivative 5e-6 (Y, X) is recovered exactly too)
    dudx = 1e-3 + 6e-6 * Xc + 8e-7 * Xc * Yc + 5e-6 * Yc
    dudy = 2e-4 - 4e-6 * Yc + 4e-7 * Xc * Xc + 5e-6 * Xc
    dvdx = 1e-6 * Yc * Yc
    dvdy = -2e-3 + 2e-6 * Xc * Yc
    for key, want in (("dudx", dudx), ("dudy", dudy), ("dvdx", dvdx), ("dvdy", dvdy)):
        assert np.max(np.abs(r[key][interior] - want[interior])) < 1e-12, key


def test_holes_are_skipped_and_degenerate_windows_have_no_strain():
    nx, ny, step = 15, 13, 5
    X, Y = _grid(nx, ny, step)
    u = 1e-3 * X + 3e-3 * Y
    v = 2e-3 * X - 1e-3 * Y
    st = np.zeros((ny, nx), np.uint8)
    rng = np.random.default_rng(3)
    st[rng.random((ny, nx)) < 0.2] = 5          # rejected points
    r = SO.strain_field(u.ravel(), v.ravel(), st.ravel(), nx, ny, step, 5, SO.BILINEAR, SO.GREEN_LAGRANGE)
    ok = r["valid"]
    assert not ok[st.ravel() != 0].any()         # a rejected centre has no strain
    assert ok.sum() > 0.7 * (st == 0).sum()
    assert np.max(np.abs(r["dudy"][ok] - 3e-3)) < 1e-13
    assert np.isnan(r["exx"][~ok]).all()
    # a single valid row: the y column of the design is zero, no fit
    st2 = np.full((ny, nx), 5, np.uint8)
    st2[6, :] = 0
    r2 = SO.strain_field(u.ravel(), v.ravel(), st2.ravel(), nx, ny, step, 5, SO.BILINEAR, SO.GREEN_LAGRANGE)
    assert not r2["valid"].any()


def test_vsg_eq7():
    assert SO.vsg(9, 10, 21) == 101
    assert SO.vsg(1, 7, 31) == 31


def test_uniaxial_stretch_closed_forms():
    lam = 1.0 + 3e-2
    F = np.diag([lam, 1.0])
    want = {SO.GREEN_LAGRANGE: 0.5 * (lam * lam - 1.0), SO.HENCKY: np.log(lam),
            SO.EULER_ALMANSI: 0.5 * (1.0 - 1.0 / (lam * lam)), SO.BIOT_RIGHT: lam - 1.0,
            SO.BIOT_LEFT: lam - 1.0}
    for m, w in want.items():
        E = SO.strain_tensor(F, m)
        assert abs(E[0, 0] - w) < 1e-15 and abs(E[1, 1]) < 1e-15 and abs(E[0, 1]) < 1e-15, m


def test_simple_shear_green_lagrange_and_rotation_invariance():
    g = 0.02
    E = SO.strain_tensor(np.array([[1.0, g], [0.0, 1.0]]), SO.GREEN_LAGRANGE)
    assert np.allclose(E, [[0.0, g / 2], [g / 2, g * g / 2]], atol=1e-16)
    th = 0.3
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    for m in SO.MEASURES:
        assert np.max(np.abs(SO.strain_tensor(R, m))) < 1e-14, m
    # F = R U: right measures see U only, left ones its rotation R U R^T
    U = np.array([[1.02, 0.004], [0.004, 0.99]])
    for m in (SO.GREEN_LAGRANGE, SO.HENCKY, SO.BIOT_RIGHT):
        assert np.allclose(SO.strain_tensor(R @ U, m), SO.strain_tensor(U, m), atol=1e-14), m
    assert np.allclose(SO.strain_tensor(R @ U, SO.BIOT_LEFT), R @ (U - np.eye(2)) @ R.T, atol=1e-14)


def test_measures_match_library_matrix_functions():
    rng = np.random.default_rng(5)
    for _ in range(20):
        F = np.eye(2) + rng.uniform(-0.08, 0.08, (2, 2))
        C, B = F.T @ F, F @ F.T
        I = np.eye(2)
        want = {SO.GREEN_LAGRANGE: 0.5 * (C - I), SO.HENCKY: 0.5 * sla.logm(C).real,
                SO.EULER_ALMANSI: 0.5 * (I - sla.inv(B)), SO.BIOT_RIGHT: sla.sqrtm(C).real - I,
                SO.BIOT_LEFT: sla.sqrtm(B).real - I}
        for m, w in want.items():
            assert np.max(np.abs(SO.strain_tensor(F, m) - w)) < 1e-13, m


def test_planted_mistakes_are_caught(monkeypatch):
    nx, ny, step = 11, 11, 4
    X, Y = _grid(nx, ny, step)
    u, v = 2e-3 * X, 1e-3 * Y
    st = np.zeros(nx * ny, np.uint8)
    # coordinates in grid units instead of pixels: the gradient comes out step times too large
    real_basis = SO.basis
    monkeypatch.setattr(SO, "basis", lambda x, y, kind: real_basis(np.asarray(x) / step, np.asarray(y) / step,
                                                                    kind))
    r = SO.strain_field(u.ravel(), v.ravel(), st, nx, ny, step, 5, SO.BILINEAR, SO.GREEN_LAGRANGE)
    assert np.max(np.abs(r["dudx"] - 2e-3)) > 1e-3
    monkeypatch.setattr(SO, "basis", real_basis)
    # Euler-Almansi from F^T F instead of F F^T differs under shear
    F = np.array([[1.0, 0.05], [0.0, 1.0]])
    wrong = 0.5 * (np.eye(2) - np.linalg.inv(F.T @ F))
    assert np.max(np.abs(SO.strain_tensor(F, SO.EULER_ALMANSI) - wrong)) > 1e-3
