"""Multi-window FFT initialiser (Sec. 2.2, Eq. 1; MAD of Sec. 4) on the GPU against
its oracle: Eq. 1 over explicit windows of every kind the library runs (odd subset
sizes, powers of two in shared memory, powers of two through the global work
buffer), the MAD rule bit for bit, the whole coarse-to-fine field, and
correlations whose seeds start from it.

Tolerances: the integer peak must match unless the oracle's own top two values are
within 2e-5 (FP32 transforms round R at about 1e-6); R at the peak within 2e-5; the
Gaussian sub-pixel offsets within 1e-4 px (the fit divides log differences of R by
its curvature)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import dic_oracle as O
from oracle import fft_oracle as F

from parity_util import GPU_PARAMS, ORACLE_PARAMS, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TIE = 2e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_2601_12941_gb300 as P
    from paper_2601_12941_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    P.load()
    return P


def _speckle(W, H, seed, fld=synth.IDENTITY, dtype="u8", noise=2.0, tag=1):
    sp = synth.Speckle(seed=seed, density=0.03, sigma=(1.5, 3.0), cell=16)
    return synth.render(synth.ImageSpec(sp, field=fld, gray_max=250.0, noise=noise, noise_tag=tag), W, H, dtype)


def _shifted_pair(seed, du, dv, N, dtype="u8"):
    big = _speckle(N + 150, N + 150, seed, dtype=dtype)
    o = 70
    return (np.ascontiguousarray(big[o:o + N, o:o + N]),
            np.ascontiguousarray(big[o - dv:o + N - dv, o - du:o + N - du]))


def _gpu_windows(pkg, c, L, origins, subpixel):
    from paper_2601_12941_gb300 import binding as B

    org = torch.as_tensor(np.asarray(origins, np.int32).reshape(-1, 4), device="cuda")
    n = org.shape[0]
    u, v, pk = (torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3))
    B.dic_fftcc_windows(c.h, L, org, subpixel, u, v, pk)
    torch.cuda.synchronize()
    return u.cpu().numpy(), v.cpu().numpy(), pk.cpu().numpy()


def _oracle_windows(ref, dfm, L, origins, subpixel):
    """Per window: u, v, peak, and whether the oracle's top two R values are a near tie."""
    ref = np.asarray(ref, np.float64)
    dfm = np.asarray(dfm, np.float64)
    out = []
    for (x0, y0, gx0, gy0) in origins:
        R = F.fftcc(ref[y0:y0 + L, x0:x0 + L], dfm[gy0:gy0 + L, gx0:gx0 + L])
        dx, dy, pk = F.peak(R, subpixel)
        s = np.sort(R.ravel())
        out.append(((gx0 - x0) + dx, (gy0 - y0) + dy, pk, s[-1] - s[-2] < TIE, R))
    return out


def _random_origins(rng, W, H, L, n, spread):
    org = []
    for _ in range(n):
        x0 = int(rng.integers(0, W - L + 1))
        y0 = int(rng.integers(0, H - L + 1))
        gx0 = int(np.clip(x0 + rng.integers(-spread, spread + 1), 0, W - L))
        gy0 = int(np.clip(y0 + rng.integers(-spread, spread + 1), 0, H - L))
        org.append((x0, y0, gx0, gy0))
    return org


@pytest.mark.parametrize("L,n,subpixel", [(3, 200, False), (9, 200, True), (21, 300, True), (31, 200, True),
                                          (41, 120, False), (61, 40, True),
                                          (16, 300, True), (32, 200, True), (64, 60, True),
                                          (128, 12, False), (256, 6, False), (512, 3, False)])
def test_eq1_over_windows_matches_oracle(pkg, L, n, subpixel):
    W, H = 700, 640
    fld = synth.affine_field(W, H, u0=3.3, v0=-2.6, exx=4e-3, eyy=-3e-3, exy=2e-3)
    ref = _speckle(W, H, 21)
    dfm = _speckle(W, H, 21, fld=fld, tag=2)
    rng = np.random.default_rng(L)
    origins = _random_origins(rng, W, H, L, n, spread=min(L // 3, 12))
    c = pkg.Correlation(ref, dfm, None, 21, 10, "affine")
    gu, gv, gp = _gpu_windows(pkg, c, L, origins, subpixel)
    c.close()
    ora = _oracle_windows(ref, dfm, L, origins, subpixel)
    ties = 0
    for k, (ou, ov, opk, tie, R) in enumerate(ora):
        if tie:
            ties += 1
            # another valid arg-max: the oracle's R there is within the tie margin
            ix = int(round(-(gu[k] - (origins[k][2] - origins[k][0])))) % L
            iy = int(round(-(gv[k] - (origins[k][3] - origins[k][1])))) % L
            assert R[iy, ix] >= R.max() - TIE
            continue
        if subpixel:
            assert abs(gu[k] - ou) < 1e-4 and abs(gv[k] - ov) < 1e-4, (k, gu[k], ou, gv[k], ov)
        else:
            assert (gu[k], gv[k]) == (ou, ov), (k, gu[k], ou, gv[k], ov)
        assert abs(gp[k] - opk) < 2e-5, (k, gp[k], opk)
    assert ties <= max(2, n // 50)


@pytest.mark.parametrize("L", [31, 32, 64, 128])
@pytest.mark.parametrize("dtype", ["u16", "bf16", "f32", "f64"])
def test_gray_types_over_windows_match_oracle(pkg, dtype, L):
    """Every gray element type through each window path: the tensor-core windows (31,
    32), the shared-memory FFT (64) and the row kernels of the work-buffer path (128)
    load the window with the element type fixed once per window or row."""
    W, H = 420, 380
    fld = synth.affine_field(W, H, u0=2.6, v0=-1.9, exx=3e-3, eyy=-2e-3, exy=1e-3)
    kind = "u8" if dtype == "bf16" else dtype
    ref = _speckle(W, H, 31, dtype=kind)
    dfm = _speckle(W, H, 31, fld=fld, dtype=kind, tag=2)
    if dtype == "bf16":                  # integer gray levels below 256 are exact in BF16
        ref_in = torch.from_numpy(ref.astype(np.float32)).to(torch.bfloat16).cuda()
        dfm_in = torch.from_numpy(dfm.astype(np.float32)).to(torch.bfloat16).cuda()
    else:
        ref_in, dfm_in = ref, dfm
    rng = np.random.default_rng(100 + L)
    origins = _random_origins(rng, W, H, L, 40, spread=min(L // 3, 10))
    subpixel = L <= 64
    c = pkg.Correlation(ref_in, dfm_in, None, 21, 10, "affine")
    gu, gv, gp = _gpu_windows(pkg, c, L, origins, subpixel)
    c.close()
    ora = _oracle_windows(ref, dfm, L, origins, subpixel)
    ties = 0
    for k, (ou, ov, opk, tie, R) in enumerate(ora):
        if tie:
            ties += 1
            continue
        if subpixel:
            assert abs(gu[k] - ou) < 1e-4 and abs(gv[k] - ov) < 1e-4, (k, gu[k], ou, gv[k], ov)
        else:
            assert (gu[k], gv[k]) == (ou, ov), (k, gu[k], ou, gv[k], ov)
        assert abs(gp[k] - opk) < 2e-5, (k, gp[k], opk)
    assert ties <= 2


@pytest.mark.parametrize("scale", [1e-12, 1e-6, 1e6, 1e12])
def test_extreme_gray_ranges_match_oracle(pkg, scale):
    """Floating-point gray levels far from the usual range (scaled by 1e-12 .. 1e12):
    Eq. 1 does not depend on the scale, and the tensor-core windows (31, 32 px) take
    their power-of-two operand scales from the data, so they must give the oracle's
    result at any scale where the FP32 window sums of squares stay finite and normal."""
    W, H = 300, 280
    fld = synth.affine_field(W, H, u0=1.7, v0=-2.4, exx=2e-3, eyy=-1e-3, exy=5e-4)
    ref = _speckle(W, H, 41, dtype="f64") * scale
    dfm = _speckle(W, H, 41, fld=fld, dtype="f64", tag=2) * scale
    c = pkg.Correlation(ref, dfm, None, 21, 10, "affine")
    for L, subpixel in ((31, True), (32, True), (64, True)):
        rng = np.random.default_rng(7 + L)
        origins = _random_origins(rng, W, H, L, 30, spread=8)
        gu, gv, gp = _gpu_windows(pkg, c, L, origins, subpixel)
        ora = _oracle_windows(ref, dfm, L, origins, subpixel)
        for k, (ou, ov, opk, tie, R) in enumerate(ora):
            if tie:
                continue
            assert abs(gu[k] - ou) < 1e-4 and abs(gv[k] - ov) < 1e-4, (L, k, gu[k], ou, gv[k], ov)
            assert abs(gp[k] - opk) < 2e-5, (L, k, gp[k], opk)
    c.close()


def test_flat_and_skipped_windows(pkg):
    W, H = 400, 360
    ref = _speckle(W, H, 5)
    dfm = _speckle(W, H, 5, tag=2)
    ref[0:140, 0:140] = 77                        # a flat reference patch
    dfm[200:340, 220:360] = 200                   # a flat deformed patch
    c = pkg.Correlation(ref, dfm, None, 21, 10, "affine")
    for L in (31, 64, 128):
        origins = [(0, 0, 40, 30), (100, 40, 220, 200), (-1, 0, 0, 0), (W - L, H - L, 20, 20),
                   (W - L + 1, 0, 0, 0)]               # the last is outside the image: skipped
        gu, gv, gp = _gpu_windows(pkg, c, L, origins, False)
        ora = _oracle_windows(ref, dfm, L, origins[:2], False)
        for k in range(2):                        # flat: no shift, peak 0 on both sides
            assert (gu[k], gv[k], gp[k]) == (ora[k][0], ora[k][1], 0.0) and ora[k][2] == 0.0
        assert (gu[2], gv[2], gp[2]) == (0.0, 0.0, 0.0) and (gu[4], gv[4], gp[4]) == (0.0, 0.0, 0.0)
        o3 = _oracle_windows(ref, dfm, L, origins[3:4], False)[0]
        assert gu[3] == o3[0] and gv[3] == o3[1]
    c.close()


def test_mad_rule_is_bit_exact(pkg):
    from paper_2601_12941_gb300 import binding as B

    rng = np.random.default_rng(9)
    for nx, ny in [(1, 1), (2, 3), (17, 13), (64, 40)]:
        u = rng.integers(-3, 4, (ny, nx)).astype(np.float32) + 20
        v = rng.integers(-2, 3, (ny, nx)).astype(np.float32) - 7
        out = rng.random((ny, nx)) < 0.05
        u[out] += rng.integers(5, 40, out.sum())
        valid = (rng.random((ny, nx)) > 0.1).astype(np.uint8)
        sub = rng.random((ny, nx)) < 0.3
        u[sub] += rng.random(sub.sum()).astype(np.float32)          # some sub-pixel values too
        for tau in (3.0, 0.0):
            t = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), device="cuda")
            uo, vo = torch.empty(nx * ny, device="cuda"), torch.empty(nx * ny, device="cuda")
            rep = torch.empty(nx * ny, dtype=torch.uint8, device="cuda")
            B.dic_mad_filter(t(u), t(v), t(valid), nx, ny, tau, 0.5, uo, vo, rep)
            torch.cuda.synchronize()
            fu, fv, frep = F.mad_filter(u.astype(np.float64), v.astype(np.float64), valid.astype(bool), tau, 0.5)
            assert np.array_equal(rep.cpu().numpy().reshape(ny, nx).astype(bool), frep)
            assert np.array_equal(uo.cpu().numpy().reshape(ny, nx), fu.astype(np.float32))
            assert np.array_equal(vo.cpu().numpy().reshape(ny, nx), fv.astype(np.float32))


@pytest.mark.parametrize("du,dv,N,D,S,step,roi", [(37, -23, 512, 80, 21, 8, False), (12, 9, 384, 60, 31, 10, True),
                                                  (-5, 3, 256, 10, 21, 6, False), (0, 0, 200, 0, 17, 7, False)])
def test_field_matches_oracle_on_integer_shifts(pkg, du, dv, N, D, S, step, roi):
    ref, dfm = _shifted_pair(3, du, dv, N)
    mask = None
    if roi:
        mask = np.zeros((N, N), np.uint8)
        mask[40:N - 30, 25:N - 50] = 1
    ora = F.multiwindow(ref, dfm, mask, S, step, D, subpixel=False)
    c = pkg.Correlation(ref, dfm, mask, S, step, "affine")
    g = c.fft_field(max_displacement=D, subpixel=False)
    assert g["windows"] == [lv["L"] for lv in ora["levels"]]
    gu, gv = g["u"].cpu().numpy(), g["v"].cpu().numpy()
    assert np.array_equal(g["status"].cpu().numpy(), ora["status"].astype(np.uint8))
    ok = ora["status"] == O.OK
    assert np.array_equal(gu[ok], ora["u"][ok].astype(np.float32))
    assert np.array_equal(gv[ok], ora["v"][ok].astype(np.float32))
    assert np.array_equal(g["replaced"].cpu().numpy().astype(bool), ora["replaced"])
    assert np.abs(g["peak"].cpu().numpy()[ok] - ora["peak"][ok]).max() < 2e-5
    c.close()


def test_smooth_field_level_by_level(pkg):
    # a smooth field with sub-pixel residuals: each level of the GPU is fed the
    # oracle's windows and guesses, so a legitimate near-tie flip cannot cascade
    W = H = 480
    fld = synth.affine_field(W, H, u0=21.4, v0=-13.2, exx=6e-3, eyy=-4e-3, exy=3e-3)
    ref = _speckle(W, H, 31)
    dfm = _speckle(W, H, 31, fld=fld, tag=2)
    ora = F.multiwindow(ref, dfm, None, 21, 8, 50, subpixel=True)
    c = pkg.Correlation(ref, dfm, None, 21, 8, "affine")
    r = 10
    for li, lv in enumerate(ora["levels"]):
        L, nx, ny = lv["L"], lv["nx"], lv["ny"]
        last = li == len(ora["levels"]) - 1
        if last:
            xs, ys = O.grid(W, H, 21, 8)
            X, Y = np.meshgrid(xs - r, ys - r)
        else:
            X, Y = np.meshgrid(np.arange(nx) * L, np.arange(ny) * L)
        gx = np.clip(X + lv["guess_u"], 0, W - L).astype(int)
        gy = np.clip(Y + lv["guess_v"], 0, H - L).astype(int)
        origins = np.stack([X.ravel(), Y.ravel(), gx.ravel(), gy.ravel()], 1)
        gu, gv, gp = _gpu_windows(pkg, c, L, origins, last)
        o = _oracle_windows(ref, dfm, L, origins, last)
        tie = np.array([t[3] for t in o])
        ou, ov = lv["raw_u"].ravel(), lv["raw_v"].ravel()
        tol = 1e-4 if last else 0.0
        bad = ~tie & ((np.abs(gu - ou) > tol) | (np.abs(gv - ov) > tol))
        assert not bad.any(), (L, np.flatnonzero(bad)[:5])
        assert tie.sum() <= max(2, len(tie) // 100)
    c.close()
    # the whole GPU pipeline agrees with the oracle everywhere but at most a handful
    # of points downstream of such a flip
    c = pkg.Correlation(ref, dfm, None, 21, 8, "affine")
    g = c.fft_field(max_displacement=50, subpixel=True)
    gu, gv = g["u"].cpu().numpy(), g["v"].cpu().numpy()
    far = (np.abs(gu - ora["u"]) > 1e-4) | (np.abs(gv - ora["v"]) > 1e-4)
    assert far.mean() < 0.01
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fft_seeded_correlation_matches_oracle(pkg, precision):
    W = H = 256
    fld = synth.affine_field(W, H, u0=37.4, v0=-21.7, exx=1e-3, eyy=-5e-4)
    ref = _speckle(W, H, 9, noise=1.0)
    dfm = _speckle(W, H, 9, fld=fld, noise=1.0, tag=2)
    seeds = [(128, 128)]
    prm = dict(init="fft", max_displacement=100)
    ora = oracle.correlate(ref, dfm, None, 21, 8, "affine", seeds, dict(ORACLE_PARAMS, **prm))
    c = pkg.Correlation(ref, dfm, None, 21, 8, "affine", precision=precision, **dict(GPU_PARAMS[precision], **prm))
    c.run(seeds)
    gpu = c.results()
    c.close()
    stats = compare(gpu, ora, W, H, 21)
    assert stats["accepted"] > 0.5 * stats["points"]
    # the integer search cannot start this seed
    from paper_2601_12941_gb300 import DicError

    c = pkg.Correlation(ref, dfm, None, 21, 8, "affine", precision=precision)
    with pytest.raises(DicError):
        c.run(seeds)
    c.close()
