"""Full-size workloads on the GPU, checked point by point on a sample.

The 2048 x 2048 u16 quadratic sine pair and the 32768 x 32768 u8 gigapixel pair
run whole on the GPU with the kernels and launch configuration the benchmark
uses. The oracle then correlates a seeded sample of points one at a time, each
from a start it derives from the analytic displacement field (never from GPU
output), on host-rendered images or crops; the two must agree within the parity
tolerances. Over all points, the propagation must satisfy the wave invariants,
and the device-rendered input must equal the host-rendered one wherever the
oracle reads it.
"""
import numpy as np
import pytest

import synth
from oracle import dic_oracle as O
from synth import workloads as wl

from parity_util import GPU_PARAMS, ORACLE_PARAMS, TOL_P, TOL_UV

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_2601_12941_gb300 as P
    from paper_2601_12941_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    P.load()
    return P


def wave_invariants(res):
    """Wave k of every attempted non-seed point is 1 + the smallest wave of its
    accepted 4-neighbours (so waves are BFS distances over accepted points), no
    point next to an accepted one is left unattempted, and unattempted points are
    reported not reached."""
    nx, ny = int(res["nx"]), int(res["ny"])
    st = np.asarray(res["status"]).reshape(ny, nx).astype(np.int64)
    wv = np.asarray(res["wave"]).reshape(ny, nx).astype(np.int64)
    ok = st == O.OK
    big = np.int64(1) << 40
    acc_w = np.where(ok, wv, big)
    best = np.full((ny, nx), big)
    best[:, 1:] = np.minimum(best[:, 1:], acc_w[:, :-1])
    best[:, :-1] = np.minimum(best[:, :-1], acc_w[:, 1:])
    best[1:, :] = np.minimum(best[1:, :], acc_w[:-1, :])
    best[:-1, :] = np.minimum(best[:-1, :], acc_w[1:, :])
    attempted = wv >= 0
    inner = attempted & (wv > 0)
    assert np.array_equal(wv[inner], best[inner] + 1), "a wave index is not a BFS distance"
    inroi = st != O.NOT_IN_ROI
    assert not (inroi & ~attempted & (best < big)).any(), "an accepted point left a neighbour unattempted"
    assert (st[~attempted & inroi] == O.NOT_REACHED).all()


def _dev(a):
    return torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()


def _sine_taylor_start(fld, xc, yc, h=0.5):
    """The analytic field's second-order expansion at the centre in Eq. 5's
    parameters (no 1/2 factor on the quadratic terms), by central differences."""
    X = np.array([xc, xc + h, xc - h, xc, xc, xc + h, xc - h, xc + h, xc - h], float)
    Y = np.array([yc, yc, yc, yc + h, yc - h, yc + h, yc + h, yc - h, yc - h], float)
    out = []
    for f in synth.displacement(fld, X, Y):
        fx, fy = (f[1] - f[2]) / (2 * h), (f[3] - f[4]) / (2 * h)
        fxx, fyy = (f[1] - 2 * f[0] + f[2]) / h ** 2, (f[3] - 2 * f[0] + f[4]) / h ** 2
        fxy = (f[5] - f[6] - f[7] + f[8]) / (4 * h * h)
        out.append((f[0], fx, fy, 0.5 * fxx, fxy, 0.5 * fyy))
    (u, ux, uy, uxx, uxy, uyy), (v, vx, vy, vxx, vxy, vyy) = out
    return [u, v, ux, uy, vx, vy, uxx, uxy, uyy, vxx, vxy, vyy]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sine_2048_u16_quadratic_full_size(pkg, precision):
    """The 2048^2 quadratic workload in both precisions. Periods above ~80 px
    (x > 500): the 12-parameter warp follows the sine and the minimum near the
    analytic start is unique, so the oracle, started there, must give the GPU's
    status and parameters. Shorter periods (150 < x <= 500, T 31-80 px): the cost
    has several minima within a fraction of a pixel (the oracle's roots from the
    analytic start move by up to 0.5 px), so which one a point reaches depends on
    its start (the neighbour's warp on the GPU); there each accepted GPU point is
    checked to be a valid answer: a stationary point of the cost (one oracle
    Gauss-Newton step from it moves it by less than the parity tolerances) whose
    correlation coefficient clears the cut-off."""
    w = wl.sine_2048_u16()
    W, H, S = w.width, w.height, w.subset_size
    ref = synth.render(w.ref, W, H, "u16")
    dfm = synth.render(w.deformed, W, H, "u16")
    c = pkg.Correlation(_dev(ref), _dev(dfm), None, S, w.subset_step, w.shape, precision=precision,
                        search_radius=w.search_radius, **GPU_PARAMS[precision])
    c.run(list(w.seeds))
    res = c.results()
    c.close()
    wave_invariants(res)
    ok = res["status"] == O.OK
    assert ok.mean() > 0.95
    refp, defp = O.Plane(ref), O.Plane(dfm)
    rng = np.random.default_rng(7)
    cand = np.flatnonzero((res["x"] > 500) & (res["wave"] >= 0))
    pick = rng.choice(cand, 40, replace=False)
    errs = []
    for q in pick:
        xc, yc = int(res["x"][q]), int(res["y"][q])
        # start: the analytic field's displacement at the centre, rounded
        u, v = synth.displacement(w.field, np.array([float(xc)]), np.array([float(yc)]))
        ora = O.icgn(refp, defp, xc, yc, S, "quadratic", [round(u[0]), round(v[0])], ORACLE_PARAMS)
        assert (ora["status"] == O.OK) == bool(ok[q]), (q, ora["status"], res["status"][q])
        if ora["status"] == O.OK:
            d = np.abs(res["p"][q] - ora["p"])
            assert d[:2].max() <= TOL_UV and d[2:].max() <= TOL_P, (q, d)
            assert abs(float(res["zncc"][q]) - ora["zncc"]) <= 1e-5, q
            errs.append(d[:2].max())
    # short periods: validity of the GPU's root
    short = np.flatnonzero((res["x"] > 150) & (res["x"] <= 500) & ok)
    n_moved = 0
    for q in rng.choice(short, 30, replace=False):
        xc, yc = int(res["x"][q]), int(res["y"][q])
        one = O.icgn(refp, defp, xc, yc, S, "quadratic", list(res["p"][q]), dict(ORACLE_PARAMS, max_iter=1))
        assert one["status"] in (O.OK, O.MAX_ITER), (q, one["status"])
        d = np.abs(one["p"] - res["p"][q])
        assert d[:2].max() <= TOL_UV and d[2:].max() <= TOL_P, (q, d)
        assert one["zncc"] >= 0.70 and abs(float(res["zncc"][q]) - one["zncc"]) <= 1e-5, q
        # and the oracle's own start lands on a root of the same quality
        ana = O.icgn(refp, defp, xc, yc, S, "quadratic", _sine_taylor_start(w.field, xc, yc), ORACLE_PARAMS)
        n_moved += int(ana["status"] != O.OK or np.abs(ana["p"][:2] - res["p"][q][:2]).max() > TOL_UV)
    print("sine 2048 %s: %d accepted of %d, sampled max |du,dv| %.2e; short periods: 30 valid roots, "
          "%d of them not the root the analytic start reaches" % (precision, ok.sum(), ok.size, max(errs), n_moved))


def test_gigapixel_32768_u8_full_size(pkg):
    w = wl.gigapixel_u8()
    W, H, S, r = w.width, w.height, w.subset_size, (w.subset_size - 1) // 2
    ref = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    dfm = torch.empty_like(ref)
    synth.render_gpu(w.ref, ref)
    synth.render_gpu(w.deformed, dfm)
    c = pkg.Correlation(ref, dfm, None, S, w.subset_step, w.shape, precision="mixed",
                        search_radius=w.search_radius, **GPU_PARAMS["mixed"])
    c.run(list(w.seeds))
    res = c.results()
    c.close()
    wave_invariants(res)
    ok = res["status"] == O.OK
    assert ok.mean() > 0.99
    fld = w.field
    rng = np.random.default_rng(11)
    X = res["x"].astype(np.float64) - fld.cx
    Y = res["y"].astype(np.float64) - fld.cy
    # subsets away from the slip line Y' = X' (a jump inside the subset has no
    # single affine root) and from the image edges
    far = np.abs(Y - X) / np.sqrt(2.0) > r * np.sqrt(2.0) + 8
    inside = (res["x"] > 200) & (res["x"] < W - 200) & (res["y"] > 200) & (res["y"] < H - 200)
    pick = rng.choice(np.flatnonzero(far & inside & (res["wave"] >= 0)), 30, replace=False)
    pad = 48 + r + 16
    errs = []
    for q in pick:
        xc, yc = int(res["x"][q]), int(res["y"][q])
        x0, y0, side = xc - pad, yc - pad, 2 * pad + 1
        rc, roff = synth.render_crop(w.ref, W, H, x0, y0, side, side, "u8")
        dc, doff = synth.render_crop(w.deformed, W, H, x0, y0, side, side, "u8")
        # the device-rendered input equals the host-rendered crop the oracle reads
        assert np.array_equal(dc, dfm[doff[1]:doff[1] + dc.shape[0], doff[0]:doff[0] + dc.shape[1]].cpu().numpy())
        assert np.array_equal(rc, ref[roff[1]:roff[1] + rc.shape[0], roff[0]:roff[0] + rc.shape[1]].cpu().numpy())
        refp = O.Plane(rc, roff[0], roff[1], W, H)
        defp = O.Plane(dc, doff[0], doff[1], W, H)
        # start: the analytic affine field at the centre (displacement and gradient)
        u, v = synth.displacement(fld, np.array([float(xc)]), np.array([float(yc)]))
        jump = fld.jump * np.sqrt(0.5) if (yc - fld.cy) > (xc - fld.cx) else 0.0
        p0 = [u[0], v[0], fld.exx, fld.exy, fld.eyx, fld.eyy]
        ora = O.icgn(refp, defp, xc, yc, S, "affine", p0, ORACLE_PARAMS)
        assert (ora["status"] == O.OK) == bool(ok[q]), (q, ora["status"], res["status"][q])
        if ora["status"] == O.OK:
            d = np.abs(res["p"][q] - ora["p"])
            assert d[:2].max() <= TOL_UV and d[2:].max() <= TOL_P, (q, d, jump)
            errs.append(d[:2].max())
    print("gigapixel: %d accepted of %d, waves %d, sampled max |du,dv| %.2e"
          % (ok.sum(), ok.size, res["n_waves"], max(errs)))


def _small_pair():
    W, H = 170, 150
    sp = synth.Speckle(seed=99, density=0.0305, sigma=(1.5, 3.0), cell=16)
    fld = synth.affine_field(W, H, u0=0.9, v0=-1.4, exx=1e-3, eyy=1e-3)
    ref = synth.render(synth.ImageSpec(sp, gray_max=255.0, noise_tag=1), W, H, "u8")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=255.0, noise_tag=2), W, H, "u8")
    return W, H, ref, dfm


@pytest.mark.parametrize("S,shape,thr", [(7, "rigid", 1e-5), (61, "affine", 1e-8), (61, "quadratic", 1e-8)])
def test_subset_size_limits_match_oracle(pkg, S, shape, thr):
    """Smallest useful and largest supported subsets (rigid 7 x 7 converges
    linearly, so both sides stop at 1e-5 there)."""
    import oracle
    from parity_util import compare

    W, H, ref, dfm = _small_pair()
    step = 4 if S < 20 else 9
    seeds = [(85, 75)]
    ora = oracle.correlate(ref, dfm, None, S, step, shape, seeds,
                           dict(conv_threshold=thr, max_iter=100, search_radius=3))
    c = pkg.Correlation(_dev(ref), _dev(dfm), None, S, step, shape, precision="mixed", search_radius=3,
                        conv_threshold=max(thr, 1e-5), max_iter=100)
    c.run(seeds)
    gpu = c.results()
    c.close()
    stats = compare(gpu, ora, W, H, S)
    assert stats["accepted"] > 0.5 * stats["points"]


def test_three_pixel_subsets_reject_the_seed_like_the_oracle(pkg):
    """A 3 x 3 subset never meets the threshold: both sides stop at max_iter, the
    front dies at the seed and the call reports that no seed was accepted."""
    import oracle
    from paper_2601_12941_gb300 import DicError

    W, H, ref, dfm = _small_pair()
    ora = oracle.correlate(ref, dfm, None, 3, 4, "rigid", [(85, 75)],
                           dict(conv_threshold=1e-4, max_iter=60, search_radius=3))
    c = pkg.Correlation(_dev(ref), _dev(dfm), None, 3, 4, "rigid", precision="mixed", search_radius=3,
                        conv_threshold=1e-4, max_iter=60)
    with pytest.raises(DicError) as e:
        c.run([(85, 75)])
    assert e.value.code == -5
    gpu = c.results()
    c.close()
    assert np.array_equal(gpu["status"], ora["status"].astype(np.uint8))
    assert np.array_equal(gpu["wave"], ora["wave"])
