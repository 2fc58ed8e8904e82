"""CUDA library against the FP64 oracle, element by element, through the C-ABI.

Sizes are ones the oracle finishes in seconds while still spanning many blocks,
several propagation waves and ragged image sizes. Tolerances: |du|, |dv| <= 1e-3 px
and |dp_2..11| <= 1e-5 on points both accept, the same accepted/rejected set and
the same wave index except at borderline points (see parity_util)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import dic_oracle as O
from synth import workloads as wl

from parity_util import GPU_PARAMS, ORACLE_PARAMS, compare

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


def _pair(W, H, fld, dtype="u8", seed=101, gray=255.0, noise=0.0, density=0.0305, sigma=(1.5, 3.0)):
    sp = synth.Speckle(seed=seed, density=density, sigma=sigma, cell=16)
    ref = synth.ImageSpec(sp, gray_max=gray, noise=noise, noise_tag=1)
    dfm = synth.ImageSpec(sp, field=fld, gray_max=gray, noise=noise, noise_tag=2)
    return synth.render(ref, W, H, dtype), synth.render(dfm, W, H, dtype)


_ORACLE_CACHE = {}


def _oracle(key, *args):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle.correlate(*args)
    return _ORACLE_CACHE[key]


def _run(pkg, ref, dfm, roi, S, step, shape, seeds, precision, device=True, **kw):
    prm = dict(GPU_PARAMS[precision])
    prm.update(kw)
    if device:
        ref_t = torch.from_numpy(ref.view(np.int16) if ref.dtype == np.uint16 else ref).cuda()
        dfm_t = torch.from_numpy(dfm.view(np.int16) if dfm.dtype == np.uint16 else dfm).cuda()
    else:
        ref_t, dfm_t = ref, dfm
    c = pkg.Correlation(ref_t, dfm_t, roi, S, step, shape, precision=precision, **prm)
    c.run(seeds)
    res = c.results()
    c.close()
    return res


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_prefilter_matches_oracle_coefficients(pkg, precision, dtype):
    W, H = 203, 157   # ragged: neither a multiple of the 32-pixel tile
    ref, dfm = _pair(W, H, synth.affine_field(W, H, u0=0.5), dtype=dtype)
    c = pkg.Correlation(ref, dfm, None, 21, 9, "affine", precision=precision)
    c.run([(100, 80)])
    from paper_2601_12941_gb300 import binding as B

    for which, img in ((0, ref), (1, dfm)):
        ptr, ld, es = pkg.dic_get_coefficients(c.h, which)
        typestr = np.dtype(np.float64 if es == 8 else np.float32).str
        dev = torch.as_tensor(B._DeviceArray(ptr, (H, ld), typestr), device="cuda")
        got = dev[:, :W].double().cpu().numpy()
        want = O.bspline_coefficients(img.astype(np.float64))
        rel = np.abs(got - want).max() / np.abs(want).max()
        assert rel < (1e-13 if precision == "fp64" else 2e-6), rel
    c.close()


@pytest.mark.parametrize("dtype", ["u8", "u16", "bf16", "f32", "f64"])
def test_prefilter_strips_match_oracle_for_every_gray_type(pkg, dtype):
    """The FP32 prefilter on an image wide and tall enough for interior strips (16-byte
    vector loads), edge strips (mirrored columns) and a partial last block of rows,
    for every gray type the library reads; a width of 700 (rows not 16-byte aligned)
    takes the element-by-element path everywhere."""
    from paper_2601_12941_gb300 import binding as B

    for W, H in ((704, 600), (700, 531)):
        gray = 4095.0 if dtype == "u16" else 255.0
        kind = {"u8": "u8", "bf16": "u8", "u16": "u16", "f32": "f32", "f64": "f64"}[dtype]
        ref, dfm = _pair(W, H, synth.affine_field(W, H, u0=0.5), dtype=kind, gray=gray, noise=0.01 * gray)
        if dtype == "bf16":
            dev_ref = torch.from_numpy(ref).cuda().to(torch.bfloat16)
            dev_dfm = torch.from_numpy(dfm).cuda().to(torch.bfloat16)
        else:
            dev_ref = torch.from_numpy(ref.view(np.int16) if ref.dtype == np.uint16 else ref).cuda()
            dev_dfm = torch.from_numpy(dfm.view(np.int16) if dfm.dtype == np.uint16 else dfm).cuda()
        c = pkg.Correlation(dev_ref, dev_dfm, None, 21, 9, "affine", precision="mixed")
        c.run([(W // 2, H // 2)])
        for which, img in ((0, ref), (1, dfm)):
            ptr, ld, es = pkg.dic_get_coefficients(c.h, which)
            dev = torch.as_tensor(B._DeviceArray(ptr, (H, ld), np.dtype(np.float32).str), device="cuda")
            got = dev[:, :W].double().cpu().numpy()
            want = O.bspline_coefficients(img.astype(np.float64))
            rel = np.abs(got - want).max() / np.abs(want).max()
            assert rel < 2e-6, (W, H, which, rel)
        c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fp64_solve"])
def test_affine_256_u8_matches_oracle(pkg, precision):
    w = wl.affine_256_u8()
    ref = synth.render(w.ref, w.width, w.height, w.dtype)
    dfm = synth.render(w.deformed, w.width, w.height, w.dtype)
    prm = dict(ORACLE_PARAMS, search_radius=w.search_radius)
    ora = _oracle("affine256", ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds, prm)
    gpu = _run(pkg, ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds, precision,
               search_radius=w.search_radius)
    stats = compare(gpu, ora, w.width, w.height, w.subset_size, precision=precision)
    assert stats["accepted"] > 2000
    if precision == "fp64":
        assert stats["max_uv"] < 1e-8 and stats["max_p"] < 1e-9
    print(precision, stats)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fp64_solve"])
def test_quadratic_sine_u16_matches_oracle(pkg, precision):
    W, H = 230, 190
    w = wl.sine_2048_u16(W, H)
    ref = synth.render(w.ref, W, H, "u16")
    dfm = synth.render(w.deformed, W, H, "u16")
    S, step = 31, 7
    prm = dict(ORACLE_PARAMS, search_radius=w.search_radius)
    ora = _oracle("sine230", ref, dfm, None, S, step, "quadratic", w.seeds, prm)
    gpu = _run(pkg, ref, dfm, None, S, step, "quadratic", w.seeds, precision,
               search_radius=w.search_radius)
    stats = compare(gpu, ora, W, H, S, precision=precision)
    assert stats["accepted"] > 0.8 * stats["points"]
    print(precision, stats)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fp64_solve"])
def test_rigid_matches_oracle(pkg, precision):
    W, H = 150, 133
    ref, dfm = _pair(W, H, synth.affine_field(W, H, u0=-3.4, v0=1.3), dtype="u8")
    prm = dict(ORACLE_PARAMS, search_radius=6)
    ora = _oracle("rigid150", ref, dfm, None, 15, 4, "rigid", [(75, 66)], prm)
    gpu = _run(pkg, ref, dfm, None, 15, 4, "rigid", [(75, 66)], precision, search_radius=6)
    compare(gpu, ora, W, H, 15, precision=precision)


@pytest.mark.parametrize("S", [41, 21])
@pytest.mark.parametrize("dtype", ["u16", "f32", "f64"])
def test_gray_types_at_both_block_sizes_match_oracle(pkg, dtype, S):
    """Gray levels of each element type through the 128-thread kernel (subset 41: the
    u16 and f32 gray tiles share the gradient region, the f64 tile has its own) and the
    64-thread kernel (subset 21)."""
    W, H = 170, 150
    gray = 4095.0 if dtype == "u16" else 255.0
    fld = synth.affine_field(W, H, u0=1.3, v0=-0.8, exx=1.5e-3, eyy=-1e-3, exy=4e-4)
    ref, dfm = _pair(W, H, fld, dtype=dtype, gray=gray, noise=0.01 * gray)
    prm = dict(ORACLE_PARAMS, search_radius=4)
    seeds = [(W // 2, H // 2)]
    ora = oracle.correlate(ref, dfm, None, S, 7, "affine", seeds, prm)
    gpu = _run(pkg, ref, dfm, None, S, 7, "affine", seeds, "mixed", search_radius=4)
    compare(gpu, ora, W, H, S)


def test_roi_hole_two_seeds_and_out_of_roi_seed(pkg):
    W, H = 180, 160
    fld = synth.affine_field(W, H, u0=1.6, v0=-2.2, exx=2e-3, eyy=-1e-3, exy=5e-4, eyx=5e-4)
    ref, dfm = _pair(W, H, fld, dtype="u16", gray=4095.0, noise=0.01 * 4095)
    roi = np.ones((H, W), bool)
    roi[60:100, 70:110] = False
    roi[:, 150:] = False
    seeds = [(40, 40), (120, 130), (85, 80)]    # the last lies in the hole
    prm = dict(ORACLE_PARAMS, search_radius=5)
    ora = oracle.correlate(ref, dfm, roi, 17, 5, "affine", seeds, prm)
    gpu = _run(pkg, ref, dfm, roi, 17, 5, "affine", seeds, "mixed", search_radius=5)
    stats = compare(gpu, ora, W, H, 17)
    assert (np.asarray(gpu["status"]) == O.NOT_IN_ROI).sum() == (ora["status"] == O.NOT_IN_ROI).sum() > 0
    assert (np.asarray(gpu["wave"]) == 0).sum() == 2
    print(stats)


def test_host_and_device_inputs_and_results_agree(pkg):
    W, H = 120, 100
    ref, dfm = _pair(W, H, synth.affine_field(W, H, u0=0.7, v0=0.2), dtype="u8")
    a = _run(pkg, ref, dfm, None, 15, 5, "affine", [(60, 50)], "mixed", device=True)
    b = _run(pkg, ref, dfm, None, 15, 5, "affine", [(60, 50)], "mixed", device=False)
    for k in ("p", "status", "wave", "iters"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]))
    c = pkg.Correlation(ref, dfm, None, 15, 5, "affine")
    c.run([(60, 50)])
    host = c.results()
    dev = c.results(on_device=True)
    for k in ("p", "u", "v", "zncc", "status", "wave", "iters", "x", "y"):
        assert np.array_equal(np.asarray(host[k]), dev[k].cpu().numpy(), equal_nan=k == "zncc")
    c.close()


def test_repeat_runs_are_deterministic_and_nan_flag(pkg):
    W, H = 140, 120
    ref, dfm = _pair(W, H, synth.affine_field(W, H, u0=2.2, v0=0.4, exx=1e-3), dtype="u8")
    c = pkg.Correlation(ref, dfm, None, 21, 6, "affine")
    c.run([(70, 60)])
    r1 = c.results()
    c.run([(70, 60)])
    r2 = c.results()
    for k in ("p", "status", "wave", "iters", "zncc"):
        assert np.array_equal(r1[k], r2[k], equal_nan=True)
    c.set_params(nan_unconverged=1)
    c.run([(70, 60)])
    r3 = c.results()
    ok = r3["status"] == 0
    assert np.isnan(r3["u"][~ok]).all() and np.array_equal(r3["u"][ok], r1["u"][ok])
    c.close()


def test_flat_image_and_seed_errors(pkg):
    from paper_2601_12941_gb300 import DicError

    flat = np.full((64, 64), 77, np.uint8)
    c = pkg.Correlation(flat, flat, None, 15, 5, "affine")
    with pytest.raises(DicError) as e:
        c.run([(32, 32)])
    assert e.value.code == -5     # DIC_ENOSEED
    r = c.results()
    q = int(np.flatnonzero(r["wave"] == 0)[0])
    assert r["status"][q] == O.FLAT_SUBSET
    c.close()
    ref, dfm = _pair(64, 64, synth.IDENTITY)
    roi = np.zeros((64, 64), bool)
    roi[:, :32] = True
    c = pkg.Correlation(ref, dfm, roi, 15, 5, "affine")
    with pytest.raises(DicError) as e:
        c.run([(50, 32)])          # seed outside the ROI
    assert e.value.code == -5
    with pytest.raises(DicError) as e:
        c.run([])
    assert e.value.code == -1
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_strain_uses_global_fallback_and_matches_oracle(pkg, precision):
    """35% stretch: the warped 21 x 21 subset spans more coefficients than the
    shared-memory window holds, so samples read the global plane."""
    W, H = 160, 150
    fld = synth.affine_field(W, H, u0=0.6, v0=-0.4, exx=0.35, eyy=0.3)
    ref, dfm = _pair(W, H, fld, dtype="f32", seed=77)
    prm = dict(ORACLE_PARAMS, search_radius=3)
    ora = _oracle("strain160", ref, dfm, None, 21, 6, "affine", [(80, 75)], prm)
    gpu = _run(pkg, ref, dfm, None, 21, 6, "affine", [(80, 75)], precision, search_radius=3)
    stats = compare(gpu, ora, W, H, 21, precision=precision)
    assert stats["accepted"] >= 4
    print(precision, stats)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fp64_solve"])
def test_bf16_gray_levels_equal_the_u8_run_and_match_oracle(pkg, precision):
    """Gray levels stored as BF16 (the gigapixel workload's storage type): a BF16
    tensor holding u8 values represents them exactly, so every result equals the u8
    run's bit for bit, and both match the oracle."""
    W, H = 190, 170
    fld = synth.affine_field(W, H, u0=-1.3, v0=2.1, exx=1.2e-3, eyy=-6e-4, exy=3e-4, eyx=3e-4)
    ref, dfm = _pair(W, H, fld, dtype="u8", seed=202, noise=2.0)
    seeds = [(95, 85)]
    prm = dict(ORACLE_PARAMS, search_radius=4)
    ora = _oracle("bf16_190", ref, dfm, None, 21, 5, "affine", seeds, prm)
    a = _run(pkg, ref, dfm, None, 21, 5, "affine", seeds, precision, search_radius=4)
    rb = torch.from_numpy(ref).cuda().to(torch.bfloat16)
    db = torch.from_numpy(dfm).cuda().to(torch.bfloat16)
    assert torch.equal(rb.float(), torch.from_numpy(ref).cuda().float())
    c = pkg.Correlation(rb, db, None, 21, 5, "affine", precision=precision, search_radius=4,
                        **GPU_PARAMS[precision])
    c.run(seeds)
    b = c.results()
    c.close()
    for k in ("p", "zncc", "status", "wave", "iters"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=k == "zncc"), k
    stats = compare(b, ora, W, H, 21, precision=precision)
    assert stats["accepted"] > 0.9 * stats["points"]
    print(precision, stats)


@pytest.mark.parametrize("W,H,S,step,seed", [
    (40, 40, 21, 10, (20, 20)),      # 2 x 2 grid
    (25, 25, 21, 10, (12, 12)),      # one point
    (260, 26, 21, 6, (12, 12)),      # one row of 40 points, seeded at its left end: 40 waves
    (24, 200, 21, 5, (12, 190)),     # one column of 36 points, seeded at its bottom end
])
def test_tiny_grids_and_one_row_strips_match_oracle(pkg, W, H, S, step, seed):
    """Grids with fewer points than the first wave batches, and strips with as many
    waves as points: the wave loop must finish on the empty front. The field moves
    every subset at least 1.3 px away from the top and left edges (centres start at
    r, so an unmoved subset there starts at row or column 0, outside the sampling
    bounds)."""
    fld = synth.affine_field(W, H, u0=1.5, v0=1.5, exx=1e-3)
    ref, dfm = _pair(W, H, fld, dtype="u8", seed=303)
    prm = dict(ORACLE_PARAMS, search_radius=2)
    ora = oracle.correlate(ref, dfm, None, S, step, "affine", [seed], prm)
    assert (ora["status"] == O.OK).sum() >= max(1, 0.9 * len(ora["status"]))
    for precision in ("fp64", "mixed"):
        gpu = _run(pkg, ref, dfm, None, S, step, "affine", [seed], precision, search_radius=2)
        stats = compare(gpu, ora, W, H, S, precision=precision)
        assert stats["accepted"] >= max(1, 0.9 * stats["points"]), stats


def test_acceptance_is_decided_at_the_warp_of_the_last_pass(pkg):
    """R8: the in-bounds test belongs to the last iteration's sampling pass. A
    point whose single pass lies inside the bounds is accepted although the update
    carries its subset past the right edge; the GPU agrees with the oracle."""
    from scipy import ndimage

    W, H = 64, 40
    rng = np.random.default_rng(3)
    base = ndimage.gaussian_filter(rng.random((H, W + 8)), 1.5) * 200.0
    ref = np.ascontiguousarray(base[:, 4:4 + W]).astype(np.float32)
    dfm = np.ascontiguousarray(base[:, 1:1 + W]).astype(np.float32)
    S, r = 11, 5
    step = 17                            # centres x = 5, 22, 39, 56 and y = 5, 22
    seed = (W - 2 - r - 1, 22)           # x = 56: at p = 0 its last column is x = W - 3
    prm = dict(max_iter=1, conv_threshold=10.0, zncc_min=-1.0, search_radius=0)
    ora = oracle.correlate(ref.astype(np.float64), dfm.astype(np.float64), None, S, step, "affine", [seed], prm)
    q = int(np.flatnonzero(np.asarray(ora["wave"]) == 0)[0])
    assert ora["status"][q] == O.OK and ora["p"][q][0] > 1.0
    for precision in ("fp64", "mixed"):
        c = pkg.Correlation(torch.from_numpy(ref).cuda(), torch.from_numpy(dfm).cuda(), None, S, step, "affine",
                            precision=precision, **prm)
        c.run([seed])
        g = c.results()
        c.close()
        assert g["status"][q] == O.OK and g["iters"][q] == 1
        assert abs(g["p"][q][0] - ora["p"][q][0]) < 1e-4
