"""Bicubic convolution interpolation (DIC_BICUBIC; oracle reading R14) on the GPU
against the oracle: the coefficient plane bit for bit, whole correlations in both
precisions, with another cost and with Levenberg-Marquardt, and exact recovery of
an integer shift."""
import numpy as np
import pytest

import oracle
import synth
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


def _run(pkg, ref, dfm, S, step, shape, seeds, precision, R, **kw):
    c = pkg.Correlation(ref, dfm, None, S, step, shape, interp="bicubic", precision=precision, search_radius=R,
                        **dict(GPU_PARAMS[precision], **kw))
    c.run(seeds)
    r = c.results()
    c.close()
    return r


def _affine_pair(dtype=None):
    w = wl.affine_256_u8()
    dt = dtype or w.dtype
    return w, synth.render(w.ref, w.width, w.height, dt), synth.render(w.deformed, w.width, w.height, dt)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bicubic_affine_matches_oracle(pkg, precision):
    w, ref, dfm = _affine_pair()
    ora = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds,
                           dict(ORACLE_PARAMS, search_radius=w.search_radius, interp="bicubic"))
    gpu = _run(pkg, ref, dfm, w.subset_size, w.subset_step, w.shape, w.seeds, precision, w.search_radius)
    stats = compare(gpu, ora, w.width, w.height, w.subset_size)
    assert stats["accepted"] > 2000
    if precision == "fp64":
        assert stats["max_uv"] < 1e-8


@pytest.mark.parametrize("cost,optimizer", [("nssd", "gn"), ("znssd", "lm")])
def test_bicubic_with_other_cost_and_optimizer(pkg, cost, optimizer):
    w, ref, dfm = _affine_pair()
    ora = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds,
                           dict(ORACLE_PARAMS, search_radius=w.search_radius, interp="bicubic", cost=cost,
                                optimizer=optimizer))
    gpu = _run(pkg, ref, dfm, w.subset_size, w.subset_step, w.shape, w.seeds, "mixed", w.search_radius,
               cost=cost, optimizer=optimizer)
    stats = compare(gpu, ora, w.width, w.height, w.subset_size)
    assert stats["accepted"] > 2000


def test_bicubic_quadratic_u16_mixed(pkg):
    W, H = 230, 190
    fld = synth.sine_field(W, 0.5, 10.0, 300.0)
    sp = synth.Speckle(seed=77, density=0.0305, sigma=(1.5, 3.0), cell=16)
    G = 4095.0
    ref = synth.render(synth.ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=1), W, H, "u16")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=2), W, H, "u16")
    seeds = [(115, 95)]
    ora = oracle.correlate(ref, dfm, None, 31, 4, "quadratic", seeds,
                           dict(ORACLE_PARAMS, search_radius=4, interp="bicubic"))
    gpu = _run(pkg, ref, dfm, 31, 4, "quadratic", seeds, "mixed", 4)
    stats = compare(gpu, ora, W, H, 31)
    assert stats["accepted"] > 0.8 * stats["points"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_bicubic_plane_is_the_gray_image(pkg, precision, dtype):
    from paper_2601_12941_gb300 import binding as B

    W, H = 203, 157   # ragged
    sp = synth.Speckle(seed=5, density=0.03, sigma=(1.5, 3.0), cell=16)
    ref = synth.render(synth.ImageSpec(sp, gray_max=250.0, noise=2.0, noise_tag=1), W, H, dtype)
    dfm = synth.render(synth.ImageSpec(sp, field=synth.affine_field(W, H, u0=0.5), gray_max=250.0, noise=2.0,
                                       noise_tag=2), W, H, dtype)
    c = pkg.Correlation(ref, dfm, None, 21, 9, "affine", interp="bicubic", precision=precision)
    c.run([(100, 80)])
    for which, img in ((0, ref), (1, dfm)):
        ptr, ld, es = pkg.dic_get_coefficients(c.h, which)
        typestr = np.dtype(np.float64 if es == 8 else np.float32).str
        dev = torch.as_tensor(B._DeviceArray(ptr, (H, ld), typestr), device="cuda")
        got = dev[:, :W].cpu().numpy()
        assert np.array_equal(got, img.astype(got.dtype))
    c.close()


def test_bicubic_integer_shift_is_exact(pkg):
    sp = synth.Speckle(seed=7, density=0.03, sigma=(1.5, 3.0), cell=16)
    big = synth.render(synth.ImageSpec(sp, gray_max=255.0), 230, 230, "u8")
    ref = np.ascontiguousarray(big[5:205, 5:205])
    dfm = np.ascontiguousarray(big[5 + 2:205 + 2, 5 - 3:205 - 3])       # moves by (+3, -2)
    r = _run(pkg, ref, dfm, 21, 10, "affine", [(100, 100)], "mixed", 6)
    ok = r["status"] == 0
    assert ok.sum() > 0.8 * len(ok)
    assert np.abs(r["u"][ok] - 3.0).max() < 1e-5 and np.abs(r["v"][ok] + 2.0).max() < 1e-5
    assert np.abs(r["p"][ok][:, 2:]).max() < 1e-6
