"""Levenberg-Marquardt (Sec. 2.2; oracle reading R13) on the GPU against the oracle
running the same damping schedule, in both precisions and with each cost, and
against the GPU's own Gauss-Newton root."""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads as wl

from parity_util import GPU_PARAMS, ORACLE_PARAMS, TOL_P, TOL_UV, compare

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
    c = pkg.Correlation(ref, dfm, None, S, step, shape, precision=precision, search_radius=R,
                        **dict(GPU_PARAMS[precision], **kw))
    c.run(seeds)
    r = c.results()
    c.close()
    return r


def _affine_pair():
    w = wl.affine_256_u8()
    return w, synth.render(w.ref, w.width, w.height, w.dtype), synth.render(w.deformed, w.width, w.height, w.dtype)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cost", ["znssd", "nssd", "ssd"])
def test_lm_matches_oracle(pkg, precision, cost):
    w, ref, dfm = _affine_pair()
    ora = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds,
                           dict(ORACLE_PARAMS, search_radius=w.search_radius, cost=cost, optimizer="lm"))
    gpu = _run(pkg, ref, dfm, w.subset_size, w.subset_step, w.shape, w.seeds, precision, w.search_radius,
               cost=cost, optimizer="lm")
    stats = compare(gpu, ora, w.width, w.height, w.subset_size)
    assert stats["accepted"] > 2000
    if precision == "fp64":
        assert stats["max_uv"] < 1e-8


def test_lm_quadratic_mixed_matches_oracle(pkg):
    W, H = 230, 190
    fld = synth.sine_field(W, 0.5, 10.0, 300.0)
    sp = synth.Speckle(seed=77, density=0.0305, sigma=(1.5, 3.0), cell=16)
    G = 4095.0
    ref = synth.render(synth.ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=1), W, H, "u16")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=2), W, H, "u16")
    seeds = [(115, 95)]
    ora = oracle.correlate(ref, dfm, None, 31, 4, "quadratic", seeds,
                           dict(ORACLE_PARAMS, search_radius=4, optimizer="lm"))
    gpu = _run(pkg, ref, dfm, 31, 4, "quadratic", seeds, "mixed", 4, optimizer="lm")
    stats = compare(gpu, ora, W, H, 31)
    assert stats["accepted"] > 0.8 * stats["points"]


def test_lm_and_gauss_newton_reach_the_same_root(pkg):
    w, ref, dfm = _affine_pair()
    gn = _run(pkg, ref, dfm, w.subset_size, w.subset_step, w.shape, w.seeds, "fp64", w.search_radius)
    lm = _run(pkg, ref, dfm, w.subset_size, w.subset_step, w.shape, w.seeds, "fp64", w.search_radius,
              optimizer="lm")
    both = (gn["status"] == 0) & (lm["status"] == 0)
    assert both.sum() > 2000
    assert np.abs(gn["p"][both][:, :2] - lm["p"][both][:, :2]).max() < TOL_UV
    assert np.abs(gn["p"][both][:, 2:] - lm["p"][both][:, 2:]).max() < TOL_P


def test_unknown_optimizer_is_rejected(pkg):
    from paper_2601_12941_gb300 import DicError, binding as B

    img = np.zeros((64, 64), np.uint8)
    h, _ = B.dic_create(img, img, None, 21, 5, B.DIC_AFFINE)
    p = B.dic_default_params()
    p.optimizer = 2
    with pytest.raises(DicError):
        B.dic_set_params(h, p)
    B.dic_destroy(h)
