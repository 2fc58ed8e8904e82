"""Cost functions (Eq. 2-4) on the GPU against the oracle: NSSD and SSD next to the
default ZNSSD, in both precisions, including a pair with a gain and offset change
where the three costs converge to different roots."""
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


def _run(pkg, ref, dfm, S, step, shape, seeds, precision, cost, R):
    c = pkg.Correlation(ref, dfm, None, S, step, shape, precision=precision, cost=cost, search_radius=R,
                        **GPU_PARAMS[precision])
    c.run(seeds)
    r = c.results()
    c.close()
    return r


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cost", ["nssd", "ssd"])
def test_affine_256_costs_match_oracle(pkg, precision, cost):
    w = wl.affine_256_u8()
    ref = synth.render(w.ref, w.width, w.height, w.dtype)
    dfm = synth.render(w.deformed, w.width, w.height, w.dtype)
    ora = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds,
                           dict(ORACLE_PARAMS, search_radius=w.search_radius, cost=cost))
    gpu = _run(pkg, ref, dfm, w.subset_size, w.subset_step, w.shape, w.seeds, precision, cost, w.search_radius)
    stats = compare(gpu, ora, w.width, w.height, w.subset_size)
    assert stats["accepted"] > 2000
    if precision == "fp64":
        assert stats["max_uv"] < 1e-8


# SSD has neither invariance: under a strong gain its optimisation runs to the
# iteration cap at many points, where FP32 and FP64 may legitimately part; it gets a
# mild offset instead
@pytest.mark.parametrize("cost,gain,offset", [("znssd", 1.25, 12.0), ("nssd", 1.25, 12.0), ("ssd", 1.0, 2.0)])
def test_gain_and_offset_pair_each_cost_matches_its_own_root(pkg, cost, gain, offset):
    W, H = 200, 170
    fld = synth.affine_field(W, H, u0=1.6, v0=-0.9, exx=2e-3, eyy=-1e-3)
    sp = synth.Speckle(seed=404, density=0.0305, sigma=(1.5, 3.0), cell=16)
    ref = synth.render(synth.ImageSpec(sp, gray_max=200.0, noise=2.0, noise_tag=1), W, H, "f32")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=200.0, noise=2.0, noise_tag=2), W, H, "f32")
    dfm = (gain * dfm + offset).astype(np.float32)          # gain and offset on the deformed image
    seeds = [(W // 2, H // 2)]
    ora = oracle.correlate(ref, dfm, None, 21, 6, "affine", seeds, dict(ORACLE_PARAMS, search_radius=6, cost=cost))
    gpu = _run(pkg, ref, dfm, 21, 6, "affine", seeds, "mixed", cost, 6)
    stats = compare(gpu, ora, W, H, 21)
    assert stats["accepted"] > 0.8 * stats["points"]


def test_quadratic_sine_nssd_mixed(pkg):
    W, H = 230, 190
    fld = synth.sine_field(W, 0.5, 10.0, 300.0)
    sp = synth.Speckle(seed=77, density=0.0305, sigma=(1.5, 3.0), cell=16)
    G = 4095.0
    ref = synth.render(synth.ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=1), W, H, "u16")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=2), W, H, "u16")
    seeds = [(115, 95)]
    ora = oracle.correlate(ref, dfm, None, 31, 4, "quadratic", seeds, dict(ORACLE_PARAMS, search_radius=4, cost="nssd"))
    gpu = _run(pkg, ref, dfm, 31, 4, "quadratic", seeds, "mixed", "nssd", 4)
    stats = compare(gpu, ora, W, H, 31)
    assert stats["accepted"] > 0.8 * stats["points"]


def test_unknown_cost_is_rejected(pkg):
    from paper_2601_12941_gb300 import DicError, binding as B

    img = np.zeros((64, 64), np.uint8)
    h, _ = B.dic_create(img, img, None, 21, 5, B.DIC_AFFINE)
    p = B.dic_default_params()
    p.cost = 3
    with pytest.raises(DicError):
        B.dic_set_params(h, p)
    B.dic_destroy(h)
