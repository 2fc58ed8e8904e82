"""The 128-thread kernels (subsets above 31) of every variant against the oracle: the
other costs, Levenberg-Marquardt, Keys bicubic, FP64 solves on the mixed path and the
quadratic shape in both precisions, at subset 41. The 64-thread kernels (subsets up to
31) carry the same variants in the cost, optimiser and interpolant tests; these kernels
differ in their block size, register budget and shared-memory layout (the gray tile
shares the gradient region)."""
import numpy as np
import pytest

import oracle
import synth

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


@pytest.fixture(scope="module")
def pair():
    W, H = 200, 180
    fld = synth.affine_field(W, H, u0=1.9, v0=-1.2, exx=2e-3, eyy=-1.5e-3, exy=6e-4)
    sp = synth.Speckle(seed=141, density=0.0305, sigma=(1.5, 3.0), cell=16)
    ref = synth.render(synth.ImageSpec(sp, field=synth.IDENTITY, gray_max=255.0, noise=0.0, noise_tag=1), W, H, "u8")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=255.0, noise=0.0, noise_tag=2), W, H, "u8")
    return W, H, ref, dfm


@pytest.mark.parametrize("shape,cost,optimizer,interp,precision", [
    ("affine", "nssd", "gn", "bspline3", "mixed"),
    ("affine", "ssd", "lm", "bspline3", "mixed"),
    ("affine", "znssd", "lm", "bspline3", "mixed"),
    ("affine", "znssd", "gn", "bicubic", "mixed"),
    ("affine", "znssd", "gn", "bspline3", "mixed_fp64_solve"),
    ("quadratic", "znssd", "gn", "bspline3", "mixed"),
    ("quadratic", "znssd", "gn", "bspline3", "fp64"),
])
def test_subset_41_variants_match_oracle(pkg, pair, shape, cost, optimizer, interp, precision):
    W, H, ref, dfm = pair
    S, step, R = 41, 8, 4
    seeds = [(W // 2, H // 2)]
    prm = dict(ORACLE_PARAMS, search_radius=R, cost=cost, optimizer=optimizer, interp=interp)
    ora = oracle.correlate(ref, dfm, None, S, step, shape, seeds, prm)
    c = pkg.Correlation(ref, dfm, None, S, step, shape, interp=interp, precision=precision, search_radius=R,
                        **dict(GPU_PARAMS[precision], cost=cost, optimizer=optimizer))
    c.run(seeds)
    gpu = c.results()
    c.close()
    stats = compare(gpu, ora, W, H, S, precision=precision)
    assert stats["accepted"] > 0.9 * len(ora["status"])
