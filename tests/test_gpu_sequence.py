"""Sequence mode: several deformed frames against one resident reference, each frame
started from the previous frame's accepted warps (oracle reading R11). The oracle
chains its own results and the library chains its own; every frame must match
point by point."""
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


def _frames(W, H, n, e_step=4e-3, nu=0.3):
    sp = synth.Speckle(seed=555, density=0.0305, sigma=(1.5, 3.0), cell=16)
    G = 65535.0
    ref = synth.render(synth.ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=100), W, H, "u16")
    out = []
    for k in range(1, n + 1):
        e = e_step * k
        fld = synth.affine_field(W, H, exx=e, eyy=-nu * e)
        out.append(synth.render(synth.ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=100 + k),
                                W, H, "u16"))
    return ref, out


def _dev(a):
    return torch.from_numpy(a.view(np.int16)).cuda()


@pytest.mark.parametrize("S,shape", [(21, "affine"), (31, "quadratic")])
def test_sequence_frames_match_oracle(pkg, S, shape):
    W, H, step = 260, 220, 8
    ref, frames = _frames(W, H, 3)
    seeds = [(130, 110)]
    prm = dict(ORACLE_PARAMS, search_radius=8)
    c = pkg.Correlation(_dev(ref), _dev(frames[0]), None, S, step, shape, precision="mixed",
                        search_radius=8, **GPU_PARAMS["mixed"])
    prev = None
    for k, img in enumerate(frames):
        if k == 0:
            c.run(seeds)
            ora = oracle.correlate(ref, img, None, S, step, shape, seeds, prm)
        else:
            c.set_deformed(_dev(img))
            c.run_next()
            ora = oracle.correlate_sequence(ref, img, None, S, step, shape, prev, prm)
        gpu = c.results()
        stats = compare(gpu, ora, W, H, S)
        assert stats["accepted"] > 0.8 * stats["points"], (k, stats)
        if k > 0:
            # every point accepted before starts in wave 0
            assert ((gpu["wave"] == 0) == (prev_gpu_status == 0)).all()
        prev = ora
        prev_gpu_status = gpu["status"].copy()
    c.close()


def test_sequence_needs_an_earlier_correlation(pkg):
    from paper_2601_12941_gb300 import DicError

    ref, frames = _frames(64, 64, 1)
    c = pkg.Correlation(_dev(ref), _dev(frames[0]), None, 15, 5, "affine")
    with pytest.raises(DicError) as e:
        c.run_next()
    assert e.value.code == -6
    c.close()
