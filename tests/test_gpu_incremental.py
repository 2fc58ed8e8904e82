"""Incremental reference updating (readings I1-I4) on the GPU against the oracle:
each frame's correlation against the current reference element by element, and
the total warps from the first frame (composed on the device) within the parity
tolerances; no update leaves the totals equal to the frame's own warps."""
import numpy as np
import pytest

import synth
from oracle import dic_oracle as O
from oracle import incremental_oracle as I

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


def _frames(W, H, strains, u0=1.3, v0=-0.7, seed=17, dtype="u16"):
    sp = synth.Speckle(seed=seed, density=0.03, sigma=(1.5, 3.0), cell=16)
    out = []
    for k, e in enumerate(strains):
        fld = synth.affine_field(W, H, u0=u0 * k, v0=v0 * k, exx=e, eyy=-0.4 * e, exy=0.3 * e)
        out.append(synth.render(synth.ImageSpec(sp, field=fld, gray_max=4000.0, noise=8.0, noise_tag=k + 1), W, H,
                                dtype))
    return out


def _gpu_sequence(pkg, frames, S, step, shape, seeds, precision, update_after):
    c = pkg.Correlation(frames[0], frames[1], None, S, step, shape, precision=precision, **GPU_PARAMS[precision])
    out = []
    for k in range(1, len(frames)):
        if k == 1:
            c.run(seeds)
        else:
            c.set_deformed(frames[k])
            c.run_next()
        out.append((c.results(), c.totals()))
        if k in update_after:
            c.update_reference()
    c.close()
    return out


def _compare_totals(tg, to, tol_uv, tol_p):
    sg, so = np.asarray(tg["status"]).astype(int), np.asarray(to["status"]).astype(int)
    assert (sg != so).sum() <= max(2, len(so) // 100), "total status differs at %d points" % (sg != so).sum()
    both = (sg == O.OK) & (so == O.OK)
    assert both.sum() > 0.5 * len(so)
    assert np.abs(tg["p"][both][:, :2] - to["p"][both][:, :2]).max() < tol_uv
    if tg["p"].shape[1] > 2:
        assert np.abs(tg["p"][both][:, 2:] - to["p"][both][:, 2:]).max() < tol_p
    return both.sum()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_updated_sequence_matches_oracle(pkg, precision):
    W = H = 200
    frames = _frames(W, H, [0.0, 0.04, 0.08, 0.12])
    seeds = [(100, 100)]
    ora = I.correlate_incremental(frames, None, 21, 10, O.AFFINE, seeds, ORACLE_PARAMS, update_after=(1, 2))
    gpu = _gpu_sequence(pkg, frames, 21, 10, "affine", seeds, precision, update_after=(1, 2))
    tol_uv = 1e-8 if precision == "fp64" else TOL_UV
    tol_p = 1e-9 if precision == "fp64" else TOL_P
    for (rg, tg), (ro, to) in zip(gpu, ora):
        compare(rg, ro, W, H, 21)
        _compare_totals(tg, to, tol_uv, tol_p)
    # the last totals are the composed 12 % stretch
    tg = gpu[-1][1]
    ok = tg["status"] == O.OK
    assert abs(np.median(tg["p"][ok][:, 2]) - 0.12) < 2e-3


def test_no_update_totals_are_the_frames_own_warps(pkg):
    W = H = 200
    frames = _frames(W, H, [0.0, 0.02, 0.04])
    gpu = _gpu_sequence(pkg, frames, 21, 10, "affine", [(100, 100)], "mixed", update_after=())
    for res, tot in gpu:
        ok = res["status"] == O.OK
        assert np.array_equal(tot["status"] == O.OK, ok)
        assert np.array_equal(tot["p"][ok], res["p"][ok])
        assert tot["n_updates"] == 0


def test_rigid_updates_match_oracle(pkg):
    W = H = 180
    frames = _frames(W, H, [0.0, 0.0, 0.0], u0=2.6, v0=-1.9)
    seeds = [(90, 90)]
    ora = I.correlate_incremental(frames, None, 21, 10, O.RIGID, seeds, ORACLE_PARAMS, update_after=(1,))
    gpu = _gpu_sequence(pkg, frames, 21, 10, "rigid", seeds, "mixed", update_after=(1,))
    for (rg, tg), (ro, to) in zip(gpu, ora):
        compare(rg, ro, W, H, 21)
        _compare_totals(tg, to, TOL_UV, TOL_P)
    assert gpu[-1][1]["n_updates"] == 1


def test_quadratic_update_is_rejected(pkg):
    from paper_2601_12941_gb300 import DicError

    frames = _frames(160, 160, [0.0, 0.01])
    c = pkg.Correlation(frames[0], frames[1], None, 21, 10, "quadratic")
    c.run([(80, 80)])
    with pytest.raises(DicError):
        c.update_reference()
    c.close()
