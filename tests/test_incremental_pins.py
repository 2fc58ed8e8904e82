"""Pins of the incremental reference-updating oracle (readings I1-I4) to things
other than itself: the composed warp maps points exactly as the two warps applied
in turn, no update reproduces the plain sequence bit for bit, and a large
stretch applied in steps is recovered against the analytic field and against
direct correlation with the first frame. CPU only."""
import numpy as np
import pytest

import synth
from oracle import dic_oracle as O
from oracle import incremental_oracle as I

RNG = np.random.default_rng(2012)


def test_composition_maps_points_like_the_two_warps_in_turn():
    for _ in range(20):
        ua = RNG.uniform(-5, 5, 2)
        Aa = RNG.uniform(-0.1, 0.1, (2, 2))
        p_q = RNG.uniform(-0.1, 0.1, 6)
        p_q[:2] = RNG.uniform(-3, 3, 2)
        X = RNG.uniform(50, 150, 2)
        xq = np.round(X + ua) + RNG.integers(-1, 2, 2)              # a grid point near x_r
        (u, v), A = I.compose(ua, Aa, p_q, X + ua - xq)
        Aq = I.gradient_matrix(p_q)
        for dx in RNG.uniform(-10, 10, (5, 2)):
            y = X + ua + (np.eye(2) + Aa) @ dx                      # frame 0 -> reference r
            z = xq + p_q[:2] + (np.eye(2) + Aq) @ (y - xq)           # reference r -> frame k
            total = X + np.array([u, v]) + (np.eye(2) + A) @ dx
            assert np.abs(z - total).max() < 1e-11


def _frames(W, H, strains, u0=1.3, v0=-0.7, seed=17):
    sp = synth.Speckle(seed=seed, density=0.03, sigma=(1.5, 3.0), cell=16)
    out = []
    for k, e in enumerate(strains):
        fld = synth.affine_field(W, H, u0=u0 * k, v0=v0 * k, exx=e, eyy=-0.4 * e)
        out.append(synth.render(synth.ImageSpec(sp, field=fld, gray_max=250.0), W, H, "f64"))
    return out


PRM = dict(conv_threshold=1e-8, max_iter=100)


def test_no_update_reproduces_the_plain_sequence():
    W = H = 160
    frames = _frames(W, H, [0.0, 0.01, 0.02, 0.03])
    seeds = [(80, 80)]
    inc = I.correlate_incremental(frames, None, 21, 10, O.AFFINE, seeds, PRM, update_after=())
    prev = None
    for k in range(1, len(frames)):
        if prev is None:
            res = O.correlate(frames[0], frames[k], None, 21, 10, O.AFFINE, seeds, PRM)
        else:
            res = O.correlate_sequence(frames[0], frames[k], None, 21, 10, O.AFFINE, prev, PRM)
        prev = res
        r, tot = inc[k - 1]
        ok = res["status"] == O.OK
        assert np.array_equal(tot["status"] == O.OK, ok)
        assert np.array_equal(tot["p"][ok], res["p"][ok])


def test_stepwise_stretch_is_recovered_with_updates():
    W = H = 200
    strains = [0.0, 0.04, 0.08, 0.12, 0.16]
    frames = _frames(W, H, strains)
    seeds = [(100, 100)]
    inc = I.correlate_incremental(frames, None, 21, 10, O.AFFINE, seeds, PRM, update_after=(1, 2, 3))
    res, tot = inc[-1]
    ok = tot["status"] == O.OK
    assert ok.sum() > 0.5 * len(ok)
    xs, ys = O.grid(W, H, 21, 10)
    X = np.tile(xs, len(ys)).astype(float)
    Y = np.repeat(ys, len(xs)).astype(float)
    fld = synth.affine_field(W, H, u0=1.3 * 4, v0=-0.7 * 4, exx=0.16, eyy=-0.064)
    u, v = synth.displacement(fld, X[ok], Y[ok])
    assert np.abs(tot["u"][ok] - u).max() < 2e-2 and np.abs(tot["v"][ok] - v).max() < 2e-2
    # the composed gradient is the product of the steps: exx 0.16, eyy -0.064 overall
    assert np.abs(tot["p"][ok][:, 2] - 0.16).max() < 2e-3 and np.abs(tot["p"][ok][:, 5] + 0.064).max() < 2e-3
    assert np.abs(tot["p"][ok][:, 3]).max() < 2e-3 and np.abs(tot["p"][ok][:, 4]).max() < 2e-3
    # and the last reference is frame 3: its own correlation is the small last step
    assert np.abs(np.median(res["p"][res["status"] == O.OK][:, 2]) - (1.16 / 1.12 - 1)) < 2e-3


def test_updated_and_direct_totals_agree():
    W = H = 200
    frames = _frames(W, H, [0.0, 0.02, 0.04, 0.06])
    seeds = [(100, 100)]
    a = I.correlate_incremental(frames, None, 21, 10, O.AFFINE, seeds, PRM, update_after=(1, 2))
    b = I.correlate_incremental(frames, None, 21, 10, O.AFFINE, seeds, PRM, update_after=())
    ta, tb = a[-1][1], b[-1][1]
    ok = (ta["status"] == O.OK) & (tb["status"] == O.OK)
    assert ok.sum() > 0.6 * len(ok)
    assert np.abs(ta["p"][ok][:, :2] - tb["p"][ok][:, :2]).max() < 1e-2
    assert np.abs(ta["p"][ok][:, 2:] - tb["p"][ok][:, 2:]).max() < 1e-3


def test_rigid_updates_and_quadratic_is_rejected():
    W = H = 160
    frames = _frames(W, H, [0.0, 0.0, 0.0], u0=2.6, v0=-1.9)
    inc = I.correlate_incremental(frames, None, 21, 10, O.RIGID, [(80, 80)], PRM, update_after=(1,))
    tot = inc[-1][1]
    ok = tot["status"] == O.OK
    assert ok.sum() > 0.6 * len(ok)
    assert np.abs(tot["u"][ok] - 5.2).max() < 2e-2 and np.abs(tot["v"][ok] + 3.8).max() < 2e-2
    with pytest.raises(ValueError):
        I.correlate_incremental(frames, None, 21, 10, O.QUADRATIC, [(80, 80)], PRM, update_after=(1,))


def test_nearest_index_ties_go_low_and_out_of_range_is_none():
    assert I.nearest_index(2.5, 10) == 2 and I.nearest_index(2.51, 10) == 3 and I.nearest_index(-0.49, 10) == 0
    assert I.nearest_index(-0.5, 10) is None                 # the tie goes to -1, outside the grid
    assert I.nearest_index(9.5, 10) == 9 and I.nearest_index(9.51, 10) is None


def test_roi_points_stay_out_and_totals_follow_the_field():
    W = H = 200
    frames = _frames(W, H, [0.0, 0.03, 0.06])
    roi = np.zeros((H, W), np.uint8)
    roi[15:185, 20:170] = 1
    seeds = [(100, 100)]
    inc = I.correlate_incremental(frames, roi, 21, 10, O.AFFINE, seeds, PRM, update_after=(1,))
    inroi = O.roi_points(roi, W, H, 21, 10).ravel()
    for res, tot in inc:
        assert (tot["status"][~inroi] == O.NOT_IN_ROI).all() and (res["status"][~inroi] == O.NOT_IN_ROI).all()
        assert not tot["p"][~inroi].any()
    tot = inc[-1][1]
    ok = tot["status"] == O.OK
    assert ok.sum() > 0.6 * inroi.sum()
    # the composed gradient of two 3 % steps is the 6 % field
    assert np.abs(tot["p"][ok][:, 2] - 0.06).max() < 2e-3 and np.abs(tot["p"][ok][:, 5] + 0.024).max() < 2e-3
