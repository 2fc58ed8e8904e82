"""Allocation-free correlation: dic_correlate_static against dic_correlate.

Some callers cannot allocate device memory at the moment they correlate, for
example code that runs inside a memory allocator's own callback, a real-time loop
that must not wait on the driver's allocation locks, or an application that has
handed all device memory to its own pool. dic_correlate_static serves them: it
takes device images and caller-owned device outputs, and keeps every
intermediate buffer in one fixed-size device array of the library. This file
checks, through the C-ABI, that its results equal those of the handle-based
dic_correlate within the parity tolerances, on two calls in a row (the second
call finds the first call's leftovers in the shared array), for every shape
function, for u8, u16 and BF16 gray levels, several seeds (some snapped at the
image edges), a non-default stream, tiny grids and a one-row strip; and that a
problem above the fixed limits, or an output too short for the grid, is refused
with a clear message. It is collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_UV = 1e-3
TOL_P = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_2601_12941_gb300 as P
    from paper_2601_12941_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    P.load()
    return P


def _pair(W, H, dtype="u8", u0=1.8, v0=-0.9):
    gray = 255.0 if dtype in ("u8", "bf16") else 4095.0
    sp = synth.Speckle(seed=4242, density=0.0305, sigma=(1.5, 3.0), cell=16)
    fld = synth.affine_field(W, H, u0=u0, v0=v0, exx=1.5e-3, exy=3e-4, eyx=3e-4, eyy=-8e-4)
    kind = "u16" if dtype == "u16" else "u8"
    ref = synth.render(synth.ImageSpec(sp, gray_max=gray, noise=0.008 * gray, noise_tag=1), W, H, kind)
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=gray, noise=0.008 * gray, noise_tag=2), W, H, kind)

    def dev(a):
        t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
        return t.to(torch.bfloat16) if dtype == "bf16" else t

    return dev(ref), dev(dfm)


def _outputs(n, nparams):
    # filled with junk so that a value the call forgot to write shows up
    f64 = dict(dtype=torch.float64, device="cuda")
    return dict(u=torch.full((n,), 7.0, **f64), v=torch.full((n,), 7.0, **f64),
                p=torch.full((n, nparams), 7.0, **f64),
                zncc=torch.full((n,), 7.0, dtype=torch.float32, device="cuda"),
                iters=torch.full((n,), 77, dtype=torch.int32, device="cuda"),
                converged=torch.full((n,), 7, dtype=torch.uint8, device="cuda"),
                status=torch.full((n,), 77, dtype=torch.uint8, device="cuda"),
                wave=torch.full((n,), 77, dtype=torch.int32, device="cuda"))


def _handle_results(pkg, ref, dfm, S, step, shape, seeds, **kw):
    c = pkg.Correlation(ref, dfm, None, S, step, shape, precision="mixed", **kw)
    try:
        c.run(seeds)
    except pkg.DicError:
        pass
    want = c.results()
    c.close()
    return want


def _check_equal(got, want, call):
    ok = want["status"] == 0
    assert np.array_equal(got["status"], want["status"]), call
    assert np.array_equal(got["wave"], want["wave"]), call
    assert np.abs(got["p"][ok, :2] - want["p"][ok, :2]).max() <= TOL_UV, call
    if got["p"].shape[1] > 2:
        assert np.abs(got["p"][ok, 2:] - want["p"][ok, 2:]).max() <= TOL_P, call
    assert np.array_equal(got["u"][ok], got["p"][ok, 0]), call
    assert np.array_equal(got["v"][ok], got["p"][ok, 1]), call
    assert np.allclose(got["zncc"][ok], want["zncc"][ok], atol=1e-6, rtol=0), call
    assert np.array_equal(got["iters"][ok], want["iters"][ok]), call
    assert np.array_equal(got["converged"], want["converged"]), call


def _static(pkg, ref, dfm, S, step, shape, prm, seeds, n, stream=None):
    nparams = pkg.N_PARAMS[pkg.SHAPES[shape]]
    out = _outputs(n, nparams)
    sp = stream.cuda_stream if stream is not None else 0
    accepted = pkg.binding.dic_correlate_static(ref, dfm, S, step, pkg.SHAPES[shape], prm, seeds, out, sp)
    (stream or torch.cuda.current_stream()).synchronize()
    return accepted, {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("shape,dtype", [("affine", "u8"), ("rigid", "u16"), ("quadratic", "u8"),
                                         ("affine", "bf16")])
def test_static_entry_matches_the_handle_entry_on_two_calls(pkg, shape, dtype):
    W, H, S, step, seeds = 236, 190, 21, 5, [(118, 95)]
    ref, dfm = _pair(W, H, dtype)
    kw = dict(conv_threshold=1e-5, max_iter=100, search_radius=6)
    prm = pkg.params(precision="mixed", **kw)
    want = _handle_results(pkg, ref, dfm, S, step, shape, seeds, **kw)
    n = int(want["n_points"])
    for call in range(2):
        accepted, got = _static(pkg, ref, dfm, S, step, shape, prm, seeds, n)
        assert accepted == int(want["n_accepted"]) > 0.8 * n, call
        _check_equal(got, want, call)


def test_static_entry_with_several_seeds_at_the_edges_and_on_a_side_stream(pkg):
    """Seeds outside the grid snap to its corners (ties to the lower index) like the
    handle path's; the call runs on a non-default stream."""
    W, H, S, step = 236, 190, 21, 5
    ref, dfm = _pair(W, H, "u8")
    seeds = [(0, 0), (W - 1, H - 1), (118, 95), (W - 1, 3)]
    kw = dict(conv_threshold=1e-5, max_iter=100, search_radius=6)
    prm = pkg.params(precision="mixed", **kw)
    want = _handle_results(pkg, ref, dfm, S, step, "affine", seeds, **kw)
    assert (want["wave"] == 0).sum() == 4
    side = torch.cuda.Stream()
    for call in range(2):
        accepted, got = _static(pkg, ref, dfm, S, step, "affine", prm, seeds, int(want["n_points"]), side)
        assert accepted == int(want["n_accepted"]), call
        _check_equal(got, want, call)


@pytest.mark.parametrize("W,H,step,seed", [(40, 40, 10, (20, 20)), (260, 26, 6, (12, 12))])
def test_static_entry_on_tiny_grids_and_strips(pkg, W, H, step, seed):
    """A 2 x 2 grid and a one-row strip of 40 points (40 waves): the wave loop ends on
    the empty front, as in the handle path."""
    ref, dfm = _pair(W, H, "u8", u0=1.5, v0=1.5)
    kw = dict(conv_threshold=1e-5, max_iter=100, search_radius=2)
    prm = pkg.params(precision="mixed", **kw)
    want = _handle_results(pkg, ref, dfm, 21, step, "affine", [seed], **kw)
    n = int(want["n_points"])
    assert int(want["n_accepted"]) >= 0.9 * n
    for call in range(2):
        accepted, got = _static(pkg, ref, dfm, 21, step, "affine", prm, [seed], n)
        assert accepted == int(want["n_accepted"]), call
        _check_equal(got, want, call)


def test_static_entry_refuses_short_or_mistyped_outputs(pkg):
    from paper_2601_12941_gb300 import DicError

    W, H, S, step = 236, 190, 21, 5
    ref, dfm = _pair(W, H, "u8")
    prm = pkg.params(precision="mixed", search_radius=6)
    nx, ny = pkg.binding.grid_size(W, H, S, step)
    out = _outputs(nx * ny - 1, 6)
    with pytest.raises(DicError) as e:
        pkg.binding.dic_correlate_static(ref, dfm, S, step, pkg.DIC_AFFINE, prm, [(118, 95)], out)
    assert e.value.code == -1 and "elements" in str(e.value)
    out = _outputs(nx * ny, 6)
    out["zncc"] = out["zncc"].double()
    with pytest.raises(DicError) as e:
        pkg.binding.dic_correlate_static(ref, dfm, S, step, pkg.DIC_AFFINE, prm, [(118, 95)], out)
    assert "dtype" in str(e.value)


def test_static_entry_refuses_problems_above_its_limits(pkg):
    from paper_2601_12941_gb300 import DicError

    big = torch.zeros((1200, 1200), dtype=torch.uint8, device="cuda")
    prm = pkg.params(precision="mixed")
    nx, ny = pkg.binding.grid_size(1200, 1200, 21, 5)
    out = _outputs(nx * ny, 6)
    with pytest.raises(DicError) as e:
        pkg.binding.dic_correlate_static(big, big, 21, 5, pkg.DIC_AFFINE, prm, [(600, 600)], out)
    assert e.value.code == -1 and "static limit" in str(e.value)
