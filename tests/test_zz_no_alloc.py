"""Allocation-free correlation: dic_correlate_static against dic_correlate.

Some callers cannot allocate device memory at the moment they correlate, for
example code that runs inside a memory allocator's own callback, a real-time loop
that must not wait on the driver's allocation locks, or an application that has
handed all device memory to its own pool. dic_correlate_static serves them: it
takes device images and caller-owned device outputs, and keeps every
intermediate buffer in one fixed-size device array of the library. This file
checks, through the C-ABI, that its results equal those of the handle-based
dic_correlate within the parity tolerances, on two calls in a row (the second
call finds the first call's leftovers in the shared array), and that a problem
above the fixed limits is refused with a clear message. It is collected last.
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


def _pair(W, H):
    sp = synth.Speckle(seed=4242, density=0.0305, sigma=(1.5, 3.0), cell=16)
    fld = synth.affine_field(W, H, u0=1.8, v0=-0.9, exx=1.5e-3, exy=3e-4, eyx=3e-4, eyy=-8e-4)
    ref = synth.render(synth.ImageSpec(sp, gray_max=255.0, noise=2.0, noise_tag=1), W, H, "u8")
    dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=255.0, noise=2.0, noise_tag=2), W, H, "u8")
    return torch.from_numpy(ref).cuda(), torch.from_numpy(dfm).cuda()


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


def test_static_entry_matches_the_handle_entry_on_two_calls(pkg):
    W, H, S, step, seeds = 236, 190, 21, 5, [(118, 95)]
    ref, dfm = _pair(W, H)
    prm = pkg.params(precision="mixed", conv_threshold=1e-5, max_iter=100, search_radius=6)
    c = pkg.Correlation(ref, dfm, None, S, step, "affine", precision="mixed", conv_threshold=1e-5,
                        max_iter=100, search_radius=6)
    c.run(seeds)
    want = c.results()
    c.close()
    n, nparams = int(want["n_points"]), int(want["n_params"])
    for call in range(2):
        out = _outputs(n, nparams)
        accepted = pkg.binding.dic_correlate_static(ref, dfm, S, step, pkg.DIC_AFFINE, prm, seeds, out)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        assert accepted == int(want["n_accepted"]) > 0.8 * n, call
        assert np.array_equal(got["status"], want["status"]), call
        assert np.array_equal(got["wave"], want["wave"]), call
        ok = want["status"] == 0
        assert np.abs(got["p"][ok, :2] - want["p"][ok, :2]).max() <= TOL_UV
        assert np.abs(got["p"][ok, 2:] - want["p"][ok, 2:]).max() <= TOL_P
        assert np.array_equal(got["u"][ok], got["p"][ok, 0])
        assert np.allclose(got["zncc"][ok], want["zncc"][ok], atol=1e-6, rtol=0)
        assert np.array_equal(got["iters"][ok], want["iters"][ok])


def test_static_entry_refuses_problems_above_its_limits(pkg):
    from paper_2601_12941_gb300 import DicError

    big = torch.zeros((1200, 1200), dtype=torch.uint8, device="cuda")
    prm = pkg.params(precision="mixed")
    out = _outputs(1, 6)
    with pytest.raises(DicError) as e:
        pkg.binding.dic_correlate_static(big, big, 21, 5, pkg.DIC_AFFINE, prm, [(600, 600)], out)
    assert e.value.code == -1 and "static limit" in str(e.value)
