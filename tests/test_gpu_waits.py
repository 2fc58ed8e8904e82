"""The bounded-wait path of the wave kernel, without a fault or a hang.

Every tile load of the wave kernel completes on an mbarrier whose wait is bounded;
a wait that runs out sets an error flag, lets the copy in flight land (a second
bounded wait), ends its block, and the call returns DIC_ETIMEOUT. The test hook
dic_test_expire_tile_waits makes the first wait give up at once (a wait that can
never succeed), so the whole error path runs while every copy still completes. The
handle must then give correct results again once normal waits are restored."""
import numpy as np
import pytest

import synth

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


def test_expired_tile_waits_return_timeout_and_the_handle_recovers(pkg):
    from paper_2601_12941_gb300 import DicError
    from paper_2601_12941_gb300 import binding as B

    W, H = 256, 224
    sp = synth.Speckle(seed=515, density=0.0305, sigma=(1.5, 3.0), cell=16)
    fld = synth.affine_field(W, H, u0=1.2, v0=-0.7, exx=1e-3)
    ref = torch.from_numpy(synth.render(synth.ImageSpec(sp, gray_max=255.0, noise_tag=1), W, H, "u8")).cuda()
    dfm = torch.from_numpy(synth.render(synth.ImageSpec(sp, field=fld, gray_max=255.0, noise_tag=2), W, H,
                                        "u8")).cuda()
    seeds = [(128, 112)]
    with pkg.Correlation(ref, dfm, None, 21, 6, "affine", precision="mixed", search_radius=3) as fresh:
        fresh.run(seeds)
        want = fresh.results()
    c = pkg.Correlation(ref, dfm, None, 21, 6, "affine", precision="mixed", search_radius=3)
    try:
        B.dic_test_expire_tile_waits(True)
        with pytest.raises(DicError) as e:
            c.run(seeds)
        assert e.value.code == B.DIC_ETIMEOUT and "in time" in str(e.value)
        # the seed's block gave up before correlating it: nothing was accepted
        assert (c.results()["status"] == 0).sum() == 0
    finally:
        B.dic_test_expire_tile_waits(False)
    torch.cuda.synchronize()
    c.run(seeds)
    got = c.results()
    c.close()
    assert int(want["n_accepted"]) > 0.9 * int(want["n_points"])
    for k in ("p", "zncc", "status", "wave", "iters"):
        assert np.array_equal(np.asarray(got[k]), np.asarray(want[k]), equal_nan=k == "zncc"), k
