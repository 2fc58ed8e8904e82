"""Strain post-processing (Sec. 2.3) on the GPU against the strain oracle: the same
displacement fields in, the valid masks bit for bit and the displacement gradient
and strain components within 1e-6 (FP32 arithmetic on centred displacements; the
components are at most a few 1e-2 here)."""
import numpy as np
import pytest

from oracle import strain_oracle as SO

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-6
KEYS = ("dudx", "dudy", "dvdx", "dvdy", "exx", "eyy", "exy")


@pytest.fixture(scope="module")
def pkg():
    import paper_2601_12941_gb300 as P
    from paper_2601_12941_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    P.load()
    return P


def _field(nx, ny, step, scale, seed, hole_frac):
    """Smooth displacement field with noise on the grid, and a status array with
    random rejected points and a rectangular hole."""
    rng = np.random.default_rng(seed)
    j, i = np.mgrid[0:ny, 0:nx]
    X, Y = i * step + 17.0, j * step + 11.0
    u = 2.5 + scale * (0.6 * X - 0.2 * Y) / 100 + scale * 3e-4 * (X * X - 0.5 * X * Y) / 100
    v = -1.25 + scale * (0.15 * X + 0.4 * Y) / 100 + scale * 2e-4 * Y * Y / 100
    u = u + 0.01 * rng.standard_normal(u.shape)
    v = v + 0.01 * rng.standard_normal(v.shape)
    st = np.zeros((ny, nx), np.uint8)
    st[rng.random((ny, nx)) < hole_frac] = 5
    st[ny // 3:ny // 3 + 4, nx // 2:nx // 2 + 6] = 1
    return u.ravel(), v.ravel(), st.ravel()


def _gpu(pkg, u, v, st, nx, ny, step, window, basis, measure):
    from paper_2601_12941_gb300 import binding as B

    out = B.strain_outputs(nx * ny)
    B.dic_strain_field(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), torch.from_numpy(st).cuda(), nx, ny,
                       step, window, basis, measure, out)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in out.items()}


def _compare(g, o):
    vg, vo = g["valid"].astype(bool), o["valid"]
    assert np.array_equal(vg, vo), "valid masks differ at %d points" % (vg != vo).sum()
    for k in KEYS:
        assert np.isnan(g[k][~vg]).all(), k
        err = np.abs(g[k][vg].astype(np.float64) - o[k][vg])
        assert err.max() <= TOL, "%s: max error %.3g" % (k, err.max())
    return vg.sum()


@pytest.mark.parametrize("basis", [SO.BILINEAR, SO.BIQUADRATIC])
@pytest.mark.parametrize("window", [3, 5, 9, 15])
def test_strain_matches_oracle_all_measures(pkg, basis, window):
    nx, ny, step = 47, 38, 5
    u, v, st = _field(nx, ny, step, 1.0, seed=window, hole_frac=0.04)
    for measure in SO.MEASURES:
        o = SO.strain_field(u, v, st, nx, ny, step, window, basis, measure)
        g = _gpu(pkg, u, v, st, nx, ny, step, window, basis, measure)
        n = _compare(g, o)
        assert n > 0.6 * nx * ny


@pytest.mark.parametrize("measure", SO.MEASURES)
def test_large_strain_measures_differ_and_match(pkg, measure):
    # strains of a few 1e-2: the five measures differ by more than the tolerance
    nx, ny, step = 30, 24, 7
    u, v, st = _field(nx, ny, step, 8.0, seed=11, hole_frac=0.0)
    o = SO.strain_field(u, v, st, nx, ny, step, 7, SO.BIQUADRATIC, measure)
    g = _gpu(pkg, u, v, st, nx, ny, step, 7, SO.BIQUADRATIC, measure)
    _compare(g, o)
    gl = SO.strain_field(u, v, st, nx, ny, step, 7, SO.BIQUADRATIC, SO.GREEN_LAGRANGE)
    if measure != SO.GREEN_LAGRANGE:
        ok = o["valid"]
        assert np.nanmax(np.abs(o["exx"][ok] - gl["exx"][ok])) > 1e-4


def test_degenerate_windows_and_edges(pkg):
    nx, ny, step = 20, 16, 4
    u, v, _ = _field(nx, ny, step, 1.0, seed=3, hole_frac=0.0)
    st = np.full(nx * ny, 5, np.uint8)
    st[8 * nx:9 * nx] = 0                       # one accepted row: no bilinear fit anywhere
    g = _gpu(pkg, u, v, st, nx, ny, step, 5, SO.BILINEAR, SO.GREEN_LAGRANGE)
    assert not g["valid"].any()
    st2 = np.zeros(nx * ny, np.uint8)           # everything accepted: edges clip their windows
    o = SO.strain_field(u, v, st2, nx, ny, step, 9, SO.BIQUADRATIC, SO.HENCKY)
    g2 = _gpu(pkg, u, v, st2, nx, ny, step, 9, SO.BIQUADRATIC, SO.HENCKY)
    assert _compare(g2, o) == nx * ny


def test_strain_of_a_correlation(pkg):
    import synth
    from synth import workloads as WL

    w = WL.affine_256_u8()
    ref = synth.render(w.ref, w.width, w.height, w.dtype)
    dfm = synth.render(w.deformed, w.width, w.height, w.dtype)
    c = pkg.Correlation(ref, dfm, None, w.subset_size, w.subset_step, w.shape, search_radius=w.search_radius)
    c.run(w.seeds)
    r = c.results()
    g = {k: t.cpu().numpy() for k, t in c.strain(9, "biquadratic", "green_lagrange").items()}
    c.close()
    o = SO.strain_field(r["u"], r["v"], r["status"], r["nx"], r["ny"], w.subset_step, 9, SO.BIQUADRATIC,
                        SO.GREEN_LAGRANGE)
    _compare(g, o)
    # the imposed field: exx = 1e-3, eyy = -5e-4, symmetric shear 2e-4 (small-strain
    # limit of Green-Lagrange)
    ok = g["valid"].astype(bool)
    assert abs(np.median(g["exx"][ok]) - 1e-3) < 2e-4
    assert abs(np.median(g["eyy"][ok]) + 5e-4) < 2e-4
