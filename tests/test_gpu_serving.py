"""Serving on the GPU: the device-memory estimates match the library's allocations,
a re-gridded handle (resident reference) gives the same results as a fresh one,
every job's result is the same alone and in a concurrent mix, admission keeps the
device footprint within the budget, and a served job still matches the oracle."""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads as WL

from parity_util import GPU_PARAMS, ORACLE_PARAMS, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("u", "v", "p", "zncc", "iters", "status", "wave")


@pytest.fixture(scope="module")
def pkg():
    import paper_2601_12941_gb300 as P
    from paper_2601_12941_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    P.load()
    return P


def _pool():
    """Three references (two sizes, u8 and u16) and their speckle patterns."""
    out = []
    for i, (W, H, dt) in enumerate([(256, 256, "u8"), (384, 320, "u16"), (300, 300, "u8")]):
        G = 255.0 if dt == "u8" else 65535.0
        sp = synth.Speckle(seed=900 + i, density=0.0305, sigma=(1.5, 3.0), cell=16)
        ref = synth.render(synth.ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=1), W, H, dt)
        out.append((W, H, dt, G, sp, ref))
    return out


def _jobs(pool):
    """Eight jobs over the pool: own deformation, subset size, step and shape each."""
    rng = np.random.default_rng(77)
    specs = [(0, 21, 5, "affine"), (1, 31, 6, "quadratic"), (0, 15, 4, "quadratic"), (2, 25, 7, "affine"),
             (1, 41, 8, "affine"), (0, 33, 6, "affine"), (2, 17, 3, "quadratic"), (1, 19, 5, "affine")]
    jobs = []
    for j, (i, S, step, shape) in enumerate(specs):
        W, H, dt, G, sp, ref = pool[i]
        u0, v0 = rng.uniform(-3.0, 3.0, size=2)
        e = rng.uniform(-5e-3, 5e-3, size=4)
        fld = synth.affine_field(W, H, u0=u0, v0=v0, exx=e[0], exy=e[1], eyx=e[2], eyy=e[3])
        dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=50 + j), W, H, dt)
        jobs.append(dict(pool=i, ref=ref, deformed=dfm, S=S, step=step, shape=shape, seeds=[(W // 2, H // 2)]))
    return jobs


def _alone(pkg, job, prm):
    c = pkg.Correlation(job["ref"], job["deformed"], None, job["S"], job["step"], job["shape"], **prm)
    c.run(job["seeds"])
    r = c.results()
    c.close()
    return r


def _same(a, b, names):
    for k in names:
        x, y = np.asarray(a[k]), np.asarray(b[k])
        assert x.shape == y.shape, k
        if x.dtype.kind == "f":
            assert np.array_equal(x, y, equal_nan=True), k
        else:
            assert np.array_equal(x, y), k


def test_device_bytes_match_estimates(pkg):
    from paper_2601_12941_gb300 import binding as B

    W, H, dt, G, sp, ref = _pool()[1]
    dfm = synth.render(synth.ImageSpec(sp, field=synth.affine_field(W, H, u0=1.2), gray_max=G, noise_tag=7),
                       W, H, dt)
    roi = np.zeros((H, W), np.uint8)
    roi[20:-20, 30:-30] = 1
    cases = [(ref, dfm, None, 21, 5, "affine", "mixed", 1),
             (torch.from_numpy(ref.view(np.int16)).cuda(), dfm, roi, 31, 3, "quadratic", "fp64", 3),
             (ref, torch.from_numpy(dfm.view(np.int16)).cuda(), None, 15, 2, "rigid", "mixed", 2)]
    for r_img, d_img, m, S, step, shape, prec, ns in cases:
        seeds = [(W // 2 + 8 * k, H // 2) for k in range(ns)]
        prm = B.params(precision=prec)
        ri, _ = B.make_image(r_img)
        di, _ = B.make_image(d_img)
        est = B.dic_estimate_device_bytes(ri, di, m is not None, S, step, B.SHAPES[shape], prm, ns)
        c = pkg.Correlation(r_img, d_img, m, S, step, shape, precision=prec)
        c.run(seeds)
        assert c.device_bytes() == est, (S, shape, prec)
        # re-grid for other settings: the prediction holds exactly as well
        for S2, step2, shape2, prec2, ns2 in [(41, 7, "affine", prec, 1), (17, 1, "quadratic", "mixed", 4)]:
            prm2 = B.params(precision=prec2)
            di2, _ = B.make_image(dfm)
            pred = B.dic_estimate_regrid_bytes(c.h, di2, False, S2, step2, B.SHAPES[shape2], prm2, ns2)
            c.set_subsets(S2, step2, shape2)
            c.set_deformed(dfm)
            c.set_params(precision=prec2)
            c.run([(W // 2 + 8 * k, H // 2) for k in range(ns2)])
            assert c.device_bytes() == pred, (S2, shape2, prec2)
        c.close()


def test_regridded_handle_equals_fresh_handle(pkg):
    pool = _pool()
    jobs = [j for j in _jobs(pool) if j["pool"] == 0]
    prm = dict(precision="mixed")
    c = pkg.Correlation(jobs[0]["ref"], jobs[0]["deformed"], None, jobs[0]["S"], jobs[0]["step"],
                        jobs[0]["shape"], **prm)
    c.run(jobs[0]["seeds"])
    for job in jobs[1:] + jobs[:1]:
        c.set_subsets(job["S"], job["step"], job["shape"])
        with pytest.raises(pkg.DicError):
            c.results()                     # results are dropped by the re-grid
        c.set_deformed(job["deformed"])
        c.run(job["seeds"])
        _same(c.results(), _alone(pkg, job, prm), FIELDS)
    c.close()


def test_each_job_same_alone_and_in_the_mix(pkg):
    from paper_2601_12941_gb300.serve import Job, Server

    pool = _pool()
    jobs = _jobs(pool)
    prm = dict(precision="mixed")
    alone = [_alone(pkg, j, prm) for j in jobs]
    with Server(workers=4, hbm_budget=2 << 30) as srv:
        # twice through: the second pass reuses the cached handle of each reference
        futs = [srv.submit(Job(j["ref"], j["deformed"], j["seeds"], j["S"], j["step"], j["shape"], params=prm,
                               ref_key=("pool", j["pool"]), fields=FIELDS)) for j in jobs + jobs]
        res = [f.result(timeout=300) for f in futs]
        st = srv.stats()
    for k, r in enumerate(res):
        _same(r.fields, alone[k % len(jobs)], FIELDS)
        assert r.n_accepted > 0.8 * r.n_points
    assert st["completed"] == 2 * len(jobs) and st["cache_hits"] >= 1
    assert st["cache_hits"] + st["cache_misses"] == 2 * len(jobs)
    assert st["peak_busy_workers"] >= 2 and st["peak_bytes"] <= st["budget_bytes"]


def test_device_bytes_match_estimates_with_fft_seeds_and_bicubic(pkg):
    from paper_2601_12941_gb300 import binding as B

    W, H, dt, G, sp, ref = _pool()[1]
    dfm = synth.render(synth.ImageSpec(sp, field=synth.affine_field(W, H, u0=9.6, v0=-5.2), gray_max=G,
                                       noise_tag=8), W, H, dt)
    ri, _ = B.make_image(ref)
    di, _ = B.make_image(dfm)
    seeds = [(W // 2, H // 2)]
    # FFT-seeded (windows up to 128 px: the global work-buffer path is allocated too)
    prm = B.params(init="fft", max_displacement=100)
    est = B.dic_estimate_device_bytes(ri, di, False, 21, 5, B.DIC_AFFINE, prm, 1)
    c = pkg.Correlation(ref, dfm, None, 21, 5, "affine", init="fft", max_displacement=100)
    c.run(seeds)
    assert c.device_bytes() == est
    assert (c.results()["status"] == 0).sum() > 0
    # re-grid with the integer search: the FFT arrays stay held and are counted
    prm2 = B.params(search_radius=12)
    pred = B.dic_estimate_regrid_bytes(c.h, di, False, 31, 7, B.DIC_AFFINE, prm2, 2)
    c.set_subsets(31, 7, "affine")
    c.set_deformed(dfm)
    c.set_params(init="search", search_radius=12)
    c.run([(W // 2, H // 2), (W // 2 + 40, H // 2)])
    assert c.device_bytes() == pred
    # and back to FFT seeds with a larger window set
    prm3 = B.params(init="fft", max_displacement=300)
    pred = B.dic_estimate_regrid_bytes(c.h, di, False, 21, 4, B.DIC_AFFINE, prm3, 1)
    c.set_subsets(21, 4, "affine")
    c.set_deformed(dfm)
    c.set_params(init="fft", max_displacement=300)
    c.run(seeds)
    assert c.device_bytes() == pred
    c.close()
    # the bicubic interpolant holds the same planes as the spline
    est = B.dic_estimate_device_bytes(ri, di, False, 21, 5, B.DIC_AFFINE, B.params(search_radius=12), 1)
    c = pkg.Correlation(ref, dfm, None, 21, 5, "affine", interp="bicubic", search_radius=12)
    c.run(seeds)
    assert c.device_bytes() == est
    c.close()


def test_admission_keeps_footprint_within_budget(pkg):
    from paper_2601_12941_gb300.serve import AdmissionError, Job, LibdicEngine, Server

    W, H, dt, G, sp, ref = _pool()[0]
    mk = []
    for k in range(4):
        fld = synth.affine_field(W, H, u0=0.4 * k, v0=-0.3 * k, exx=1e-3 * k)
        dfm = synth.render(synth.ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=70 + k), W, H, dt)
        # distinct keys: every job after the first must evict the previous job's handle
        mk.append(Job(ref, dfm, [(W // 2, H // 2)], 21, 5, "affine", params=dict(precision="mixed"),
                      ref_key=("job", k)))
    est = LibdicEngine().estimate(mk[0])
    budget = int(1.5 * est)                  # room for one job at a time
    with Server(workers=4, hbm_budget=budget) as srv:
        futs = [srv.submit(j) for j in mk]
        too_big = srv.submit(Job(np.zeros((4096, 4096), np.uint8), np.zeros((4096, 4096), np.uint8),
                                 [(2048, 2048)], 21, 1, "quadratic"))
        res = [f.result(timeout=300) for f in futs]
        with pytest.raises(AdmissionError):
            too_big.result(timeout=60)
        st = srv.stats()
    assert st["rejected"] == 1 and st["completed"] == len(mk)
    assert st["peak_bytes"] <= budget and st["peak_busy_workers"] == 1
    assert st["memory_waits"] >= 1 and st["evictions"] == len(mk) - 1
    assert all(r.device_bytes == est for r in res)


def test_served_job_matches_oracle(pkg):
    from paper_2601_12941_gb300.serve import Job, Server

    w = WL.affine_256_u8()
    ref = synth.render(w.ref, w.width, w.height, w.dtype)
    dfm = synth.render(w.deformed, w.width, w.height, w.dtype)
    with Server(workers=2, hbm_budget=1 << 30) as srv:
        r = srv.submit(Job(ref, dfm, w.seeds, w.subset_size, w.subset_step, w.shape,
                           params=dict(precision="fp64", search_radius=w.search_radius, **GPU_PARAMS["fp64"]),
                           fields=("p", "zncc", "iters", "status", "wave"))).result(timeout=120)
    ora = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape, w.seeds,
                           dict(ORACLE_PARAMS, search_radius=w.search_radius))
    stats = compare(r.fields, ora, w.width, w.height, w.subset_size)
    assert stats["accepted"] > 2000
