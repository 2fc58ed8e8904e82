"""Throughput of the subset-correlation hot path on the gigapixel affine pair.

One step = one pair correlated end to end on the device: B-spline prefilter of
both images, seed search, and every propagation wave (reference precompute, IC-GN
iterations, final ZNCC, frontier claims), results left on the device. The inputs
(32768 x 32768 u8, 1.07 GB each) are resident in HBM before the timed region and
are larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--size 32768] [--no-fp64] [--no-cpu] [--no-e2e]

Under torchrun (N > 1) every rank correlates its own pair (independent replicas,
weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("converged subset-points/sec (1 Gpx pair, affine) vs plain FP64 GPU; "
          "p50/p99 pair latency")
UNIT = "points/s"
FP32_LANES_PER_SM = 128
# Algorithmic FP32 flops of the wave kernel (FMA = 2), the method's reporting count:
# per pixel and sampling pass of IC-GN (warp, B-spline weights, the 4 x 4 contraction,
# sum g and sum g^2, sum SD g: 64 rigid, 84 affine, 108 quadratic), per pixel of a
# separate final ZNCC pass (72), and n(n+1) per pixel for the reference precompute
# (J^T J). The Gauss-Newton kernel takes the ZNCC from its converging pass instead of
# a separate pass, with one more sum (sum f'g', 2 flops) in every pass: the executed
# count is n(n+1) + passes x (count + 2) per pixel, passes = iterations (+1 for a pass
# that left the sampling bounds).
FLOP_ITER = {2: 64, 6: 84, 12: 108}
FLOP_FINAL = 72
FLOP_COEFF_SUM = 2
PT_OUT_OF_BOUNDS = 3

# DRAM bytes (read + write) per attempted point of the wave kernel, from one ncu
# capture of the current kernel (a mid-run wave of 2,560 points on the 6144^2 version
# of the workload: 30.65 MB per launch); None when the kernel has changed since
WAVE_DRAM_BYTES_PER_POINT = 11972

# Tensor work of the FFT window kernel per window (split-FP16 products, three per
# m16n8k16 step, of the 32-padded window: 192 for the forward rows, 192 for the
# columns, 96 for the inverse rows, 48 for the real column pass) and FLOPs per
# m16n8k16 product; FP16 runs at the bf16 dense rate, so the measured bf16 peak is the
# denominator.
TC_MMAS_PER_WINDOW = 528
TC_FLOPS_PER_MMA = 2 * 16 * 8 * 16


def measured_peaks():
    """The generated peaks file ({} when absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


MEASURED = measured_peaks()


def sm_count():
    """Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount)."""
    import torch

    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def sm_max_mhz():
    """Maximum SM clock: the generated peaks file, else nvidia-smi, else 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, KeyError, ValueError):
        pass
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip().splitlines()
        return float(out[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return 2070.0, "nominal"


def fp32_peak():
    """FP32 peak in TFLOP/s: SM count (from the device) x 128 FP32 lanes x 2 (FMA) x
    the maximum SM clock; derived from unit counts and clocks (no measured FP32
    peak exists for this pool). Returns (peak, note, sms, mhz)."""
    sms = sm_count()
    mhz, src = sm_max_mhz()
    return (sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            "derived: %d SMs (device attribute) x %d FP32 lanes x 2 (FMA) x %.0f MHz (%s)"
            % (sms, FP32_LANES_PER_SM, mhz, src), sms, mhz)


def survey_flops(iters, status, wave, S, nparams):
    """The method's fixed reporting count: (iters x per-pass + final pass) S^2 + n(n+1) S^2."""
    attempted = wave >= 0
    it = iters[attempted].astype(np.float64)
    px = float(S * S)
    return float(np.sum((it * FLOP_ITER[nparams] + FLOP_FINAL) * px + px * nparams * (nparams + 1)))


def executed_flops(iters, status, wave, S, nparams, final_pass=False):
    """Work the Gauss-Newton kernel executes: n(n+1) S^2 per attempted point plus
    (per-pass count + 2) S^2 per sampling pass; final_pass: one more pass per
    attempted point (Levenberg-Marquardt)."""
    attempted = wave >= 0
    passes = iters[attempted].astype(np.float64) + (status[attempted] == PT_OUT_OF_BOUNDS)
    if final_pass:
        passes = passes + 1.0
    px = float(S * S)
    return float(np.sum(passes * (FLOP_ITER[nparams] + FLOP_COEFF_SUM) * px + px * nparams * (nparams + 1)))


def wave_roofline(res, S, nparams, kernel_ms, final_pass=False):
    """Roofline of the wave kernels of one correlation: executed TFLOP/s over the
    summed wave-kernel time, against the derived FP32 peak; the fixed reporting
    count beside it."""
    peak, note, sms, mhz = fp32_peak()
    ex = executed_flops(res["iters"], res["status"], res["wave"], S, nparams, final_pass)
    sv = survey_flops(res["iters"], res["status"], res["wave"], S, nparams)
    t = kernel_ms / 1e3
    return {"bound": "alu", "achieved": ex / t / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": ex / t / 1e12 / peak,
            "frac_survey_count": sv / t / 1e12 / peak, "kernel_ms": kernel_ms, "sm_count": sms, "sm_max_mhz": mhz,
            "peak_note": note, "algorithmic_gflop": ex / 1e9, "survey_count_gflop": sv / 1e9}


class Clocks:
    """nvidia-smi samples while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            rows = open(self.path).read().strip().splitlines()
        except OSError:
            rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in rows:
            f = [x.strip() for x in row.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if self.path:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        under = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": float(np.median(under)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """Host-side aggregation over the replicas of a multi-GPU run (one process per
    GPU, each correlating its own pair): a barrier, the slowest rank's time and the
    sum of the work. `dist` is torch.distributed or None; `device` holds the
    reduction buffers (cuda for NCCL, cpu for gloo)."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX) if self.dist is not None else float(x)

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM) if self.dist is not None else float(x)


def aggregate(ranks, local_ms_per_step, local_accepted):
    """(ms_per_step, value): the slowest rank's time per step and the points all
    ranks accepted per second of that time (weak scaling)."""
    ms = ranks.max(local_ms_per_step)
    return ms, ranks.sum(local_accepted) / (ms / 1e3)


def run_ours(args):
    import torch

    import paper_2601_12941_gb300 as P
    import synth
    from synth import workloads as wl

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = wl.gigapixel_u8(args.size)
    ref = torch.empty((w.height, w.width), dtype=torch.uint8, device="cuda")
    dfm = torch.empty_like(ref)
    synth.render_gpu(w.ref, ref)
    synth.render_gpu(w.deformed, dfm)
    torch.cuda.synchronize()
    seeds = list(w.seeds)
    nparams = P.N_PARAMS[P.SHAPES[w.shape]]

    ranks = Ranks(dist, "cuda")

    def barrier():
        ranks.barrier()
        torch.cuda.synchronize()

    max_over_ranks = ranks.max
    sum_over_ranks = ranks.sum

    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    wave_launches = []

    def timed_steps(c, steps, warmup):
        for _ in range(warmup):
            c.set_reference(ref)
            c.set_deformed(dfm)
            c.run(seeds, sp)
        barrier()
        lat = []
        kern = 0.0
        launches = 0
        wave_launches.clear()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.set_reference(ref)
            c.set_deformed(dfm)
            c.run(seeds, sp)
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
            tm = c.timing()
            kern += tm["icgn_kernel_ms"]
            launches += tm["n_wave_launches"] + 7   # 2 prefilter, reset, 2 seed search, commit, finalize
            wave_launches.append(tm["n_wave_launches"])
        ev1.record(stream)
        barrier()
        total_ms = ev0.elapsed_time(ev1)
        return total_ms, lat, kern, launches

    c = P.Correlation(ref, dfm, None, w.subset_size, w.subset_step, w.shape, precision="mixed",
                      search_radius=w.search_radius, profile=1)
    with Clocks(local) as clk:
        total_ms, lat, kern_ms, launches = timed_steps(c, args.steps, args.warmup)
    clocks = clk.summary()
    res = c.results()
    accepted = int(res["n_accepted"])
    attempted = int((res["wave"] >= 0).sum())
    ms_per_step, value = aggregate(ranks, total_ms / args.steps, accepted)
    kern_avg = kern_ms / args.steps
    tm = c.timing()
    roof = wave_roofline(res, w.subset_size, nparams, kern_avg)
    per_launch = attempted / (sum(wave_launches) / len(wave_launches))
    roof.update({"kernel": "wave_kernel<float, 6, 128, 0> (fused reference precompute, IC-GN, ZNCC, claims)",
                 "traffic": WAVE_DRAM_BYTES_PER_POINT * per_launch if WAVE_DRAM_BYTES_PER_POINT else None,
                 "traffic_note": "bytes per launch: DRAM bytes per attempted point (ncu capture of the 6144^2 "
                                 "case) x attempted points per wave launch; the kernel is ALU-bound",
                 "kernel_ms_per_step": kern_avg, "share_of_step": kern_avg / (total_ms / args.steps),
                 "achieved_note": "achieved = executed FP32 flops of the step's wave kernels / their summed "
                                  "CUDA-event durations (%d launches per step)" % (sum(wave_launches) / len(wave_launches))})
    # prefilter of both images: HBM-bound, 1 B read + 4 B written per pixel and image
    hbm, hbm_note = hbm_peak_gbs()
    pf_bytes = 2.0 * (1 + 4) * w.width * w.height
    pf_gbs = pf_bytes / (tm["prefilter_ms"] / 1e3) / 1e9 if tm["prefilter_ms"] > 0 else None

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name + ": %dx%d u8 SEM-like speckle pair (0.5-1.5 px dots), "
                                  "affine field plus 0.8 px slip on the diagonal, subset %d, step %d, "
                                  "affine, %d seeds, search radius %d"
                                  % (w.width, w.height, w.subset_size, w.subset_step, len(seeds),
                                     w.search_radius),
                      "points": int(res["n_points"]), "accepted": accepted, "attempted": attempted,
                      "waves": int(res["n_waves"]),
                      "precision": "DIC_MIXED: u8 gray levels; FP32 spline coefficients, samples, sums, "
                                   "Jacobi-scaled Hessian inverse, solve and ZNCC normalisation; FP64 results "
                                   "(config 3 as written, BF16 gray and FP64 solves: see config3_as_written)",
                      "controls": "max_iter 40, threshold 0.01, zncc_min 0.70",
                      "l2": "no flush: each step reads two 1.07 GB gray planes and writes two 4.3 GB coefficient planes, above the 129 MB L2",
                      "parallelism": "replicas x%d" % world},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "gpu_launches": launches,
           "roofline": roof,
           "prefilter": {"bound": "hbm", "kernel": "prefilter_iir_kernel<u8> (2 images)", "ms_per_step": tm["prefilter_ms"],
                         "achieved": pf_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": pf_gbs / hbm if pf_gbs else None, "peak_note": hbm_note,
                         "algorithmic_bytes_per_pixel": 5},
           "stages_ms": {k: tm[k] for k in ("prefilter_ms", "setup_ms", "waves_ms", "seed_kernel_ms")},
           "clocks": clocks}

    if not args.no_e2e:
        # right after the headline steps, on the same handle and in the same state of the GPU
        with Clocks(local) as clk_e2e:
            out["e2e"] = e2e_leg(args, c, ref, dfm, seeds, stream, barrier, max_over_ranks, sum_over_ranks)
        out["e2e"]["clocks"] = clk_e2e.summary()
        c.set_reference(ref)
        c.set_deformed(dfm)

    if not args.no_fp64:
        c64 = P.Correlation(ref, dfm, None, w.subset_size, w.subset_step, w.shape, precision="fp64",
                            search_radius=w.search_radius, profile=1)
        t64, lat64, k64, _ = timed_steps(c64, args.fp64_steps, 1)
        r64 = c64.results()
        v64 = sum_over_ranks(int(r64["n_accepted"])) / (max_over_ranks(t64 / args.fp64_steps) / 1e3)
        out["fp64_plain"] = {"value": v64, "unit": UNIT, "ms_per_step": t64 / args.fp64_steps,
                             "steps": args.fp64_steps, "wave_kernel_ms": k64 / args.fp64_steps,
                             "speedup_of_mixed": value / v64 if v64 else None}
        out["vs_fp64_plain"] = value / v64 if v64 else None
        c64.close()
    if not args.no_variants:
        out["config3_as_written"] = config3_leg(args, P, ref, dfm, w, seeds, stream, timed_steps)

    if rank == 0 and not args.no_oracle_error:
        # the oracle's error report of the headline step's result (host work, after the timing)
        out["oracle_error"] = oracle_error_gigapixel(res, w, args.oracle_points)

    if not args.no_strain:
        out["strain"] = strain_leg(c, w, stream)
    if not args.no_fft:
        out["fft_init"] = fft_leg(ref, dfm, stream, reps=args.fft_reps, kernel_reps=args.fft_kernel_reps)
    if not args.no_variants:
        out["variants"] = variants_leg(ref, dfm, w, seeds, stream)
    c.close()
    del ref, dfm
    torch.cuda.empty_cache()

    if not args.no_configs:
        out["config1"] = config1_leg(P, stream, rank == 0 and not args.no_oracle_error)
        out["config2"] = config2_leg(P, stream, rank == 0 and not args.no_oracle_error)
    if args.seq_frames > 0:
        out["sequence"] = sequence_leg(args, stream)
        if not args.no_configs:
            out["sequence_subsets"] = [sequence_variant_leg(args, stream, S, shape, frames)
                                       for S, shape, frames in ((31, "affine", 100), (41, "affine", 100),
                                                                (21, "quadratic", 100), (41, "quadratic", 50))]
    if args.serve_jobs > 0 and world == 1:
        out["serving"] = serving_leg(args)

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(w, out["cpu_baseline"])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def config3_leg(args, P, ref, dfm, w, seeds, stream, timed_steps):
    """Config 3 as its description reads: gray levels in BF16 (the u8 pair converted on
    the device, outside the timed region; u8 values are exact in BF16), coefficients
    in FP32, and the Hessian inverse, the solve and the final ZNCC normalisation in
    FP64 (DIC_MIXED_FP64_SOLVE). Same grid, seeds and controls as the headline."""
    import torch

    rb = ref.to(torch.bfloat16)
    db = dfm.to(torch.bfloat16)
    torch.cuda.synchronize()
    c = P.Correlation(rb, db, None, w.subset_size, w.subset_step, w.shape, precision="mixed_fp64_solve",
                      search_radius=w.search_radius, profile=1)
    steps = max(2, min(args.steps, 5))
    t, lat, kern, _ = timed_steps(c, steps, 1)
    r = c.results()
    tm = c.timing()
    c.close()
    acc = int(r["n_accepted"])
    out = {"precision": "DIC_MIXED_FP64_SOLVE: BF16 gray levels, FP32 coefficients, samples and sums; FP64 Hessian "
                        "inverse, solve (one refinement step) and ZNCC normalisation",
           "steps": steps, "ms_per_step": t / steps, "points_per_s": acc / (t / steps / 1e3), "accepted": acc,
           "prefilter_ms": tm["prefilter_ms"],
           "roofline": wave_roofline(r, w.subset_size, 6, kern / steps)}
    if not args.no_oracle_error:
        out["oracle_error"] = oracle_error_gigapixel(r, w, max(60, args.oracle_points // 4))
    del rb, db
    return out


def oracle_error_gigapixel(res, w, n_points, seed=2026):
    """Error of a 1 Gpx result against the FP64 oracle on a seeded sample of points:
    each sampled point is correlated by the oracle from the analytic field (start:
    the field's displacement and gradient at the centre) on host-rendered crops, to
    its converged root (threshold 1e-8, 100 iterations); the GPU result was taken at
    the bench's controls. Three fifths of the sample lie away from the slip line, the
    rest near it (their subsets just clear it); subsets that cross the line have no
    single affine root and are counted apart (status agreement only)."""
    import oracle
    import synth
    from oracle import dic_oracle as O

    fld = w.field
    S, r = w.subset_size, (w.subset_size - 1) // 2
    X = res["x"].astype(np.float64) - fld.cx
    Y = res["y"].astype(np.float64) - fld.cy
    dist = np.abs(Y - X) / np.sqrt(2.0)
    clear = r * np.sqrt(2.0) + 1.0
    inside = (res["x"] > 200) & (res["x"] < w.width - 200) & (res["y"] > 200) & (res["y"] < w.height - 200)
    att = res["wave"] >= 0
    rng = np.random.default_rng(seed)
    far = np.flatnonzero(inside & att & (dist > clear + 40))
    near = np.flatnonzero(inside & att & (dist > clear) & (dist <= clear + 40))
    cross = np.flatnonzero(inside & att & (dist <= clear - 2.0))
    n_near = n_points * 2 // 5
    pick = np.concatenate([rng.choice(far, n_points - n_near, replace=False),
                           rng.choice(near, min(n_near, len(near)), replace=False)])
    pad = 48 + r + 16
    du, dp, agree, both = [], [], 0, 0
    t0 = time.perf_counter()

    def run_point(q, p0):
        xc, yc = int(res["x"][q]), int(res["y"][q])
        x0, y0, side = xc - pad, yc - pad, 2 * pad + 1
        rc, roff = synth.render_crop(w.ref, w.width, w.height, x0, y0, side, side, w.dtype)
        dc, doff = synth.render_crop(w.deformed, w.width, w.height, x0, y0, side, side, w.dtype)
        refp = O.Plane(rc, roff[0], roff[1], w.width, w.height)
        defp = O.Plane(dc, doff[0], doff[1], w.width, w.height)
        return O.icgn(refp, defp, xc, yc, S, "affine", p0, dict(conv_threshold=1e-8, max_iter=100))

    for q in pick:
        xc, yc = float(res["x"][q]), float(res["y"][q])
        u, v = synth.displacement(fld, np.array([xc]), np.array([yc]))
        ora = run_point(q, [u[0], v[0], fld.exx, fld.exy, fld.eyx, fld.eyy])
        g_ok = res["status"][q] == 0
        o_ok = ora["status"] == O.OK
        agree += int(g_ok == o_ok)
        if g_ok and o_ok:
            both += 1
            d = np.abs(np.asarray(res["p"][q]) - ora["p"])
            du.append(d[:2].max())
            dp.append(d[2:].max())
    cross_pick = rng.choice(cross, min(20, len(cross)), replace=False) if len(cross) else []
    cross_agree = 0
    for q in cross_pick:
        xc, yc = float(res["x"][q]), float(res["y"][q])
        u, v = synth.displacement(fld, np.array([xc]), np.array([yc]))
        ora = run_point(q, [u[0], v[0], fld.exx, fld.exy, fld.eyx, fld.eyy])
        cross_agree += int((res["status"][q] == 0) == (ora["status"] == O.OK))
    du, dp = np.array(du), np.array(dp)
    return {"sample": "%d points (%d away from the slip line, %d near it), oracle from the analytic field on "
                      "host-rendered crops, converged to 1e-8" % (len(pick), n_points - n_near, len(pick) - (n_points - n_near)),
            "both_accepted": both, "status_agreement": "%d/%d" % (agree, len(pick)),
            "max_uv_px": float(du.max()) if both else None, "mean_uv_px": float(du.mean()) if both else None,
            "max_p2_5": float(dp.max()) if both else None, "mean_p2_5": float(dp.mean()) if both else None,
            "crossing_slip_line_status_agreement": "%d/%d" % (cross_agree, len(cross_pick)),
            "note": "the GPU stopped at the bench's threshold (0.01 on ||dp||), the oracle at 1e-8: the error "
                    "includes the unconverged remainder the paper's threshold leaves",
            "oracle_seconds": time.perf_counter() - t0}


def pair_leg(P, ref, dfm, w, precision, stream, steps, warmup=2):
    """One workload pair timed on the device (reference and deformed set, prefilter,
    seed search, every wave), results left on the device; returns the last result."""
    import torch

    c = P.Correlation(ref, dfm, None, w.subset_size, w.subset_step, w.shape, precision=precision,
                      search_radius=w.search_radius, profile=1)
    for _ in range(warmup):
        c.set_reference(ref)
        c.set_deformed(dfm)
        c.run(list(w.seeds), stream.cuda_stream)
    stream.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    kern = 0.0
    lat = []
    a.record(stream)
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.set_reference(ref)
        c.set_deformed(dfm)
        c.run(list(w.seeds), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
        kern += c.timing()["icgn_kernel_ms"]
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    r = c.results()
    c.close()
    nparams = P.N_PARAMS[P.SHAPES[w.shape]]
    acc = int(r["n_accepted"])
    return r, {"precision": precision, "steps": steps, "ms_per_step": ms, "points_per_s": acc / (ms / 1e3),
               "accepted": acc, "points": int(r["n_points"]), "waves": int(r["n_waves"]),
               "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
               "roofline": wave_roofline(r, w.subset_size, nparams, kern / steps)}


def _parity_stats(gpu, ora):
    """Status agreement and parameter errors of a whole-grid GPU result against the
    oracle's correlation of the same pair (same controls)."""
    sg, so = np.asarray(gpu["status"]).astype(int), np.asarray(ora["status"]).astype(int)
    both = (sg == 0) & (so == 0)
    pg, po = np.asarray(gpu["p"])[both], np.asarray(ora["p"])[both]
    d = np.abs(pg - po)
    return {"status_agreement": "%d/%d" % (int((sg == so).sum()), len(so)), "both_accepted": int(both.sum()),
            "max_uv_px": float(d[:, :2].max()) if both.any() else None,
            "mean_uv_px": float(d[:, :2].mean()) if both.any() else None,
            "max_p2": float(d[:, 2:].max()) if both.any() and d.shape[1] > 2 else None,
            "max_zncc": float(np.abs(np.asarray(gpu["zncc"], np.float64)[both] - ora["zncc"][both]).max())
            if both.any() else None}


def config1_leg(P, stream, with_oracle):
    """Config 1: the 256^2 u8 affine pair (2,304 points, subset 21, step 5, one seed),
    the plain FP64 form and the mixed form, each against the oracle's correlation of
    the whole pair at the same (Sec. 4 default) controls."""
    import torch

    import oracle
    import synth
    from synth import workloads as wl

    w = wl.affine_256_u8()
    ref_h = synth.render(w.ref, w.width, w.height, "u8")
    dfm_h = synth.render(w.deformed, w.width, w.height, "u8")
    ref, dfm = torch.from_numpy(ref_h).cuda(), torch.from_numpy(dfm_h).cuda()
    out = {"workload": "%s: %dx%d u8, subset %d, step %d, affine, 1 seed, Sec. 4 default controls"
                       % (w.name, w.width, w.height, w.subset_size, w.subset_step)}
    ora = None
    if with_oracle:
        t0 = time.perf_counter()
        ora = oracle.correlate(ref_h, dfm_h, None, w.subset_size, w.subset_step, w.shape, list(w.seeds),
                               dict(search_radius=w.search_radius))
        out["oracle_seconds"] = time.perf_counter() - t0
    for prec in ("fp64", "mixed"):
        r, d = pair_leg(P, ref, dfm, w, prec, stream, steps=20)
        if ora is not None:
            d["oracle_error"] = _parity_stats(r, ora)
        out[prec] = d
    return out


def config2_leg(P, stream, with_oracle, n_oracle=40):
    """Config 2: the 2048^2 u16 sine pair (1,018,081 points, subset 31, step 2,
    quadratic), FP64 and mixed; oracle error on a seeded sample of points with periods
    above 80 px (x > 500), each correlated by the oracle from the analytic field's
    rounded displacement to its converged root."""
    import torch

    import synth
    from oracle import dic_oracle as O
    from synth import workloads as wl

    w = wl.sine_2048_u16()
    ref_h = synth.render(w.ref, w.width, w.height, "u16")
    dfm_h = synth.render(w.deformed, w.width, w.height, "u16")
    ref = torch.from_numpy(ref_h.view(np.int16)).cuda()
    dfm = torch.from_numpy(dfm_h.view(np.int16)).cuda()
    out = {"workload": "%s: %dx%d u16 (12-bit), v = 0.5 sin(2 pi y / T(x)), T 10-300 px, 1%% noise, subset %d, "
                       "step %d, quadratic, Sec. 4 default controls"
                       % (w.name, w.width, w.height, w.subset_size, w.subset_step)}
    refp = dfp = None
    if with_oracle:
        refp, dfp = O.Plane(ref_h), O.Plane(dfm_h)
    for prec, steps in (("fp64", 2), ("mixed", 5)):
        r, d = pair_leg(P, ref, dfm, w, prec, stream, steps=steps, warmup=1)
        if refp is not None:
            rng = np.random.default_rng(17)
            cand = np.flatnonzero((r["x"] > 500) & (r["status"] == 0))
            errs, perr, agree = [], [], 0
            for q in rng.choice(cand, n_oracle, replace=False):
                xc, yc = int(r["x"][q]), int(r["y"][q])
                u, v = synth.displacement(w.field, np.array([float(xc)]), np.array([float(yc)]))
                ora = O.icgn(refp, dfp, xc, yc, w.subset_size, "quadratic", [round(u[0]), round(v[0])],
                             dict(conv_threshold=1e-8, max_iter=100))
                agree += int(ora["status"] == O.OK)
                if ora["status"] == O.OK:
                    dd = np.abs(np.asarray(r["p"][q]) - ora["p"])
                    errs.append(dd[:2].max())
                    perr.append(dd[2:].max())
            d["oracle_error"] = {"sample": "%d accepted points with x > 500, oracle converged to 1e-8" % n_oracle,
                                 "oracle_accepts": "%d/%d" % (agree, n_oracle),
                                 "max_uv_px": float(max(errs)) if errs else None,
                                 "mean_uv_px": float(np.mean(errs)) if errs else None,
                                 "max_p2_11": float(max(perr)) if perr else None}
        out[prec] = d
    out["speedup_of_mixed"] = out["mixed"]["points_per_s"] / out["fp64"]["points_per_s"]
    return out


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (generated file), else the
    recipe's fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def strain_leg(c, w, stream, window=9, basis="biquadratic", measure="green_lagrange", reps=20):
    """Sec. 2.3 strain of the step's displacement field (10.7 M points): one kernel
    over the grid, HBM-bound. Algorithmic bytes per point: u, v (FP64) and status
    read once, seven FP32 components and the valid flag written: 46 B."""
    import torch

    from paper_2601_12941_gb300 import binding as B

    r = c.results(on_device=True)
    n = int(r["n_points"])
    outs = B.strain_outputs(n)
    args = (r["u"], r["v"], r["status"], r["nx"], r["ny"], w.subset_step, window, basis, measure, outs,
            stream.cuda_stream)
    for _ in range(3):
        B.dic_strain_field(*args)
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.dic_strain_field(*args)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms))
    bytes_per_point = 2 * 8 + 1 + 7 * 4 + 1
    gbs = bytes_per_point * n / (t / 1e3) / 1e9
    peak, note = hbm_peak_gbs()
    valid = int(outs["valid"].sum().item())
    return {"window": window, "basis": basis, "measure": measure,
            "vsg_px": (window - 1) * w.subset_step + w.subset_size, "points": n, "valid": valid,
            "ms": t, "points_per_s": n / (t / 1e3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_note": note, "algorithmic_bytes_per_point": bytes_per_point}}


def variants_leg(ref, dfm, w, seeds, stream, steps=2):
    """The next-row variants on the same 1.07 Gpx pair and grid as the headline step:
    the NSSD and SSD costs (Eq. 2-3), Levenberg-Marquardt, and Keys bicubic
    interpolation, each through the generic kernel instantiations. One warm-up step
    and `steps` timed steps each (reference and deformed set, prefilter, seeds, every
    wave)."""
    import torch

    import paper_2601_12941_gb300 as P

    out = {}
    for label, kw in (("nssd", dict(cost="nssd")), ("ssd", dict(cost="ssd")), ("lm", dict(optimizer="lm")),
                      ("bicubic", dict(interp="bicubic"))):
        interp = kw.pop("interp", "bspline3")
        c = P.Correlation(ref, dfm, None, w.subset_size, w.subset_step, w.shape, interp=interp, precision="mixed",
                          search_radius=w.search_radius, profile=1, **kw)
        c.run(seeds, stream.cuda_stream)
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        kern = 0.0
        a.record(stream)
        for _ in range(steps):
            c.set_reference(ref)
            c.set_deformed(dfm)
            c.run(seeds, stream.cuda_stream)
            kern += c.timing()["icgn_kernel_ms"]
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        r = c.results()
        acc = int(r["n_accepted"])
        out[label] = {"ms_per_step": ms, "points_per_s": acc / (ms / 1e3), "accepted": acc,
                      "wave_kernel_ms": kern / steps,
                      "mean_iterations": float(r["iters"][r["status"] == 0].mean()) if acc else None}
        c.close()
        torch.cuda.empty_cache()
    return out


def fft_launches(levels):
    """Kernel launches of one FFT field: per level the origins, the correlation and the
    MAD filter, the correlation taking 4 launches at 128-512 px (rows, paired columns,
    inverse rows, finish) and 6 above (two transposes more); one status launch."""
    return 1 + 3 * len(levels) + sum(3 if L <= 512 else 5 for L in levels if L > 64)


def fft_leg(ref, dfm, stream, S=31, step=15, D=2000, border=None, reps=3, kernel_reps=3):
    """Multi-window FFT initialiser (Sec. 2.2, Eq. 1; MAD) on the 1 Gpx pair with the
    SEM study's settings (Sec. 4): subset 31, step 15, maximum displacement 2000 px
    (windows 2048 .. 32, then 31), a 1000 px border outside the ROI, Gaussian
    sub-pixel fit. The last level (one 31 x 31 window per grid point: the DFT matrix
    products on the tensor cores, split-FP16 mma.sync) is timed alone through
    dic_fftcc_windows on the same number of windows. Its roofline counts the tensor
    work it executes, TC_MMAS_PER_WINDOW m16n8k16 products of 2 x 16 x 8 x 16 FLOPs,
    against the measured bf16 dense peak (FP16 and bf16 share the rate); the method's
    own count, 22 S^3 + 2 S^2 FP32 FLOPs per window
    (the forward 2-D DFT, 2 S^3 complex multiply-adds of 8 FLOPs; the inverse of the
    Hermitian cross power, (S+1)/2 rows of S^2 complex multiply-adds and a real
    column pass of S^2 (S-1)/2 two-FMA terms), is given beside it."""
    import torch

    import paper_2601_12941_gb300 as P
    from paper_2601_12941_gb300 import binding as B

    H, W = ref.shape
    if border is None:
        border = int(round(1000 * W / 32768))             # the SEM study's 1000 px at 32768 px
    roi = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    roi[border:H - border, border:W - border] = 1
    c = P.Correlation(ref, dfm, roi, S, step, "affine")
    c.fft_field(max_displacement=D, stream_ptr=stream.cuda_stream)          # warm-up (allocates)
    stream.synchronize()
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g = c.fft_field(max_displacement=D, stream_ptr=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms))
    ok = g["status"] == 0
    n_ok = int(ok.sum().item())
    # the dominant kernel alone: the last level's windows (the in-ROI subsets)
    r = (S - 1) // 2
    xs = torch.arange(g["nx"], device="cuda") * step
    ys = torch.arange(g["ny"], device="cuda") * step
    X, Y = torch.meshgrid(xs, ys, indexing="xy")
    org = torch.stack([X.ravel(), Y.ravel(), X.ravel(), Y.ravel()], 1).to(torch.int32)[ok]
    org = org.contiguous()
    n = org.shape[0]
    u, v, pk = (torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3))
    if kernel_reps > 0:
        B.dic_fftcc_windows(c.h, S, org, True, u, v, pk, stream.cuda_stream)
    kms = []
    for _ in range(kernel_reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.dic_fftcc_windows(c.h, S, org, True, u, v, pk, stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        kms.append(a.elapsed_time(b))
    k = float(np.median(kms)) if kms else float("nan")
    flops = (22.0 * S ** 3 + 2.0 * S ** 2) * n
    achieved = flops / (k / 1e3) / 1e12
    tc_flops = float(TC_MMAS_PER_WINDOW * TC_FLOPS_PER_MMA) * n
    tc_achieved = tc_flops / (k / 1e3) / 1e12
    f16_peak = MEASURED.get("bf16_tflops", 1912.3)
    levels = g["windows"]
    launches = fft_launches(levels)
    c.close()
    del roi
    return {"workload": "sem_fft_%d_u8: %dx%d u8 pair, subset %d, step %d, max displacement %d px, %d px border "
                        "outside the ROI, Gaussian sub-pixel fit" % (W, W, H, S, step, D, border),
            "windows": levels, "points_in_roi": n_ok, "ms": t, "points_per_s": n_ok / (t / 1e3),
            "gpu_launches": launches,
            "last_level_ms": k, "last_level_share": k / t,
            "roofline": {"bound": "tensor",
                         "kernel": "fftcc_tc_kernel (split-FP16 mma.sync m16n8k16, one warp per window)",
                         "achieved": tc_achieved, "peak": f16_peak, "unit": "TFLOP/s", "frac": tc_achieved / f16_peak,
                         "executed_flops_per_window": TC_MMAS_PER_WINDOW * TC_FLOPS_PER_MMA,
                         "peak_note": "FP16 dense at the bf16 rate, of measured: bf16 burst %.1f TFLOP/s "
                                      "(MEASURED_PEAKS.json)" % MEASURED.get("bf16_tflops", float("nan")),
                         "algorithmic_fp32": {"flops_per_window": 22 * S ** 3 + 2 * S ** 2, "achieved": achieved,
                                              "peak": fp32_peak()[0], "frac": achieved / fp32_peak()[0],
                                              "peak_note": fp32_peak()[1]}}}


def e2e_leg(args, c, ref, dfm, seeds, stream, barrier, max_over_ranks, sum_over_ranks):
    """Same metric through the C-ABI with host images (pinned) copied in and host
    results copied out inside the timed region."""
    import torch

    href = torch.empty(ref.shape, dtype=ref.dtype, pin_memory=True)
    hdef = torch.empty(dfm.shape, dtype=dfm.dtype, pin_memory=True)
    href.copy_(ref)
    hdef.copy_(dfm)
    nref, ndef = href.numpy(), hdef.numpy()
    steps = max(1, min(args.steps, 3))
    c.set_params(profile=0)
    c.set_reference(nref)
    c.set_deformed(ndef)
    c.run(seeds, stream.cuda_stream)
    r = c.results(copy=False)
    barrier()
    t0 = time.perf_counter()
    parts = np.zeros(3)
    for _ in range(steps):
        ta = time.perf_counter()
        c.set_reference(nref)
        c.set_deformed(ndef)
        tb = time.perf_counter()
        c.run(seeds, stream.cuda_stream)
        tc = time.perf_counter()
        r = c.results(copy=False)   # the handle's pinned host buffers, filled by the C call
        parts += (tb - ta, tc - tb, time.perf_counter() - tc)
    barrier()
    el = max_over_ranks((time.perf_counter() - t0) / steps)
    n = int(r["n_points"])
    d2h = sum(np.asarray(r[k]).nbytes for k in ("x", "y", "u", "v", "p", "zncc", "iters", "converged", "status", "wave"))
    up, run, back = parts / steps
    return {"value": sum_over_ranks(int(r["n_accepted"])) / el, "unit": UNIT,
            "ms_per_step": el * 1e3, "h2d_bytes_per_step": int(nref.nbytes + ndef.nbytes),
            "d2h_bytes_per_step": int(d2h), "points": n,
            "split_ms": {"upload": up * 1e3, "correlate": run * 1e3, "readback": back * 1e3},
            "h2d_gbs": (nref.nbytes + ndef.nbytes) / up / 1e9, "d2h_gbs": d2h / back / 1e9}


def run_sequence(stream, S, shape, frames, oracle_points=20):
    """Frames of the incremental uniaxial sequence (4096 x 3000 u16, strain ramping
    to 2e-2 over 200 frames, 1% noise), step 10, subset S and shape function given:
    frame 1 from the seed, every later frame from the previous frame's field
    (dic_correlate_sequence) against the resident frame-0 reference. Per-frame
    latency covers the deformed prefilter and every wave; frames are rendered outside
    the timed region. The frames of a shorter run are those of the 200-frame ramp
    (frame k has strain 0.02 k / 199). Oracle error: a seeded sample of points of the
    last frame, each correlated by the oracle from the analytic field on
    host-rendered crops to its converged root."""
    import torch

    import paper_2601_12941_gb300 as P
    import synth
    from oracle import dic_oracle as O
    from synth import workloads as wl

    w0 = wl.sequence_frame(1, subset_size=S, shape=shape)
    ref = torch.empty((w0.height, w0.width), dtype=torch.int16, device="cuda")
    dfm = torch.empty_like(ref)
    synth.render_gpu(w0.ref, ref)
    synth.render_gpu(w0.deformed, dfm)
    c = P.Correlation(ref, dfm, None, w0.subset_size, w0.subset_step, w0.shape, precision="mixed",
                      search_radius=w0.search_radius, profile=1)
    c.run(list(w0.seeds), stream.cuda_stream)
    nparams = P.N_PARAMS[P.SHAPES[shape]]
    lat, acc, kern, flops = [], [], [], []
    for k in range(2, frames + 1):
        synth.render_gpu(wl.sequence_frame(k, subset_size=S, shape=shape).deformed, dfm)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.set_deformed(dfm)
        c.run_next(stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
        kern.append(c.timing()["icgn_kernel_ms"])
        rr = c.results()
        acc.append(int(rr["n_accepted"]))
        flops.append(executed_flops(rr["iters"], rr["status"], rr["wave"], S, nparams))
    r = c.results()
    c.close()
    lat = np.array(lat)
    peak, note, _, _ = fp32_peak()
    achieved = float(np.sum(flops)) / (float(np.sum(kern)) / 1e3) / 1e12
    out = {"frames": frames, "size": [w0.width, w0.height], "subset": S, "step": w0.subset_step,
           "shape": shape, "points_per_frame": int(r["n_points"]), "accepted_last_frame": int(r["n_accepted"]),
           "frame_ms_p50": float(np.percentile(lat, 50)), "frame_ms_p99": float(np.percentile(lat, 99)),
           "points_per_s": float(np.sum(acc) / (np.sum(lat) / 1e3)),
           "wave_kernel_ms_p50": float(np.percentile(kern, 50)),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "peak_note": note},
           "note": "frame 1 from the seed (not timed); frames 2..%d timed" % frames}
    if oracle_points:
        wl_last = wl.sequence_frame(frames, subset_size=S, shape=shape)
        fld = wl_last.field
        rng = np.random.default_rng(31 + S)
        ok = np.flatnonzero((r["status"] == 0) & (r["x"] > 100) & (r["x"] < w0.width - 100)
                            & (r["y"] > 100) & (r["y"] < w0.height - 100))
        pad = (S - 1) // 2 + 80
        errs, perr, agree = [], [], 0
        pick = rng.choice(ok, min(oracle_points, len(ok)), replace=False)
        for q in pick:
            xc, yc = int(r["x"][q]), int(r["y"][q])
            x0, y0, side = xc - pad, yc - pad, 2 * pad + 1
            rc, roff = synth.render_crop(wl_last.ref, w0.width, w0.height, x0, y0, side, side, "u16")
            dc, doff = synth.render_crop(wl_last.deformed, w0.width, w0.height, x0, y0, side, side, "u16")
            u, v = synth.displacement(fld, np.array([float(xc)]), np.array([float(yc)]))
            p0 = [u[0], v[0], fld.exx, fld.exy, fld.eyx, fld.eyy] + [0.0] * (nparams - 6)
            ora = O.icgn(O.Plane(rc, roff[0], roff[1], w0.width, w0.height),
                         O.Plane(dc, doff[0], doff[1], w0.width, w0.height), xc, yc, S, shape, p0,
                         dict(conv_threshold=1e-8, max_iter=100))
            agree += int(ora["status"] == O.OK)
            if ora["status"] == O.OK:
                d = np.abs(np.asarray(r["p"][q]) - ora["p"])
                errs.append(d[:2].max())
                perr.append(d[2:].max())
        out["oracle_error"] = {"sample": "%d accepted points of frame %d, oracle from the analytic field, "
                                         "converged to 1e-8" % (len(pick), frames),
                               "oracle_accepts": "%d/%d" % (agree, len(pick)),
                               "max_uv_px": float(max(errs)) if errs else None,
                               "mean_uv_px": float(np.mean(errs)) if errs else None,
                               "max_p2": float(max(perr)) if perr else None}
    return out


def sequence_leg(args, stream):
    """Config 4 at subset 21, affine, 200 frames (see run_sequence), and the same
    sequence with incremental reference updating."""
    out = run_sequence(stream, 21, "affine", args.seq_frames, 0 if args.no_oracle_error else 20)
    out["updating"] = sequence_updating_leg(args, stream)
    return out


def sequence_variant_leg(args, stream, S, shape, frames):
    """Config 4 at another subset size or shape function (see run_sequence)."""
    return run_sequence(stream, S, shape, min(frames, args.seq_frames), 0 if args.no_oracle_error else 10)


def sequence_updating_leg(args, stream, every=50):
    """The same sequence with incremental reference updating: the total warps from
    frame 0 taken after every frame (dic_get_total_results) and the reference updated
    to the current frame every `every` frames (dic_update_reference). Two frame buffers
    alternate: an updated reference keeps borrowing its frame's buffer."""
    import torch

    import paper_2601_12941_gb300 as P
    import synth
    from synth import workloads as wl

    n = args.seq_frames
    w0 = wl.sequence_frame(1)
    ref = torch.empty((w0.height, w0.width), dtype=torch.int16, device="cuda")
    bufs = [torch.empty_like(ref), torch.empty_like(ref)]
    synth.render_gpu(w0.ref, ref)
    synth.render_gpu(w0.deformed, bufs[0])
    c = P.Correlation(ref, bufs[0], None, w0.subset_size, w0.subset_step, w0.shape, precision="mixed",
                      search_radius=w0.search_radius, profile=0)
    c.run(list(w0.seeds), stream.cuda_stream)
    cur = 0
    lat, upd, tot_ms = [], [], []
    for k in range(2, n + 1):
        if (k - 1) % every == 0:                        # frame k - 1 becomes the reference
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.update_reference(stream.cuda_stream)
            b.record(stream)
            b.synchronize()
            upd.append(a.elapsed_time(b))
            cur ^= 1                                    # the old frame buffer is now the reference's
        synth.render_gpu(wl.sequence_frame(k).deformed, bufs[cur])
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.set_deformed(bufs[cur])
        c.run_next(stream.cuda_stream)
        m.record(stream)
        t = c.totals(on_device=True, stream_ptr=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
        tot_ms.append(m.elapsed_time(b))
    ok = int((t["status"] == 0).sum().item())
    exx = float(t["p"][t["status"] == 0][:, 2].median().item())
    n_up = t["n_updates"]
    c.close()
    return {"every": every, "updates": n_up, "frame_ms_p50": float(np.percentile(lat, 50)),
            "frame_ms_p99": float(np.percentile(lat, 99)), "totals_ms_p50": float(np.percentile(tot_ms, 50)),
            "update_ms_p50": float(np.percentile(upd, 50)) if upd else None,
            "total_points_last_frame": ok, "total_exx_median_last_frame": exx,
            "note": "per frame: deformed prefilter, waves against the current reference, total warps from "
                    "frame 0; updates timed apart"}


def serving_leg(args):
    """A finite stream of mixed jobs with Poisson arrivals through the Server: pooled
    references (8, side log-uniform in [512, 16384], u8 or u16), per-job subset
    size, step, shape and affine field. Inputs are rendered on the device and staged
    in pinned host memory before the stream starts; a job's latency runs from its
    submission to its u, v, zncc and status on the host (upload, prefilter of
    whichever image is new, seed search, every wave, read-back)."""
    import torch

    import synth
    from paper_2601_12941_gb300.serve import Job, Server
    from synth import workloads as wl

    jobs = wl.serving_stream(n_jobs=args.serve_jobs, rate=args.serve_rate)

    def stage(spec, w):
        dt = torch.uint8 if w.dtype == "u8" else torch.int16
        d = torch.empty((w.height, w.width), dtype=dt, device="cuda")
        synth.render_gpu(spec, d)
        h = torch.empty(d.shape, dtype=dt, pin_memory=True)
        h.copy_(d)
        a = h.numpy()
        return a.view(np.uint16) if w.dtype == "u16" else a

    refs, inputs = {}, []
    for j in jobs:
        if j.ref_index not in refs:
            refs[j.ref_index] = stage(j.workload.ref, j.workload)
        inputs.append(stage(j.workload.deformed, j.workload))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    done = []
    with Server(workers=args.serve_workers) as srv:
        budget = srv.budget
        t0 = time.perf_counter()
        futs = []
        for j, dfm in zip(jobs, inputs):
            delay = t0 + j.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            w = j.workload
            futs.append(srv.submit(Job(refs[j.ref_index], dfm, list(w.seeds), w.subset_size, w.subset_step, w.shape,
                                       params=dict(precision="mixed", search_radius=w.search_radius),
                                       ref_key=("pool", j.ref_index))))
        failed = 0
        for j, f in zip(jobs, futs):
            try:
                r = f.result()
            except Exception:
                failed += 1
                continue
            r.fields = None
            done.append((j, r))
        st = srv.stats()
    if not done:
        return {"jobs": len(jobs), "failed": failed}
    t_end = max(r.t_end for _, r in done)
    wall = t_end - t0
    lat = np.array([r.latency_s for _, r in done])
    queue = np.array([r.queue_s for _, r in done])
    acc = sum(r.n_accepted for _, r in done)
    px = sum(r.n_points * j.workload.subset_size ** 2 for j, r in done)
    return {"jobs": len(jobs), "completed": len(done), "failed": failed, "workers": args.serve_workers,
            "offered_rate_jobs_per_s": args.serve_rate, "arrival_span_s": jobs[-1].arrival_s,
            "wall_s": wall, "achieved_jobs_per_s": len(done) / wall,
            "achieved_points_per_s": acc / wall, "subset_px_per_s": px / wall,
            "mean_points_per_job": float(np.mean([r.n_points for _, r in done])),
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "queue_s_p50": float(np.percentile(queue, 50)),
            "budget_gb": budget / 1e9, "peak_gb": st["peak_bytes"] / 1e9,
            "cache_hits": st["cache_hits"], "cache_misses": st["cache_misses"], "evictions": st["evictions"],
            "memory_waits": st["memory_waits"], "rejected": st["rejected"],
            "note": "the offered rate exceeds what one GPU sustains on this mix, so the stream runs "
                    "saturated: achieved_jobs_per_s is the capacity, the highest arrival rate at which "
                    "p99 latency can stay bounded"}


def cpu_baseline(w, seconds):
    """The FP64 oracle as it stands, one host thread, on a crop of the same pair:
    square crops around the first seed, grown until a run takes `seconds`."""
    import oracle
    import synth

    cx, cy = w.seeds[0]
    side = 200
    best = None
    while True:
        x0, y0 = cx - side // 2, cy - side // 2
        ref, _ = synth.render_crop(w.ref, w.width, w.height, x0, y0, side, side, w.dtype)
        dfm, _ = synth.render_crop(w.deformed, w.width, w.height, x0, y0, side, side, w.dtype)
        t = time.perf_counter()
        res = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape,
                               [(side // 2, side // 2)], dict(search_radius=w.search_radius))
        el = time.perf_counter() - t
        acc = int((res["status"] == 0).sum())
        best = dict(value=acc / el, unit=UNIT, cores=1, kind="oracle", nproc=os.cpu_count(), cpu_model=cpu_model(),
                    sample="%dx%d crop centred on the first seed of the same pair, %d points, %d accepted, %.1f s"
                    % (side, side, len(res["status"]), acc, el), seconds=el)
        if el >= seconds or side >= 1600:
            return best
        side = int(side * min(2.0, max(1.2, (seconds / max(el, 1e-3)) ** 0.5)))


def _oracle_crop_job(job):
    """One crop of the 1 Gpx pair through the oracle (runs in a spawned worker)."""
    import oracle
    import synth
    from synth import workloads as wl

    size, cx, cy, side = job
    w = wl.gigapixel_u8(size)
    x0, y0 = cx - side // 2, cy - side // 2
    ref, _ = synth.render_crop(w.ref, w.width, w.height, x0, y0, side, side, w.dtype)
    dfm, _ = synth.render_crop(w.deformed, w.width, w.height, x0, y0, side, side, w.dtype)
    t = time.perf_counter()
    res = oracle.correlate(ref, dfm, None, w.subset_size, w.subset_step, w.shape, [(side // 2, side // 2)],
                           dict(search_radius=w.search_radius))
    return int((res["status"] == 0).sum()), time.perf_counter() - t


def cpu_model():
    """The host CPU's model name (lscpu or /proc/cpuinfo), or the platform's."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline_all_cores(w, single):
    """The oracle on every host core: one crop per core (the single-thread leg's crop
    size, centred on different blocks of the pair), in a pool of spawned processes
    (no fork after the GPU was used); value = accepted points of all crops / wall
    time of the batch, pool start-up excluded."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    side = int(single["sample"].split("x")[0])
    b = w.width // 8
    centres = [(b // 2 + (i % 8) * b, b // 2 + ((i // 8) % 8) * b) for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_crop_job, [(w.width, cx, cy, 64) for cx, cy in centres])   # warm the workers
        t = time.perf_counter()
        res = pool.map(_oracle_crop_job, [(w.width, cx, cy, side) for cx, cy in centres])
        wall = time.perf_counter() - t
    acc = sum(a for a, _ in res)
    return {"value": acc / wall, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "nproc": cores, "sample": "%d crops of %dx%d (one per core, centred on different blocks of the same "
                                      "pair), %d accepted points, %.1f s wall" % (cores, side, side, acc, wall),
            "speedup_over_one_core": (acc / wall) / single["value"] if single.get("value") else None}


def run_reference(args):
    """The oracle (the only reference there is: the paper ships no code) on the
    host cores, on bounded crops of the same workload."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    from synth import workloads as wl

    w = wl.gigapixel_u8(args.size)
    per_step = max(3.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(w, per_step)
    vals, secs = [], []
    for _ in range(args.steps):
        b = cpu_baseline(w, per_step)
        vals.append(b["value"])
        secs.append(b["seconds"])
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": w.name + " (bounded crops, see cpu_baseline.sample)",
                      "parallelism": "host, 1 thread"},
           "cpu_baseline": dict(b, value=v),
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_fft_only(args):
    """The FFT initialiser leg alone on the synthetic pair of --size (profiling)."""
    import torch

    import synth
    from synth import workloads as wl

    w = wl.gigapixel_u8(args.size)
    ref = torch.empty((w.height, w.width), dtype=torch.uint8, device="cuda")
    dfm = torch.empty_like(ref)
    synth.render_gpu(w.ref, ref)
    synth.render_gpu(w.deformed, dfm)
    torch.cuda.synchronize()
    out = fft_leg(ref, dfm, torch.cuda.Stream(), reps=args.fft_reps, kernel_reps=args.fft_kernel_reps)
    print(json.dumps({"fft_init": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=32768)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-strain", action="store_true")
    ap.add_argument("--no-fft", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--fft-only", action="store_true",
                    help="run only the FFT initialiser leg on the pair of --size (profiling)")
    ap.add_argument("--fft-reps", type=int, default=3, help="timed fields of the FFT leg (after one warm-up)")
    ap.add_argument("--fft-kernel-reps", type=int, default=3,
                    help="timed runs of the last level alone (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 comparator")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 256^2, 2048^2 and extra sequence legs")
    ap.add_argument("--no-oracle-error", action="store_true", help="skip the oracle error reports")
    ap.add_argument("--oracle-points", type=int, default=200,
                    help="sampled points of the 1 Gpx oracle error report")
    ap.add_argument("--serve-jobs", type=int, default=500,
                    help="jobs in the serving stream (0: skip the serving leg)")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="Poisson arrival rate, jobs/s")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--seq-frames", type=int, default=200,
                    help="frames of the 4096 x 3000 sequence leg (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.fft_only:
        run_fft_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
