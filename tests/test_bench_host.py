"""The work counts bench.py divides by, checked on the CPU against counts written out
by hand: the wave kernel's executed and reporting FLOPs, the tensor products of the FFT
window kernel, and the launch count of an FFT field."""
import numpy as np

import bench


def test_wave_flop_counts_by_hand():
    S, n = 21, 6
    px = S * S
    iters = np.array([2, 3, 1, 0, 5], np.int32)
    status = np.array([0, 0, bench.PT_OUT_OF_BOUNDS, 1, 0], np.uint8)
    wave = np.array([0, 1, 2, -1, 3], np.int32)          # the fourth point was never attempted
    per_pass = bench.FLOP_ITER[n] + bench.FLOP_COEFF_SUM
    # passes: iterations, plus one for the pass that left the sampling bounds
    passes = [2, 3, 1 + 1, 5]
    want = sum(p * per_pass * px + px * n * (n + 1) for p in passes)
    assert bench.executed_flops(iters, status, wave, S, n) == want
    # Levenberg-Marquardt: one more (final) pass per attempted point
    assert bench.executed_flops(iters, status, wave, S, n, final_pass=True) == want + 4 * per_pass * px
    # the fixed reporting count: iterations x per-pass + the final ZNCC pass, plus J^T J
    want_s = sum((i * bench.FLOP_ITER[n] + bench.FLOP_FINAL) * px + px * n * (n + 1) for i in (2, 3, 1, 5))
    assert bench.survey_flops(iters, status, wave, S, n) == want_s


def test_fft_window_kernel_product_count():
    # split-FP16 products (three per m16n8k16 step) of the 32-padded window:
    # rows (64 x 64) x (64 x 32), columns (32 x 64) x (64 x 64), inverse rows
    # (64 x 64) x (64 x 16), real column pass (32 x 32) x (32 x 32)
    def products(m, n, k):
        return (m // 16) * (n // 8) * (k // 16) * 3

    total = products(64, 32, 64) + products(32, 64, 64) + products(64, 16, 64) + products(32, 32, 32)
    assert total == bench.TC_MMAS_PER_WINDOW == 528
    assert bench.TC_FLOPS_PER_MMA == 2 * 16 * 8 * 16


def test_fft_field_launch_count():
    # the SEM settings' levels: 2048 .. 32 px, then the 31 px subsets; per level the
    # origins, the correlation and the MAD filter, the correlation taking 6 launches
    # at 1024 and 2048 px and 4 at 128-512 px; one status launch
    levels = [2048, 1024, 512, 256, 128, 64, 32, 31]
    corr = {2048: 6, 1024: 6, 512: 4, 256: 4, 128: 4, 64: 1, 32: 1, 31: 1}
    want = 1 + sum(2 + corr[L] for L in levels)
    assert bench.fft_launches(levels) == want == 44
