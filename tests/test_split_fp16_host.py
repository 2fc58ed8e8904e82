"""The FFT window kernel multiplies operands split into an FP16 high part and an FP16
remainder (x = hi + lo, both rounded to FP16) and keeps hi*hi + hi*lo + lo*hi with FP32
accumulation, after scaling each data operand by a power of two so that its largest
value lies in [2^13, 2^14). Checked here in numpy (float16 rounding, float32 sums)
against float64 products: the scheme keeps about 22 significant bits relative to the
largest term, and without the scaling large or small operands leave the FP16 range."""
import numpy as np


def _split(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float32), lo.astype(np.float32)


def _scale_exp(m):
    return 13 - int(np.floor(np.log2(m))) if m > 0 else 0


def _split_product(a, b, scale=True):
    """a (M x K) times b (K x N) the kernel's way: a and b scaled by powers of two, split,
    three partial products summed in float32, the scales undone."""
    ea = _scale_exp(np.abs(a).max()) if scale else 0
    eb = _scale_exp(np.abs(b).max()) if scale else 0
    ah, al = _split((a * 2.0 ** ea).astype(np.float32))
    bh, bl = _split((b * 2.0 ** eb).astype(np.float32))
    acc = (ah @ bh).astype(np.float32) + (ah @ bl).astype(np.float32) + (al @ bh).astype(np.float32)
    return acc.astype(np.float64) * 2.0 ** (-ea - eb)


def test_split_products_keep_about_22_bits():
    rng = np.random.default_rng(3)
    for scale_a in (1e-9, 1.0, 255.0, 1e9):
        a = rng.uniform(-1, 1, (32, 64)) * scale_a
        L = 31
        k = np.arange(64) % 32
        w = np.exp(-2j * np.pi * np.outer(k, k) / L)       # DFT-like entries, |w| <= 1
        b = np.real(w)
        exact = a @ b
        got = _split_product(a, b)
        err = np.abs(got - exact).max() / (np.abs(a).max() * np.abs(b).max() * a.shape[1])
        assert err < 2.0 ** -20, (scale_a, err)


def test_without_scaling_large_values_overflow_fp16():
    a = np.full((16, 16), 1e6)
    b = np.eye(16)
    with np.errstate(over="ignore", invalid="ignore"):
        got = _split_product(a, b, scale=False)
    assert not np.isfinite(got).all()
    assert np.allclose(_split_product(a, b), a @ b, rtol=1e-6)


def test_dropping_the_remainder_terms_is_caught():
    # the high parts alone keep only FP16's 11 bits: the bound above must fail
    rng = np.random.default_rng(4)
    a = rng.uniform(-1, 1, (32, 64)) * 255.0
    b = rng.uniform(-1, 1, (64, 32))
    ea, eb = _scale_exp(np.abs(a).max()), _scale_exp(np.abs(b).max())
    ah, _ = _split((a * 2.0 ** ea).astype(np.float32))
    bh, _ = _split((b * 2.0 ** eb).astype(np.float32))
    got = (ah @ bh).astype(np.float64) * 2.0 ** (-ea - eb)
    err = np.abs(got - a @ b).max() / (np.abs(a).max() * np.abs(b).max() * a.shape[1])
    assert err > 2.0 ** -20
