"""Error bounds of the two split-product arithmetics (CPU, no GPU).

The tensor-core kernels multiply FP64 operands as split products: each
operand is truncated to FP32 and split into narrow slices whose pairwise
products are summed. This test restates both splits from their definitions
in numpy (bit operations on IEEE values) and checks the per-product error
bounds the mixed-precision tolerances are derived from:

  * BF16x3: x = s0 + s1 + s2 exactly (three 8-bit slices of the 24-bit FP32
    significand); six products with i + j <= 2; relative error of a*b at most
    2 * 2^-23 (truncation of both operands) + 3 * 2^-24 (dropped products);
  * TF32x3: hi = x rounded to 11 significant bits (to nearest, ties away),
    lo = the remainder rounded likewise; hi*hi + hi*lo + lo*hi; relative error
    at most 2 * 2^-23 + 2 * 2^-22 (rounding of lo) + 2^-22 (lo*lo dropped).
"""
import numpy as np


def f64_to_f32_trunc(x):
    """FP64 -> FP32 by truncating the significand (the kernels' conversion)."""
    b = x.view(np.uint64)
    sign = (b >> np.uint64(63)).astype(np.uint32) << np.uint32(31)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    mant = ((b >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.uint32)
    assert np.all((e > 0) & (e < 255))  # normal range only in this test
    return (sign | (e.astype(np.uint32) << np.uint32(23)) | mant).view(np.float32)


def bf16_rn(x):
    """FP32 -> BF16 (as FP32) rounded to nearest even."""
    b = x.view(np.uint32).astype(np.uint64)
    r = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32)


def tf32_rna(x):
    """FP32 -> TF32 (as FP32) rounded to nearest, ties away from zero."""
    b = x.view(np.uint32).astype(np.uint64)
    return ((b + np.uint64(0x1000)) & np.uint64(0xFFFFE000)).astype(np.uint32).view(np.float32)


def _samples(n=200000, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=n) * np.exp(rng.uniform(-8, 8, n))
    b = rng.normal(size=n) * np.exp(rng.uniform(-8, 8, n))
    return a, b


def test_bf16x3_split_is_exact_and_bounded():
    a, b = _samples()
    fa, fb = f64_to_f32_trunc(a), f64_to_f32_trunc(b)

    def split(x):
        s0 = bf16_rn(x)
        r1 = (x - s0).astype(np.float32)
        s1 = bf16_rn(r1)
        s2 = bf16_rn((r1 - s1).astype(np.float32))
        return [s.astype(np.float64) for s in (s0, s1, s2)]

    sa, sb = split(fa), split(fb)
    assert np.array_equal(sa[0] + sa[1] + sa[2], fa.astype(np.float64))  # exact split
    prod = sum(sa[i] * sb[j] for i in range(3) for j in range(3 - i))
    rel = np.abs(prod - a * b) / np.abs(a * b)
    assert rel.max() <= 2 * 2.0 ** -23 + 3 * 2.0 ** -24


def test_tf32x3_split_is_bounded():
    a, b = _samples(seed=1)
    fa, fb = f64_to_f32_trunc(a), f64_to_f32_trunc(b)

    def split(x):
        hi = tf32_rna(x)
        lo = tf32_rna((x - hi).astype(np.float32))
        return hi.astype(np.float64), lo.astype(np.float64)

    (ah, al), (bh, bl) = split(fa), split(fb)
    prod = ah * bh + ah * bl + al * bh
    rel = np.abs(prod - a * b) / np.abs(a * b)
    bound = 2 * 2.0 ** -23 + 2 * 2.0 ** -22 + 2.0 ** -22
    assert rel.max() <= bound
    assert rel.max() > 2 * 2.0 ** -23  # coarser than the BF16 split, as the tolerances assume
