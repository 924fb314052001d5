"""The exact three-part 16-bit split that the tensor-core passes rely on
(the stage-2 operands M^T, Omega2 and Q2; the stage-1 projection's Q1; the
similarity Gram's U): v = hi + mid + lo with each part a BF16 value, rounded to
nearest from the remainder of the parts before it.  Emulated here with numpy
bit operations (round to nearest even on the upper 16 bits of an FP32 word),
so that the claim the kernels build on is checked without a GPU:

* the split is exact for FP32 values away from the subnormal range;
* every product of two parts is exact in FP32 (8 x 8 significant bits), so a
  sum of the nine part products over a long reduction carries only the FP32
  accumulation error of the plain FP32 product."""
import numpy as np


def bf16_rne(x):
    """FP32 -> nearest BF16 value (ties to even), returned as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def split3(v):
    v = np.asarray(v, dtype=np.float32)
    h = bf16_rne(v)
    r1 = (v - h).astype(np.float32)
    m = bf16_rne(r1)
    lo = bf16_rne((r1 - m).astype(np.float32))
    return h, m, lo


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even neighbour 1
    assert bf16_rne(np.float32(1 + 2.0 ** -8)) == np.float32(1.0)
    assert bf16_rne(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)
    assert bf16_rne(np.float32(1 + 2.0 ** -8 + 2.0 ** -20)) == np.float32(1 + 2.0 ** -7)
    assert bf16_rne(np.float32(-3.0)) == np.float32(-3.0)


def test_split_is_exact_over_a_wide_exponent_range():
    rng = np.random.default_rng(7)
    v = (rng.standard_normal(200_000) * np.exp2(rng.integers(-60, 60, 200_000))).astype(np.float32)
    h, m, lo = split3(v)
    # every part is a BF16 value
    for p in (h, m, lo):
        assert np.all((p.view(np.uint32) & 0xFFFF) == 0)
    # the three parts add up to v exactly (the sum in FP64 is exact)
    total = h.astype(np.float64) + m.astype(np.float64) + lo.astype(np.float64)
    np.testing.assert_array_equal(total, v.astype(np.float64))


def test_part_products_are_exact_and_the_split_product_is_fp32_accurate():
    rng = np.random.default_rng(11)
    n = 4096
    a = rng.standard_normal(n).astype(np.float32)
    b = (rng.standard_normal(n) * 3.0).astype(np.float32)
    pa, pb = split3(a), split3(b)
    # each part product is exactly representable in FP32
    for x in pa:
        for y in pb:
            prod64 = x.astype(np.float64) * y.astype(np.float64)
            np.testing.assert_array_equal(prod64.astype(np.float32).astype(np.float64), prod64)
    # sum over the reduction in FP32 of all nine part products per term, as the
    # FP32 tensor-core accumulator does, against the exact FP64 dot product
    acc = np.float32(0.0)
    for i in range(n):
        t = np.float32(0.0)
        for x in pa:
            for y in pb:
                t = np.float32(t + np.float32(x[i]) * np.float32(y[i]))
        acc = np.float32(acc + t)
    exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    bound = n * 2.0 ** -24 * float(np.sum(np.abs(a.astype(np.float64) * b.astype(np.float64))))
    assert abs(float(acc) - exact) <= bound
