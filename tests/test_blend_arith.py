"""FP32 arithmetic the blend kernels rely on, emulated on the CPU with one rounding per
instruction as the GPU performs it (no GPU, no library call).

* The alpha >= 1/255 decision of the forward blend is taken as a factor
  sat(fma(s, 2^31, 1 - kSMin 2^31)) on the FMA pipe, where s = alpha / 0.99 and
  kSMin = FP32(1/(255 * 0.99)).  It must equal the comparison s >= kSMin for every FP32 s in
  [0, 1] (the backward takes the comparison itself, and both passes must decide alike).
  Checked for every float within 2^20 ulps of kSMin, every float below 2^-8 down to 2^-12,
  the binade edges, and random floats over [0, 1].
* The 0.99 clamp is applied as alpha = 0.99 sat(o' 2^p2) with o' = FP32(o / 0.99); this stays
  within 3 ulps of the literal FP32 min(0.99, o 2^p2) of the 3DGS compositing rule the paper
  renders with (Sec. 3.2), over random opacities in [1/255, 1] and factors 2^p2 in (0, 1].
"""
import numpy as np

F = np.float32
K_ALPHA_MAX = F(0.99)
K_S_MIN = F(1.0 / (255.0 * 0.99))          # (float)(1.0 / (255.0 * 0.99)) in the kernels
K_IN_C = F(F(1.0) - K_S_MIN * F(2.0 ** 31))  # 1.0f - kSMin * 0x1p31f
K_INV_ALPHA_MAX = F(F(1.0) / K_ALPHA_MAX)    # 1.0f / kAlphaMax


def fma_sat(s, b, c):
    """fma.rn.sat.f32: the exact product-sum rounded once to FP32, then clamped to [0, 1].
    s * 2^31 + c is exact in FP64 here (24 + 31 bits of the product within 53)."""
    r = (s.astype(np.float64) * float(b) + float(c)).astype(np.float32)
    return np.clip(r, F(0.0), F(1.0))


def mul_sat(a, b):
    """mul.rn.sat.f32: the FP32 product (exact in FP64, rounded once), clamped to [0, 1]."""
    r = (a.astype(np.float64) * b.astype(np.float64)).astype(np.float32)
    return np.clip(r, F(0.0), F(1.0))


def floats_between(lo, hi):
    """Every FP32 value in [lo, hi] (non-negative)."""
    a = np.array([lo], np.float32).view(np.uint32)[0]
    b = np.array([hi], np.float32).view(np.uint32)[0]
    return np.arange(a, b + 1, dtype=np.uint32).view(np.float32)


def test_constants_are_exact():
    assert F(2.0 ** -8) <= K_S_MIN < F(2.0 ** -7)
    k = float(K_S_MIN) * 2.0 ** 31
    assert k == int(k) and k < 2 ** 24          # kSMin 2^31 is an integer below 2^24
    assert float(K_IN_C) == 1.0 - k             # so 1 - kSMin 2^31 is exact in FP32


def test_in_factor_equals_the_comparison():
    bits = np.array([K_S_MIN], np.float32).view(np.uint32)[0]
    near = np.arange(bits - 2 ** 20, bits + 2 ** 20, dtype=np.uint32).view(np.float32)
    low = floats_between(F(2.0 ** -12), F(2.0 ** -8))
    rng = np.random.default_rng(0)
    rand = rng.random(2_000_000, dtype=np.float32)
    edges = np.array([0.0, 2.0 ** -126, 2.0 ** -9, 2.0 ** -8, 2.0 ** -7, 0.5, 1.0], np.float32)
    for s in (near, low, rand, edges):
        f = fma_sat(s, F(2.0 ** 31), K_IN_C)
        assert np.all((f == 0.0) | (f == 1.0))
        assert np.array_equal(f == 1.0, s >= K_S_MIN)


def test_saturated_alpha_matches_the_clamp():
    rng = np.random.default_rng(1)
    n = 2_000_000
    o = rng.uniform(1.0 / 255.0, 1.0, n).astype(np.float32)
    ex = rng.uniform(0.0, 1.0, n).astype(np.float32)
    ex[: n // 10] = F(1.0)                            # the centre, where the clamp acts most
    o[n // 10: n // 5] = rng.uniform(0.98, 1.0, n // 10).astype(np.float32)
    o_s = (o.astype(np.float64) * float(K_INV_ALPHA_MAX)).astype(np.float32)
    s = mul_sat(o_s, ex)
    alpha = (s.astype(np.float64) * float(K_ALPHA_MAX)).astype(np.float32)
    raw = (o.astype(np.float64) * ex.astype(np.float64)).astype(np.float32)
    ref = np.minimum(K_ALPHA_MAX, raw)
    ulp = np.spacing(ref)
    assert np.all(np.abs(alpha.astype(np.float64) - ref.astype(np.float64)) <= 3 * ulp.astype(np.float64))
    # the clamp is active (s = 1) exactly where the product o' 2^p2 reaches 1, i.e. where
    # o 2^p2 reaches 0.99 up to those few ulps
    active = s == F(1.0)
    assert np.all(raw[active] >= K_ALPHA_MAX * F(1.0 - 2.0 ** -21))
    assert np.all(raw[~active] <= K_ALPHA_MAX * F(1.0 + 2.0 ** -21))
