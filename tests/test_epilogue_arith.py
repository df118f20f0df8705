"""Host model of the tensor-core epilogue's cross-segment arithmetic (csrc/tc_gemm.cuh), in IEEE FP32.

The kernel adds each segment's FP32 result v_g, times the segment's power-of-two weight w_g, into a
two-float sum (hi, lo) with TwoSum, and adds the run's correction sum into lo. Since the paired-pipe
form it keeps (hi, lo) in units of the current weight wc and rescales them when the weight changes,
multiplying by wc once at the end. These tests emulate both orders in numpy float32 (every operation
rounded to nearest, as the f32 and f32x2 instructions are) and check that they give the same bits, and
that the two-float sum is exact against an FP64 reference where it must be.
"""
import numpy as np
import pytest

f32 = np.float32


def two_sum(hi, lo, x):
    s = (hi + x).astype(f32)
    bv = (s - hi).astype(f32)
    e = ((hi - (s - bv).astype(f32)).astype(f32) + (x - bv).astype(f32)).astype(f32)
    return s, (lo + e).astype(f32)


def weighted_first(segs, weights, corr, run_last):
    """The earlier form: every segment's value multiplied by its weight before the TwoSum."""
    hi = (weights[0] * segs[0]).astype(f32)
    lo = np.zeros_like(hi)
    for g in range(len(segs)):
        if g > 0:
            hi, lo = two_sum(hi, lo, (weights[g] * segs[g]).astype(f32))
        if run_last[g]:
            lo = (lo + (weights[g] * corr[g]).astype(f32)).astype(f32)
    return hi, lo


def weight_folded(segs, weights, corr, run_last):
    """The current form: sums in units of the current weight, rescaled exactly when it changes."""
    wc = weights[0]
    hi = segs[0].copy()
    lo = np.zeros_like(hi)
    for g in range(len(segs)):
        if g > 0:
            if weights[g] != wc:
                r = f32(wc / weights[g])
                hi = (hi * r).astype(f32)
                lo = (lo * r).astype(f32)
                wc = weights[g]
            hi, lo = two_sum(hi, lo, segs[g])
        if run_last[g]:
            lo = (lo + corr[g]).astype(f32)
    return (hi * f32(wc)).astype(f32), (lo * f32(wc)).astype(f32)


def _job(rng, nseg, ncol):
    segs = [rng.standard_normal(ncol).astype(f32) * f32(2.0 ** rng.integers(-3, 4)) for _ in range(nseg)]
    corr = [(s * f32(2.0 ** -8) * rng.standard_normal(ncol).astype(f32)).astype(f32) for s in segs]
    # runs of equal weight (the weights of the contraction's q classes: 1 and 2, and the FP16 scale steps)
    weights, run_last = [], []
    w = f32(2.0 ** rng.integers(-2, 3))
    for g in range(nseg):
        weights.append(w)
        change = g + 1 < nseg and rng.random() < 0.2
        run_last.append(change or g == nseg - 1 or rng.random() < 0.3)
        if change:
            w = f32(w * f32(2.0 ** rng.choice([-1, 1, 2])))
    return segs, weights, corr, run_last


@pytest.mark.parametrize("seed", range(8))
def test_weight_folding_gives_the_same_bits(seed):
    rng = np.random.default_rng(seed)
    segs, weights, corr, run_last = _job(rng, int(rng.integers(1, 40)), 256)
    a = weighted_first(segs, weights, corr, run_last)
    b = weight_folded(segs, weights, corr, run_last)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


def test_two_sum_is_error_free():
    """hi + lo carries the exact FP64 sum of FP32 values with no corrections (TwoSum's defining property)."""
    rng = np.random.default_rng(11)
    segs = [rng.standard_normal(4096).astype(f32) * f32(2.0 ** rng.integers(-12, 12)) for _ in range(3)]
    hi, lo = segs[0].copy(), np.zeros(4096, f32)
    for x in segs[1:]:
        hi, lo = two_sum(hi, lo, x)
    exact = sum(x.astype(np.float64) for x in segs)
    # two additions: the low word's own roundings are at most 2^-24 of |lo| each
    err = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - exact)
    assert np.all(err <= 2.0 ** -23 * np.abs(lo.astype(np.float64)) + 1e-300)


def test_two_float_sum_beats_fp32_over_many_segments():
    """Across 450 segments (the NiO-shaped contraction's K = 57 600 in 128-K segments) the two-float sum
    stays near FP64 while a plain FP32 sum drifts by ~sqrt(n) 2^-24."""
    rng = np.random.default_rng(3)
    segs = [rng.standard_normal(2048).astype(f32) for _ in range(450)]
    exact = sum(x.astype(np.float64) for x in segs)
    hi, lo = segs[0].copy(), np.zeros(2048, f32)
    plain = segs[0].copy()
    for x in segs[1:]:
        hi, lo = two_sum(hi, lo, x)
        plain = (plain + x).astype(f32)
    scale = np.abs(exact).max()
    e2 = np.abs(hi.astype(np.float64) + lo - exact).max() / scale
    e1 = np.abs(plain.astype(np.float64) - exact).max() / scale
    assert e2 < 1e-12
    assert e1 > 1e3 * e2
