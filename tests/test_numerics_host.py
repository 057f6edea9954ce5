"""Host checks of the arithmetic the tensor kernels rely on (no GPU).

The 3xTF32 products split every FP32 value x into a head rounded to TF32 and
an exact tail (Ootomo and Yokota, IJHPCA 2022).  The kernels round the head
with an integer trick on the bit pattern (add half a TF32 unit to the
magnitude bits, clear the low 13 bits); these tests check, over random and
edge-case bit patterns, that this is round-to-nearest with ties away from
zero to 10 fraction bits and that the tail is exact, using float64 arithmetic
that is independent of the trick."""
import numpy as np


def _trick(x32):
    b = x32.view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def _reference(x32):
    """Nearest value with 11 significant bits (10 fraction bits), ties away
    from zero, computed in float64 from the value itself."""
    x = x32.astype(np.float64)
    a = np.abs(x)
    out = np.zeros_like(x)
    nz = a > 0
    e = np.floor(np.log2(a[nz]))
    e = np.maximum(e, -126.0)                  # below FP32's normal range the spacing stays 2^-136
    q = np.exp2(e - 10.0)                      # TF32 spacing at this binade
    r = np.floor(a[nz] / q + 0.5) * q          # exact in float64
    out[nz] = np.sign(x[nz]) * r
    return out


def test_tf32_head_is_round_to_nearest_ties_away():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2 ** 32, size=400_000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < np.float32(3.0e38))]
    # exact ties and neighbours of binade edges
    ties = (np.arange(1, 2000, dtype=np.uint32) << np.uint32(13)) | np.uint32(0x1000)
    edges = np.array([0x3F7FF000, 0x3F7FEFFF, 0x3F7FF001, 0x00001000, 0x00800000, 0x007FF000],
                     dtype=np.uint32)
    x = np.concatenate([x, (ties + np.uint32(0x3F800000)).view(np.float32),
                        (ties + np.uint32(0x3F800000) | np.uint32(0x80000000)).view(np.float32),
                        edges.view(np.float32)])
    hi = _trick(x)
    np.testing.assert_array_equal(hi.astype(np.float64), _reference(x))


def test_tf32_tail_is_exact():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200_000) * np.exp2(rng.integers(-60, 60, 200_000))).astype(np.float32)
    hi = _trick(x)
    lo = (x - hi).astype(np.float32)
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), x.astype(np.float64))
    # the tail is at most half a TF32 unit of the head's binade
    big = np.abs(x) > 1e-30
    assert np.all(np.abs(lo[big]) <= np.abs(x[big]) * 2.0 ** -11 * 1.0000001)
