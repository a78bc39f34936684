"""The branch-free projection rounds a column by one FP32 addition: for a
power-of-two width W = 2^k and turns t in [-1/2, 1/2], the pattern of
t + 1.5 * 2^(23 - k) (FP32, round to nearest even) ends in round(t * W) mod W
(ties to even), and NaN gives 0.  This is an identity of IEEE FP32
arithmetic, checked here with numpy's float32 addition (the GPU's FADD rounds
the same way); the GPU parity tests check the kernels themselves."""
import numpy as np
import pytest


@pytest.mark.parametrize("k", [4, 7, 8, 9, 10, 11, 12, 13])
def test_one_addition_rounding_is_round_half_even_mod_w(k):
    W = 1 << k
    magic = np.float32(1.5 * 2.0 ** 23 / W)
    rng = np.random.default_rng(k)
    t = rng.uniform(-0.5, 0.5, 100000).astype(np.float32)
    ties = ((np.arange(-W // 2, W // 2) + 0.5) / W).astype(np.float32)        # exact half columns
    near = np.nextafter(ties, np.float32(1.0))                                  # one ulp above a tie
    edges = np.float32([0.5, -0.5, 0.0, -0.0, 1.0 / W, -1.0 / W])
    t = np.concatenate([t, ties, near, edges])
    u = (t + magic).astype(np.float32).view(np.int32) & (W - 1)
    ref = np.mod(np.rint(t.astype(np.float64) * W).astype(np.int64), W)
    np.testing.assert_array_equal(u, ref)
    nan = np.array([np.float32(np.nan) + magic], np.float32).view(np.int32)[0] & (W - 1)
    assert nan == 0
