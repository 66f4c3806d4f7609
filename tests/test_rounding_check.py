"""The comparison the reduced-precision GPU tests use (gpu_common's
expected_readback / assert_rounded_like_oracle), exercised on the CPU: a
stand-in for the GPU that rounds a slightly perturbed value (FP32-sized
errors) with the right rule passes, one that rounds to nearest where
stochastic rounding is wanted (or the reverse), or with another node's random
bits, fails."""
import numpy as np
import pytest

from gpu_common import W, assert_rounded_like_oracle, expected_readback

PRECISIONS = ["fp16dev", "fp16dev_sr", "bf16dev", "bf16dev_sr"]


def _case(seed, n=20000):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, 19, n)
    post = W[i] * (1 + 0.02 * rng.standard_normal(n))
    src = rng.integers(0, 5000, n)
    noisy = post + 4 * np.spacing(post.astype(np.float32)).astype(np.float64) * rng.standard_normal(n)
    return i, post, src, noisy


@pytest.mark.parametrize("precision", PRECISIONS)
def test_the_right_rounding_passes(precision):
    i, post, src, noisy = _case(1)
    want, step, dist = expected_readback(post, i, src, precision, 1234, 0)
    got, _, _ = expected_readback(noisy, i, src, precision, 1234, 0)
    assert assert_rounded_like_oracle(got, want, step, dist) > 0.9


@pytest.mark.parametrize("precision", PRECISIONS)
def test_the_other_rounding_mode_fails(precision):
    i, post, src, noisy = _case(2)
    want, step, dist = expected_readback(post, i, src, precision, 1234, 0)
    other = precision[:-3] if precision.endswith("_sr") else precision + "_sr"
    bad, _, _ = expected_readback(noisy, i, src, other, 1234, 0)
    with pytest.raises(AssertionError):
        assert_rounded_like_oracle(bad, want, step, dist)


@pytest.mark.parametrize("precision", ["fp16dev_sr", "bf16dev_sr"])
def test_other_random_bits_fail(precision):
    i, post, src, noisy = _case(3)
    want, step, dist = expected_readback(post, i, src, precision, 1234, 0)
    for bad_src, seed, step_no in ((src + 1, 1234, 0), (src, 1235, 0), (src, 1234, 1)):
        bad, _, _ = expected_readback(noisy, i, bad_src, precision, seed, step_no)
        with pytest.raises(AssertionError):
            assert_rounded_like_oracle(bad, want, step, dist)
