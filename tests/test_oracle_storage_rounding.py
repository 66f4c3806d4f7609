"""Pins of the oracle's reduced-precision storage rounding (an extension of
the method: the populations' deviations from rest stored as FP16 / BF16).

Round to nearest is pinned to numpy's float16 conversion and torch's
bfloat16 conversion (both IEEE round-to-nearest-even), over normal and
subnormal magnitudes, both signs and exact ties.  Stochastic rounding is
pinned by brute force over all 65536 random numbers: every result is one of
the two grid neighbours, grid values are left unchanged, and the mean over r
is the input itself (unbiased rounding) wherever the input's fraction of a
grid step is a multiple of 2^-16, as for every FP32 input in the normal
range.
"""
import numpy as np
import pytest

from oracle import oracle as orc


def _fp32_samples(rng, n, lo_exp, hi_exp):
    mag = np.exp2(rng.uniform(lo_exp, hi_exp, n))
    x = (mag * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    return x.astype(np.float64)


def test_nearest_fp16_matches_numpy():
    rng = np.random.default_rng(1)
    # normal and subnormal FP16 magnitudes (2^-24 .. 2^-14 .. 2^10)
    x = np.concatenate([_fp32_samples(rng, 20000, -26, 10), rng.standard_normal(2000) * 1e-3])
    want = x.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(orc.round_storage(x, "fp16"), want)


def test_nearest_fp16_ties_go_to_even():
    k = np.arange(0, 2048, dtype=np.float64)
    for scale in (2.0 ** -24, 2.0 ** -20, 2.0 ** -3):  # subnormal and normal steps
        x = (2 * k + 1) * scale / 2  # exactly half-way between grid values
        x = x[np.abs(x) < 65504]
        np.testing.assert_array_equal(orc.round_storage(x, "fp16"), x.astype(np.float16).astype(np.float64))


def test_nearest_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([_fp32_samples(rng, 20000, -140, 20), rng.standard_normal(2000) * 1e-3])
    # exact ties: FP32 values whose low 16 bits are 0x8000
    bits = (rng.integers(0x30000000, 0x40000000, 500, dtype=np.uint32) & np.uint32(0xffff0000)) | np.uint32(0x8000)
    x = np.concatenate([x, bits.view(np.float32).astype(np.float64)])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(orc.round_storage(x, "bf16"), want)


def _neighbours(x, fmt):
    """The two grid values around x (towards and away from zero), by a
    route other than the oracle's: a sorted table of all positive finite
    grid values, built from the format's bit patterns."""
    if fmt == "fp16":
        grid = np.arange(0, 0x7c00, dtype=np.uint16).view(np.float16).astype(np.float64)
    else:
        torch = pytest.importorskip("torch")
        b = np.arange(0, 0x7f80, dtype=np.int32).astype(np.int16)
        grid = torch.from_numpy(b).view(torch.bfloat16).to(torch.float64).numpy()
    a = np.abs(x)
    i = np.searchsorted(grid, a, side="right") - 1
    lo = grid[i]
    hi = np.where(grid[i] == a, grid[i], grid[np.minimum(i + 1, grid.size - 1)])
    return np.sign(x) * lo, np.sign(x) * hi


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_stochastic_is_unbiased_over_all_random_numbers(fmt):
    rng = np.random.default_rng(3)
    lo_exp = -13 if fmt == "fp16" else -120  # the normal range of the format
    x = _fp32_samples(rng, 300, lo_exp, 8)
    r = np.arange(65536, dtype=np.uint32)
    lo, hi = _neighbours(x, fmt)
    for k in range(x.size):
        y = orc.round_storage(np.full(65536, x[k]), fmt, r)
        assert np.all((y == lo[k]) | (y == hi[k])), x[k]
        assert y.mean() == x[k], (x[k], y.mean())
        # rounding away from zero exactly for the smallest r
        away = np.abs(y) > np.abs(lo[k])
        n_away = int(away.sum())
        assert np.all(away[:n_away]) and not np.any(away[n_away:])


def test_stochastic_fp16_subnormal_step():
    # 3.25 steps of 2^-24: 4 steps for r < 2^14, else 3
    x = np.full(65536, 3.25 * 2.0 ** -24)
    y = orc.round_storage(x, "fp16", np.arange(65536, dtype=np.uint32))
    assert np.all(y[:16384] == 4 * 2.0 ** -24) and np.all(y[16384:] == 3 * 2.0 ** -24)
    # a deviation below the smallest subnormal: 0 or the smallest subnormal,
    # with mean within 2^-16 of a step of x
    x = np.full(65536, 0.3 * 2.0 ** -24)
    y = orc.round_storage(x, "fp16", np.arange(65536, dtype=np.uint32))
    assert set(np.unique(y)) <= {0.0, 2.0 ** -24}
    assert abs(y.mean() - x[0]) <= 2.0 ** -24 * 2.0 ** -16


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_stochastic_keeps_grid_values_and_is_odd(fmt):
    rng = np.random.default_rng(4)
    x = orc.round_storage(rng.standard_normal(5000) * 1e-3, fmt)  # grid values
    r = rng.integers(0, 65536, x.size, dtype=np.uint32)
    np.testing.assert_array_equal(orc.round_storage(x, fmt, r), x)
    z = rng.standard_normal(5000) * 1e-3
    np.testing.assert_array_equal(orc.round_storage(-z, fmt, r), -orc.round_storage(z, fmt, r))
    assert orc.round_storage(np.zeros(3), fmt, r[:3]).tolist() == [0.0, 0.0, 0.0]


def test_random_bits_layout():
    # population i: Philox call i / 8 of counter (node, step, 2, i / 8), word
    # (i / 2) mod 4, low half for even i
    seed = (7 << 32) | 12345
    nodes = np.array([0, 1, 4095, 2 ** 24 + 3], dtype=np.uint32)
    got = orc.sr_bits(seed, nodes, 17)
    for k, node in enumerate(nodes):
        words = [orc.philox4x32_10([int(node), 17, 2, q], [12345, 7]) for q in range(3)]
        for i in range(19):
            w = int(words[i // 8][(i // 2) % 4])
            assert got[k, i] == ((w & 0xffff) if i % 2 == 0 else (w >> 16))
    # distinct from the fluid-noise stream (counter word 2 = 0)
    assert not np.array_equal(orc.philox4x32_10([0, 17, 0, 0], [12345, 7]), orc.philox4x32_10([0, 17, 2, 0], [12345, 7]))
