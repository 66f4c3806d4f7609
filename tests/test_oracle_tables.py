"""Pins of the oracle's building blocks: D3Q19 tables, mode basis, Philox.

Each check compares the oracle with something other than itself: the
definition of the velocity set (Sec. 2, Fig. 1a), the isotropy identities of
a lattice with c_s^2 = 1/3, exact rational norms worked out by hand, and an
independent Philox4x32-10 implementation (Triton's, run on the CPU by its
interpreter).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest


def test_velocity_set_is_nearest_and_next_nearest(orc):
    # Sec. 2: 19 vectors including c_0 = 0, connecting a site to its 6 nearest
    # and 12 next-nearest neighbours: exactly the vectors of {-1,0,1}^3 with
    # |c|^2 <= 2.
    c, w = orc.d3q19()
    want = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) <= 2}
    got = {tuple(int(x) for x in row) for row in c}
    assert len(got) == 19 and got == want
    assert tuple(c[0]) == (0, 0, 0)
    # every vector has its opposite in the set
    for row in c:
        assert tuple(-row) in got


def test_weights_isotropy(orc):
    c, w = orc.d3q19()
    cf = c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ cf, 0.0, atol=1e-16)
    second = np.einsum("i,ia,ib->ab", w, cf, cf)
    np.testing.assert_allclose(second, np.eye(3) / 3.0, atol=1e-16)  # c_s^2 = 1/3
    third = np.einsum("i,ia,ib,ic->abc", w, cf, cf, cf)
    np.testing.assert_allclose(third, 0.0, atol=1e-16)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(fourth, iso, atol=1e-16)  # c_s^4 (dd + dd + dd)


def test_mode_basis_orthogonal_with_hand_norms(orc):
    c, w = orc.d3q19()
    e, b = orc.modes()
    # rows 0..3 are the moments of Eqs. (1) and (2)
    np.testing.assert_array_equal(e[0], np.ones(19))
    np.testing.assert_array_equal(e[1:4], c.T.astype(float))
    gram = np.einsum("i,ki,li->kl", w, e, e)
    np.testing.assert_allclose(gram - np.diag(np.diag(gram)), 0.0, atol=1e-15)
    # norms worked out by hand from the weights 1/3, 1/18, 1/36
    F = Fraction
    hand = [F(1), F(1, 3), F(1, 3), F(1, 3), F(2, 3), F(4, 3), F(4, 9), F(1, 9), F(1, 9), F(1, 9),
            F(2, 3), F(2, 3), F(2, 3), F(2, 9), F(2, 9), F(2, 9), F(2), F(4, 3), F(4, 9)]
    np.testing.assert_allclose(b, [float(x) for x in hand], rtol=1e-15)
    np.testing.assert_allclose(np.diag(gram), b, rtol=1e-15)
    # invertibility: f -> m -> f round trip with f_i = w_i sum_k e_ki m_k / b_k
    f = np.linspace(0.01, 0.2, 19)
    m = e @ f
    back = w * (e.T @ (m / b))
    np.testing.assert_allclose(back, f, rtol=1e-13)


def test_uniform_transform(orc):
    # u = (x + 1/2) 2^-32, xi = sqrt(12)(u - 1/2): symmetric about 0, inside
    # (-sqrt 3, sqrt 3), unit variance over the full 32-bit range.
    s3 = np.sqrt(3.0)
    lo = orc.uniform_unit(0)
    hi = orc.uniform_unit(0xFFFFFFFF)
    assert -s3 < lo < -s3 + 1e-9 and s3 - 1e-9 < hi < s3
    assert abs(lo + hi) < 1e-15
    xs = np.arange(0, 2**32, 2**16, dtype=np.uint64) + 2**15
    vals = np.array([orc.uniform_unit(int(x)) for x in xs[::16]])
    assert abs(vals.mean()) < 1e-3
    assert abs((vals ** 2).mean() - 1.0) < 2e-3


def test_uniform16_transform(orc):
    # 16-bit variates: the 65536 levels (h + 1/2) 2^-16 are symmetric about
    # 1/2, so the mean over all levels is exactly 0 and the variance is
    # 1 - 2^-32; only the low 16 bits are used.
    vals = np.array([orc.uniform_unit16(h) for h in range(65536)])
    assert abs(vals.mean()) < 1e-15
    assert abs((vals ** 2).mean() - (1.0 - 2.0 ** -32)) < 1e-12
    assert orc.uniform_unit16(0x12345) == orc.uniform_unit16(0x2345)
    assert vals.min() > -np.sqrt(3.0) and vals.max() < np.sqrt(3.0)


_TRITON_SCRIPT = r"""
import json, sys
import numpy as np
import torch, triton, triton.language as tl

@triton.jit
def kern(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

req = json.loads(sys.stdin.read())
res = []
for seed in req["seeds"]:
    ctr = np.array(req["counters"], dtype=np.uint32)
    n = ctr.shape[0]
    cin = torch.tensor(ctr.view(np.int32).reshape(-1))
    out = torch.zeros(4 * n, dtype=torch.int32)
    kern[(1,)](cin, out, seed, N=n)
    res.append(out.numpy().view(np.uint32).reshape(n, 4).tolist())
print(json.dumps(res))
"""


def _triton_philox(counters, seeds):
    """Philox4x32-10 from Triton's own implementation, run on the CPU by its
    interpreter in a child process (the interpreter must be chosen before
    Triton is first imported)."""
    import json
    import subprocess
    import sys

    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(
        {"counters": [[int(x) for x in c] for c in counters], "seeds": [int(s) for s in seeds]}),
        capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return np.array(json.loads(out.stdout.strip().splitlines()[-1]), dtype=np.uint64)


def test_philox_matches_independent_implementation(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    counters = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [12345, 678, 0, 3], [5, 2**31, 1, 0]]
    counters += [list(x) for x in rng.integers(0, 2**32, size=(11, 4), dtype=np.uint64)]
    seeds = (1, 0x1234567890ABCDEF, 2**64 - 1)
    refs = _triton_philox(counters, seeds)
    for seed, ref in zip(seeds, refs):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for ctr, want in zip(counters, ref):
            got = orc.philox4x32_10(ctr, key)
            np.testing.assert_array_equal(got, want)


def test_philox_outputs_look_uniform(orc):
    # weak statistical sanity on 4096 outputs (bit balance, no stuck lanes)
    outs = np.array([orc.philox4x32_10([i, 7, 0, 0], [1, 0]) for i in range(1024)], dtype=np.uint64)
    bits = ((outs[..., None] >> np.arange(32, dtype=np.uint64)) & 1).astype(float)
    frac = bits.mean(axis=(0, 1))
    assert np.all(np.abs(frac - 0.5) < 0.04)
