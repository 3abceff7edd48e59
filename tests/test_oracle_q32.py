"""Pins of the oracle's Q32.32 fixed-point variant (the paper's arithmetic, Section 4.1):
the fixed-point product and exponential against exact integer / 40-digit arithmetic,
the z-scoring of Eq. 3 (scale and shift invariance, Eq. 4 for h), agreement with the
binary64 functional far below the fixed-point resolution's effect, and the error
scale of the paper's Table 4 on h."""
import math

import numpy as np
import pytest

import oracle
import synthdata

mp = pytest.importorskip("mpmath")


def test_product_is_truncated_high_part():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a = int(rng.integers(-(1 << 45), 1 << 45))
        b = int(rng.integers(-(1 << 45), 1 << 45))
        assert oracle.q32_mul(a, b) == (a * b) >> 32      # Python: floor division, exact
    assert oracle.q32_mul(-1, 1) == -1                     # toward minus infinity
    assert oracle.q32_mul(1 << 32, 7 << 32) == 7 << 32


def test_exponential_is_floored_exactly():
    mp.mp.dps = 40
    for w in [0, 1, 12345, 1 << 31, 3 << 32, (25 << 32) // 3, 40 << 32, 44 << 32]:
        ref = int(mp.floor(mp.exp(-mp.mpf(w) / 2 ** 33) * 2 ** 32))
        assert oracle.q32_exp_half(w) == ref, w


@pytest.mark.parametrize("r", [4, 6])
def test_matches_binary64_to_fixed_point_resolution(r):
    x = synthdata.normal_mixture(31, 1000, [0.5, 0.5], [-1.0, 1.0], [0.5, 0.7]) * 3.0 + 7.0
    mean, var = oracle.moments(x)
    g = 0.4 if r == 6 else 0.3
    got, abs_he = oracle.psi_q32(x, r, g, mean, math.sqrt(var))
    ref = oracle.psi(x, r, g)
    # A term He_r(u) e with e = exp(-u^2/2) truncated to 2^-32 is off by at most
    # |He_r(u)| 2^-32, plus ~|He_r|'s own truncations times e and the final product
    # (a few units of 2^-32): sum over the pairs, in the normalisation of Eqs. 6-7.
    n = x.size
    pairs = n * (n - 1) / 2
    bound = 2 * (abs_he + 64 * pairs) * 2.0 ** -32 / (math.sqrt(2 * math.pi) * n * n * g ** (r + 1))
    assert abs(got - ref) <= bound
    assert abs(got - ref) <= 1e-4 * abs(ref)
    assert abs(got - ref) > 0.0                       # the fixed point is really used
    assert abs_he > 0.0


@pytest.mark.parametrize("r", [4, 6])
def test_z_scoring_makes_it_affine_invariant(r):
    """With z = (x - mean)/sigma (Eq. 3) a power-of-two scale and a shift leave every
    Q32.32 value unchanged, so psi scales exactly like the functional does."""
    x = synthdata.student_t3(32, 400)
    m, v = oracle.moments(x)
    a, _ = oracle.psi_q32(x, r, 0.5, m, math.sqrt(v))
    y = 4.0 * x
    m4, v4 = oracle.moments(y)
    b, _ = oracle.psi_q32(y, r, 2.0, m4, math.sqrt(v4))
    assert b == a * 4.0 ** -(r + 1)


@pytest.mark.parametrize("n", [128, 256, 512, 1024])
def test_h_error_is_on_the_scale_of_table_4(n):
    """Table 4 reports relative errors of h between ~3e-8 and ~4e-6 for its Q32.32
    implementations; the same arithmetic on the pair sums lands in that range."""
    x = synthdata.normal(33 + n, n)
    a = oracle.plugin(x)
    b = oracle.plugin_q32(x)
    assert b["status"] == 0
    rel = abs(b["h"] - a["h"]) / a["h"]
    assert 0.0 < rel < 1e-5
