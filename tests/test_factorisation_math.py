"""The mathematics the binary32 pair kernel rests on, checked on the CPU.

- The factorisation of the pair Gaussian over a tile pair: with a_i = a0 + alpha_i,
  b_j = b0 + beta_j and Delta = a0 - b0,
      exp(-(a_i - b_j)^2 / 2) = R_i C_j exp(alpha_i beta_j),
      R_i = exp(-alpha_i (Delta + alpha_i / 2)),
      C_j = exp(beta_j (Delta - beta_j / 2) - Delta^2 / 2),
  exactly (checked in 50-digit arithmetic).
- The truncation of the coupling factor exp(p) by 1 + p (|p| <= 4e-6) and by
  1 + p + p^2/2 (|p| <= 1e-3): relative errors at most p^2/2 = 8.0e-12 and p^3/6 =
  1.7e-10 (to first order; the checks allow the next order).
- The degree-8 polynomial for 2^f on [-1/2, 1/2] in the kernel source, with its
  coefficients as the kernel holds them (binary32) and evaluated exactly: relative
  error at most 1.3e-9 and mean error below 2e-10 in size.  The polynomial itself
  (coefficients of unlimited precision) is good to about 1e-12; storing the linear
  coefficient ln 2 in binary32 moves it by d = 1.9e-9 (2.7e-9 relative), so the
  relative error is close to d f 2^-f, largest (1.3e-9) at f = -1/2.  A binary32 FMA
  evaluation adds its own rounding (2^-24 per step) on top of this.
- The shifted Hermite forms the factorised path evaluates straight from u:
  He_4 = (u^2 - 3)^2 - 6 and He_6 = ((u^2 - 5)^2 - 30)(u^2 - 5) - 40, against the
  probabilists' Hermite polynomials of numpy's HermiteE basis, with the shifts and
  constants read from the kernel source; and their binary32 evaluation (emulated
  with exact products, one rounding per FMA) unbiased and within 1e-6 of the
  largest term.
"""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNELS = os.path.join(ROOT, "paper_1505_02100_gb300", "csrc", "kde_kernels.cu")


def test_factorisation_identity_is_exact():
    mpmath.mp.dps = 50
    rng = np.random.default_rng(11)
    for _ in range(200):
        a0, b0 = (mpmath.mpf(float(v)) for v in rng.uniform(-20, 20, 2))
        alpha, beta = (mpmath.mpf(float(v)) for v in rng.uniform(-0.5, 0.5, 2))
        delta = a0 - b0
        u = (a0 + alpha) - (b0 + beta)
        lhs = mpmath.exp(-u * u / 2)
        R = mpmath.exp(-alpha * (delta + alpha / 2))
        C = mpmath.exp(beta * (delta - beta / 2) - delta * delta / 2)
        rhs = R * C * mpmath.exp(alpha * beta)
        assert abs(lhs - rhs) <= mpmath.mpf(10) ** -40 * lhs


@pytest.mark.parametrize("order,pmax,bound", [(1, 4.0e-6, 8.01e-12), (2, 1.0e-3, 1.67e-10)])
def test_coupling_truncation_bounds(order, pmax, bound):
    mpmath.mp.dps = 40
    worst = mpmath.mpf(0)
    for k in range(-200, 201):
        p = mpmath.mpf(pmax) * k / 200
        series = 1 + p + (p * p / 2 if order == 2 else 0)
        worst = max(worst, abs(mpmath.exp(p) - series) / mpmath.exp(p))
    assert worst <= bound, worst
    # and the bound is reached at the edge, so the kernel's thresholds are the binding ones
    assert worst >= bound / 2


def _exp2_coefficients():
    src = open(KERNELS).read()
    body = re.search(r"float exp2_reduced\(float f\) \{(.*?)\n\}", src, re.S).group(1)
    nums = re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)
    return [Fraction(float(np.float32(v))) for v in nums]   # highest power first, binary32 values


def test_exp2_polynomial_accuracy_on_the_reduced_range():
    coeffs = _exp2_coefficients()
    assert len(coeffs) == 8                 # q(f) of degree 7, then 2^f ~ q(f) f + 1: degree 8
    mpmath.mp.dps = 40
    errs = []
    for k in range(-512, 513):
        f = Fraction(k, 1024)
        q = coeffs[0]
        for c in coeffs[1:]:
            q = q * f + c
        p = q * f + 1
        exact = mpmath.power(2, mpmath.mpf(f.numerator) / f.denominator)
        errs.append(float((mpmath.mpf(p.numerator) / p.denominator - exact) / exact))
    errs = np.array(errs)
    assert errs[512] == 0.0                 # p(0) = 1 exactly
    assert np.abs(errs).max() <= 1.3e-9, np.abs(errs).max()
    assert abs(errs.mean()) <= 2e-10, errs.mean()
    # the linear coefficient is ln 2 rounded to binary32; that rounding sets the error's size
    c1 = coeffs[-1]
    assert c1 == Fraction(float(np.float32(np.log(2.0))))
    dc1 = float(c1) - float(mpmath.log(2))
    model = abs(dc1) * 0.5 * 2.0 ** 0.5             # |d f 2^-f| at f = -1/2
    assert 0.9 * model <= np.abs(errs).max() <= 1.05 * model


def _hermite_u_constants():
    src = open(KERNELS).read()
    body = re.search(r"float hermite_u\(float u\) \{(.*?)\n\}", src, re.S).group(1)
    blocks = {}
    for r, blk in re.findall(r"if \(RORD == (\d+)\) \{(.*?)\n  \}", body, re.S):
        blocks[int(r)] = [float(v) for v in re.findall(r"(-?\d+\.\d+)f", blk)]
    return blocks


def _shifted(r, c, u):
    """The kernel's evaluation order in exact rational arithmetic."""
    t = u * u + Fraction(c[0])
    if r == 4:
        return t * t + Fraction(c[1])
    return (t * t + Fraction(c[1])) * t + Fraction(c[2])


def test_shifted_hermite_forms_are_the_hermite_polynomials():
    from numpy.polynomial import hermite_e as H
    consts = _hermite_u_constants()
    assert consts == {4: [-3.0, -6.0], 6: [-5.0, -30.0, -40.0]}
    for r in (4, 6):
        power = [Fraction(int(round(v))) for v in H.herme2poly([0] * r + [1])]
        assert all(Fraction(v) == p for v, p in zip(H.herme2poly([0] * r + [1]), power))
        for k in range(-40, 41):                      # degree r: r + 1 points fix it; use 81
            u = Fraction(k, 7)
            want = sum(p * u ** i for i, p in enumerate(power))
            assert _shifted(r, consts[r], u) == want, (r, u)


def _f32_fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c).astype(np.float32)


@pytest.mark.parametrize("r", [4, 6])
def test_shifted_hermite_binary32_error(r):
    from numpy.polynomial import hermite_e as H
    c = _hermite_u_constants()[r]
    u = np.random.default_rng(5).uniform(0.0, 9.0, 2_000_000).astype(np.float32)
    t = _f32_fma(u, u, c[0])                           # u*u is exact in binary64
    h = _f32_fma(t, t, c[1]) if r == 4 else _f32_fma(_f32_fma(t, t, c[1]), t, c[2])
    ud = u.astype(np.float64)
    exact = H.hermeval(ud, [0] * r + [1])
    g = np.exp(-ud * ud / 2)
    err = (h.astype(np.float64) - exact) * g
    scale = np.abs(exact * g).max()
    assert np.abs(err).max() <= 1e-6 * scale, np.abs(err).max() / scale
    # unbiased: the mean is within a few standard errors of zero
    assert abs(err.mean()) <= 5 * err.std() / np.sqrt(err.size)
