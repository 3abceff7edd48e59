"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values printed
in Algorithm 1 (golden fixtures), derivatives taken numerically at 40 digits,
integral identities, exact rational arithmetic, invariances, a long double brute
force, and closed-form expectations for normal data.  A dropped term, a wrong
sign, index or exponent, or a mishandled diagonal in the oracle fails at least
one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthdata
from conftest import read_golden_table

mp = pytest.importorskip("mpmath")


def _constants():
    return {row[0]: eval(row[1], {"math": math}) for row in read_golden_table("algorithm1_constants.txt")}


def _mp_phi(u):
    return mp.exp(-u * u / 2) / mp.sqrt(2 * mp.pi)


# --------------------------------------------------------------------------
# Kernel derivatives K^(r) (Algorithm 1, Steps IV and VI)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [4, 6, 8, 10])
@pytest.mark.parametrize("u", [0.0, 0.3, -1.0, 1.7, 2.5, -4.0, 6.25, 9.0])
def test_kernel_deriv_is_rth_derivative_of_gaussian(r, u):
    """K^(r)(u) equals d^r/du^r of the Gaussian kernel, taken numerically (no Hermite form)."""
    mp.mp.dps = 40
    ref = float(mp.diff(_mp_phi, mp.mpf(u), r))
    got = oracle.kernel_deriv(r, u)
    assert abs(got - ref) <= 1e-14 * max(abs(ref), 1e-3 * math.exp(-u * u / 2)) + 1e-300


def test_kernel_deriv_at_zero_matches_printed_constants():
    """K^(6)(0) and K^(4)(0) as printed in Steps III and V."""
    c = _constants()
    assert oracle.kernel_deriv(6, 0.0) == pytest.approx(c["K6_0"], rel=1e-15)
    assert oracle.kernel_deriv(4, 0.0) == pytest.approx(c["K4_0"], rel=1e-15)


def test_printed_polynomials_are_hermite_derivatives():
    """The golden polynomial coefficients (Steps IV, VI) reproduce the numerical derivative."""
    mp.mp.dps = 40
    for row in read_golden_table("kernel_polynomials.txt"):
        r = int(row[0])
        coef = [float(v) for v in row[1].split()]
        for u in (0.2, 1.1, 2.9):
            p = np.polyval(coef, u) * math.exp(-u * u / 2) / math.sqrt(2 * math.pi)
            assert p == pytest.approx(float(mp.diff(_mp_phi, mp.mpf(u), r)), rel=1e-13, abs=1e-16)


@pytest.mark.parametrize("r", [4, 6, 8, 10])
def test_kernel_deriv_moment_identities(r):
    """Integration by parts: int K^(r) = 0 and int u^r K^(r)(u) du = r! for even r."""
    from scipy.integrate import quad
    f0, _ = quad(lambda u: oracle.kernel_deriv(r, u), -40, 40, limit=400, epsabs=1e-13)
    fr, _ = quad(lambda u: u ** r * oracle.kernel_deriv(r, u), -40, 40, limit=400, epsabs=1e-11)
    assert abs(f0) < 1e-11
    assert fr == pytest.approx(math.factorial(r), rel=1e-10)


# --------------------------------------------------------------------------
# The functional psi_r(g) (Steps IV and VI, Eqs. 6-7)
# --------------------------------------------------------------------------

def _psi_by_derivative(x, r, g):
    """psi_r(g) = d^r/dt^r of n^-2 sum_ij phi_g(t + X_i - X_j) at t = 0, phi_g(y) = phi(y/g)/g.

    This uses only the Gaussian itself: no Hermite polynomial, no g^-(r+1) factor and
    no separate diagonal term.
    """
    mp.mp.dps = 40
    xs = [mp.mpf(float(v)) for v in x]
    gg = mp.mpf(float(g))
    n = len(xs)
    d = [xi - xj for xi in xs for xj in xs]

    def F(t):
        return mp.fsum(_mp_phi((t + dij) / gg) for dij in d) / (gg * n * n)

    return float(mp.diff(F, mp.mpf(0), r))


@pytest.mark.parametrize("form", [oracle.FORM_FULL, oracle.FORM_SYMMETRIC])
@pytest.mark.parametrize("r", [4, 6, 8, 10])
@pytest.mark.parametrize("case", ["two", "three", "toy8"])
def test_psi_equals_rth_derivative_of_pair_density(form, r, case, toy8):
    x = {"two": [0.0, 1.0], "three": [0.0, 1.0, 3.0], "toy8": list(toy8)}[case]
    for g in (0.37, 1.0, 2.3):
        ref = _psi_by_derivative(x, r, g)
        assert oracle.psi(x, r, g, form=form, threads=1) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("r", [4, 6, 8, 10])
def test_psi_is_integral_of_squared_kde_derivative(r, toy8):
    """Convolution identity: psi_r(sqrt(2) b) = (-1)^(r/2) int (f_b^(r/2)(x))^2 dx,
    f_b the Gaussian KDE of the data with bandwidth b (Eq. 1)."""
    from scipy.integrate import quad
    x = np.asarray(toy8)
    b = 0.6
    k = r // 2
    n = x.size
    mp.mp.dps = 30

    def fk(t):
        # derivative of order k of the KDE, taken numerically at 30 digits
        return float(mp.diff(lambda s: mp.fsum(_mp_phi((s - mp.mpf(float(xi))) / b)
                                               for xi in x) / (n * b), mp.mpf(t), k))

    integral, _ = quad(lambda t: fk(t) ** 2, x.min() - 12 * b, x.max() + 12 * b, limit=200,
                       epsabs=1e-14, epsrel=1e-11)
    ref = (-1) ** k * integral
    assert oracle.psi(x, r, math.sqrt(2) * b, threads=1) == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("r", [4, 6, 8, 10])
def test_full_and_symmetric_forms_agree(r):
    """Step IV/VI printed double sum vs Eqs. (6)-(7) (2 * sum_{i<j} + n K^(r)(0))."""
    x = synthdata.normal(11, 700) * 1.7 + 0.3
    g = 0.41
    a = oracle.psi(x, r, g, form=oracle.FORM_FULL)
    b = oracle.psi(x, r, g, form=oracle.FORM_SYMMETRIC)
    assert a == pytest.approx(b, rel=1e-13)


@pytest.mark.parametrize("n", [2, 5, 17, 64])
def test_long_double_brute_force_agrees(n):
    x = synthdata.normal(100 + n, n) * 3.0 + 1e4
    ref = oracle.plugin_ld(x)
    got = oracle.plugin(x)
    assert got["status"] == oracle.OK == ref["status"]
    for k in ("sigma", "psi8", "g1", "psi6", "g2", "psi4", "h"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12), k
    for r, g in ((6, got["g1"]), (4, got["g2"])):
        assert oracle.psi(x, r, g, form=oracle.FORM_FULL) == pytest.approx(
            oracle.psi_ld(x, r, g), rel=1e-13)


def test_long_double_is_wider_than_double():
    assert oracle.long_double_bits() >= 64


def test_thread_count_does_not_change_bits():
    x = synthdata.student_t3(5, 3001)
    a = oracle.psi(x, 6, 0.3, threads=1)
    b = oracle.psi(x, 6, 0.3, threads=7)
    assert a == b


@pytest.mark.parametrize("r", [4, 6])
def test_block_sums_partition_the_triangle(r):
    """Blocks of the i<j triangle add up to the off-diagonal sum of Eq. (6)/(7)."""
    n, g = 301, 0.55
    x = synthdata.normal(21, n)
    edges = [0, 90, 200, n]
    tot = 0.0
    for a in range(3):
        for b in range(a, 3):
            s, t = oracle.psi_block(x, edges[a], edges[a + 1], edges[b], edges[b + 1], r, g)
            assert t >= abs(s)
            tot += s
    psi = oracle.psi(x, r, g)
    off = (psi * n * n * g ** (r + 1) - n * oracle.kernel_deriv(r, 0.0)) / 2
    assert tot == pytest.approx(off, rel=1e-12)


# --------------------------------------------------------------------------
# Algorithm 1 end to end
# --------------------------------------------------------------------------

def test_step1_moments_exact_rational():
    """Step I (unbiased variance, divisor n-1) against exact rational arithmetic."""
    x = synthdata.normal(3, 50) * 2.5 + 1e4
    fx = [Fraction(float(v)) for v in x]
    mean = sum(fx) / len(fx)
    var = sum((v - mean) ** 2 for v in fx) / (len(fx) - 1)
    m, v = oracle.moments(x)
    assert m == pytest.approx(float(mean), rel=1e-15)
    assert v == pytest.approx(float(var), rel=1e-13)
    assert v == pytest.approx(np.var(x, ddof=1), rel=1e-12)


def test_step2_psi8_is_normal_scale_functional():
    """Step II: psi8^NS = int (f^(4))^2 dx for the N(0, sigma^2) density."""
    x = synthdata.normal(8, 257) * 0.8
    res = oracle.plugin(x)
    s = mp.mpf(res["sigma"])
    mp.mp.dps = 30

    def f(t):
        return mp.exp(-t * t / (2 * s * s)) / (s * mp.sqrt(2 * mp.pi))

    val = mp.quad(lambda t: mp.diff(f, t, 4) ** 2, [-mp.inf, 0, mp.inf])
    assert res["psi8"] == pytest.approx(float(val), rel=1e-12)


def test_pilot_bandwidths_cancel_leading_bias():
    """Steps III and V choose g so that the two leading bias terms of psi_r cancel:
    n^-1 g^-(r+1) K^(r)(0) + g^2 mu2 psi_{r+2} / 2 = 0, with K^(r)(0) and
    mu2 = int u^2 K(u) du taken numerically."""
    from scipy.integrate import quad
    mp.mp.dps = 40
    mu2 = quad(lambda u: u * u * math.exp(-u * u / 2) / math.sqrt(2 * math.pi), -40, 40)[0]
    k6 = float(mp.diff(_mp_phi, 0, 6))
    k4 = float(mp.diff(_mp_phi, 0, 4))
    x = synthdata.normal(9, 500)
    n = x.size
    res = oracle.plugin(x)
    t1 = k6 / (n * res["g1"] ** 7)
    assert t1 + 0.5 * res["g1"] ** 2 * mu2 * res["psi8"] == pytest.approx(0.0, abs=1e-12 * abs(t1))
    t2 = k4 / (n * res["g2"] ** 5)
    assert t2 + 0.5 * res["g2"] ** 2 * mu2 * res["psi6"] == pytest.approx(0.0, abs=1e-12 * abs(t2))


def test_step7_h_minimises_amise():
    """Step VII: h is the stationary point of AMISE(h) = R(K)/(n h) + h^4 mu2^2 psi4 / 4,
    with R(K) = int K^2 taken numerically."""
    from scipy.integrate import quad
    from scipy.optimize import minimize_scalar
    RK = quad(lambda u: math.exp(-u * u) / (2 * math.pi), -40, 40)[0]
    x = synthdata.normal(10, 400)
    n = x.size
    res = oracle.plugin(x)
    h, psi4 = res["h"], res["psi4"]
    assert -RK / (n * h * h) + h ** 3 * psi4 == pytest.approx(0.0, abs=1e-12 * RK / (n * h * h))
    opt = minimize_scalar(lambda hh: RK / (n * hh) + hh ** 4 * psi4 / 4, bounds=(h / 4, 4 * h),
                          method="bounded", options={"xatol": 1e-10})
    assert opt.x == pytest.approx(h, rel=1e-6)


def test_toy8_chain_with_independent_functionals(toy8):
    """Whole chain on the toy dataset: Step I exact, Steps IV/VI by the derivative identity,
    scalar steps with the printed constants."""
    c = _constants()
    x = list(toy8)
    n = len(x)
    fx = [Fraction(v) for v in x]
    mean = sum(fx) / n
    sigma = math.sqrt(float(sum((v - mean) ** 2 for v in fx) / (n - 1)))
    psi8 = c["PSI8_NS_COEF"] / sigma ** 9
    g1 = (-2 * c["K6_0"] / (c["MU2"] * psi8 * n)) ** (1 / 9)
    psi6 = _psi_by_derivative(x, 6, g1)
    g2 = (-2 * c["K4_0"] / (c["MU2"] * psi6 * n)) ** (1 / 7)
    psi4 = _psi_by_derivative(x, 4, g2)
    h = (c["RK"] / (c["MU2"] ** 2 * psi4 * n)) ** (1 / 5)
    res = oracle.plugin(np.array(x))
    for k, v in dict(sigma=sigma, psi8=psi8, g1=g1, psi6=psi6, g2=g2, psi4=psi4, h=h).items():
        assert res[k] == pytest.approx(v, rel=1e-13), k


def _dyadic(z, bits=20):
    return np.round(z * 2.0 ** bits) / 2.0 ** bits


@pytest.mark.parametrize("b", [1e4, -3.5])
def test_translation_invariance(b):
    x = _dyadic(synthdata.normal(12, 600))
    h0 = oracle.plugin(x)["h"]
    assert oracle.plugin(x + b)["h"] == pytest.approx(h0, rel=1e-13)


@pytest.mark.parametrize("a", [2.0 ** -3, 2.0 ** 5, -1.0, 3.0])
def test_scale_equivariance(a):
    """h(a X) = |a| h(X): catches any wrong exponent among Steps II-VII."""
    x = synthdata.lognormal(13, 500)
    r0 = oracle.plugin(x)
    r1 = oracle.plugin(a * x)
    assert r1["h"] == pytest.approx(abs(a) * r0["h"], rel=1e-13)
    assert r1["g1"] == pytest.approx(abs(a) * r0["g1"], rel=1e-13)
    assert r1["psi6"] == pytest.approx(abs(a) ** -7 * r0["psi6"], rel=1e-12)
    assert r1["psi4"] == pytest.approx(abs(a) ** -5 * r0["psi4"], rel=1e-12)


def test_permutation_invariance():
    x = synthdata.normal_mixture(14, 800, [0.3, 0.7], [-2, 1], [0.5, 1.0])
    perm = np.argsort(synthdata.uniform(15, x.size))
    assert oracle.plugin(x[perm])["h"] == pytest.approx(oracle.plugin(x)["h"], rel=1e-13)


@pytest.mark.parametrize("family", ["normal", "t3", "lognormal", "uniform", "bimodal"])
def test_signs_psi6_negative_psi4_positive(family):
    n = 1500
    x = {"normal": lambda: synthdata.normal(16, n),
         "t3": lambda: synthdata.student_t3(17, n),
         "lognormal": lambda: synthdata.lognormal(18, n),
         "uniform": lambda: synthdata.uniform(19, n),
         "bimodal": lambda: synthdata.bimodal_offset(n, 20)}[family]()
    res = oracle.plugin(x)
    assert res["status"] == oracle.OK
    assert res["psi6"] < 0 < res["psi4"]


@pytest.mark.parametrize("r,g", [(4, 0.4), (6, 0.5)])
def test_expectation_for_normal_data(r, g):
    """E psi_r(g) = K^(r)(0) [n^-1 g^-(r+1) + (1 - n^-1)(g^2 + 2 sigma^2)^(-(r+1)/2)]
    for N(mu, sigma^2) data (X_i - X_j ~ N(0, 2 sigma^2); Gaussian convolution)."""
    n, sigma, reps = 1000, 1.3, 30
    k0 = oracle.kernel_deriv(r, 0.0)
    expect = k0 * (1 / (n * g ** (r + 1)) + (1 - 1 / n) * (g * g + 2 * sigma ** 2) ** (-(r + 1) / 2))
    vals = np.array([oracle.psi(sigma * synthdata.normal(1000 + s, n) + 2.0, r, g)
                     for s in range(reps)])
    se = vals.std(ddof=1) / math.sqrt(reps)
    assert abs(vals.mean() - expect) < 4 * se + 1e-3 * abs(expect)


def test_h_approaches_normal_reference_bandwidth():
    """For normal data h tends to the AMISE-optimal (4/(3n))^(1/5) sigma."""
    n = 12000
    ratios = []
    for s in range(2):
        x = 2.0 * synthdata.normal(2000 + s, n)
        res = oracle.plugin(x)
        ratios.append(res["h"] / ((4 / (3 * n)) ** 0.2 * 2.0))
    assert np.mean(ratios) == pytest.approx(1.0, abs=0.05)


def test_error_statuses():
    assert oracle.plugin([1.0])["status"] == oracle.ERR_INVALID
    assert oracle.plugin([2.0, 2.0, 2.0])["status"] == oracle.ERR_DEGENERATE
    assert oracle.plugin([0.0, float("nan"), 1.0])["status"] == oracle.ERR_INVALID
    with pytest.raises(ValueError):
        oracle.psi([0.0, 1.0], 5, 1.0)
    with pytest.raises(ValueError):
        oracle.psi([0.0, 1.0], 4, -1.0)
