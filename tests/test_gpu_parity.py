"""GPU path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances are the stated accuracy bar: relative 1e-5 for the FP32 pair path and
1e-11 for the all-FP64 path, on psi6, psi4 and h (and every other scalar of
Algorithm 1).  sigma, psi8 and g1 come from binary64 moments on both paths.
"""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import synthdata

pytestmark = pytest.mark.gpu

FIELDS = ("sigma", "psi8", "g1", "psi6", "g2", "psi4", "h")
TOL = {0: 1e-5, 1: 1e-11}          # KDE_FP32, KDE_FP64
SCALAR_TOL = 1e-13                 # sigma, psi8, g1: binary64 on both sides


@pytest.fixture(scope="module")
def kde():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_02100_gb300 as k
    return k


def _rel(a, b):
    return abs(a - b) / abs(b)


def _check_result(got, ref, prec, label=""):
    assert got["status"] == 0, (label, got["status"])
    for f in FIELDS:
        tol = SCALAR_TOL if f in ("sigma", "psi8", "g1") else TOL[prec]
        assert _rel(got[f], ref[f]) <= tol, (label, prec, f, got[f], ref[f], _rel(got[f], ref[f]))


@pytest.mark.parametrize("prec", [1, 0])
def test_single_normal_n1024(kde, prec):
    """n = 1024 iid N(0,1), seed 0: every scalar of Algorithm 1."""
    import torch
    x = synthdata.single_normal(1024, 0)
    ref = oracle.plugin(x, form=oracle.FORM_FULL)
    got = kde.kde_plugin_h(torch.tensor(x, device="cuda"), prec)
    _check_result(got, ref, prec, "n1024")


SWEEP_N = [2, 3, 4, 5, 7, 31, 33, 127, 128, 129, 255, 256, 257, 300, 511, 512, 513,
           1023, 1024, 1025, 2047, 2049, 4097, 16383, 16385, 20000]


@pytest.mark.parametrize("n", SWEEP_N)
def test_plugin_sweep_ragged_and_tile_edges(kde, n):
    """Sizes around every tile side (256, 512) and the small-n switch, both precisions."""
    x = synthdata.normal_mixture(300 + n, n, [0.6, 0.4], [0.0, 2.5], [1.0, 0.4]) * 3.0 - 7.0
    ref = oracle.plugin(x)
    for prec in (1, 0):
        _check_result(kde.kde_plugin_h(x, prec), ref, prec, f"n={n}")


@pytest.mark.parametrize("r", [4, 6])
@pytest.mark.parametrize("n", [2, 3, 257, 1000, 5000])
def test_psi_given_g(kde, n, r):
    x = synthdata.student_t3(400 + n, n)
    ref_plugin = oracle.plugin(x)
    g = ref_plugin["g2"] if r == 4 else ref_plugin["g1"]
    ref = oracle.psi(x, r, g, form=oracle.FORM_FULL)
    for prec in (1, 0):
        assert _rel(kde.kde_psi(x, r, g, prec), ref) <= TOL[prec]
    # a few other bandwidths: psi_r(g) is smooth in g
    for gg in (0.3 * g, 3.0 * g):
        ref = oracle.psi(x, r, gg)
        assert _rel(kde.kde_psi(x, r, gg, 1), ref) <= 1e-11
        assert _rel(kde.kde_psi(x, r, gg, 0), ref) <= 1e-4


def test_bimodal_offset_n65536(kde):
    """n = 65536, 0.5 N(-1, 0.25) + 0.5 N(1, 0.25) + 1e4: FP32 path vs FP64 path vs oracle."""
    import torch
    x = synthdata.bimodal_offset()
    ref = oracle.plugin(x)
    xd = torch.tensor(x, device="cuda")
    r64 = kde.kde_plugin_h(xd, 1)
    r32 = kde.kde_plugin_h(xd, 0)
    _check_result(r64, ref, 1, "bimodal fp64")
    _check_result(r32, ref, 0, "bimodal fp32")
    assert abs(r32["mean"] - 1e4) < 0.05


def _golden_large():
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_golden
    return make_golden.load("large")


@pytest.mark.parametrize("r", [6, 4])
@pytest.mark.parametrize("family", ["t3", "lognormal", "uniform"])
def test_large_n_sampled_slots(kde, family, r):
    """n = 2^20: per-chunk partial sums of the timed FP32 kernel checked one by one
    against the oracle's block sums over the same pairs, at psi6(g1) and psi4(g2)
    (the oracle's pilots for this sample).

    Bound: every binary32 term carries a few rounding errors of relative size
    2^-24, independent from term to term, so a chunk's error grows like the root
    of the sum of squared terms; |He_r(u) exp(-u^2/2)| <= |He_r(0)| bounds that
    by |He_r(0)| sum|terms|.  The test allows 32 x 2^-24 x sqrt(|He_r(0)| sum|terms|)
    plus 4 x 2^-24 |sum| -- for a tile pair of 2.6e5 terms some 1e4 times tighter
    than 1e-5 of sum|terms|."""
    x = np.sort(synthdata.large_sample(family))     # the library tiles the sorted sample
    n = x.size
    ref = _golden_large()[family]
    g = ref["g1"] if r == 6 else ref["g2"]
    slots, info = kde.kde_psi_slots(x, r, g, 0)
    T, C, ntp = info["tile"], info["chunk"], info["n_tile_pairs"]
    nt = (n + T - 1) // T
    assert ntp == nt * (nt + 1) // 2 and slots.size == info["n_slots"]

    def tile_pair(p):
        # row-major upper triangle
        I = 0
        while (I + 1) * nt - (I + 1) * I // 2 <= p:
            I += 1
        return I, I + (p - (I * nt - I * (I - 1) // 2))

    eps = 2.0 ** -24
    he0 = 15.0 if r == 6 else 3.0
    rng = np.random.default_rng(5 + r)
    picks = sorted(set([0, slots.size - 1] + list(rng.integers(0, slots.size, 6))))
    checked = 0
    for c in picks:
        s_ref, a_ref = 0.0, 0.0
        for p in range(c * C, min((c + 1) * C, ntp)):
            I, J = tile_pair(p)
            s, a = oracle.psi_block(x, I * T, min((I + 1) * T, n), J * T, min((J + 1) * T, n), r, g)
            s_ref += s
            a_ref += a
        scale = math.sqrt(2 * math.pi)   # slots hold sums of He_r(u) exp(-u^2/2)
        want, mag = s_ref * scale, a_ref * scale
        bound = 32 * eps * math.sqrt(he0 * mag) + 4 * eps * abs(want)
        assert abs(slots[c] - want) <= bound, (c, slots[c], want, bound)
        checked += mag > 0
    assert checked >= 2


def test_large_n_fp32_vs_fp64_and_expectation(kde):
    """n = 2^20 normal: FP32 and FP64 GPU paths agree to 1e-5 on psi6, psi4, h, and
    psi6(g1) is near the closed-form normal expectation."""
    import torch
    n = 1 << 20
    x = synthdata.normal(31, n) * 1.7 + 4.0
    xd = torch.tensor(x, device="cuda")
    r32 = kde.kde_plugin_h(xd, 0)
    r64 = kde.kde_plugin_h(xd, 1)
    for f in ("psi6", "g2", "psi4", "h"):
        assert _rel(r32[f], r64[f]) <= 1e-5, f
    g, s = r64["g1"], 1.7
    k0 = -15 / math.sqrt(2 * math.pi)
    expect = k0 * (1 / (n * g ** 7) + (1 - 1 / n) * (g * g + 2 * s * s) ** -3.5)
    assert _rel(r64["psi6"], expect) < 0.02


@pytest.mark.parametrize("r", [4, 6])
def test_clamp_variant_with_far_outlier(kde, r):
    """A point so far out at the given g that max|w| >= 3e5: the FP32 kernel clamps
    -w^2 (else its Hermite factor would overflow to inf * 0); its terms vanish."""
    x = synthdata.normal(41, 3000)
    x[17] = 1.0e6
    ref = oracle.psi(x, r, 0.3)
    assert _rel(kde.kde_psi(x, r, 0.3, 1), ref) <= TOL[1]
    assert _rel(kde.kde_psi(x, r, 0.3, 0), ref) <= TOL[0]


@pytest.mark.parametrize("scale", [1e-30, 1e-8, 1e8, 1e30])
def test_extreme_scales(kde, scale):
    x = synthdata.normal(42, 777) * scale
    ref = oracle.plugin(x)
    for prec in (1, 0):
        _check_result(kde.kde_plugin_h(x, prec), ref, prec, f"scale {scale}")


def test_two_points_exact_forms(kde):
    ref = oracle.plugin([0.0, 1.0])
    for prec in (1, 0):
        _check_result(kde.kde_plugin_h([0.0, 1.0], prec), ref, prec, "n=2")


def test_error_statuses(kde):
    r = kde.kde_plugin_h(np.full(100, 3.25), 0, check=False)
    assert r["status"] == kde.KDE_ERR_DEGENERATE
    assert r["mean"] == 3.25 and r["sigma"] == 0.0 and math.isnan(r["h"])
    x = synthdata.normal(43, 500)
    x[100] = float("nan")
    r = kde.kde_plugin_h(x, 0, check=False)
    assert r["status"] == kde.KDE_ERR_INVALID and math.isnan(r["h"])
    x[100] = float("inf")
    assert kde.kde_plugin_h(x, 1, check=False)["status"] == kde.KDE_ERR_INVALID
    with pytest.raises(kde.KdeError):
        kde.kde_plugin_h([1.0], 0)
    # the library stays usable after errors
    ref = oracle.plugin(synthdata.normal(44, 300))
    _check_result(kde.kde_plugin_h(synthdata.normal(44, 300), 0), ref, 0, "after errors")


def test_deterministic_and_input_location_independent(kde):
    import torch
    x = synthdata.student_t3(45, 30001)
    xd = torch.tensor(x, device="cuda")
    runs = [kde.kde_plugin_h(xd, 0) for _ in range(5)] + [kde.kde_plugin_h(x, 0)]
    for r in runs[1:]:
        assert r == runs[0]


def test_device_output_async_and_stream(kde):
    import torch
    x = synthdata.normal(46, 4000)
    xd = torch.tensor(x, device="cuda")
    s = torch.cuda.Stream()
    out = torch.empty(kde.RESULT_BYTES // 8, dtype=torch.float64, device="cuda")
    psi_out = torch.empty(1, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        kde.kde_plugin_h(xd, 0, out=out, stream=s)
        kde.kde_psi(xd, 4, 0.3, 0, out=psi_out, stream=s)
    s.synchronize()
    host = kde.kde_plugin_h(x, 0)
    vals = out.cpu().numpy()
    for i, f in enumerate(kde.RESULT_FIELDS):
        assert vals[i] == host[f]
    assert psi_out.item() == kde.kde_psi(x, 4, 0.3, 0)


def test_float32_input(kde):
    x32 = synthdata.lognormal(47, 9000).astype(np.float32)
    ref = oracle.plugin(x32.astype(np.float64))
    for prec in (1, 0):
        _check_result(kde.kde_plugin_h(x32, prec), ref, prec, "f32 input")


@pytest.mark.parametrize("prec", [0, 1])
def test_permutation_invariance_is_bitwise(kde, prec):
    """The device sorts every sample first, so any input order gives the same bits."""
    x = synthdata.student_t3(48, 5001)
    perm = np.argsort(synthdata.uniform(49, x.size))
    assert kde.kde_plugin_h(x, prec) == kde.kde_plugin_h(x[perm], prec) == kde.kde_plugin_h(np.sort(x), prec)
