"""Pins of the oracle's l-stage plug-in (Algorithm 1 generalised to l estimated
functionals): the reduction to Algorithm 1 at l = 2, the normal-scale functional
against an integral, and each pilot bandwidth against the bias balance it solves."""
import math

import numpy as np
import pytest

import oracle
import synthdata

mp = pytest.importorskip("mpmath")


def test_two_stages_is_algorithm_1():
    x = synthdata.normal_mixture(21, 900, [0.3, 0.7], [-1.0, 2.0], [0.5, 1.1])
    a = oracle.plugin(x)
    b = oracle.plugin_stages(x, 2)
    assert b["status"] == 0 and a["status"] == 0
    for key, (r, kind) in {"psi8": (8, "psi"), "g1": (6, "g"), "psi6": (6, "psi"),
                           "g2": (4, "g"), "psi4": (4, "psi")}.items():
        assert b[kind][r] == pytest.approx(a[key], rel=1e-14), key
    assert b["h"] == pytest.approx(a["h"], rel=1e-14)
    assert math.isnan(b["g"][8]) and math.isnan(b["psi"][10])


@pytest.mark.parametrize("stages", [1, 2, 3, 4])
def test_normal_scale_functional_is_an_integral(stages):
    """psi_r^NS = (-1)^(r/2) int (phi_sigma^(r/2))^2 for the top order r = 2l + 4."""
    x = synthdata.normal(22, 300) * 1.3 + 2.0
    res = oracle.plugin_stages(x, stages)
    r = 2 * stages + 4
    s = mp.mpf(res["sigma"])
    mp.mp.dps = 30
    f = lambda t: mp.diff(lambda y: mp.npdf(y, 0, s), t, r // 2) ** 2
    ref = (-1) ** (r // 2) * mp.quad(f, [-mp.inf, 0, mp.inf])
    assert res["psi"][r] == pytest.approx(float(ref), rel=1e-10)


@pytest.mark.parametrize("stages", [1, 2, 3, 4])
def test_each_pilot_balances_the_leading_bias(stages):
    """g_r makes n^-1 g^-(r+1) K^(r)(0) + g^2 psi_{r+2} / 2 vanish (mu2 = 1)."""
    x = synthdata.student_t3(23, 2000)
    res = oracle.plugin_stages(x, stages)
    assert res["status"] == 0
    n = x.size
    for r in range(2 * stages + 2, 2, -2):
        g = res["g"][r]
        a = oracle.kernel_deriv(r, 0.0) / (n * g ** (r + 1))
        b = 0.5 * g * g * res["psi"][r + 2]
        assert abs(a + b) <= 1e-12 * abs(a), r
        # and psi_r is the functional at that pilot
        assert res["psi"][r] == pytest.approx(oracle.psi(x, r, g), rel=1e-14)
    assert res["h"] == pytest.approx((1 / (2 * math.sqrt(math.pi)) / (res["psi"][4] * n)) ** 0.2,
                                     rel=1e-14)


def test_stage_count_limits():
    x = synthdata.normal(24, 100)
    assert oracle.plugin_stages(x, 0)["status"] == oracle.ERR_INVALID
    assert oracle.plugin_stages(x, 5)["status"] == oracle.ERR_INVALID
    assert oracle.plugin_stages(np.full(10, 2.0), 3)["status"] == oracle.ERR_DEGENERATE
