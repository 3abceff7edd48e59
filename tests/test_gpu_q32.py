"""The Q32.32 fixed-point variant (the paper's arithmetic, Section 4.1) through the
C ABI: against the oracle's fixed-point functional within the bound its arithmetic
allows, against the binary64 oracle on the scale of Table 4, order-independent bit
for bit (integer sums), and refused where it is not defined."""
import math

import numpy as np
import pytest

import oracle
import synthdata

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kde():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_02100_gb300 as k
    return k


def _bound(x, r, g, abs_he, sigma):
    """|psi_GPU - psi_oracle|: the GPU's exp (polynomial, shift) is within ~10 units of
    2^-32 of the exactly truncated one, times |He_r|; a one-unit difference of a z value
    moves a term by at most ~16 (sigma/g) units; normalised as in Eqs. 6-7."""
    n = x.size
    pairs = n * (n - 1) / 2
    units = 16.0 * abs_he + 16.0 * (sigma / g + 1.0) * pairs
    return 2.0 * units * 2.0 ** -32 / (math.sqrt(2 * math.pi) * n * n * g ** (r + 1))


@pytest.mark.parametrize("r", [4, 6])
@pytest.mark.parametrize("n", [2, 255, 256, 257, 3000, 20000])
def test_psi_matches_fixed_point_oracle(kde, r, n):
    x = synthdata.normal_mixture(900 + n, n, [0.5, 0.5], [-1.0, 1.0], [0.5, 0.7]) * 2.0 + 3.0
    mean, var = oracle.moments(x)
    sigma = math.sqrt(var)
    g = 0.35 if r == 6 else 0.25
    ref, abs_he = oracle.psi_q32(x, r, g, mean, sigma)
    got = kde.kde_psi(x, r, g, kde.KDE_Q32)
    assert abs(got - ref) <= _bound(x, r, g, abs_he, sigma), (got, ref)


@pytest.mark.parametrize("n", [128, 1024, 20000])
def test_plugin_against_both_oracles(kde, n):
    x = synthdata.normal(910 + n, n) * 1.5 + 2.0
    q = oracle.plugin_q32(x)
    f = oracle.plugin(x)
    got = kde.kde_plugin_h(x, kde.KDE_Q32)
    assert got["status"] == 0
    # Step IV at the same g1: within the arithmetic's bound
    _, abs_he = oracle.psi_q32(x, 6, q["g1"], q["mean"], q["sigma"])
    assert abs(got["psi6"] - q["psi6"]) <= _bound(x, 6, q["g1"], abs_he, q["sigma"])
    # Steps V-VII inherit that difference (g2 moves with psi6)
    for key in ("g2", "psi4", "h"):
        assert abs(got[key] - q[key]) <= 1e-6 * abs(q[key]), key
    # the paper's Table 4 scale: relative error of h against binary64 below ~1e-5
    assert abs(got["h"] - f["h"]) <= 1e-5 * f["h"]


def test_order_independent_bitwise_and_batch(kde):
    x = synthdata.student_t3(920, 7001)
    perm = np.argsort(synthdata.uniform(921, x.size))
    a = kde.kde_plugin_h(x, kde.KDE_Q32)
    assert a == kde.kde_plugin_h(x[perm], kde.KDE_Q32)
    xs = [synthdata.normal(930 + k, nn) for k, nn in enumerate((700, 4000, 12345))]
    off = np.concatenate([[0], np.cumsum([v.size for v in xs])])
    for v, b in zip(xs, kde.kde_plugin_h_batch(np.concatenate(xs), off, kde.KDE_Q32)):
        assert b == kde.kde_plugin_h(v, kde.KDE_Q32)


def test_refusals(kde):
    x = synthdata.normal(940, 500)
    with pytest.raises(kde.KdeError):
        kde.kde_psi(x, 8, 0.5, kde.KDE_Q32)
    with pytest.raises(kde.KdeError):
        kde.kde_plugin_h_stages(x, 3, kde.KDE_Q32)
    assert kde.kde_plugin_h_stages(x, 2, kde.KDE_Q32)["h"] == kde.kde_plugin_h(x, kde.KDE_Q32)["h"]
    r = kde.kde_plugin_h(np.full(64, 2.0), kde.KDE_Q32, check=False)
    assert r["status"] == kde.KDE_ERR_DEGENERATE
    with kde.Server(hbm_budget_bytes=64 << 20, max_inflight=2) as srv:
        with pytest.raises(kde.KdeError):
            srv.submit(x.astype(np.float32), kde.KDE_Q32)
