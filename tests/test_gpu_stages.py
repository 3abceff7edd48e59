"""The l-stage plug-in (l = 1..4; Algorithm 1 is l = 2) and psi_r for r = 8, 10
through the C ABI, against the oracle: relative 1e-5 (FP32 path) and 1e-11 (FP64)."""
import math

import numpy as np
import pytest

import oracle
import synthdata

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-11}


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


@pytest.mark.parametrize("stages", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [3000, 40000])
def test_stages_match_oracle(kde, stages, n):
    x = synthdata.normal_mixture(800 + n, n, [0.4, 0.6], [-1.0, 1.2], [0.6, 0.9]) + 5.0
    ref = oracle.plugin_stages(x, stages)
    assert ref["status"] == 0
    top = 2 * stages + 4
    for prec in (1, 0):
        got = kde.kde_plugin_h_stages(x, stages, prec)
        assert got["status"] == 0 and got["stages"] == stages
        assert _rel(got["sigma"], ref["sigma"]) <= 1e-13
        assert _rel(got["psi"][top], ref["psi"][top]) <= 1e-13          # normal scale
        assert math.isnan(got["g"][top])
        for r in range(4, top, 2):
            assert _rel(got["psi"][r], ref["psi"][r]) <= TOL[prec], (prec, r)
            assert _rel(got["g"][r], ref["g"][r]) <= TOL[prec], (prec, r)
        assert _rel(got["h"], ref["h"]) <= TOL[prec], prec
        for r in range(top + 2, 16, 2):
            assert math.isnan(got["psi"][r])


def test_two_stages_is_kde_plugin_h(kde):
    x = synthdata.student_t3(810, 25000)
    for prec in (0, 1):
        a = kde.kde_plugin_h(x, prec)
        b = kde.kde_plugin_h_stages(x, 2, prec)
        assert (b["psi"][8], b["g"][6], b["psi"][6], b["g"][4], b["psi"][4], b["h"]) == \
            (a["psi8"], a["g1"], a["psi6"], a["g2"], a["psi4"], a["h"])


@pytest.mark.parametrize("r", [8, 10])
@pytest.mark.parametrize("n", [2, 513, 5000])
def test_psi_high_orders(kde, r, n):
    x = synthdata.normal(820 + n, n) * 2.0 - 1.0
    g = 0.7 if r == 8 else 0.9
    ref = oracle.psi(x, r, g)
    for prec in (1, 0):
        assert _rel(kde.kde_psi(x, r, g, prec), ref) <= TOL[prec], prec
    assert _rel(kde.kde_psi_static(x, r, g, 0), ref) <= TOL[0]


def test_stage_errors(kde):
    x = synthdata.normal(830, 100)
    with pytest.raises(kde.KdeError):
        kde.kde_plugin_h_stages(x, 0, 0)
    with pytest.raises(kde.KdeError):
        kde.kde_plugin_h_stages(x, 5, 0)
    with pytest.raises(kde.KdeError):
        kde.kde_psi(x, 12, 0.5, 0)
    r = kde.kde_plugin_h_stages(np.full(50, 1.5), 3, 0, check=False)
    assert r["status"] == kde.KDE_ERR_DEGENERATE
