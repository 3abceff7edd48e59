"""kde_psi_static, the allocation-free variant of kde_psi, against kde_psi.

It runs the same kernels on the same plan in a fixed scratch area, so its
results must agree with kde_psi within the parity tolerances (relative 1e-5
FP32, 1e-11 FP64); two calls in a row check that no state leaks between calls.
Collected last so that it also runs after every other GPU test.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("r", [4, 6])
@pytest.mark.parametrize("n", [2, 777, 20000, 65536])
def test_static_matches_kde_psi_twice(kde, n, r, prec):
    x = synthdata.normal_mixture(900 + n, n, [0.5, 0.5], [-1.0, 1.0], [0.5, 0.5]) + 3.0
    g = 0.35 if r == 6 else 0.2
    ref = kde.kde_psi(x, r, g, prec)
    first = kde.kde_psi_static(x, r, g, prec)
    second = kde.kde_psi_static(x, r, g, prec)
    assert _rel(first, ref) <= TOL[prec], (first, ref)
    assert _rel(second, ref) <= TOL[prec], (second, ref)


def test_static_device_input_and_output(kde):
    import torch
    x = synthdata.student_t3(950, 40000)
    xd = torch.tensor(x, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        kde.kde_psi_static(xd, 6, 0.3, 0, out=out[0:1], stream=s)
        kde.kde_psi_static(xd, 4, 0.2, 0, out=out[1:2], stream=s)
    s.synchronize()
    got = out.cpu().numpy()
    assert _rel(got[0], kde.kde_psi(x, 6, 0.3, 0)) <= TOL[0]
    assert _rel(got[1], kde.kde_psi(x, 4, 0.2, 0)) <= TOL[0]


def test_static_rejects_sizes_beyond_its_scratch(kde):
    x = synthdata.normal(951, kde.STATIC_MAX_N + 1)
    with pytest.raises(kde.KdeError) as ei:
        kde.kde_psi_static(x, 6, 0.3, 0)
    assert ei.value.status == kde.KDE_ERR_INVALID
    assert "static scratch limit" in str(ei.value)
    with pytest.raises(kde.KdeError):
        kde.kde_psi_static(np.zeros(1), 6, 0.3, 0)
    # still usable afterwards
    y = synthdata.normal(952, 5000)
    assert _rel(kde.kde_psi_static(y, 4, 0.25, 1), kde.kde_psi(y, 4, 0.25, 1)) <= TOL[1]
