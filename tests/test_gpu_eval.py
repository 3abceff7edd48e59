"""Density estimate (Eq. 1, Gaussian kernel of Eq. 2) through the C ABI against the
oracle: relative 1e-5 (FP32 path) and 1e-11 (FP64 path) at every point, with an
absolute floor far below the FP32 underflow of terms beyond ~13 bandwidths."""
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


def _check(got, ref, prec, label=""):
    floor = 1e-30 * ref.max()
    err = np.abs(got - ref)
    bad = err > TOL[prec] * np.abs(ref) + floor
    assert not bad.any(), (label, prec, int(bad.sum()), float((err / np.maximum(ref, 1e-300)).max()))


@pytest.mark.parametrize("n", [1, 2, 1023, 1024, 1025, 5000])
@pytest.mark.parametrize("m", [1, 511, 512, 513, 2000])
def test_eval_sweep_tiles_and_ragged(kde, n, m):
    x = synthdata.normal_mixture(700 + n, n, [0.5, 0.5], [-1.0, 1.5], [0.6, 0.4]) * 2.0 + 3.0
    h = 0.23
    t = np.linspace(x.min() - 4 * h, x.max() + 4 * h, m)
    ref = oracle.kde_eval(x, h, t)
    for prec in (1, 0):
        _check(kde.kde_eval(x, h, t, prec), ref, prec, f"n={n} m={m}")


def test_eval_with_plugin_bandwidth_offset_data(kde):
    x = synthdata.bimodal_offset(n=20000)
    h = kde.kde_plugin_h(x, 0)["h"]
    t = synthdata.uniform(77, 3001) * 6.0 - 3.0 + 1e4
    ref = oracle.kde_eval(x, h, t)
    for prec in (1, 0):
        _check(kde.kde_eval(x, h, t, prec), ref, prec, "bimodal+1e4")


def test_eval_full_size_sampled_points(kde):
    """n = 2^20 t3 sample, 8192 points: 64 of them checked against the oracle."""
    x = synthdata.large_sample("t3")
    h = 0.05
    t = np.linspace(-8.0, 8.0, 8192)
    got = kde.kde_eval(x, h, t, 0)
    pick = np.sort(synthdata.uniform(78, 64) * t.size).astype(int)
    _check(got[pick], oracle.kde_eval(x, h, t[pick]), 0, "t3 2^20")


def test_eval_far_outlier_and_range_limit(kde):
    x = synthdata.normal(79, 3000)
    h = 0.2
    x[5] = 5.0e6 * h                   # within the FP32 range limit (1e7 bandwidths)
    t = np.array([0.0, 0.5, x[5], x[5] + 0.3 * h, 2.5e6 * h])
    ref = oracle.kde_eval(x, h, t)
    for prec in (1, 0):
        _check(kde.kde_eval(x, h, t, prec), ref, prec, "outlier")
    x[5] = 3.0e7 * h                   # beyond it: FP32 refuses, FP64 computes
    with pytest.raises(kde.KdeError) as ei:
        kde.kde_eval(x, h, t, 0)
    assert ei.value.status == kde.KDE_ERR_INVALID
    _check(kde.kde_eval(x, h, t, 1), oracle.kde_eval(x, h, t), 1, "far outlier fp64")


def test_eval_errors_and_determinism(kde):
    import torch
    x = synthdata.student_t3(80, 4000)
    t = np.linspace(-3, 3, 700)
    with pytest.raises(kde.KdeError):
        kde.kde_eval(x, 0.0, t, 0)
    y = x.copy()
    y[3] = np.nan
    with pytest.raises(kde.KdeError):
        kde.kde_eval(y, 0.3, t, 0)
    with pytest.raises(kde.KdeError):
        kde.kde_eval(y, 0.3, t, 1)
    a = kde.kde_eval(x, 0.3, t, 0)
    b = kde.kde_eval(torch.tensor(x, device="cuda"), 0.3, torch.tensor(t, device="cuda"), 0)
    assert np.array_equal(a, b)
    out = torch.empty(t.size, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        kde.kde_eval(torch.tensor(x, device="cuda"), 0.3, torch.tensor(t, device="cuda"), 0,
                     out=out, stream=s)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), a)
