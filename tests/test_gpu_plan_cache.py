"""Plans kept across calls on one stream.

Each stream's workspace keeps the plan (tiling, work-list) of its last call and
rebuilds it only when the sizes, precision, mode, g or a sample's tile
configuration change.  Calls that alternate between plans, or change the tile
configuration in between, must give bit for bit what a fresh workspace (a new
stream) gives, and those results match the oracle.
"""
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


def _fresh(kde, fn):
    import torch
    s = torch.cuda.Stream()
    out = fn(s)
    s.synchronize()
    return out


def test_alternating_sizes_and_data_on_one_stream(kde):
    import torch
    s = torch.cuda.Stream()
    a = synthdata.student_t3(61, 20000)
    b = synthdata.normal(62, 7001)
    c = synthdata.lognormal(63, 20000)           # same n as a, other values
    seq = [a, b, a, c, c, b, a]
    got = [kde.kde_plugin_h(x, kde.KDE_FP32, stream=s) for x in seq]
    for x, r in zip(seq, got):
        assert r == _fresh(kde, lambda st: kde.kde_plugin_h(x, kde.KDE_FP32, stream=st))
    ref = oracle.plugin(c)
    for f in ("psi6", "psi4", "h"):
        assert abs(got[3][f] - ref[f]) <= 1e-5 * abs(ref[f]), (f, got[3][f], ref[f])
    torch.cuda.synchronize()


def test_tile_configuration_change_between_calls(kde, monkeypatch):
    import torch
    s = torch.cuda.Stream()
    x = synthdata.student_t3(64, 30001)
    first = kde.kde_plugin_h(x, kde.KDE_FP32, stream=s)
    for cfg in ("3", "1", "0"):
        monkeypatch.setenv("KDE_FP32_TILE_CONFIG", cfg)
        got = kde.kde_plugin_h(x, kde.KDE_FP32, stream=s)
        assert got == _fresh(kde, lambda st: kde.kde_plugin_h(x, kde.KDE_FP32, stream=st)), cfg
        assert abs(got["h"] - first["h"]) <= 1e-5 * first["h"]
    monkeypatch.delenv("KDE_FP32_TILE_CONFIG")
    assert kde.kde_plugin_h(x, kde.KDE_FP32, stream=s) == first
    torch.cuda.synchronize()


def test_psi_with_changing_g_and_order(kde):
    import torch
    s = torch.cuda.Stream()
    x = synthdata.normal(65, 12000)
    calls = [(6, 0.3), (6, 0.31), (4, 0.31), (6, 0.3), (4, 0.5)]
    for prec in (kde.KDE_FP32, kde.KDE_FP64):
        got = [kde.kde_psi(x, r, g, prec, stream=s) for r, g in calls]
        for (r, g), v in zip(calls, got):
            assert v == _fresh(kde, lambda st: kde.kde_psi(x, r, g, prec, stream=st)), (prec, r, g)
        tol = 1e-5 if prec == kde.KDE_FP32 else 1e-11
        for (r, g), v in zip(calls[:2], got[:2]):
            ref = oracle.psi(x, r, g)
            assert abs(v - ref) <= tol * abs(ref), (prec, r, g, v, ref)
    torch.cuda.synchronize()


def test_batch_then_single_then_batch(kde):
    import torch
    s = torch.cuda.Stream()
    specs = synthdata.batch_specs(12, 66, 256, 9000)
    xs = [synthdata.sample_from_spec(sp) for sp in specs]
    packed = np.concatenate(xs)
    offs = np.concatenate([[0], np.cumsum([v.size for v in xs])])
    b1 = kde.kde_plugin_h_batch(packed, offs, kde.KDE_FP32, stream=s)
    one = kde.kde_plugin_h(xs[3], kde.KDE_FP32, stream=s)
    b2 = kde.kde_plugin_h_batch(packed, offs, kde.KDE_FP32, stream=s)
    assert b1 == b2
    assert one == b1[3]
    torch.cuda.synchronize()
