"""Tile-configuration autotuner: valid choices, used by every plan, parity kept,
and clearing restores the built-in rule."""
import numpy as np
import pytest

import oracle
import synthdata

pytestmark = pytest.mark.gpu

SIZES = (1 << 10, 1 << 12, 1 << 14, 1 << 16, 1 << 18)


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
def test_autotune_table_is_used_and_cleared(kde, prec):
    before = [kde.kde_tile_config(n, prec) for n in SIZES + (1 << 21,)]
    try:
        chosen = kde.kde_autotune(prec)
        count = 5 if prec == 0 else 3
        assert len(chosen) == 5 and all(0 <= c < count for c in chosen)
        for n, c in zip(SIZES, chosen):
            assert kde.kde_tile_config(n, prec)[0] == c
            assert kde.kde_tile_config(n + n // 3, prec)[0] == c      # same size class
        assert kde.kde_tile_config(1 << 21, prec)[0] == chosen[-1]
        # results under the tuned configurations still meet the parity bar
        tol = 1e-5 if prec == 0 else 1e-11
        for n in (1500, 5000, 70000):
            x = synthdata.normal_mixture(500 + n, n, [0.3, 0.7], [-2.0, 1.0], [0.7, 1.2])
            ref = oracle.plugin(x)
            got = kde.kde_plugin_h(x, prec)
            for f in ("psi6", "psi4", "h"):
                assert _rel(got[f], ref[f]) <= tol, (n, f)
        # batch and single calls consult the same table: bitwise equal
        xs = [synthdata.student_t3(600 + k, n) for k, n in enumerate((3000, 17000, 40000))]
        off = np.concatenate([[0], np.cumsum([x.size for x in xs])])
        batch = kde.kde_plugin_h_batch(np.concatenate(xs), off, prec)
        for x, b in zip(xs, batch):
            assert b == kde.kde_plugin_h(x, prec)
    finally:
        kde.kde_autotune_clear(prec)
    assert [kde.kde_tile_config(n, prec) for n in SIZES + (1 << 21,)] == before
