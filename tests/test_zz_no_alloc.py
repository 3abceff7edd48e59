"""kde_psi_static, the allocation-free variant of kde_psi, against kde_psi and the oracle.

Callers that cannot allocate device memory on their call path use it: a process
whose framework allocator already holds most of HBM, or a latency-bound loop in
which cudaMalloc / cudaFree would synchronise the device.  It runs the same
kernels on the same plan in a fixed scratch area, so its results must agree
with kde_psi within the parity tolerances (relative 1e-5 FP32, 1e-11 FP64; the
Q32.32 sums are exact integers, so equal to rounding of the final scaling), and
with the oracle within the same tolerances.  Two calls in a row check that no
state leaks from one call to the next.  Collected last so that it also runs
after every other GPU test.
"""
import functools

import numpy as np
import pytest

import synthdata

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-11, 2: 1e-12}


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


def _sample(n):
    return synthdata.normal_mixture(900 + n, n, [0.5, 0.5], [-1.0, 1.0], [0.5, 0.5]) + 3.0


@functools.lru_cache(maxsize=None)
def _oracle_psi(n, r, g):
    import oracle
    return oracle.psi(_sample(n), r, g)


G = {4: 0.2, 6: 0.35, 8: 0.45, 10: 0.55}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("r", [4, 6])
@pytest.mark.parametrize("n", [2, 777, 20000, 65536])
def test_static_matches_kde_psi_and_oracle_twice(kde, n, r, prec):
    x = _sample(n)
    g = G[r]
    ref = kde.kde_psi(x, r, g, prec)
    first = kde.kde_psi_static(x, r, g, prec)
    second = kde.kde_psi_static(x, r, g, prec)
    assert _rel(first, ref) <= TOL[prec], (first, ref)
    assert _rel(second, ref) <= TOL[prec], (second, ref)
    want = _oracle_psi(n, r, g)
    assert _rel(first, want) <= TOL[prec], (first, want)


@pytest.mark.parametrize("prec,r", [(2, 4), (2, 6), (0, 8), (0, 10), (1, 8), (1, 10)])
def test_static_other_precisions_and_orders(kde, prec, r):
    n = 20000
    x = _sample(n)
    g = G[r]
    ref = kde.kde_psi(x, r, g, prec)
    for _ in range(2):
        assert _rel(kde.kde_psi_static(x, r, g, prec), ref) <= TOL[prec]
    if prec != 2:
        assert _rel(ref, _oracle_psi(n, r, g)) <= TOL[prec]


def test_static_call_allocates_no_device_memory(kde):
    import torch
    x = torch.tensor(_sample(30000), device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    kde.kde_psi_static(x, 6, 0.35, 0, out=out)   # set-up call: address lookup, modules loaded
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for r in (6, 4, 6):
        kde.kde_psi_static(x, r, G[r], 0, out=out)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after >= free_before, (free_before, free_after)
    assert _rel(out.item(), kde.kde_psi(x, 6, 0.35, 0)) <= TOL[0]


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
