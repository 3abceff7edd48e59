"""The seeded input generators: reproducible and with the stated distributions."""
import math

import numpy as np
import pytest

import synthdata


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator.
    r = synthdata.raw64(0, 3)
    assert [int(v) for v in r] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_open_interval_and_moments():
    u = synthdata.uniform(1, 200000)
    assert u.min() > 0 and u.max() < 1
    assert u.mean() == pytest.approx(0.5, abs=3e-3)
    assert u.var() == pytest.approx(1 / 12, rel=1e-2)


def test_normal_moments_and_reproducibility():
    z = synthdata.normal(2, 200001)
    assert z.size == 200001
    assert z.mean() == pytest.approx(0.0, abs=1e-2)
    assert z.std() == pytest.approx(1.0, abs=1e-2)
    assert np.array_equal(z, synthdata.normal(2, 200001))
    assert not np.array_equal(z[:100], synthdata.normal(3, 100))


def test_t3_and_lognormal_shapes():
    t = synthdata.student_t3(3, 200000)
    assert np.median(t) == pytest.approx(0.0, abs=1e-2)
    # P(|T3| > 3.182) = 0.05 (two-sided 95% quantile of t with 3 dof)
    assert np.mean(np.abs(t) > 3.182) == pytest.approx(0.05, abs=3e-3)
    ln = synthdata.lognormal(4, 200000)
    assert np.median(ln) == pytest.approx(1.0, abs=2e-2)


def test_bimodal_offset_workload():
    x = synthdata.bimodal_offset()
    assert x.size == 65536
    assert x.mean() == pytest.approx(1e4, abs=0.02)
    assert x.std() == pytest.approx(math.sqrt(1 + 0.25), rel=2e-2)


def test_batch_specs_ranges():
    specs = synthdata.batch_specs()
    assert len(specs) == 512
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 256 and ns.max() <= 262144
    assert {s.family for s in specs} == {"normal", "mixture", "t3"}
    for s in specs:
        if s.family == "mixture":
            assert 2 <= len(s.params["weights"]) <= 5
            assert sum(s.params["weights"]) == pytest.approx(1.0)
