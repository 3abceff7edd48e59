"""The stored oracle values (tests/golden/plugin_*.txt) against the closed forms of
Algorithm 1 and against the oracle itself.

The GPU tests of the large, batched and served workloads compare with values that
tests/golden/make_golden.py wrote from ``oracle/``.  These CPU tests check, for every
stored record, that
- its scalars satisfy the closed-form steps that link them: Step II (psi8 from sigma),
  Step III (g1 from psi8), Step V (g2 from psi6) and Step VII (h from psi4);
- its n is the n of the seeded input it was written for;
- for the smaller records, re-running the oracle on the same seeded input gives the
  stored numbers back to the last printed digit (the files hold ``%.17g``).
"""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import synthdata

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

SQ2PI = math.sqrt(2.0 * math.pi)
SQPI = math.sqrt(math.pi)


def _chain(rec):
    n = rec["n"]
    psi8 = 105.0 / (32.0 * SQPI * rec["sigma"] ** 9)                      # Step II
    g1 = (30.0 / SQ2PI / (psi8 * n)) ** (1.0 / 9.0)                       # Step III, -2 K6(0) = 30/sqrt(2 pi)
    g2 = (6.0 / SQ2PI / (-rec["psi6"] * n)) ** (1.0 / 7.0)               # Step V, -2 K4(0) = -6/sqrt(2 pi)
    h = (1.0 / (2.0 * SQPI) / (rec["psi4"] * n)) ** 0.2                   # Step VII, R(K) = 1/(2 sqrt(pi))
    return {"psi8": psi8, "g1": g1, "g2": g2, "h": h}


def _inputs(kind):
    if kind == "large":
        return {fam: (lambda fam=fam: synthdata.large_sample(fam)) for fam in synthdata.LARGE_FAMILIES}
    if kind == "batch":
        return {str(s.index): (lambda s=s: synthdata.sample_from_spec(s)) for s in synthdata.batch_specs()}
    specs = synthdata.server_specs()[:1000]
    return {str(s.index): (lambda s=s: synthdata.sample_from_spec(s, np.float32).astype(np.float64))
            for s in specs}


@pytest.mark.parametrize("kind", ["large", "batch", "serve"])
def test_stored_scalars_follow_the_closed_form_steps(kind):
    gold = make_golden.load(kind)
    assert gold
    for key, rec in gold.items():
        assert rec["status"] == 0, (kind, key)
        assert rec["psi6"] < 0 < rec["psi4"], (kind, key)
        want = _chain(rec)
        for f in ("psi8", "g1", "g2", "h"):
            assert abs(rec[f] - want[f]) <= 1e-13 * abs(want[f]), (kind, key, f, rec[f], want[f])


@pytest.mark.parametrize("kind", ["large", "batch", "serve"])
def test_stored_records_match_their_seeded_inputs(kind):
    gold = make_golden.load(kind)
    specs = {"batch": {str(s.index): s.n for s in synthdata.batch_specs()},
             "serve": {str(s.index): s.n for s in synthdata.server_specs()[:1000]},
             "large": {fam: 1 << 20 for fam in synthdata.LARGE_FAMILIES}}[kind]
    for key, rec in gold.items():
        assert specs[key] == rec["n"], (kind, key)
    if kind == "batch":
        assert len(gold) == 512
    if kind == "serve":
        assert set(make_golden.load_file("serve")) == {k for k, n in specs.items() if n <= 65536}
        mid = {k for k, n in specs.items() if 65536 < n <= 262144}
        assert set(gold) - set(make_golden.load_file("serve")) == mid
    if kind == "large":
        assert set(gold) == set(synthdata.LARGE_FAMILIES)


@pytest.mark.parametrize("kind", ["batch", "serve"])
def test_small_records_are_what_the_oracle_writes(kind):
    """The stored values are the oracle's: re-run it on the smallest records."""
    gold = make_golden.load(kind)
    make = _inputs(kind)
    smallest = sorted(gold, key=lambda k: gold[k]["n"])[:12]
    for key in smallest:
        res = oracle.plugin(make[key]())
        for f in make_golden.FIELDS:
            assert float(f"{res[f]:.17g}") == gold[key][f], (kind, key, f, res[f], gold[key][f])
