"""The oracle reproduces its stored outputs (tests/golden/oracle_fixtures.json):
a regression record of its arithmetic on small seeded inputs, written by
tests/golden/make_golden.py, which calls only the oracle and the input
generators.  A change to the oracle's results shows here first; the fixture
is then rewritten by that script in the same commit, whose message names the
passage that justifies the change.  The same fixture holds a digest of every
synthetic workload, so that a measured workload cannot change unnoticed."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")

_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
make_golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(make_golden)

with open(make_golden.FIXTURE) as _f:
    FIXTURE = json.load(_f)

# rounding-level agreement: the oracle's sums are ordered, so only libm may move the last bits
RTOL = 1e-11


@pytest.mark.parametrize("name", sorted(make_golden.SCENES))
def test_synthetic_workloads_unchanged(name):
    """The seeded generators still produce the recorded workloads, array for
    array (point counts, coordinates, features, true motions, parameters)."""
    assert make_golden.scene_digest(name) == FIXTURE["scenes"][name]


def test_fixture_matches_the_generator_cases():
    assert FIXTURE["xi"] == make_golden.XI
    stored = [{k: v for k, v in c.items() if k != "expected"} for c in FIXTURE["cases"]]
    assert stored == make_golden.CASES
    for c in FIXTURE["cases"]:
        assert c["cite"] and ("Eq." in c["cite"] or "Sec." in c["cite"])


def _close(got, want, path):
    if isinstance(want, dict):
        assert set(got) == set(want), path
        for k in want:
            _close(got[k], want[k], f"{path}.{k}")
    elif isinstance(want, list):
        g, w = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
        assert g.shape == w.shape, path
        scale = max(np.abs(w).max(), 1e-300)
        assert np.abs(g - w).max() <= RTOL * scale, path
    elif isinstance(want, int) and not isinstance(want, bool):
        assert got == want, path
    else:
        assert got == pytest.approx(want, rel=RTOL), path


@pytest.mark.parametrize("idx", range(len(make_golden.CASES)), ids=[c["name"] for c in make_golden.CASES])
def test_oracle_reproduces_fixture(idx):
    case = FIXTURE["cases"][idx]
    _close(make_golden.compute(case), case["expected"], case["name"])
