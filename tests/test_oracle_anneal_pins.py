"""Pins of the oracle's annealing trigger and stopping test by closed-form
trajectories.

Sec. IV of the paper decays the lengthscale by 2 % when the indicator has
stabilised; it defines neither the test for "stabilised" nor when to stop.
The reading both sides implement is stated in tests/anneal_closed_form.py.
Here it is pinned on problems whose whole registration follows from a
scalar formula (one pair of points on an axis, translated; two
point-symmetric pairs, rotated): the indicator of every iteration, every
step and so every decision is computed in 30-digit arithmetic from that
formula alone, and the oracle must reproduce the iteration count, the
iterations at which the lengthscale decays, each iteration's lengthscale
and indicator, and the final pose.

Each case is also shown to tell the reading apart from plausible
misreadings (an absolute tolerance, a comparison two iterations back, a
reference kept across a decay, an "or" in the stopping test, a stop that
ignores the lengthscale floor): on the same closed form each gives another
decay sequence or stop, so an oracle with any of them fails here.
"""
import math

import numpy as np
import pytest

import anneal_closed_form as acf
import oracle

pytest.importorskip("mpmath")

# trace columns: ell, F, i_theta, |g|, F'', t, |t omega|, |t v|, decayed, pairs, rows 0-2 of T_k
C_ELL, C_ITH, C_SROT, C_STR, C_DEC, C_T0 = 0, 2, 6, 7, 8, 10


def _run_oracle(case):
    X, Z, kw = acf.points(case)
    return oracle.register(X, Z, np.eye(4), **kw)


@pytest.mark.parametrize("case", sorted(acf.CASES))
def test_case_decisions_are_far_from_their_thresholds(case):
    """Every indicator comparison of the closed-form run is at least 2 % of
    the tolerance away from the threshold, so the rounding of any FP64 (or
    the GPU's FP32) evaluation cannot flip a decision."""
    tr = acf.trajectory(**acf.CASES[case])
    margins = [abs(it["margin"]) for it in tr if it["margin"] is not None]
    assert len(margins) >= 10
    assert min(margins) > 0.02


@pytest.mark.parametrize("case", sorted(acf.CASES))
def test_case_tells_the_reading_from_misreadings(case):
    c = acf.CASES[case]
    ref = acf.summary(acf.trajectory(**c))
    differs = {v: acf.summary(acf.trajectory(variant=v, **c)) != ref
               for v in ("abs", "km2", "keep", "or", "nofloor")}
    # together the cases separate every misreading; each case separates these
    expect = {"trans_anneal": ("abs", "km2", "keep", "nofloor"),
              "trans_floor_early": ("abs", "km2", "or"),
              "rot_anneal": ("abs", "km2", "keep", "nofloor")}[case]
    for v in expect:
        assert differs[v], v


@pytest.mark.parametrize("case", sorted(acf.CASES))
def test_oracle_annealing_and_stop_follow_the_closed_form(case):
    c = acf.CASES[case]
    ref = acf.trajectory(**c)
    T, info, tr = _run_oracle(case)
    n, decays = acf.summary(ref)
    assert tr.shape[0] == n == info["iters"]
    assert info["status"] == 0                          # stopped by the test, not the cap
    assert list(np.nonzero(tr[:, C_DEC])[0]) == decays
    for k, it in enumerate(ref):
        assert tr[k, C_ELL] == pytest.approx(it["ell"], rel=1e-12, abs=0.0), k
        assert tr[k, C_ITH] == pytest.approx(it["i"], rel=1e-12, abs=0.0), k
        step = tr[k, C_STR] if c["kind"] == "trans" else tr[k, C_SROT]
        assert step == pytest.approx(abs(it["step"]), rel=1e-9, abs=1e-14), k
    assert info["ell_final"] == pytest.approx(ref[-1]["ell"], rel=1e-12)
    # the final pose: the offset (angle) left after the last step
    left = ref[-1]["u"] - ref[-1]["step"]
    if c["kind"] == "trans":
        assert T[0, 3] == pytest.approx(c["u0"] - left, abs=1e-12)
        assert np.allclose(T[:3, :3], np.eye(3), atol=0.0)
    else:
        assert math.atan2(T[1, 0], T[0, 0]) == pytest.approx(c["u0"] - left, abs=1e-12)
        assert np.abs(T[:3, 3]).max() < 1e-14


def test_decay_needs_a_fresh_reference_in_the_closed_form():
    """After the pair is aligned the indicator is constant, and the reading
    decays exactly every second iteration (one to take the reference at the
    new lengthscale, one to compare), down to the floor."""
    ref = acf.trajectory(**acf.CASES["trans_anneal"])
    _, decays = acf.summary(ref)
    late = [k for k in decays if ref[k]["u"] < 1e-9]
    assert len(late) >= 2 and all(b - a == 2 for a, b in zip(late, late[1:]))
