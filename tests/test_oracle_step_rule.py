"""Pins of the oracle's registration loop: the step rule, the pose update
and its composition order, the trust region, the annealing trigger and the
stopping test.

The paper names a step size (Sec. III-B) and cites gradient ascent on the Lie
group (Sec. I) but prints no rule.  The rule taken: the ascent direction is
the gradient in a metric on se(3) written about the moved centroid of Z
(rotations weighted by the cloud's mean squared radius plus l^2), so it does
not depend on where the coordinate origin lies; the step is a Newton step
along that direction (t = F' / -F'' where F'' < 0, else the trust region's
edge), never beyond the trust region: no point of Z moves more than half a
lengthscale (or max_step_trans), no rotation exceeds max_step_rot.  On
problems whose objective along the ascent direction has one variable, the
Newton step and its iterates are computed here from that closed form alone,
with no call into the oracle's arithmetic:

- one pair of points on the x axis, offset delta: the direction is a pure
  translation along x and F(s) = exp(-(delta - s)^2 / 2 l^2), so the Newton
  step is s* = delta l^2 / (l^2 - delta^2) while delta < l;
- two pairs placed point-symmetrically about a centre q, Z = R_z(-phi) X
  about q: the translational gradient cancels, the direction is a rotation
  about q and F(theta) = 2 exp(-a (1 - cos(phi - theta))), a = r^2 / l^2, so
  the Newton step is sin(phi) / (cos(phi) - a sin(phi)^2).

The whole registration is equivariant under a common rigid motion of both
clouds (the objective is invariant, Sec. III; the rule names no origin),
which a direction taken about the coordinate origin would break.  The
annealing trigger and stopping test are readings of Sec. IV (the paper
defines neither).  They are pinned by closed-form annealed trajectories in
tests/test_oracle_anneal_pins.py; the tests here add checks of the same rule
along registrations of a cube scene.
"""
import math

import numpy as np
import pytest

import oracle
import scenes

ELL = 0.5
# trace columns: ell, F, i_theta, |g|, F'', t, |t omega|, |t v|, decayed, pairs, rows 0-2 of T_k
C_ELL, C_ITH, C_GN, C_FPP, C_T, C_SROT, C_STR, C_DEC, C_NP, C_T0 = 0, 2, 3, 4, 5, 6, 7, 8, 9, 10


def axial_pair(delta):
    X = np.array([[1.0 + delta, 0.0, 0.0]])
    Z = np.array([[1.0, 0.0, 0.0]])
    return X, Z


def rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def symmetric_pairs(r, phi, q=(0.0, 0.0, 0.0)):
    q = np.asarray(q, dtype=np.float64)
    X = np.array([[r, 0.0, 0.0], [-r, 0.0, 0.0]])
    Z = (rz(-phi) @ X.T).T
    return X + q, Z + q


def newton_translation(delta, ell=ELL):
    return delta * ell ** 2 / (ell ** 2 - delta ** 2)


def newton_rotation(u, a):
    return math.sin(u) / (math.cos(u) - a * math.sin(u) ** 2)


def test_translation_newton_step():
    delta = 0.3 * ELL
    T, info, tr = oracle.register(*axial_pair(delta), np.eye(4), ell=ELL, max_iters=1)
    assert T[0, 3] == pytest.approx(newton_translation(delta), rel=1e-12)
    assert T[1, 3] == 0.0 and T[2, 3] == 0.0
    assert np.allclose(T[:3, :3], np.eye(3), atol=0.0)
    # F'' along g is |g|^2 times the closed-form second derivative of F(s) at s = 0
    g = delta / ELL ** 2 * math.exp(-delta ** 2 / (2 * ELL ** 2))
    fss = (delta ** 2 / ELL ** 4 - 1 / ELL ** 2) * math.exp(-delta ** 2 / (2 * ELL ** 2))
    assert tr[0, C_GN] == pytest.approx(g, rel=1e-12)
    assert tr[0, C_FPP] == pytest.approx(g * g * fss, rel=1e-12)


def test_translation_newton_iterates():
    """Repeated steps follow the scalar Newton iteration on the remaining
    offset: the pose each iteration starts from carries the sum of the
    earlier steps."""
    delta = 0.3 * ELL
    T, info, tr = oracle.register(*axial_pair(delta), np.eye(4), ell=ELL, max_iters=4,
                                  step_tol_rot=0.0, step_tol_trans=0.0)
    rem, moved = delta, 0.0
    for k in range(tr.shape[0]):
        assert tr[k, C_T0 + 3] == pytest.approx(moved, abs=1e-15)   # T_k[0, 3]
        s = newton_translation(rem)
        moved += s
        rem -= s
    assert T[0, 3] == pytest.approx(moved, abs=1e-15)
    # Newton's quadratic convergence: the offset left after three steps is at rounding level
    assert abs(T[0, 3] - delta) < 1e-12


def test_single_pair_converges_onto_its_maximiser_set():
    """For one pair of points F = exp(-|x - T z|^2 / 2 l^2) is maximal exactly
    on the poses with T z = x (a set, since rotations about the line through
    x are free); from an off-axis start the ascent, rotation included, ends
    on it and stops by its step test."""
    X = np.array([[0.4, -0.2, 0.9]])
    Z = np.array([[0.5, 0.05, 0.8]])
    T, info, tr = oracle.register(X, Z, np.eye(4), ell=ELL, max_iters=300, step_tol_rot=1e-12,
                                  step_tol_trans=1e-12)
    assert info["status"] == 0 and info["iters"] < 300
    assert tr[0, C_SROT] > 0.0                       # the path rotates as well as translates
    assert np.linalg.norm(T[:3, :3] @ Z[0] + T[:3, 3] - X[0]) < 1e-10
    assert info["F"] == pytest.approx(1.0, abs=1e-15)


def test_translation_clamp_half_lengthscale():
    delta = 0.45 * ELL                       # Newton step 0.564 l, clamped to 0.5 l
    assert newton_translation(delta) > 0.5 * ELL
    T, _, tr = oracle.register(*axial_pair(delta), np.eye(4), ell=ELL, max_iters=1)
    assert T[0, 3] == pytest.approx(0.5 * ELL, rel=1e-14)
    assert tr[0, C_STR] == pytest.approx(0.5 * ELL, rel=1e-14)


def test_translation_clamp_explicit():
    delta = 0.3 * ELL
    T, _, _ = oracle.register(*axial_pair(delta), np.eye(4), ell=ELL, max_iters=1, max_step_trans=0.05)
    assert T[0, 3] == pytest.approx(0.05, rel=1e-14)


def test_step_to_the_trust_edge_where_curvature_is_not_negative():
    delta = 1.5 * ELL                        # beyond the inflection point: F'' > 0 along the direction
    T, _, tr = oracle.register(*axial_pair(delta), np.eye(4), ell=ELL, max_iters=1)
    assert tr[0, C_FPP] > 0.0
    assert T[0, 3] == pytest.approx(0.5 * ELL, rel=1e-12)
    T, _, _ = oracle.register(*axial_pair(delta), np.eye(4), ell=ELL, max_iters=1, max_step_trans=0.03)
    assert T[0, 3] == pytest.approx(0.03, rel=1e-12)


def test_zero_gradient_takes_no_step_and_stops():
    X, _ = axial_pair(0.0)
    T, info, tr = oracle.register(X, X.copy(), np.eye(4), ell=ELL, max_iters=5)
    assert np.array_equal(T, np.eye(4))
    assert info["status"] == 0 and info["iters"] == 1 and tr[0, C_T] == 0.0


def test_rotation_newton_step():
    r, phi = 1.0, 0.05
    a = r * r / ELL ** 2
    # cutoff 3 l = 1.5 keeps each point with its own partner only (the others are 2 r apart)
    T, _, tr = oracle.register(*symmetric_pairs(r, phi), np.eye(4), ell=ELL, cutoff_mult=3.0, max_iters=1)
    assert tr[0, C_NP] == 2
    theta = math.atan2(T[1, 0], T[0, 0])
    assert theta == pytest.approx(newton_rotation(phi, a), rel=1e-12)
    assert np.abs(T[:3, 3]).max() < 1e-15
    assert np.allclose(T[:3, :3], rz(theta), atol=1e-15)


def test_update_composes_on_the_left():
    """The step is a perturbation of the pose on the left, T <- exp(t g^) T:
    with Z moved by -t0 and T_init a translation by t0, the problem at T_init
    is the symmetric one above, and the step rotates T_init's translation too."""
    r, phi = 1.0, 0.05
    a = r * r / ELL ** 2
    t0 = np.array([0.3, -0.2, 0.1])
    X, Z = symmetric_pairs(r, phi)
    T_init = np.eye(4)
    T_init[:3, 3] = t0
    T, _, _ = oracle.register(X, Z - t0, T_init, ell=ELL, cutoff_mult=3.0, max_iters=1)
    R = rz(newton_rotation(phi, a))
    assert np.allclose(T[:3, :3], R, atol=1e-14)
    assert np.allclose(T[:3, 3], R @ t0, atol=1e-14)
    assert np.abs(T[:3, 3] - t0).max() > 1e-3     # a right-composed update would keep t0


def test_rotation_newton_iterates():
    r, phi = 1.0, 0.08
    a = r * r / ELL ** 2
    _, _, tr = oracle.register(*symmetric_pairs(r, phi), np.eye(4), ell=ELL, cutoff_mult=3.0, max_iters=4,
                               step_tol_rot=0.0, step_tol_trans=0.0)
    u, total = phi, 0.0
    for k in range(tr.shape[0]):
        Tk = tr[k, C_T0:C_T0 + 12].reshape(3, 4)
        assert math.atan2(Tk[1, 0], Tk[0, 0]) == pytest.approx(total, abs=1e-14)
        s = newton_rotation(u, a)
        total += s
        u -= s


def test_rotation_clamp():
    r, phi = 1.0, 0.3
    a = r * r / ELL ** 2
    assert newton_rotation(phi, a) > 0.1 > 0.0
    T, _, tr = oracle.register(*symmetric_pairs(r, phi), np.eye(4), ell=ELL, cutoff_mult=3.0, max_iters=1)
    assert math.atan2(T[1, 0], T[0, 0]) == pytest.approx(0.1, rel=1e-13)
    T, _, _ = oracle.register(*symmetric_pairs(r, phi), np.eye(4), ell=ELL, cutoff_mult=3.0, max_iters=1,
                              max_step_rot=0.02)
    assert math.atan2(T[1, 0], T[0, 0]) == pytest.approx(0.02, rel=1e-13)


@pytest.fixture(scope="module")
def annealed_run():
    p = scenes.cube_pair(n=500, seed=11)
    kw = dict(FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.4, ell_min=0.15, cutoff_mult=3.0, max_iters=200,
              anneal=True, decay=0.9, indicator_tol=2e-3)
    return oracle.register(p.X, p.Z, np.eye(4), **kw), kw


def test_annealing_trigger_sequence(annealed_run):
    """Each decay fires exactly when the indicator is within the tolerance of
    the reference taken at the same lengthscale; a decay clears the
    reference; the lengthscale only changes by a decay, and never below its
    floor."""
    (T, info, tr), kw = annealed_run
    decays = int(tr[:, C_DEC].sum())
    assert decays >= 5 and tr[-1, C_ELL] == kw["ell_min"]
    have_ref, i_ref = False, 0.0
    for k in range(tr.shape[0]):
        ell, ith = tr[k, C_ELL], tr[k, C_ITH]
        nxt = tr[k + 1, C_ELL] if k + 1 < tr.shape[0] else None
        if ell > kw["ell_min"]:
            fire = have_ref and abs(ith - i_ref) < kw["indicator_tol"] * abs(i_ref)
            assert bool(tr[k, C_DEC]) == fire, k
            if fire:
                have_ref = False
                if nxt is not None:
                    assert nxt == pytest.approx(max(kw["decay"] * ell, kw["ell_min"]), rel=1e-15)
            else:
                have_ref, i_ref = True, ith
                if nxt is not None:
                    assert nxt == ell
        else:
            assert tr[k, C_DEC] == 0 and (nxt is None or nxt == ell)


def test_a_decay_needs_a_reference_at_the_new_lengthscale():
    """With a decay so gentle that the indicator barely moves, a reference kept
    across a decay would fire again at once; the rule asks for a fresh
    reference first, so no two decays are adjacent and they come at least
    two iterations apart."""
    p = scenes.cube_pair(n=400, seed=14)
    _, _, tr = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.3, ell_min=0.2,
                               cutoff_mult=3.0, max_iters=60, anneal=True, decay=0.9999, indicator_tol=5e-2)
    fired = np.nonzero(tr[:, C_DEC])[0]
    assert fired.size >= 10
    assert np.diff(fired).min() == 2


def test_stopping_test(annealed_run):
    """The run stops at the first iteration at the lengthscale floor whose
    step is below both tolerances, and at no earlier one."""
    (T, info, tr), kw = annealed_run
    assert info["status"] == 0 and info["iters"] == tr.shape[0]
    small = (tr[:, C_SROT] < 1e-5) & (tr[:, C_STR] < 1e-5)
    at_floor = tr[:, C_ELL] <= kw["ell_min"]
    hits = np.nonzero(small & at_floor)[0]
    assert hits.size == 1 and hits[0] == tr.shape[0] - 1
    assert info["last_step_rot"] == tr[-1, C_SROT] and info["last_step_trans"] == tr[-1, C_STR]


def test_iteration_cap_reports_not_converged():
    p = scenes.cube_pair(n=300, seed=12)
    T, info, tr = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.3,
                                  cutoff_mult=3.0, max_iters=3)
    assert info["status"] == 1 and info["iters"] == 3 == tr.shape[0]


def test_rotation_stays_orthonormal_over_long_runs():
    """Forty-odd composed updates (the rotation is re-orthonormalised every
    sixteen iterations) leave R orthonormal to rounding."""
    p = scenes.cube_pair(n=300, seed=13)
    T, info, tr = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.3,
                                  cutoff_mult=3.0, max_iters=45, step_tol_rot=0.0, step_tol_trans=0.0)
    assert info["iters"] == 45
    R = T[:3, :3]
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-13 and np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
    assert np.array_equal(T[3], [0.0, 0.0, 0.0, 1.0])


Q_FAR = (30.0, -20.0, 50.0)


def rotation_about(q, theta):
    """The pose that rotates by theta about the z axis through q."""
    R = rz(theta)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = np.asarray(q) - R @ np.asarray(q)
    return T


def test_rotation_newton_iterates_about_an_off_origin_centre():
    """The pairs point-symmetric about a centre q far from the origin: the
    ascent direction is the rotation about q (not about the origin), and
    the iterates are the closed-form Newton iterates of the centred problem."""
    r, phi = 1.0, 0.08
    a = r * r / ELL ** 2
    T, _, tr = oracle.register(*symmetric_pairs(r, phi, Q_FAR), np.eye(4), ell=ELL, cutoff_mult=3.0, max_iters=4,
                               step_tol_rot=0.0, step_tol_trans=0.0)
    u, total = phi, 0.0
    for k in range(tr.shape[0]):
        Tk = np.eye(4)
        Tk[:3, :] = tr[k, C_T0:C_T0 + 12].reshape(3, 4)
        assert np.allclose(Tk, rotation_about(Q_FAR, total), atol=1e-12), k
        assert tr[k, C_STR] < 1e-12                       # the centre does not move
        s = newton_rotation(u, a)
        total += s
        u -= s
    assert np.allclose(T, rotation_about(Q_FAR, total), atol=1e-12)


def test_rotation_trust_region_bounds_the_points_motion():
    """A rotation by s moves Z's points, at distance r from its centroid, by
    r s: the step is at most half a lengthscale of motion, 0.5 l / r, below
    max_step_rot here; where F'' >= 0 the step goes to that edge."""
    r, ell = 1.0, 0.15
    a = r * r / ell ** 2
    edge = 0.5 * ell / r
    assert edge < 0.1
    # F'' < 0 and the Newton step beyond the edge
    phi = 0.08
    assert math.cos(phi) - a * math.sin(phi) ** 2 > 0 and newton_rotation(phi, a) > edge
    T, _, tr = oracle.register(*symmetric_pairs(r, phi, Q_FAR), np.eye(4), ell=ell, cutoff_mult=3.0, max_iters=1)
    assert tr[0, C_FPP] < 0.0 and tr[0, C_SROT] == pytest.approx(edge, rel=1e-12)
    assert np.allclose(T, rotation_about(Q_FAR, edge), atol=1e-12)
    # F'' >= 0 along the rotation: the step to the edge
    phi = 0.3
    assert math.cos(phi) - a * math.sin(phi) ** 2 < 0
    T, _, tr = oracle.register(*symmetric_pairs(r, phi, Q_FAR), np.eye(4), ell=ell, cutoff_mult=3.0, max_iters=1)
    assert tr[0, C_FPP] >= 0.0 and tr[0, C_SROT] == pytest.approx(edge, rel=1e-12)


def test_registration_is_equivariant_under_a_common_rigid_motion():
    """Moving both clouds by one rigid motion G (and the start pose by
    conjugation) moves the whole trajectory the same way: T' = G T G^-1 at
    every iteration, with the same indicators, lengthscales and decisions."""
    p = scenes.cube_pair(n=400, seed=31)
    G = oracle.se3_exp(np.array([0.4, -0.7, 0.25, 12.0, -30.0, 45.0]))
    T0 = oracle.se3_exp(np.array([0.01, 0.02, -0.015, 0.03, 0.0, -0.02]))
    kw = dict(FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.3, ell_min=0.12, cutoff_mult=3.0, max_iters=40, anneal=True,
              decay=0.9, indicator_tol=2e-3)
    T, info, tr = oracle.register(p.X, p.Z, T0, **kw)
    GX = (G[:3, :3] @ p.X.astype(np.float64).T).T + G[:3, 3]
    GZ = (G[:3, :3] @ p.Z.astype(np.float64).T).T + G[:3, 3]
    Gi = np.linalg.inv(G)
    Tg, infog, trg = oracle.register(GX, GZ, G @ T0 @ Gi, **kw)
    assert infog["iters"] == info["iters"] and info["iters"] >= 10
    assert np.array_equal(trg[:, C_DEC], tr[:, C_DEC]) and tr[:, C_DEC].sum() >= 2
    np.testing.assert_allclose(trg[:, C_ELL], tr[:, C_ELL], rtol=1e-12)
    np.testing.assert_allclose(trg[:, C_ITH], tr[:, C_ITH], rtol=1e-9)
    np.testing.assert_allclose(trg[:, C_SROT], tr[:, C_SROT], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(trg[:, C_STR], tr[:, C_STR], rtol=1e-6, atol=1e-12)
    assert np.abs(Tg - G @ T @ Gi).max() < 1e-9
