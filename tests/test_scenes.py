"""The seeded synthetic inputs keep the shapes, sizes and value ranges their
recipe states (the paper's workloads stand in by these generators): point
counts, extents, feature layout and ranges, label distributions, the
ground-truth motions' bounds, and determinism under a fixed seed."""
import numpy as np
import pytest

import scenes


def rot_angle_deg(T):
    c = (np.trace(T[:3, :3]) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def check_rigid(T):
    R = T[:3, :3]
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-9) and np.linalg.det(R) == pytest.approx(1.0, abs=1e-9)
    assert np.array_equal(T[3], [0.0, 0.0, 0.0, 1.0])


def check_labels(F, start):
    lab = F[:, start:start + 19].astype(np.float64)
    assert lab.min() >= 0.0
    assert np.allclose(lab.sum(1), 1.0, atol=2e-2)   # bf16-rounded probabilities


def test_cube_pair():
    p = scenes.cube_pair()
    assert p.X.shape == (2000, 3) and p.Z.shape == (2000, 3) and p.X.dtype == np.float32
    # faces of a 4 m cube (plus 5 mm noise)
    assert np.abs(p.X).max() == pytest.approx(2.0, abs=0.05)
    assert np.all(np.abs(p.X).max(1) > 2.0 - 0.03)
    assert p.FX.shape == (2000, 3) and 0.0 <= p.FX.min() and p.FX.max() <= 1.0
    check_rigid(p.T_true)
    # Z = T_gt X with the same points: T_true maps Z back onto X
    back = scenes.apply(p.T_true, p.Z.astype(np.float64))
    assert np.abs(back - p.X).max() < 1e-5
    assert rot_angle_deg(p.T_true) == pytest.approx(5.0, abs=1e-6)
    assert np.linalg.norm(np.linalg.inv(p.T_true)[:3, 3]) == pytest.approx(0.1, abs=1e-9)


def test_street_pair():
    p = scenes.street_pair()
    assert p.X.shape == (20000, 3) and p.Z.shape == (20000, 3)
    assert p.FX.shape == (20000, 22) and p.FZ.shape == (20000, 22)
    check_labels(p.FX, 3)
    check_labels(p.FZ, 3)
    assert 0.0 <= p.FX[:, :3].min() and p.FX[:, :3].max() <= 1.0
    check_rigid(p.T_true)
    assert rot_angle_deg(p.T_true) <= 10.0 + 1e-9
    assert np.linalg.norm(p.T_true[:3, 3]) <= 0.5 + 1e-9   # |t| = |R^T t|: either direction
    # depth along the camera axis within the stated 1-40 m (noise grows as 0.002 d^2)
    d = np.linalg.norm(p.X, axis=1)
    assert d.min() > 0.8 and d.max() < 60.0
    assert p.params["cutoff_mult"] == 3.0 and p.params["ell"] == 0.3 and p.params["max_iters"] == 100


def test_room_pair():
    p = scenes.room_pair()
    assert p.X.shape[0] == 19200 and p.Z.shape[0] == 19200
    check_rigid(p.T_true)
    assert rot_angle_deg(p.T_true) <= 5.0 + 1e-9


def test_batch_pairs_sizes_and_motions():
    pairs = scenes.batch_pairs(n_pairs=8, seed=123)
    assert len(pairs) == 8
    for q in pairs:
        assert 5000 <= q.X.shape[0] <= 60000 and 5000 <= q.Z.shape[0] <= 60000
        assert q.FX.shape[1] == 22
        check_labels(q.FX, 3)
        check_rigid(q.T_true)
        assert rot_angle_deg(q.T_true) <= 8.0 + 1e-9
        # features are representable in bfloat16 (the batch stores them so)
        assert np.array_equal(scenes.bf16_round(q.FX), q.FX)


def test_generators_are_deterministic():
    a, b = scenes.street_pair(), scenes.street_pair()
    assert np.array_equal(a.X, b.X) and np.array_equal(a.FZ, b.FZ) and np.array_equal(a.T_true, b.T_true)
    c = scenes.cube_pair(seed=999)
    assert not np.array_equal(c.X, scenes.cube_pair().X)
