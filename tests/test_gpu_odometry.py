"""Frame-to-frame odometry (cvo_register_sequence) on a synthetic street
sequence: the chaining (first pair from the identity at the larger
lengthscale, later pairs warm-started from the previous motion), the
composition of absolute poses and accuracy against the generator's motions;
and parity with the oracle's own chaining on frames with a sharp optimum
(converged poses within 1e-4 rad / 1e-4 m).  Street frames are not used for
parity: their optimum is flat along some directions, so two correct
optimisers stop at points that differ by more than the pose tolerance."""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

BLOCKS = [("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]
POSE_TOL = 1e-4


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda")


def pose_err(A, B):
    D = np.linalg.inv(A) @ B
    ang = math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1.0) / 2.0)))
    return ang, float(np.linalg.norm(D[:3, 3]))


@pytest.fixture(scope="module")
def seq():
    return scenes.street_sequence(n_frames=6, n=10000)


def test_sequence_chaining_and_accuracy(seq):
    frames, C = seq
    kw = dict(blocks=BLOCKS, ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=200, anneal=True)
    h = cvo.CVO(**kw)
    fd = [(dev(P), dev(F)) for P, F in frames]
    T_rel, T_abs, infos, rc = h.register_sequence(fd, ell_first=0.6)
    assert T_rel.shape == (5, 4, 4) and T_abs.shape == (6, 4, 4) and len(infos) == 5
    # every pair equals a standalone registration with the documented start
    h2 = cvo.CVO(**kw)
    for k in range(5):
        if k == 0:
            h2.set_params(**dict(kw, ell=0.6))
            init = np.eye(4)
        else:
            h2.set_params(**kw)
            init = T_rel[k - 1]
        T, info = h2.register(fd[k][0], fd[k + 1][0], init, fd[k][1], fd[k + 1][1])
        assert np.array_equal(T, T_rel[k]), k
        assert info["iters"] == infos[k]["iters"]
    # absolute poses are the running products
    acc = np.eye(4)
    assert np.array_equal(T_abs[0], acc)
    for k in range(5):
        acc = acc @ T_rel[k]
        assert np.abs(T_abs[k + 1] - acc).max() < 1e-12
    # accuracy against the generator's motions (independent ray casts with
    # depth noise growing as 0.002 d^2, so not exact): every frame within
    # 1 deg and 10 cm
    for k in range(5):
        truth = np.linalg.inv(C[k]) @ C[k + 1]
        ang, tr = pose_err(T_rel[k], truth)
        assert ang < math.radians(1.0) and tr < 0.10, (k, math.degrees(ang), tr)


def test_sequence_matches_oracle_chaining():
    """Frames that are exact rigid copies of one box-surface cloud (a sharp
    optimum at the true motion): the GPU's chained relative poses equal the
    oracle's, and both equal the true motions, within the pose tolerance."""
    r = np.random.Generator(np.random.PCG64(41))
    W, fl = scenes.sample_box_faces(r, 1500, (4.0, 4.0, 4.0))
    F = np.concatenate([scenes.smooth_rgb(W), scenes.label_distribution(r, fl)], axis=1).astype(np.float32)
    C = [np.eye(4)]
    for _ in range(3):
        C.append(C[-1] @ scenes.random_motion(r, 4.0, 0.15))
    frames = [(scenes.apply(np.linalg.inv(Ck), W).astype(np.float32), F) for Ck in C]
    kw = dict(blocks=BLOCKS, cutoff_mult=3.0, max_iters=300)
    h = cvo.CVO(ell=0.15, **kw)
    T_rel, T_abs, infos, rc = h.register_sequence([(dev(P), dev(Fk)) for P, Fk in frames], ell_first=0.3)
    R_rel, R_abs, rinfos = oracle.register_sequence(frames, 0.3, ell=0.15, **kw)
    for k in range(3):
        assert infos[k]["status"] == 0 and rinfos[k]["status"] == 0, k
        ang, tr = pose_err(T_rel[k], R_rel[k])
        assert ang <= POSE_TOL and tr <= POSE_TOL, (k, ang, tr)
        ang, tr = pose_err(T_rel[k], np.linalg.inv(C[k]) @ C[k + 1])
        assert ang <= POSE_TOL and tr <= POSE_TOL, (k, ang, tr)
    for k in range(4):
        ang, tr = pose_err(T_abs[k], R_abs[k])
        assert ang <= 3 * POSE_TOL and tr <= 3 * POSE_TOL


def test_sequence_edge_cases(seq):
    frames, _ = seq
    h = cvo.CVO(blocks=BLOCKS, ell=0.1, cutoff_mult=3.0, max_iters=5)
    P, F = frames[0]
    # one frame: nothing to register, T_abs = I
    T_rel, T_abs, infos, rc = h.register_sequence([(dev(P), dev(F))], ell_first=0.3)
    assert T_rel.shape[0] == 0 and np.array_equal(T_abs[0], np.eye(4)) and rc == 0
    # an empty frame in the middle returns its start pose (status OK)
    e = (dev(P[:0]), dev(F[:0]))
    T_rel, T_abs, infos, rc = h.register_sequence([(dev(P), dev(F)), e, (dev(P), dev(F))], ell_first=0.3)
    assert np.array_equal(T_rel[0], np.eye(4)) and np.array_equal(T_rel[1], np.eye(4))
    with pytest.raises(cvo.CvoError):
        h.register_sequence([(dev(P), dev(F))] * 2, ell_first=-1.0)
