"""Batched registration (cvo_register_batch): pairs of uneven size registered
in one launch sequence agree with registering each pair alone.

The single-pair path is itself checked against the FP64 oracle
(test_gpu_parity.py); the batch shares its kernels but splits the sweep grid
among the pairs, so sums are grouped differently and results agree to
rounding, not bitwise.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-4


def pose_err(Ta, Tb):
    xi = oracle.se3_log(np.linalg.inv(Ta) @ Tb)
    return np.linalg.norm(xi[:3]), np.linalg.norm(xi[3:])


def small_batch(n_pairs=6, seed=4242):
    pairs = scenes.batch_pairs(n_pairs=n_pairs, seed=seed, n_range=(1500, 7000))
    out = []
    for p in pairs:
        X, Z = torch.tensor(p.X, device="cuda"), torch.tensor(p.Z, device="cuda")
        FX = torch.tensor(p.FX, device="cuda").to(torch.bfloat16)
        FZ = torch.tensor(p.FZ, device="cuda").to(torch.bfloat16)
        out.append((X, Z, np.eye(4), FX, FZ))
    return pairs, out


KW = dict(ell=0.2, cutoff_mult=3.0, max_iters=40)


def test_batch_matches_single_pairs():
    pairs, args = small_batch()
    blocks = pairs[0].blocks
    with cvo.CVO(blocks=blocks, **KW) as h:
        T_batch, infos, rc = h.register_batch(args)
        singles = [h.register(*a) for a in args]
    assert rc in (cvo.Status.OK, cvo.Status.NOT_CONVERGED)
    for k, (Ts, info_s) in enumerate(singles):
        er, et = pose_err(T_batch[k], Ts)
        assert er <= POSE_TOL and et <= POSE_TOL, (k, er, et)
        assert abs(infos[k]["iters"] - info_s["iters"]) <= 1
        assert infos[k]["F"] == pytest.approx(info_s["F"], rel=1e-4)
        assert infos[k]["pairs"] == pytest.approx(info_s["pairs"], rel=1e-3)


def test_batch_moves_towards_truth_and_masks_converged_pairs():
    pairs, args = small_batch(n_pairs=4, seed=99)
    with cvo.CVO(blocks=pairs[0].blocks, ell=0.2, cutoff_mult=3.0, max_iters=300, step_tol_rot=1e-4,
                 step_tol_trans=1e-4) as h:
        T_batch, infos, rc = h.register_batch(args)
    iters = [i["iters"] for i in infos]
    # pairs stop on their own: not all at the cap
    assert min(iters) < 300
    for k, p in enumerate(pairs):
        e0 = pose_err(np.eye(4), p.T_true)
        e1 = pose_err(T_batch[k], p.T_true)
        assert e1[0] < e0[0] and e1[1] < e0[1]


def test_batch_with_empty_pair_and_host_buffers():
    pairs, args = small_batch(n_pairs=3, seed=7)
    p = pairs[1]
    empty = (torch.zeros((0, 3), device="cuda"), args[0][1], np.eye(4),
             torch.zeros((0, 22), device="cuda", dtype=torch.bfloat16), args[0][4])
    host = (p.X, p.Z, np.eye(4), scenes.bf16_bits(p.FX), scenes.bf16_bits(p.FZ))
    with cvo.CVO(blocks=p.blocks, **KW) as h:
        T_batch, infos, rc = h.register_batch([args[0], empty, host])
        T_single, _ = h.register(*args[0])
        T_host_single, _ = h.register(*args[1])
    assert np.array_equal(T_batch[1], np.eye(4)) and infos[1]["status"] == 0 and infos[1]["iters"] == 0
    er, et = pose_err(T_batch[0], T_single)
    assert er <= POSE_TOL and et <= POSE_TOL
    er, et = pose_err(T_batch[2], T_host_single)
    assert er <= POSE_TOL and et <= POSE_TOL


def test_phased_setup_of_device_batches_equals_per_pair_setup():
    """A batch of device-resident pairs runs each setup phase for all pairs
    before one wait; a batch with a host-resident pair sets the pairs up one
    after another.  The kernels and their order per pair are the same, so the
    results are bitwise equal."""
    pairs, args = small_batch(n_pairs=4, seed=31)
    host_last = args[:3] + [(pairs[3].X, pairs[3].Z, np.eye(4), scenes.bf16_bits(pairs[3].FX),
                             scenes.bf16_bits(pairs[3].FZ))]
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        T_dev, infos_dev, _ = h.register_batch(args)
        T_mix, infos_mix, _ = h.register_batch(host_last)
    for k in range(4):
        assert np.array_equal(T_dev[k], T_mix[k]), k
        assert infos_dev[k]["F"] == infos_mix[k]["F"] and infos_dev[k]["pairs"] == infos_mix[k]["pairs"]
