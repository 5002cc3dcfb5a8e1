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


def host_last(pairs, args):
    """The same batch with its last pair in host memory."""
    q = pairs[-1]
    return args[:-1] + [(q.X, q.Z, np.eye(4), scenes.bf16_bits(q.FX), scenes.bf16_bits(q.FZ))]


def assert_bitwise_equal(a, b):
    (Ta, ia, _), (Tb, ib, _) = a, b
    for k in range(len(ia)):
        assert np.array_equal(Ta[k], Tb[k]), k
        assert ia[k]["F"] == ib[k]["F"] and ia[k]["pairs"] == ib[k]["pairs"] and ia[k]["iters"] == ib[k]["iters"], k


def test_batch_from_page_locked_host_memory(monkeypatch):
    """Host-resident inputs of a batch: page-locked ones (pulled into device
    memory by the library's own kernel), some at offsets that are not 16-byte
    aligned, and pageable ones (copied by the driver) give the bits of the
    same batch from device memory."""
    pairs, args = small_batch(n_pairs=5, seed=41)

    def shifted(t):
        # a view one row into a larger page-locked buffer
        big = torch.empty((t.shape[0] + 1,) + tuple(t.shape[1:]), dtype=t.dtype).pin_memory()
        big[1:] = t.cpu()
        return big[1:]

    host = []
    for k, (X, Z, T, FX, FZ) in enumerate(args):
        if k in (0, 2):
            host.append((X.cpu().pin_memory(), Z.cpu().pin_memory(), T, FX.cpu().pin_memory(), FZ.cpu().pin_memory()))
        elif k in (1, 4):
            host.append((shifted(X), shifted(Z), T, shifted(FX), shifted(FZ)))
        else:
            host.append((X.cpu(), Z.cpu(), T, FX.cpu(), FZ.cpu()))
    assert host[1][0].data_ptr() % 16 != 0 and host[1][3].data_ptr() % 16 != 0
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        got = h.register_batch(host)
        assert_bitwise_equal(got, h.register_batch(args))
        with monkeypatch.context() as m:
            m.setenv("CVO_BATCH_SETUP", "pairs")
            assert_bitwise_equal(got, h.register_batch(host))


def test_batch_page_locked_nonfinite_feature_rejected():
    """Page-locked inputs, pulled into device memory by the library's own
    kernel, are checked like device inputs: a NaN in one pair's features (X's,
    then Z's) returns CVO_ERR_INVALID_ARG, and the handle then registers the
    clean batch with the bits it gave before."""
    pairs, args = small_batch(n_pairs=4, seed=43)
    host = [(X.cpu().pin_memory(), Z.cpu().pin_memory(), T, FX.cpu().pin_memory(), FZ.cpu().pin_memory())
            for (X, Z, T, FX, FZ) in args]
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        ref = h.register_batch(host)
        for side in (3, 4):   # X's features, then Z's
            bad = [list(a) for a in host]
            f = bad[2][side].clone().pin_memory()
            f[f.shape[0] // 2, 5] = float("nan")
            bad[2][side] = f
            with pytest.raises(cvo.CvoError) as e:
                h.register_batch([tuple(a) for a in bad])
            assert e.value.status == cvo.Status.ERR_INVALID_ARG
        assert_bitwise_equal(ref, h.register_batch(host))


def batched_and_pairwise(h, args, monkeypatch):
    """A batch set up by the batched stages (one launch per stage for all
    pairs), and set up pair by pair (CVO_BATCH_SETUP=pairs)."""
    got = h.register_batch(args)
    with monkeypatch.context() as m:
        m.setenv("CVO_BATCH_SETUP", "pairs")
        ref = h.register_batch(args)
    return got, ref


def test_batched_setup_equals_per_pair_setup(monkeypatch):
    """The batched set-up runs the per-pair kernels' bodies on the same data
    with stable sorts, so the registrations are bitwise those of the
    pair-by-pair set-up -- here with clouds above and below the one-block
    sort's size; a batch with a host-resident pair (copied to the device
    first) gives the same bits."""
    pairs, args = small_batch(n_pairs=4, seed=31)
    pairs2 = scenes.batch_pairs(n_pairs=2, seed=32, n_range=(9000, 12000))
    for q in pairs2:
        args.append((torch.tensor(q.X, device="cuda"), torch.tensor(q.Z, device="cuda"), np.eye(4),
                     torch.tensor(q.FX, device="cuda").to(torch.bfloat16),
                     torch.tensor(q.FZ, device="cuda").to(torch.bfloat16)))
    pairs = pairs + pairs2
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        got, ref = batched_and_pairwise(h, args, monkeypatch)
        assert_bitwise_equal(got, ref)
        assert_bitwise_equal(got, h.register_batch(host_last(pairs, args)))


def test_batched_setup_over_several_launches_and_levels(monkeypatch):
    """More pairs than one batched launch takes (64), annealed over several
    grid levels: still bitwise the pair-by-pair set-up's results."""
    pairs = scenes.batch_pairs(n_pairs=70, seed=33, n_range=(200, 900))
    args = [(torch.tensor(q.X, device="cuda"), torch.tensor(q.Z, device="cuda"), np.eye(4),
             torch.tensor(q.FX, device="cuda").to(torch.bfloat16), torch.tensor(q.FZ, device="cuda").to(torch.bfloat16))
            for q in pairs]
    kw = dict(ell=0.4, ell_min=0.1, anneal=True, cutoff_mult=3.0, max_iters=30)
    with cvo.CVO(blocks=pairs[0].blocks, **kw) as h:
        assert_bitwise_equal(*batched_and_pairwise(h, args, monkeypatch))


def test_batched_setup_dense(monkeypatch):
    pairs, args = small_batch(n_pairs=3, seed=34)
    args = [(X[:600], Z[:500], T, FX[:600], FZ[:500]) for X, Z, T, FX, FZ in args]
    with cvo.CVO(blocks=pairs[0].blocks, ell=0.2, cutoff_mult=0.0, max_iters=10) as h:
        assert_bitwise_equal(*batched_and_pairwise(h, args, monkeypatch))


def test_batch_lanes_per_query():
    """The batch with 2 and 4 lanes per query (query groups of 16 and 8)
    reaches the one-lane batch's poses to rounding."""
    pairs, args = small_batch(n_pairs=4, seed=35)
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        t = h.tuning()
        T1, i1, _ = h.register_batch(args)
        for lanes in (2, 4):
            h.apply_tuning(t["cell_factor"], t["super_delta"], t["chunk_len"], lanes)
            Tl, il, _ = h.register_batch(args)
            for k in range(len(pairs)):
                er, et = pose_err(T1[k], Tl[k])
                assert er <= POSE_TOL and et <= POSE_TOL, (lanes, k, er, et)
                assert il[k]["F"] == pytest.approx(i1[k]["F"], rel=1e-4), (lanes, k)


def test_work_queue_matches_block_split_and_repeats(monkeypatch):
    """The batched sweep's work queue (CVO_BATCH_QUEUE=1: warps take items
    from a counter, each item's statistics in its own row, summed per pair in
    item order) against the default block split of the same batch: the same
    poses, F and pair counts up to the summation order, and bitwise the same
    results on a second run whatever warp took which item."""
    pairs, args = small_batch(n_pairs=6, seed=47)
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        blk = h.register_batch(args)
        with monkeypatch.context() as m:
            m.setenv("CVO_BATCH_QUEUE", "1")
            q1 = h.register_batch(args)
            q2 = h.register_batch(args)
    assert_bitwise_equal(q1, q2)
    (Tq, iq, _), (Tb, ib, _) = q1, blk
    for k in range(len(iq)):
        er, et = pose_err(Tq[k], Tb[k])
        assert er <= 1e-6 and et <= 1e-6, (k, er, et)
        assert iq[k]["F"] == pytest.approx(ib[k]["F"], rel=1e-6)
        assert abs(iq[k]["pairs"] - ib[k]["pairs"]) <= 2
        assert iq[k]["iters"] == ib[k]["iters"]


def test_pair_order_does_not_change_results(monkeypatch):
    """The batch's pairs enter the sweep largest first whatever their order
    in the call: permuting them gives each pair its pose, F and pair count
    again (to rounding with the block split; bitwise with the work queue,
    whose per-pair sums depend on the items alone)."""
    pairs, args = small_batch(n_pairs=6, seed=53)
    perm = [4, 1, 5, 0, 3, 2]
    with cvo.CVO(blocks=pairs[0].blocks, **KW) as h:
        T0, i0, _ = h.register_batch(args)
        T1, i1, _ = h.register_batch([args[k] for k in perm])
        for j, k in enumerate(perm):
            er, et = pose_err(T0[k], T1[j])
            assert er <= 1e-6 and et <= 1e-6, (k, er, et)
            assert i1[j]["F"] == pytest.approx(i0[k]["F"], rel=1e-6)
            assert i1[j]["iters"] == i0[k]["iters"]
        with monkeypatch.context() as m:
            m.setenv("CVO_BATCH_QUEUE", "1")
            Tq0, iq0, _ = h.register_batch(args)
            Tq1, iq1, _ = h.register_batch([args[k] for k in perm])
    for j, k in enumerate(perm):
        assert np.array_equal(Tq0[k], Tq1[j]), k
        assert iq0[k]["F"] == iq1[j]["F"] and iq0[k]["pairs"] == iq1[j]["pairs"], k
