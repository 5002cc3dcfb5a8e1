"""The sweep autotuners (cvo_autotune, cvo_autotune_batch): each picks a
tuning from its grid, the tuning sticks to the handle, and results under the
chosen tuning keep the oracle parity of the default one (F relative 1e-5,
gradient 1e-4 of |g|; a batch's poses within 1e-4 of the default tuning's)."""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

CELLS = (0.35, 0.5, 0.7, 1.0)
SUPERS = (1, 2, 3)
ITEM_LENS = (64, 96, 128, 192, 384, 768, 1536)
LANES = (1, 2, 4)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda")


def check_parity(h, X, Z, FX, FZ, T, kw):
    got = h.evaluate(dev(X), dev(Z), T, dev(FX), dev(FZ))
    ref = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, **kw)
    assert got["F"] == pytest.approx(ref["F"], rel=1e-5)
    gtol = 1e-4 * np.linalg.norm(ref["g"]) + 1e-7 * ref["gscale"]
    assert np.abs(got["grad"] - ref["g"]).max() <= gtol


def test_autotune_street_slice():
    p = scenes.street_pair()
    r = np.random.Generator(np.random.PCG64(3))
    ix = r.permutation(len(p.X))[:6000]
    iz = r.permutation(len(p.Z))[:6000]
    X, Z, FX, FZ = p.X[ix], p.Z[iz], p.FX[ix], p.FZ[iz]
    kw = dict(blocks=p.blocks, ell=0.2, cutoff_mult=3.0)
    h = cvo.CVO(**kw)
    assert h.tuning()["cell_factor"] == 0.5 and h.tuning()["super_delta"] == 2
    t = h.autotune(dev(X), dev(Z), p.T_true, dev(FX), dev(FZ))
    assert t["cell_factor"] in CELLS and t["super_delta"] in SUPERS
    assert t["chunk_len"] in ITEM_LENS and t["query_lanes"] in LANES and t["measured_ms"] > 0.0
    # the timed sweep did the work: no faster than the pairs it evaluates allow
    # (6,000 x 6,000 points at l = 0.2 take tens of microseconds)
    ev = h.evaluate(dev(X), dev(Z), p.T_true, dev(FX), dev(FZ))
    assert ev["pairs"] > 1e5 and t["measured_ms"] > 0.01
    cur = h.tuning()
    assert (cur["cell_factor"], cur["super_delta"], cur["chunk_len"], cur["query_lanes"]) == \
        (t["cell_factor"], t["super_delta"], t["chunk_len"], t["query_lanes"])
    check_parity(h, X, Z, FX, FZ, p.T_true, kw)
    # every tuning of the grid keeps parity (spot-check the extremes)
    for cf, sd, ip in [(0.35, 1, 48), (1.0, 3, 128)]:
        h.apply_tuning(cf, sd, ip)
        check_parity(h, X, Z, FX, FZ, p.T_true, kw)


def test_autotune_dense_and_invalid():
    p = scenes.cube_pair(n=1500)
    kw = dict(blocks=p.blocks, ell=0.1, cutoff_mult=0.0)
    h = cvo.CVO(**kw)
    t = h.autotune(dev(p.X), dev(p.Z), p.T_true, dev(p.FX), dev(p.FZ))
    # dense: no grid, so only the work split is tuned
    assert t["cell_factor"] == 0.5 and t["super_delta"] == 2 and t["chunk_len"] in ITEM_LENS
    check_parity(h, p.X, p.Z, p.FX, p.FZ, p.T_true, kw)
    with pytest.raises(cvo.CvoError):
        h.apply_tuning(0.1, 2, 8)
    with pytest.raises(cvo.CvoError):
        h.apply_tuning(0.5, 2, 8)
    with pytest.raises(cvo.CvoError):
        h.apply_tuning(0.5, 2, 128, 3)
    # empty clouds: nothing to time, the tuning is unchanged
    before = h.tuning()
    t = h.autotune(dev(p.X[:0]), dev(p.Z), p.T_true, dev(p.FX[:0]), dev(p.FZ))
    assert t["measured_ms"] == 0.0 and h.tuning() == before


def test_item_length_changes_only_the_work_split():
    """A registration with a cutoff re-plans its work items from the previous
    sweep's stream lengths (chunk_len candidates each).  The item length only
    changes how the pairs are split among warps: from the same start pose the
    first iteration finds exactly the same pairs and F to rounding, and the
    next iterations (fast annealing, so several grid levels are crossed) keep
    F and the pair counts within rounding of each other."""
    p = scenes.street_pair()
    r = np.random.Generator(np.random.PCG64(5))
    ix = r.permutation(len(p.X))[:8000]
    iz = r.permutation(len(p.Z))[:8000]
    X, Z, FX, FZ = (dev(a) for a in (p.X[ix], p.Z[iz], p.FX[ix], p.FZ[iz]))
    traces = []
    for chunk_len in (16, 64, 192):
        h = cvo.CVO(blocks=p.blocks, ell=0.4, ell_min=0.05, anneal=True, decay=0.8, indicator_tol=0.5,
                    cutoff_mult=3.0, max_iters=12)
        h.apply_tuning(0.5, 2, chunk_len)
        h.register(X, Z, np.eye(4), FX, FZ)
        traces.append(h.trace())
        h.close()
    tr0 = traces[0]
    assert len(set(tr0[:, 0])) >= 3   # the lengthscale moved through several grid levels
    for tr in traces[1:]:
        assert tr.shape == tr0.shape
        assert tr[0, 9] == tr0[0, 9]
        assert tr[0, 1] == pytest.approx(tr0[0, 1], rel=1e-6)
        np.testing.assert_allclose(tr[:, 0], tr0[:, 0], rtol=0)
        np.testing.assert_allclose(tr[:, 1], tr0[:, 1], rtol=1e-5)
        # later poses differ by rounding: a few pairs on the cutoff sphere may differ
        np.testing.assert_allclose(tr[:, 9], tr0[:, 9], rtol=1e-4)


def test_autotune_batch():
    """The batch tuner times cvo_register_batch on the pairs themselves; the
    kept tuning gives the default tuning's poses (within 1e-4 rad and m) and
    iteration counts (give or take one)."""
    pairs = scenes.batch_pairs(n_pairs=6, n_range=(3000, 9000))
    pr = pairs[0].params
    kw = dict(blocks=pairs[0].blocks, ell=pr["ell"], cutoff_mult=pr["cutoff_mult"], max_iters=pr["max_iters"])
    args = [(dev(q.X), dev(q.Z), np.eye(4), dev(q.FX).to(torch.bfloat16), dev(q.FZ).to(torch.bfloat16))
            for q in pairs]
    with cvo.CVO(**kw) as h:
        T0, inf0, _ = h.register_batch(args)
        t = h.autotune_batch(args)
        assert t["cell_factor"] in CELLS and t["super_delta"] in SUPERS and t["chunk_len"] in ITEM_LENS
        assert t["query_lanes"] in LANES
        assert t["measured_ms"] > 0.0
        cur = h.tuning()
        assert (cur["cell_factor"], cur["super_delta"], cur["chunk_len"], cur["query_lanes"]) == \
            (t["cell_factor"], t["super_delta"], t["chunk_len"], t["query_lanes"])
        T1, inf1, _ = h.register_batch(args)
        # nothing to time: the tuning is kept as it is
        assert h.autotune_batch([])["measured_ms"] == 0.0 and h.tuning() == cur
    for k in range(len(pairs)):
        xi = oracle.se3_log(np.linalg.inv(T0[k]) @ T1[k])
        assert np.linalg.norm(xi[:3]) <= 1e-4 and np.linalg.norm(xi[3:]) <= 1e-4, (k, xi)
        assert abs(inf0[k]["iters"] - inf1[k]["iters"]) <= 1, k
