"""X-row shards of one registration (cvo_shard_begin / sweep / step / end)
on one GPU: two or three handles each hold a contiguous block of X's rows
and all of Z; every iteration their sweep statistics are summed (the sum an
all-reduce over GPUs would give) and each takes the step from the sum.

Checks: the shards stay in lockstep (bitwise the same trace and pose); the
statistics at the start pose are those of one sweep over all of X (F,
gradient and indicator of the first trace row against cvo_evaluate within
the parity tolerances, the pair count exact); the sharded registration
follows the unsharded one over its first iterations; and at sampled
iterations of the sharded trajectory the FP64 oracle, stepping once from the
recorded pose and lengthscale over the whole clouds, gives the same F, pair
count and next pose."""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

F_RTOL = 1e-5
POSE_TOL = 1e-4


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda")


def trace_pose(row):
    T = np.eye(4)
    T[:3, :] = row[10:22].reshape(3, 4)
    return T


@pytest.fixture(scope="module")
def street():
    p = scenes.street_pair()
    sel = np.random.Generator(np.random.PCG64(21)).permutation(p.n)[:7000]
    return p, p.X[sel], p.Z[sel], p.FX[sel], p.FZ[sel]


KW = dict(ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=40, anneal=True)


def run_shards(blocks, X, Z, FX, FZ, nshards, T0=np.eye(4)):
    n = X.shape[0]
    hs = [cvo.CVO(blocks=blocks, **KW) for _ in range(nshards)]
    stats = [torch.zeros(cvo.SHARD_STATS, dtype=torch.float64, device="cuda") for _ in range(nshards)]
    Zd, FZd = dev(Z), dev(FZ)
    for r, h in enumerate(hs):
        lo, hi = cvo.shard_rows(n, nshards, r)
        cvo.cvo_shard_begin(h.h, dev(X[lo:hi]), Zd, n, T0, dev(FX[lo:hi]), FZd)
    total = torch.zeros(cvo.SHARD_STATS, dtype=torch.float64, device="cuda")
    for it in range(KW["max_iters"]):
        for h, s in zip(hs, stats):
            cvo.cvo_shard_sweep(h.h, s)
        torch.sum(torch.stack(stats), dim=0, out=total)
        done = [cvo.cvo_shard_step(h.h, total, wait=True) for h in hs]
        assert len(set(done)) == 1
        if done[0]:
            break
    out = []
    for h in hs:
        T, info = cvo.cvo_shard_end(h.h)
        out.append((T, info, h.trace()))
        h.close()
    return out


@pytest.mark.parametrize("nshards", [2, 3])
def test_shards_in_lockstep_and_equal_to_one_sweep(street, nshards):
    p, X, Z, FX, FZ = street
    res = run_shards(p.blocks, X, Z, FX, FZ, nshards)
    T0, i0, tr0 = res[0]
    for T, info, tr in res[1:]:
        assert np.array_equal(T, T0) and info["iters"] == i0["iters"]
        np.testing.assert_array_equal(tr, tr0)
    assert tr0.shape[0] == i0["iters"] >= 10
    # the first iteration's statistics are those of one sweep over all of X
    with cvo.CVO(blocks=p.blocks, **KW) as h:
        ev = h.evaluate(dev(X), dev(Z), np.eye(4), dev(FX), dev(FZ))
        Tu, iu = h.register(dev(X), dev(Z), np.eye(4), dev(FX), dev(FZ))
        tru = h.trace()
    assert tr0[0, 1] == pytest.approx(ev["F"], rel=F_RTOL)
    assert tr0[0, 2] == pytest.approx(ev["F"] / math.sqrt(X.shape[0] * Z.shape[0]), rel=F_RTOL)
    assert tr0[0, 9] == ev["pairs"]
    # the unsharded registration over the first iterations (column 3: the
    # slope of F along the step's direction, square-rooted)
    assert tr0[0, 3] == pytest.approx(tru[0, 3], rel=1e-4)
    k = 5
    np.testing.assert_allclose(tr0[:k, 1], tru[:k, 1], rtol=F_RTOL)
    np.testing.assert_allclose(tr0[:k, 10:22], tru[:k, 10:22], atol=POSE_TOL)


def test_sharded_trajectory_one_step_parity_with_oracle(street):
    p, X, Z, FX, FZ = street
    T_final, info, tr = run_shards(p.blocks, X, Z, FX, FZ, 2)[0]
    last = tr.shape[0] - 1
    for k in sorted({0, 2, 9, last // 2, last}):
        T_k, ell_k = trace_pose(tr[k]), tr[k, 0]
        T_next = trace_pose(tr[k + 1]) if k < last else T_final
        T1, _, otr = oracle.register(X, Z, T_k, FX=FX, FZ=FZ, blocks=p.blocks, ell=ell_k, cutoff_mult=3.0,
                                     max_iters=1)
        assert tr[k, 1] == pytest.approx(otr[0, 1], rel=F_RTOL), k
        rc2 = (3.0 * ell_k) ** 2
        band = oracle.count_band(X, Z, T_k, rc2 * (1 - 1e-5), rc2 * (1 + 1e-5))
        assert abs(tr[k, 9] - otr[0, 9]) <= band, k
        xi = oracle.se3_log(np.linalg.inv(T_next) @ T1)
        assert np.linalg.norm(xi[:3]) <= POSE_TOL and np.linalg.norm(xi[3:]) <= POSE_TOL, k


def test_register_sharded_single_shard_matches_register(street):
    """register_sharded with no all-reduce (one shard holding every row) is
    the plain registration with another loop driver: the same decisions."""
    p, X, Z, FX, FZ = street
    with cvo.CVO(blocks=p.blocks, **KW) as h:
        Ts, infs = h.register_sharded(dev(X), dev(Z), X.shape[0], np.eye(4), dev(FX), dev(FZ))
        trs = h.trace()
        Tu, infu = h.register(dev(X), dev(Z), np.eye(4), dev(FX), dev(FZ))
        tru = h.trace()
    k = min(trs.shape[0], tru.shape[0], 8)
    np.testing.assert_allclose(trs[:k, 1], tru[:k, 1], rtol=F_RTOL)
    assert infs["iters"] == trs.shape[0]


def test_shard_calls_check_their_arguments(street):
    p, X, Z, FX, FZ = street
    with cvo.CVO(blocks=p.blocks, **KW) as h:
        s = torch.zeros(cvo.SHARD_STATS, dtype=torch.float64, device="cuda")
        with pytest.raises(cvo.CvoError) as e:
            cvo.cvo_shard_sweep(h.h, s)
        assert "no shard registration" in str(e.value)
        with pytest.raises(cvo.CvoError) as e:
            cvo.cvo_shard_begin(h.h, dev(X[:10]), dev(Z), 5, np.eye(4), dev(FX[:10]), dev(FZ))
        assert "n_total" in str(e.value)
