"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Tolerances (from the arithmetic: FP32 pair terms, exact-offset geometry,
compensated cross-block sums):
  F, i_theta              relative 1e-5
  gradient components     |g_gpu - g_oracle| <= 1e-4 |g_oracle| + 1e-7 G,
                          G = sum over pairs of the norms of the gradient's
                          terms (FP32 rounding floor; |g| -> 0 at an optimum)
  second derivative       d^T H d within 1e-4 relative (plus 1e-4 |H| |d|^2)
  registered pose         |log(T_gpu^-1 T_oracle)| <= 1e-4 rad and 1e-4 m
  pair counts             differ by at most the pairs whose squared distance
                          lies within 1e-5 of the cutoff (FP32 vs FP64 test)
"""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

F_RTOL = 1e-5
G_TOL = 1e-4
G_FLOOR = 1e-7
POSE_TOL = 1e-4


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def bf16_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to("cuda").to(torch.bfloat16)


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def rand_pose(r, ang=0.2, tr=0.3):
    return oracle.se3_exp(np.concatenate([r.normal(size=3) * ang / math.sqrt(3), r.normal(size=3) * tr / math.sqrt(3)]))


def compare_eval(X, Z, FX, FZ, blocks, ell, cm, T, bf16=False, sigma=1.0, ndir=3, seed=0, tuning=None, lanes=1,
                 chunk_len=None):
    h = cvo.CVO(blocks=blocks, ell=ell, cutoff_mult=cm, sigma=sigma)
    if tuning is not None:
        cvo.cvo_set_tuning(h.h, *tuning)
    if lanes != 1 or chunk_len is not None:
        t = h.tuning()
        h.apply_tuning(t["cell_factor"], t["super_delta"], t["chunk_len"] if chunk_len is None else chunk_len, lanes)
    if FX is not None and bf16:
        fx_d, fz_d = bf16_dev(FX), bf16_dev(FZ)
        FXo, FZo = scenes.bf16_round(FX), scenes.bf16_round(FZ)
    elif FX is not None:
        fx_d, fz_d = dev(FX), dev(FZ)
        FXo, FZo = FX, FZ
    else:
        fx_d = fz_d = FXo = FZo = None
    got = h.evaluate(dev(X), dev(Z), T, fx_d, fz_d)
    kw = dict(FX=FXo, FZ=FZo, blocks=blocks, ell=ell, cutoff_mult=cm, sigma=sigma)
    ref = oracle.evaluate(X, Z, T, **kw)
    assert got["F"] == pytest.approx(ref["F"], rel=F_RTOL, abs=1e-300)
    gn = np.linalg.norm(ref["g"])
    # 1e-4 of |g|; near an optimum |g| -> 0 and the FP32 rounding of the
    # per-pair terms sets the floor: 1e-7 of the sum of their magnitudes
    gtol = G_TOL * gn + G_FLOOR * ref["gscale"]
    assert np.abs(got["grad"] - ref["g"]).max() <= gtol, (got["grad"], ref["g"], gtol)
    n, m = np.asarray(X).shape[0], np.asarray(Z).shape[0]
    assert got["i_theta"] == pytest.approx(ref["F"] / math.sqrt(n * m), rel=F_RTOL)
    if cm > 0:
        rc2 = (cm * ell) ** 2
        band = oracle.count_band(X, Z, T, rc2 * (1 - 1e-5), rc2 * (1 + 1e-5))
        assert abs(got["pairs"] - ref["npairs"]) <= band
    else:
        assert got["pairs"] == n * m
    assert got["candidates"] >= got["pairs"]
    H = got["hess"]
    r = rng(seed)
    for _ in range(ndir):
        d = r.normal(size=6) * np.array([1, 1, 1, 1, 1, 1.0])
        fpp = oracle.evaluate(X, Z, T, direction=d, **kw)["Fpp"]
        assert float(d @ H @ d) == pytest.approx(fpp, rel=1e-4, abs=1e-4 * np.abs(H).max() * float(d @ d))
    h.close()
    return got, ref


def test_cube_dense_rgb():
    p = scenes.cube_pair()
    for T in (np.eye(4), p.T_true, rand_pose(rng(1), 0.1, 0.1)):
        compare_eval(p.X, p.Z, p.FX, p.FZ, p.blocks, 0.1, 0.0, T)


def test_cutoff_semantic_ragged():
    r = rng(2)
    n, m = 1037, 999
    X = r.uniform(-0.5, 0.5, size=(n, 3)).astype(np.float32)
    Z = (X[:m] + r.normal(0, 0.02, size=(m, 3))).astype(np.float32)
    FX = np.hstack([r.uniform(0, 1, (n, 3)), r.dirichlet(np.ones(19), n)]).astype(np.float32)
    FZ = np.hstack([r.uniform(0, 1, (m, 3)), r.dirichlet(np.ones(19), m)]).astype(np.float32)
    blocks = [("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]
    compare_eval(X, Z, FX, FZ, blocks, 0.05, 3.0, rand_pose(r, 0.05, 0.03))


def test_cutoff_semantic_bf16():
    r = rng(3)
    n, m = 2100, 1900
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(m, 3)).astype(np.float32)
    FX = np.hstack([r.uniform(0, 1, (n, 3)), r.dirichlet(np.ones(19), n)]).astype(np.float32)
    FZ = np.hstack([r.uniform(0, 1, (m, 3)), r.dirichlet(np.ones(19), m)]).astype(np.float32)
    blocks = [("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]
    compare_eval(X, Z, FX, FZ, blocks, 0.1, 3.0, rand_pose(r, 0.05, 0.05), bf16=True)


SEM_BLOCKS = [("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]


def semantic_features(r, n):
    return np.hstack([r.uniform(0, 1, (n, 3)), r.dirichlet(np.ones(19), n)]).astype(np.float32)


def test_semantic_bf16_far_from_origin():
    """bfloat16 RGB + labels with a cutoff (the label products on the
    tensor-core tile) 80 m from the origin with l = 5 cm: the offsets keep
    their precision (double-float queries) there too."""
    r = rng(16)
    n = 3000
    base = np.array([60.0, -20.0, 80.0])
    X = (base + r.uniform(-1, 1, size=(n, 3))).astype(np.float32)
    Z = (X + r.normal(0, 0.01, size=X.shape)).astype(np.float32)
    FX = semantic_features(r, n)
    FZ = FX.copy()
    FZ[:, :3] = np.clip(FX[:, :3] + r.normal(0, 0.05, (n, 3)), 0, 1)
    compare_eval(X, Z, FX, FZ, SEM_BLOCKS, 0.05, 3.0, rand_pose(r, 0.002, 0.02), bf16=True)


@pytest.mark.parametrize("super_delta", [2, 4, 6])
def test_semantic_bf16_sparse_queries_wide_groups(super_delta):
    """Sparse queries over a dense cloud with octree super-cells of 2^k
    cutoff radii: a query group spans several radii, so its candidate
    stream is long and each candidate is in range of few of its queries."""
    r = rng(17 + super_delta)
    n, m = 700, 9000
    X = r.uniform(-3, 3, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-3, 3, size=(m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.15, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, tuning=(0.5, super_delta))


@pytest.mark.parametrize("n", [1, 5, 31, 33, 100])
def test_semantic_bf16_ragged_groups_and_batches(n):
    """Groups of fewer than 32 queries and staged batches of fewer than 32
    candidates on the tensor-core label tile."""
    r = rng(30 + n)
    m = 3 * n + 7
    X = r.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    Z = r.uniform(-0.3, 0.3, (m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.1, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, ndir=2)


@pytest.mark.parametrize("lanes", [2, 4])
def test_lanes_per_query_semantic_bf16(lanes):
    """Query groups of 32 / lanes queries, each query's candidates shared by
    that many lanes (bfloat16 labels on the tensor-core tile)."""
    r = rng(40 + lanes)
    n, m = 2100, 1900
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.1, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, lanes=lanes)


@pytest.mark.parametrize("lanes", [2, 4])
def test_lanes_per_query_street_f32(lanes):
    p = scenes.street_pair()
    sel = rng(7).permutation(p.n)[:5000]
    compare_eval(p.X[sel], p.Z[sel], p.FX[sel], p.FZ[sel], p.blocks, 0.3, 3.0, p.T_true, lanes=lanes)


@pytest.mark.parametrize("n", [1, 5, 17, 33])
def test_lanes_per_query_ragged(n):
    """Groups smaller than 32 / lanes and batches shorter than 2 lanes x
    candidates."""
    r = rng(60 + n)
    m = 3 * n + 7
    X = r.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    Z = r.uniform(-0.3, 0.3, (m, 3)).astype(np.float32)
    for lanes in (2, 4):
        compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.1, 3.0,
                     rand_pose(r, 0.05, 0.05), bf16=True, ndir=1, lanes=lanes)


def test_lanes_per_query_other_blocks():
    """A block list without a multi-lane sweep keeps one lane per query in
    the smaller groups: still the oracle's sums."""
    r = rng(70)
    X = r.uniform(-2, 2, size=(3001, 3)).astype(np.float32)
    Z = r.uniform(-2, 2, size=(2999, 3)).astype(np.float32)
    compare_eval(X, Z, None, None, [], 0.15, 3.0, rand_pose(r, 0.1, 0.2), lanes=4)


# Planned work items of 768 candidates or more trim the first 32 rows of a
# query group's stream by each query's ball (the set-up loops over the
# group's queries per row); shorter items, and rows past the first 32, take
# the group's box grown by a ball.  The tests above run the default
# 128-candidate items; these run the trimmed streams.
TRIM_LENS = [768, 1536]


@pytest.mark.parametrize("chunk_len", TRIM_LENS)
def test_trimmed_streams_semantic_bf16(chunk_len):
    """Rows trimmed by each query on a dense random cloud, bfloat16 labels on
    the tensor-core tile."""
    r = rng(3)
    n, m = 2100, 1900
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.1, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, chunk_len=chunk_len)


def test_trimmed_streams_far_from_origin():
    """The per-query trim's rounding margins 80 m from the origin with
    l = 5 cm."""
    r = rng(16)
    n = 3000
    base = np.array([60.0, -20.0, 80.0])
    X = (base + r.uniform(-1, 1, size=(n, 3))).astype(np.float32)
    Z = (X + r.normal(0, 0.01, size=X.shape)).astype(np.float32)
    FX = semantic_features(r, n)
    FZ = FX.copy()
    FZ[:, :3] = np.clip(FX[:, :3] + r.normal(0, 0.05, (n, 3)), 0, 1)
    compare_eval(X, Z, FX, FZ, SEM_BLOCKS, 0.05, 3.0, rand_pose(r, 0.002, 0.02), bf16=True, chunk_len=768)


@pytest.mark.parametrize("super_delta", [2, 4, 6])
def test_trimmed_streams_wide_groups(super_delta):
    """Query groups over 2^k cutoff radii: streams of more than 32 rows, the
    first 32 trimmed by each query and the rest by the box."""
    r = rng(17 + super_delta)
    n, m = 700, 9000
    X = r.uniform(-3, 3, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-3, 3, size=(m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.15, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, tuning=(0.5, super_delta), chunk_len=768)


@pytest.mark.parametrize("n", [1, 5, 31, 33, 100])
def test_trimmed_streams_ragged_groups(n):
    """Groups of fewer than 32 queries: the lanes past the group's last query
    take no part in the trim."""
    r = rng(30 + n)
    m = 3 * n + 7
    X = r.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    Z = r.uniform(-0.3, 0.3, (m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.1, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, ndir=2, chunk_len=768)


@pytest.mark.parametrize("lanes", [2, 4])
def test_trimmed_streams_lanes_per_query(lanes):
    """The trim with 2 or 4 lanes per query (each query's position held by
    all of its lanes)."""
    r = rng(50 + lanes)
    n, m = 1500, 2500
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(m, 3)).astype(np.float32)
    compare_eval(X, Z, semantic_features(r, n), semantic_features(r, m), SEM_BLOCKS, 0.1, 3.0,
                 rand_pose(r, 0.05, 0.05), bf16=True, lanes=lanes, chunk_len=768)


def test_trimmed_streams_street_f32():
    """The trim on the float32 feature path (street subsample, RGB + 19
    labels)."""
    p = scenes.street_pair()
    sel = rng(7).permutation(p.n)[:5000]
    compare_eval(p.X[sel], p.Z[sel], p.FX[sel], p.FZ[sel], p.blocks, 0.3, 3.0, p.T_true, chunk_len=768)


def test_trim_keeps_every_pair():
    """The same pair with the box's streams (384-candidate items) and the
    queries' streams (768): the same in-cutoff pair count exactly, fewer
    distance tests, the same double sum up to float32 summation order."""
    r = rng(40)
    n, m = 4000, 4000
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = (X + r.normal(0, 0.02, size=X.shape)).astype(np.float32)
    FX, FZ = semantic_features(r, n), semantic_features(r, m)
    T = rand_pose(r, 0.05, 0.05)
    out = {}
    for chunk_len in (384, 768):
        with cvo.CVO(blocks=SEM_BLOCKS, ell=0.1, cutoff_mult=3.0) as h:
            t = h.tuning()
            h.apply_tuning(t["cell_factor"], t["super_delta"], chunk_len)
            out[chunk_len] = h.evaluate(dev(X), dev(Z), T, bf16_dev(FX), bf16_dev(FZ))
    box, trim = out[384], out[768]
    assert trim["pairs"] == box["pairs"]
    assert box["pairs"] <= trim["candidates"] < box["candidates"]
    assert trim["F"] == pytest.approx(box["F"], rel=1e-6)
    assert np.abs(trim["grad"] - box["grad"]).max() <= 1e-5 * np.abs(box["grad"]).max()


def test_generic_blocks():
    r = rng(4)
    n, m = 700, 650
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(m, 3)).astype(np.float32)
    FX = np.hstack([r.uniform(0, 1, (n, 3)), r.dirichlet(np.ones(4), n)]).astype(np.float32)
    FZ = np.hstack([r.uniform(0, 1, (m, 3)), r.dirichlet(np.ones(4), m)]).astype(np.float32)
    blocks = [("se", 2, 0.3, 1.5), ("dot", 4, 1.0, 1.0), ("se", 1, 0.2, 0.8)]
    compare_eval(X, Z, FX, FZ, blocks, 0.2, 2.5, rand_pose(r, 0.1, 0.1), sigma=1.3)


def test_geometric_only_cutoff():
    r = rng(5)
    X = r.uniform(-2, 2, size=(3001, 3)).astype(np.float32)
    Z = r.uniform(-2, 2, size=(2999, 3)).astype(np.float32)
    compare_eval(X, Z, None, None, [], 0.15, 3.0, rand_pose(r, 0.1, 0.2))


def test_far_from_origin_small_lengthscale():
    """80 m from the origin with l = 5 cm: the offsets must keep full precision."""
    r = rng(6)
    base = np.array([60.0, -20.0, 80.0])
    X = (base + r.uniform(-1, 1, size=(1500, 3))).astype(np.float32)
    Z = (X + r.normal(0, 0.01, size=X.shape)).astype(np.float32)
    FX = r.uniform(0, 1, (1500, 3)).astype(np.float32)
    FZ = np.clip(FX + r.normal(0, 0.05, FX.shape), 0, 1).astype(np.float32)
    T = rand_pose(r, 0.002, 0.02)
    compare_eval(X, Z, FX, FZ, [("se", 3, 0.2, 1.0)], 0.05, 3.0, T)


def test_street_subsample():
    p = scenes.street_pair()
    sel = rng(7).permutation(p.n)[:5000]
    X, FX = p.X[sel], p.FX[sel]
    Z, FZ = p.Z[sel], p.FZ[sel]
    for T in (np.eye(4), p.T_true):
        compare_eval(X, Z, FX, FZ, p.blocks, 0.3, 3.0, T)


def test_single_points_closed_form():
    X = np.array([[0.1, -0.2, 0.3]], dtype=np.float32)
    Z = np.array([[0.15, -0.1, 0.25]], dtype=np.float32)
    got, ref = compare_eval(X, Z, None, None, [], 0.2, 0.0, np.eye(4), ndir=1)
    d2 = float(((X[0].astype(np.float64) - Z[0]) ** 2).sum())
    assert got["F"] == pytest.approx(math.exp(-d2 / (2 * 0.04)), rel=F_RTOL)


def test_empty_and_partial_groups():
    h = cvo.CVO(ell=0.3, cutoff_mult=3.0)
    X = dev(np.zeros((0, 3)))
    Z = dev(rng(8).uniform(-1, 1, (10, 3)))
    e = h.evaluate(X, Z, np.eye(4))
    assert e["F"] == 0 and e["pairs"] == 0 and not np.any(e["grad"])
    T0 = np.eye(4)
    T1, info = h.register(X, Z, T0)
    assert info["status"] == 0 and np.array_equal(T1, T0)
    h.close()
    for n in (1, 31, 33, 65):
        r = rng(9 + n)
        Xn = r.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
        Zn = r.uniform(-0.3, 0.3, (n + 7, 3)).astype(np.float32)
        compare_eval(Xn, Zn, None, None, [], 0.1, 3.0, rand_pose(r, 0.05, 0.05), ndir=1)


def test_deterministic_rerun():
    p = scenes.street_pair()
    sel = rng(10).permutation(p.n)[:8000]
    h = cvo.CVO(blocks=p.blocks, ell=0.2, cutoff_mult=3.0)
    args = (dev(p.X[sel]), dev(p.Z[sel]), p.T_true, dev(p.FX[sel]), dev(p.FZ[sel]))
    a = h.evaluate(*args)
    b = h.evaluate(*args)
    assert a["F"] == b["F"] and np.array_equal(a["grad"], b["grad"]) and np.array_equal(a["hess"], b["hess"])
    h.close()


def test_host_buffers_match_device_buffers():
    p = scenes.cube_pair(n=1500)
    h = cvo.CVO(blocks=p.blocks, ell=0.1, cutoff_mult=3.0)
    a = h.evaluate(dev(p.X), dev(p.Z), p.T_true, dev(p.FX), dev(p.FZ))
    b = h.evaluate(p.X, p.Z, p.T_true, p.FX, p.FZ)
    assert a["F"] == b["F"] and np.array_equal(a["grad"], b["grad"])
    h.close()


def test_invalid_inputs_rejected():
    h = cvo.CVO(ell=0.3, cutoff_mult=3.0)
    X = dev(rng(11).uniform(-1, 1, (50, 3)))
    bad = X.clone()
    bad[3, 1] = float("nan")
    with pytest.raises(cvo.CvoError) as e:
        h.evaluate(bad, X, np.eye(4))
    assert e.value.status == cvo.Status.ERR_INVALID_ARG
    T = np.eye(4)
    T[0, 0] = 2.0
    with pytest.raises(cvo.CvoError):
        h.evaluate(X, X, T)
    # the handle is still usable afterwards
    assert h.evaluate(X, X, np.eye(4))["F"] > 0
    h.close()


# ---- registration ------------------------------------------------------------

def pose_err(Ta, Tb):
    xi = oracle.se3_log(np.linalg.inv(Ta) @ Tb)
    return np.linalg.norm(xi[:3]), np.linalg.norm(xi[3:])


def trace_pose(row):
    T = np.eye(4)
    T[:3, :] = row[10:22].reshape(3, 4)
    return T


def one_step_parity(X, Z, FX, FZ, blocks, cm, tr, T_final, ks, anneal_kw):
    """At the GPU's own pose T_k and lengthscale l_k the oracle evaluates F and
    takes one step; the GPU's next pose must agree.  This is parity of the
    iteration map, insensitive to how trajectories drift apart over many
    iterations."""
    for k in ks:
        T_k = trace_pose(tr[k])
        ell_k = tr[k, 0]
        T_next_gpu = trace_pose(tr[k + 1]) if k + 1 < tr.shape[0] else T_final
        T1, oinfo, otr = oracle.register(X, Z, T_k, FX=FX, FZ=FZ, blocks=blocks, ell=ell_k, cutoff_mult=cm,
                                         max_iters=1, **anneal_kw)
        assert tr[k, 1] == pytest.approx(otr[0, 1], rel=F_RTOL), k
        er, et = pose_err(T_next_gpu, T1)
        assert er <= POSE_TOL and et <= POSE_TOL, (k, er, et)


def test_register_cube_dense_matches_oracle():
    """The single-pair cube workload (2,000 points, dense, <= 50 iterations):
    the GPU and the oracle stop at the same iteration on the same pose, and,
    since Z is X moved by the true motion, both end on the true pose."""
    p = scenes.cube_pair()
    kw = dict(ell=0.1, cutoff_mult=0.0, max_iters=50)
    h = cvo.CVO(blocks=p.blocks, **kw)
    T_gpu, info = h.register(dev(p.X), dev(p.Z), np.eye(4), dev(p.FX), dev(p.FZ))
    tr_gpu = h.trace()
    h.close()
    T_orc, oinfo, tr_orc = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, blocks=p.blocks, **kw)
    assert info["iters"] == oinfo["iters"] == tr_gpu.shape[0]
    er, et = pose_err(T_gpu, T_orc)
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    np.testing.assert_allclose(tr_gpu[:, 1], tr_orc[:, 1], rtol=1e-5)
    last = tr_gpu.shape[0] - 1
    one_step_parity(p.X, p.Z, p.FX, p.FZ, p.blocks, 0.0, tr_gpu, T_gpu, sorted({0, 1, last // 2, last}), {})
    # ascent: F never decreases; the registration converged onto the true pose
    assert np.all(np.diff(tr_gpu[:, 1]) > -1e-6 * tr_gpu[1:, 1])
    assert info["status"] == 0
    er, et = pose_err(T_gpu, p.T_true)
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)


def test_register_converges_to_known_transform():
    """Z = T_gt X with the same points: both converge to T_gt^-1 and agree."""
    p = scenes.cube_pair(n=1000, seed=91)
    kw = dict(ell=0.3, cutoff_mult=0.0, max_iters=400, step_tol_rot=1e-7, step_tol_trans=1e-7)
    h = cvo.CVO(blocks=p.blocks, **kw)
    T_gpu, info = h.register(dev(p.X), dev(p.Z), np.eye(4), dev(p.FX), dev(p.FZ))
    h.close()
    T_orc, oinfo, _ = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, blocks=p.blocks, **kw)
    assert info["status"] == 0 and oinfo["status"] == 0
    er, et = pose_err(T_gpu, T_orc)
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    er, et = pose_err(T_gpu, p.T_true)
    assert er <= 1e-5 and et <= 1e-5, (er, et)


def test_register_street_annealing_matches_oracle():
    """Street workload (subsampled so the oracle stays fast), annealing on."""
    p = scenes.street_pair()
    sel = rng(12).permutation(p.n)[:2500]
    X, FX, Z, FZ = p.X[sel], p.FX[sel], p.Z[sel], p.FZ[sel]
    kw = dict(ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=100, anneal=True)
    h = cvo.CVO(blocks=p.blocks, **kw)
    T_gpu, info = h.register(dev(X), dev(Z), np.eye(4), dev(FX), dev(FZ))
    tr = h.trace()
    h.close()
    assert info["iters"] == tr.shape[0]
    # one-step parity along the GPU's own trajectory
    ks = sorted(set([0, 1, 2] + list(range(5, tr.shape[0], 9)) + [tr.shape[0] - 1]))
    one_step_parity(X, Z, FX, FZ, p.blocks, 3.0, tr, T_gpu, ks, {})
    # the annealing schedule: replaying the GPU's decisions gives the same l_k
    decisions = tr[:, 8].astype(int)
    T_orc, oinfo, tro = oracle.register(X, Z, np.eye(4), FX=FX, FZ=FZ, blocks=p.blocks, replay=decisions, **kw)
    n = min(tr.shape[0], tro.shape[0])
    np.testing.assert_allclose(tr[:n, 0], tro[:n, 0], rtol=1e-12)
    # every decay fired on an indicator change below tolerance
    for k in np.nonzero(decisions)[0]:
        assert k >= 1 and tr[k - 1, 0] == tr[k, 0]
        assert abs(tr[k, 2] - tr[k - 1, 2]) < 1e-3 * abs(tr[k - 1, 2]) * (1 + 1e-6)


def test_graph_loop_equals_host_loop():
    """The registration loop as one CUDA graph (WHILE node) and the same
    kernels queued from the host give bitwise-identical results."""
    p = scenes.street_pair()
    sel = rng(13).permutation(p.n)[:6000]
    kw = dict(ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=60, anneal=True)
    h = cvo.CVO(blocks=p.blocks, **kw)
    args = (dev(p.X[sel]), dev(p.Z[sel]), np.eye(4), dev(p.FX[sel]), dev(p.FZ[sel]))
    h.set_loop("graph")
    T_graph, info_g = h.register(*args)
    tr_g = h.trace()
    h.set_loop("host")
    cvo.cvo_set_timing(h.h, True)
    T_host, info_h = h.register(*args)
    tr_h = h.trace()
    ms, n = cvo.cvo_sweep_time(h.h)
    h.close()
    assert np.array_equal(T_graph, T_host)
    assert info_g["iters"] == info_h["iters"] == n and ms > 0
    np.testing.assert_array_equal(tr_g, tr_h)


def test_persistent_loop_deterministic_and_close_to_graph():
    """The persistent kernel (dynamic work split, per-item sums in a fixed
    order) gives bitwise-equal results run to run, and agrees with the graph
    loop step by step: the first iterations' F, indicator and step match
    within the inner-product tolerance (later ones may take annealing
    decisions at other iterations, as any two rounding orders may)."""
    p = scenes.street_pair()
    sel = rng(14).permutation(p.n)[:8000]
    kw = dict(ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=60, anneal=True)
    h = cvo.CVO(blocks=p.blocks, **kw)
    args = (dev(p.X[sel]), dev(p.Z[sel]), np.eye(4), dev(p.FX[sel]), dev(p.FZ[sel]))
    h.set_loop("persistent")
    T1, i1 = h.register(*args)
    tr1 = h.trace()
    T2, i2 = h.register(*args)
    tr2 = h.trace()
    assert np.array_equal(T1, T2) and i1["iters"] == i2["iters"]
    np.testing.assert_array_equal(tr1, tr2)
    cvo.cvo_set_timing(h.h, True)
    T3, i3 = h.register(*args)
    ms, n = cvo.cvo_sweep_time(h.h)
    assert np.array_equal(T1, T3) and n == i3["iters"] and ms > 0
    cvo.cvo_set_timing(h.h, False)
    h.set_loop("graph")
    Tg, ig = h.register(*args)
    trg = h.trace()
    k = 5
    np.testing.assert_allclose(tr1[:k, 1], trg[:k, 1], rtol=1e-5)   # F
    np.testing.assert_allclose(tr1[:k, 2], trg[:k, 2], rtol=1e-5)   # indicator
    np.testing.assert_allclose(tr1[:k, 9], trg[:k, 9], rtol=1e-3)   # pairs (cutoff decisions)
    np.testing.assert_allclose(tr1[:k, 10:22], trg[:k, 10:22], atol=1e-4)   # poses the steps start from


def _trace_pose(row):
    T = np.eye(4)
    T[:3, :] = row[10:22].reshape(3, 4)
    return T


def test_persistent_loop_one_step_parity_with_oracle():
    """The persistent kernel's iterations against the oracle: at sampled
    iterations of its own trajectory the oracle takes one step from the
    recorded pose and lengthscale, and F, the pair count and the next pose
    agree (as the graph loop's full-size test checks)."""
    p = scenes.street_pair()
    sel = rng(15).permutation(p.n)[:6000]
    X, Z, FX, FZ = p.X[sel], p.Z[sel], p.FX[sel], p.FZ[sel]
    kw = dict(ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=40, anneal=True)
    with cvo.CVO(blocks=p.blocks, **kw) as h:
        h.set_loop("persistent")
        T_final, info = h.register(dev(X), dev(Z), np.eye(4), dev(FX), dev(FZ))
        tr = h.trace()
    last = tr.shape[0] - 1
    assert last >= 10
    for k in sorted({0, 1, 3, 10, last // 2, last}):
        T_k, ell_k = _trace_pose(tr[k]), tr[k, 0]
        T_next = _trace_pose(tr[k + 1]) if k < last else T_final
        T1, _, otr = oracle.register(X, Z, T_k, FX=FX, FZ=FZ, blocks=p.blocks, ell=ell_k, cutoff_mult=3.0,
                                     max_iters=1)
        assert tr[k, 1] == pytest.approx(otr[0, 1], rel=F_RTOL), k
        rc2 = (3.0 * ell_k) ** 2
        band = oracle.count_band(X, Z, T_k, rc2 * (1 - 1e-5), rc2 * (1 + 1e-5))
        assert abs(tr[k, 9] - otr[0, 9]) <= band, k
        xi = oracle.se3_log(np.linalg.inv(T_next) @ T1)
        assert np.linalg.norm(xi[:3]) <= POSE_TOL and np.linalg.norm(xi[3:]) <= POSE_TOL, k


def test_clusters_far_apart_keep_the_grid_within_its_cell_cap():
    """Two clusters 1e7 m apart with a 15 cm cutoff: the grid of Z would need
    far more than 2^31 cells at the design cell size; the setup counts cells
    in double and widens the cells until they fit, and F and the pair count
    still equal the oracle's."""
    r = rng(16)
    a = r.uniform(-0.2, 0.2, size=(24, 3))
    b = r.uniform(-0.2, 0.2, size=(24, 3))
    b[:, 0] = 1.0e7                      # exactly representable; y and z carry the detail
    X = np.concatenate([a, b]).astype(np.float32)
    Z = (X + r.normal(scale=0.01, size=X.shape)).astype(np.float32)
    Z[24:, 0] = 1.0e7
    for T in (np.eye(4), rand_pose(r, ang=0.0, tr=0.02)):
        with cvo.CVO(ell=0.05, cutoff_mult=3.0) as h:
            got = h.evaluate(dev(X), dev(Z), T)
        ref = oracle.evaluate(X.astype(np.float64), Z.astype(np.float64), T, ell=0.05, cutoff_mult=3.0)
        assert ref["npairs"] > 48
        assert got["F"] == pytest.approx(ref["F"], rel=F_RTOL)
        rc2 = 0.15 ** 2
        band = oracle.count_band(X.astype(np.float64), Z.astype(np.float64), T, rc2 * (1 - 1e-5), rc2 * (1 + 1e-5))
        assert abs(got["pairs"] - ref["npairs"]) <= band
