"""The feature-space cutoff (Sec. III-B: a pair also needs its colour
features within a multiple of the colour lengthscale) against the FP64
oracle with the same cutoff, on every feature path of the sweep: the fixed
RGB + 19-class path (float32 features), its bfloat16 tensor-core tile, and the
generic block loop; the gradient sweep; a registration.

The colours are quantised to multiples of 1/8 so that every squared colour
distance is a multiple of 1/64 and none lies near the cutoff radius
(1.6 * 0.2)^2 = 0.1024: FP32 and FP64 take every feature decision alike, and
the pair counts agree up to the geometric cutoff's boundary band alone.
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
FCM = 1.6
BLOCKS = [("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def rand_pose(r, ang=0.05, tr=0.05):
    return oracle.se3_exp(np.concatenate([r.normal(size=3) * ang / math.sqrt(3), r.normal(size=3) * tr / math.sqrt(3)]))


def quantised_rgb(r, n):
    return (r.integers(0, 9, size=(n, 3)) / 8.0).astype(np.float32)


def semantic_cloud(r, n, lo=-1.0, hi=1.0):
    X = r.uniform(lo, hi, size=(n, 3)).astype(np.float32)
    lab = r.dirichlet(np.ones(19), n)
    # label distributions rounded to bfloat16 so both feature dtypes see the same values
    F = np.hstack([quantised_rgb(r, n), scenes.bf16_round(lab)]).astype(np.float32)
    return X, F


def check_eval(X, Z, FX, FZ, blocks, ell, cm, T, fdtype=torch.float32, sigma=1.0):
    h = cvo.CVO(blocks=blocks, ell=ell, cutoff_mult=cm, sigma=sigma, feat_cutoff_mult=FCM)
    got = h.evaluate(dev(X), dev(Z), T, dev(FX, fdtype), dev(FZ, fdtype))
    h.close()
    kw = dict(FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, sigma=sigma)
    ref = oracle.evaluate(X, Z, T, feat_cutoff_mult=FCM, **kw)
    full = oracle.evaluate(X, Z, T, **kw)
    # the cutoff must bite for the comparison to mean anything
    assert ref["npairs"] < 0.8 * full["npairs"]
    assert got["F"] == pytest.approx(ref["F"], rel=F_RTOL)
    gtol = G_TOL * np.linalg.norm(ref["g"]) + G_FLOOR * ref["gscale"]
    assert np.abs(got["grad"] - ref["g"]).max() <= gtol, (got["grad"], ref["g"])
    if cm > 0:
        rc2 = (cm * ell) ** 2
        band = oracle.count_band(X, Z, T, rc2 * (1 - 1e-5), rc2 * (1 + 1e-5))
        assert abs(got["pairs"] - ref["npairs"]) <= band
    else:
        assert got["pairs"] == ref["npairs"]
    return got, ref


def test_fixed_path_float32():
    r = rng(41)
    X, FX = semantic_cloud(r, 1537)
    Z, FZ = semantic_cloud(r, 1411)
    check_eval(X, Z, FX, FZ, BLOCKS, 0.12, 3.0, rand_pose(r))


def test_tensor_core_tile_bfloat16():
    r = rng(42)
    X, FX = semantic_cloud(r, 2113)
    Z, FZ = semantic_cloud(r, 1999)
    check_eval(X, Z, FX, FZ, BLOCKS, 0.12, 3.0, rand_pose(r), fdtype=torch.bfloat16)


def test_dense_sum_counts_exact():
    r = rng(43)
    X, FX = semantic_cloud(r, 700)
    Z, FZ = semantic_cloud(r, 650)
    check_eval(X, Z, FX, FZ, BLOCKS, 0.3, 0.0, rand_pose(r))


def test_generic_blocks():
    r = rng(44)
    n, m = 800, 760
    X = r.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(m, 3)).astype(np.float32)
    FX = np.hstack([quantised_rgb(r, n)[:, :2], r.dirichlet(np.ones(4), n), quantised_rgb(r, n)[:, :1]])
    FZ = np.hstack([quantised_rgb(r, m)[:, :2], r.dirichlet(np.ones(4), m), quantised_rgb(r, m)[:, :1]])
    blocks = [("se", 2, 0.2, 1.5), ("dot", 4, 1.0, 1.0), ("se", 1, 0.2, 0.8)]
    check_eval(X, Z, FX.astype(np.float32), FZ.astype(np.float32), blocks, 0.2, 2.5, rand_pose(r, 0.1, 0.1),
               sigma=1.3)


def test_geometry_only_ignores_feature_cutoff():
    """Without feature blocks the option changes nothing, bit for bit."""
    r = rng(45)
    X = r.uniform(-1, 1, size=(1200, 3)).astype(np.float32)
    Z = r.uniform(-1, 1, size=(1100, 3)).astype(np.float32)
    T = rand_pose(r)
    out = []
    for fcm in (0.0, FCM):
        h = cvo.CVO(blocks=[], ell=0.15, cutoff_mult=3.0, feat_cutoff_mult=fcm)
        out.append(h.evaluate(dev(X), dev(Z), T))
        h.close()
    assert out[0]["F"] == out[1]["F"] and out[0]["pairs"] == out[1]["pairs"]
    assert np.array_equal(out[0]["grad"], out[1]["grad"])


def test_backward_matches_oracle():
    r = rng(46)
    X, FX = semantic_cloud(r, 900)
    Z, FZ = semantic_cloud(r, 850)
    T = rand_pose(r)
    ell = 0.3
    h = cvo.CVO(blocks=BLOCKS, ell=ell, cutoff_mult=0.0, feat_cutoff_mult=FCM)
    got = h.backward(dev(X), dev(Z), T, dev(FX), dev(FZ))
    h.close()
    got = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in got.items()}
    ref = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=ell, cutoff_mult=0.0, feat_cutoff_mult=FCM)
    full = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=ell, cutoff_mult=0.0)
    for k in ("dX", "dZ", "dFX", "dFZ"):
        scale = np.abs(ref[k]).max()
        assert np.abs(got[k] - ref[k]).max() <= G_TOL * scale, k
        # and the cutoff changed the answer well beyond the tolerance
        assert np.abs(full[k] - ref[k]).max() > 100 * G_TOL * scale, k
    assert got["dell"] == pytest.approx(ref["dell"], rel=G_TOL)


def test_register_cube_matches_oracle():
    """Dense cube registration with quantised colours: every iteration's F
    and the final pose agree with the oracle's registration."""
    p = scenes.cube_pair(n=1200, seed=97)
    FX = (np.round(p.FX * 8.0) / 8.0).astype(np.float32)
    kw = dict(ell=0.1, cutoff_mult=0.0, max_iters=30, feat_cutoff_mult=FCM)
    h = cvo.CVO(blocks=p.blocks, **kw)
    T_gpu, info = h.register(dev(p.X), dev(p.Z), np.eye(4), dev(FX), dev(FX))
    tr = h.trace()
    h.close()
    T_orc, oinfo, tro = oracle.register(p.X, p.Z, np.eye(4), FX=FX, FZ=FX, blocks=p.blocks, **kw)
    assert info["iters"] == oinfo["iters"] == tr.shape[0]
    np.testing.assert_allclose(tr[:, 1], tro[:, 1], rtol=F_RTOL)
    xi = oracle.se3_log(np.linalg.inv(T_gpu) @ T_orc)
    assert np.linalg.norm(xi[:3]) <= 1e-4 and np.linalg.norm(xi[3:]) <= 1e-4


def test_batch_with_feature_cutoff_matches_single_pairs():
    """Batched registration with the feature cutoff agrees with registering
    each pair alone with it (the batch shares the kernels, split differently)."""
    pairs = scenes.batch_pairs(n_pairs=3, seed=515, n_range=(1500, 4000))
    args = []
    for q in pairs:
        FXq = np.hstack([np.round(q.FX[:, :3] * 8.0) / 8.0, q.FX[:, 3:]]).astype(np.float32)
        FZq = np.hstack([np.round(q.FZ[:, :3] * 8.0) / 8.0, q.FZ[:, 3:]]).astype(np.float32)
        args.append((dev(q.X), dev(q.Z), np.eye(4), dev(FXq), dev(FZq)))
    with cvo.CVO(blocks=pairs[0].blocks, ell=0.2, cutoff_mult=3.0, max_iters=30, feat_cutoff_mult=FCM) as h:
        T_batch, infos, _ = h.register_batch(args)
        singles = [h.register(*a) for a in args]
    for k, (Ts, info_s) in enumerate(singles):
        xi = oracle.se3_log(np.linalg.inv(T_batch[k]) @ Ts)
        assert np.linalg.norm(xi[:3]) <= 1e-4 and np.linalg.norm(xi[3:]) <= 1e-4, k
        assert infos[k]["F"] == pytest.approx(info_s["F"], rel=1e-4)
