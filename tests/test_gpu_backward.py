"""Gradients with respect to the inputs (cvo_backward and the autograd
function) against the FP64 oracle.

What is compared:
  dX, dZ, dFX, dFZ   element by element: |gpu - oracle| <= 1e-4 * max|oracle|
                     over the array (FP32 accumulation of the per-point sums,
                     the tolerance of the se(3) gradient applied per point);
                     points with a pair whose squared distance lies within
                     1e-5 of the cutoff are left out (there FP32 and FP64 may
                     disagree on whether the pair is in the sum) and are
                     checked to be rare
  dF/dl              relative 1e-4 plus the largest term such boundary pairs
                     can contribute
At the room workload's full size (19,200 points per cloud, the launch the
library makes there) sampled rows are compared with the oracle evaluated one
point at a time, and with central differences of the oracle's F.
"""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

G_TOL = 1e-4
BAND = 1e-5


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def bf16_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to("cuda").to(torch.bfloat16)


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def rand_pose(r, ang=0.05, tr=0.05):
    return oracle.se3_exp(np.concatenate([r.normal(size=3) * ang / math.sqrt(3), r.normal(size=3) * tr / math.sqrt(3)]))


def band_masks(X, Z, T, rc2, rel=BAND, abs_d=0.0):
    """Rows of X and of Z with a pair whose squared distance is within the
    band around the cutoff (rel * rc2, or |d - rc| <= abs_d)."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Z, np.float64) @ T[:3, :3].T + T[:3, 3]
    rc = math.sqrt(rc2)
    lo = min(rc2 * (1 - rel), max(rc - abs_d, 0.0) ** 2)
    hi = max(rc2 * (1 + rel), (rc + abs_d) ** 2)
    mx = np.zeros(len(X), bool)
    mz = np.zeros(len(Y), bool)
    for a in range(0, len(X), 1024):
        d2 = ((X[a:a + 1024, None, :] - Y[None, :, :]) ** 2).sum(-1)
        b = (d2 >= lo) & (d2 <= hi)
        mx[a:a + 1024] |= b.any(1)
        mz |= b.any(0)
    return mx, mz


def check_close(got, ref, skip=None, name=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, name
    keep = np.ones(len(ref), bool) if skip is None else ~skip
    scale = np.abs(ref).max() if ref.size else 0.0
    tol = G_TOL * scale + 1e-30
    err = np.abs(got[keep] - ref[keep]).max() if keep.any() and ref.size else 0.0
    assert err <= tol, f"{name}: max error {err:.3e} > {tol:.3e} (scale {scale:.3e})"


def run_pair(X, Z, FX, FZ, blocks, ell, cm, T, bf16=False, sigma=1.0, dF=1.0, chunk_len=None):
    h = cvo.CVO(blocks=blocks, ell=ell, cutoff_mult=cm, sigma=sigma)
    if chunk_len is not None:
        t = h.tuning()
        h.apply_tuning(t["cell_factor"], t["super_delta"], chunk_len)
    if FX is not None and bf16:
        fx, fz = bf16_dev(FX), bf16_dev(FZ)
        FXo, FZo = scenes.bf16_round(FX), scenes.bf16_round(FZ)
    elif FX is not None:
        fx, fz = dev(FX), dev(FZ)
        FXo, FZo = FX, FZ
    else:
        fx = fz = FXo = FZo = None
    got = h.backward(dev(X), dev(Z), T, fx, fz, dF=dF)
    got = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in got.items()}
    ref = oracle.backward(X, Z, T, FX=FXo, FZ=FZo, blocks=blocks, ell=ell, cutoff_mult=cm, sigma=sigma)
    return got, ref, h


def compare(X, Z, FX, FZ, blocks, ell, cm, T, bf16=False, sigma=1.0, dF=1.0, chunk_len=None):
    got, ref, _ = run_pair(X, Z, FX, FZ, blocks, ell, cm, T, bf16, sigma, dF, chunk_len)
    for k in ("dX", "dZ", "dFX", "dFZ"):
        if k in ref:
            ref[k] = ref[k] * dF
    ref["dell"] *= dF
    sx = sz = None
    dell_slack = 0.0
    if cm > 0:
        rc2 = (cm * ell) ** 2
        sx, sz = band_masks(X, Z, T, rc2)
        assert sx.mean() < 0.02 and sz.mean() < 0.02
        nb = oracle.count_band(X, Z, T, rc2 * (1 - BAND), rc2 * (1 + BAND))
        # a boundary pair adds at most sigma^2 prod sigma_b^2 e^(-cm^2/2) rc^2 / l^3
        kap = sigma ** 2
        for b in blocks:
            if b[0] == "se":
                kap *= b[3] ** 2
        dell_slack = nb * abs(dF) * kap * math.exp(-cm * cm / 2) * rc2 / ell ** 3 * 25.0
    check_close(got["dX"], ref["dX"], sx, "dX")
    check_close(got["dZ"], ref["dZ"], sz, "dZ")
    if blocks:
        check_close(got["dFX"], ref["dFX"], sx, "dFX")
        check_close(got["dFZ"], ref["dFZ"], sz, "dFZ")
    assert abs(got["dell"] - ref["dell"]) <= G_TOL * abs(ref["dell"]) + dell_slack, (got["dell"], ref["dell"])
    return got, ref


def slice_pair(pair, n, seed):
    r = rng(seed)
    ix = r.permutation(len(pair.X))[:n]
    iz = r.permutation(len(pair.Z))[:n]
    FX = pair.FX[ix] if pair.FX is not None else None
    FZ = pair.FZ[iz] if pair.FZ is not None else None
    return pair.X[ix], pair.Z[iz], FX, FZ


@pytest.fixture(scope="module")
def room():
    return scenes.room_pair()


@pytest.fixture(scope="module")
def street():
    return scenes.street_pair()


@pytest.mark.parametrize("bf16", [False, True])
def test_backward_room_slice(room, bf16):
    X, Z, FX, FZ = slice_pair(room, 4000, 1)
    T = room.T_true @ rand_pose(rng(2))
    compare(X, Z, FX, FZ, room.blocks, 0.1, 3.0, T, bf16=bf16)


@pytest.mark.parametrize("bf16", [False, True])
def test_backward_room_slice_trimmed_streams(room, bf16):
    """768-candidate items: the gradient sweep's streams trimmed by each
    query's ball."""
    X, Z, FX, FZ = slice_pair(room, 4000, 1)
    T = room.T_true @ rand_pose(rng(2))
    compare(X, Z, FX, FZ, room.blocks, 0.1, 3.0, T, bf16=bf16, chunk_len=768)


@pytest.mark.parametrize("bf16", [False, True])
def test_backward_street_semantic(street, bf16):
    X, Z, FX, FZ = slice_pair(street, 3000, 3)
    T = street.T_true @ rand_pose(rng(4))
    compare(X, Z, FX, FZ, street.blocks, 0.3, 3.0, T, bf16=bf16, dF=-0.75)


def test_backward_labels_only(street):
    X, Z, FX, FZ = slice_pair(street, 2000, 5)
    T = street.T_true
    compare(X, Z, FX[:, 3:], FZ[:, 3:], [("dot", 19, 1.0, 1.0)], 0.2, 3.0, T)


def test_backward_geometric_dense():
    cube = scenes.cube_pair(n=1500)
    compare(cube.X, cube.Z, None, None, [], 0.1, 0.0, cube.T_true @ rand_pose(rng(6)), sigma=1.3)


def test_backward_generic_blocks():
    """Four blocks (two squared-exponential, two inner products): the generic
    feature path, with the inner-product factors of the other blocks."""
    r = rng(7)
    X, FX = scenes.random_cloud(r, 700, 10, extent=0.6)
    Z, FZ = scenes.random_cloud(r, 650, 10, extent=0.6)
    blocks = [("se", 2, 0.3, 1.2), ("dot", 4, 1.0, 1.0), ("se", 1, 0.5, 0.9), ("dot", 3, 1.0, 1.0)]
    T = rand_pose(r, 0.2, 0.1)
    compare(X, Z, FX, FZ, blocks, 0.15, 2.5, T, sigma=0.8)
    compare(X[:300], Z[:280], FX[:300], FZ[:280], blocks, 0.2, 0.0, T)
    compare(X, Z, FX, FZ, blocks, 0.15, 2.5, T, bf16=True)


def test_backward_tiny_and_ragged():
    """Fewer points than a warp, and sizes that leave ragged groups."""
    r = rng(8)
    for n, m in [(1, 1), (5, 3), (33, 65), (97, 31)]:
        X, FX = scenes.random_cloud(r, n, 3, extent=0.3)
        Z, FZ = scenes.random_cloud(r, m, 3, extent=0.3)
        T = rand_pose(r, 0.1, 0.05)
        compare(X, Z, FX, FZ, [("se", 3, 0.4, 1.0)], 0.2, 3.0, T)
        compare(X, Z, None, None, [], 0.2, 0.0, T)


def test_backward_edge_cases():
    r = rng(9)
    X, FX = scenes.random_cloud(r, 200, 3, extent=0.5)
    Z, FZ = scenes.random_cloud(r, 180, 3, extent=0.5)
    X[17] = (500.0, 500.0, 500.0)   # no pair in range: zero gradient
    blocks = [("se", 3, 0.3, 1.0)]
    h = cvo.CVO(blocks=blocks, ell=0.1, cutoff_mult=3.0)
    T = np.eye(4)
    d = h.backward(dev(X), dev(Z), T, dev(FX), dev(FZ))
    dX = d["dX"].cpu().numpy()
    assert np.all(dX[17] == 0.0) and np.all(d["dFX"].cpu().numpy()[17] == 0.0)
    # host inputs and outputs give the same numbers as device ones
    dh = h.backward(X, Z, T, FX, FZ)
    for k in ("dX", "dFX", "dZ", "dFZ"):
        assert np.array_equal(dh[k], d[k].cpu().numpy()), k
    assert dh["dell"] == d["dell"]
    # outputs left out are not computed; the others are unchanged
    part = h.backward(dev(X), dev(Z), T, dev(FX), dev(FZ), want=("dZ",))
    assert set(part) == {"dZ"}
    assert torch.equal(part["dZ"], d["dZ"])
    # an empty cloud: every gradient is zero
    e = h.backward(dev(X[:0]), dev(Z), T, dev(FX[:0]), dev(FZ))
    assert e["dX"].shape == (0, 3) and float(e["dZ"].abs().max()) == 0.0 and e["dell"] == 0.0
    # an invalid pose is rejected
    with pytest.raises(cvo.CvoError):
        h.backward(dev(X), dev(Z), np.diag([1.0, 1.0, -1.0, 1.0]), dev(FX), dev(FZ))


def test_backward_full_room_sampled_rows(room):
    """Full-size room pair (19,200 points each): 200 sampled rows of X and of
    Z against the oracle evaluated for one point at a time, and central
    differences of the oracle's F for some of them."""
    X, Z, FX, FZ = room.X, room.Z, room.FX, room.FZ
    blocks, ell, cm = room.blocks, 0.1, 3.0
    T = room.T_true @ rand_pose(rng(10), 0.03, 0.03)
    h = cvo.CVO(blocks=blocks, ell=ell, cutoff_mult=cm)
    d = h.backward(dev(X), dev(Z), T, dev(FX), dev(FZ))
    d = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    r = rng(11)
    ix = r.permutation(len(X))[:200]
    iz = r.permutation(len(Z))[:200]
    rc2 = (cm * ell) ** 2
    eps = 1e-5
    sx, _ = band_masks(X[ix], Z, T, rc2)
    _, sz = band_masks(X, Z[iz], T, rc2)
    assert sx.mean() < 0.05 and sz.mean() < 0.05
    # rows whose pairs all stay clear of the cutoff by 3 eps (for differences)
    fx, _ = band_masks(X[ix[:60]], Z, T, rc2, abs_d=3 * eps)
    kw = dict(blocks=blocks, ell=ell, cutoff_mult=cm)
    refx = np.array([np.concatenate([oracle.backward(X[i:i + 1], Z, T, FX=FX[i:i + 1], FZ=FZ, **kw)[k][0]
                                     for k in ("dX", "dFX")]) for i in ix])
    refz = np.array([np.concatenate([oracle.backward(X, Z[j:j + 1], T, FX=FX, FZ=FZ[j:j + 1], **kw)[k][0]
                                     for k in ("dZ", "dFZ")]) for j in iz])
    check_close(d["dX"][ix], refx[:, :3], sx, "dX rows")
    check_close(d["dFX"][ix], refx[:, 3:], sx, "dFX rows")
    check_close(d["dZ"][iz], refz[:, :3], sz, "dZ rows")
    check_close(d["dFZ"][iz], refz[:, 3:], sz, "dFZ rows")

    # central differences of the oracle's F (FP64) on 20 of the rows
    def F1(xi, fi):
        return oracle.evaluate(xi[None], Z, T, FX=fi[None], FZ=FZ, **kw)["F"]

    scale = np.abs(refx[:, :3]).max()
    rows = [i for i, s in zip(ix[:60], fx) if not s][:20]
    assert len(rows) >= 10
    for i in rows:
        x = X[i].astype(np.float64)
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a] += eps
            xm[a] -= eps
            fd = (F1(xp, FX[i].astype(np.float64)) - F1(xm, FX[i].astype(np.float64))) / (2 * eps)
            assert abs(d["dX"][i, a] - fd) <= G_TOL * scale + 1e-6 * abs(fd), (i, a, d["dX"][i, a], fd)


def test_backward_dell_finite_difference(room):
    """dF/dl against central differences of the oracle's F, with the pairs
    that cross the moving cutoff counted (none may cross)."""
    X, Z, FX, FZ = slice_pair(room, 3000, 12)
    T = room.T_true
    ell, cm = 0.1, 3.0
    got, ref, _ = run_pair(X, Z, FX, FZ, room.blocks, ell, cm, T)
    eps = 1e-7
    crossing = oracle.count_band(X, Z, T, (cm * (ell - eps)) ** 2, (cm * (ell + eps)) ** 2)
    kw = dict(FX=FX, FZ=FZ, blocks=room.blocks, cutoff_mult=cm)
    Fp = oracle.evaluate(X, Z, T, ell=ell + eps, **kw)["F"]
    Fm = oracle.evaluate(X, Z, T, ell=ell - eps, **kw)["F"]
    if crossing == 0:
        assert ref["dell"] == pytest.approx((Fp - Fm) / (2 * eps), rel=1e-5)
    assert got["dell"] == pytest.approx(ref["dell"], rel=1e-4)


def test_autograd_function(room):
    X, Z, FX, FZ = slice_pair(room, 2500, 13)
    T = room.T_true
    h = cvo.CVO(blocks=room.blocks, ell=0.1, cutoff_mult=3.0)
    Xt = dev(X).requires_grad_(True)
    Zt = dev(Z).requires_grad_(True)
    FXt = dev(FX).requires_grad_(True)
    FZt = dev(FZ).requires_grad_(True)
    ell = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    F = cvo.inner_product_fn(h, Xt, Zt, T, FXt, FZt, ell=ell)
    assert F.item() == pytest.approx(h.inner_product(dev(X), dev(Z), T, dev(FX), dev(FZ)), rel=1e-12)
    (2.5 * F).backward()
    d = h.backward(dev(X), dev(Z), T, dev(FX), dev(FZ))
    for t, k in ((Xt, "dX"), (Zt, "dZ"), (FXt, "dFX"), (FZt, "dFZ")):
        g = t.grad.double().cpu().numpy()
        want = 2.5 * d[k].double().cpu().numpy()
        assert np.abs(g - want).max() <= 1e-6 * np.abs(want).max(), k
    assert ell.grad.item() == pytest.approx(2.5 * d["dell"], rel=1e-6)
    # the indicator of Eq. (indicator_actual) is F / sqrt(N M)
    Xt.grad = None
    i = cvo.metric_fn(h, Xt, Zt, T, FXt.detach(), FZt.detach())
    # the value is the library's cvo_metric (no arithmetic in the binding)
    assert i.item() == h.metric(dev(X), dev(Z), T, dev(FX), dev(FZ))
    i.backward()
    want = d["dX"].double().cpu().numpy() / math.sqrt(len(X) * len(Z))
    assert np.abs(Xt.grad.double().cpu().numpy() - want).max() <= 1e-6 * np.abs(want).max()
    # the oracle agrees on the autograd result
    ref = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=room.blocks, ell=0.1, cutoff_mult=3.0)
    sx, _ = band_masks(X, Z, T, 0.09)
    check_close(Xt.grad.double().cpu().numpy() * math.sqrt(len(X) * len(Z)), ref["dX"], sx, "autograd dX")


def test_metric_backward_through_the_c_abi(room):
    """cvo_metric_backward gives the gradients of di * i_theta: those of
    cvo_backward scaled by 1 / sqrt(N M) (Eq. indicator_actual), against the
    oracle's input gradients; empty clouds give zeros."""
    X, Z, FX, FZ = slice_pair(room, 2000, 14)
    T = room.T_true
    h = cvo.CVO(blocks=room.blocks, ell=0.1, cutoff_mult=3.0)
    di = -1.75
    got = cvo.cvo_metric_backward(h.h, dev(X), dev(Z), T, dev(FX), dev(FZ), di=di)
    base = h.backward(dev(X), dev(Z), T, dev(FX), dev(FZ))
    s = di / math.sqrt(len(X) * len(Z))
    for k in ("dX", "dZ", "dFX", "dFZ"):
        g = got[k].double().cpu().numpy()
        want = s * base[k].double().cpu().numpy()
        assert np.abs(g - want).max() <= 1e-6 * np.abs(want).max(), k
    # the scale enters the per-query float32 terms before their sum
    assert got["dell"] == pytest.approx(s * base["dell"], rel=1e-6)
    ref = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=room.blocks, ell=0.1, cutoff_mult=3.0)
    sx, _ = band_masks(X, Z, T, 0.09)
    check_close(got["dX"].double().cpu().numpy() / s, ref["dX"], sx, "metric dX")
    e = cvo.cvo_metric_backward(h.h, dev(X[:0]), dev(Z), T, dev(FX[:0]), dev(FZ), di=di)
    assert float(e["dZ"].abs().max()) == 0.0 and e["dell"] == 0.0
