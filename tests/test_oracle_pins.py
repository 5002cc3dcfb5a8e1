"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types the oracle's formula.  Each checks the oracle
against an independent route:
  * quadrature of the Gaussian convolution identity (the SE kernel of Eq. (k)
    is, up to a constant, the L2 inner product of two narrower Gaussians), so
    F = <f_X, f_{h^-1 Z}> becomes an integral of two smoothed fields;
  * the explicit tensor product (numpy.kron) of Eq. (tensor_product);
  * scipy's k-d tree for the set of pairs inside the cutoff;
  * scipy.linalg.expm for the SE(3) exponential;
  * central finite differences of F on se(3) for the gradient and the second
    derivative;
  * the double sum, the SE(3) exponential and logarithm written out in 30- or
    40-digit arithmetic (mpmath), differentiated by mpmath for the se(3)
    gradient, the second derivative and every input gradient;
  * invariants: symmetry of the inner product, invariance under a common rigid
    motion, Cauchy-Schwarz, the Remark of Sec. III-C, the behaviour of Fig. 3,
    and recovery of a known transform.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial import cKDTree

import oracle
import scenes


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def hat(xi):
    w, v = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def expm_se3(xi):
    return scipy.linalg.expm(hat(np.asarray(xi, dtype=np.float64)))


def rand_T(r, ang=0.6, tr=0.5):
    xi = np.concatenate([r.normal(size=3) * ang / math.sqrt(3), r.normal(size=3) * tr / math.sqrt(3)])
    return expm_se3(xi)


def transform(T, P):
    return P @ T[:3, :3].T + T[:3, 3]


# ---------------------------------------------------------------------------
# 1. the inner product by quadrature (Eq. k, newscalar, scalar, double_sum)
# ---------------------------------------------------------------------------

def _grid(lo, hi, h):
    n = int(math.ceil((hi - lo) / h)) + 1
    return lo + h * np.arange(n)


def _gauss_fields(P, axes, ell):
    """exp(-|p - u|^2 / l^2) on a 3-D tensor grid, one flattened field per point."""
    gx, gy, gz = axes
    out = []
    for p in P:
        fx = np.exp(-((gx - p[0]) ** 2) / ell ** 2)
        fy = np.exp(-((gy - p[1]) ** 2) / ell ** 2)
        fz = np.exp(-((gz - p[2]) ** 2) / ell ** 2)
        out.append(np.einsum("a,b,c->abc", fx, fy, fz).ravel())
    return np.array(out)


def quad_F(X, Y, ell, sigma, fx=None, fy=None, feat=None):
    """sigma^2 (pi l^2/2)^(-3/2) * integral of sum_i a_i(u) * sum_j b_j(u) du,
    with the feature part either a 1-D squared exponential (feat=("se", l_c,
    sigma_c)) integrated on its own axis, or an inner product (feat=("dot",))."""
    lo = np.minimum(X.min(0), Y.min(0)) - 6 * ell
    hi = np.maximum(X.max(0), Y.max(0)) + 6 * ell
    h = ell / 3.0
    axes = [_grid(lo[d], hi[d], h) for d in range(3)]
    GX = _gauss_fields(X, axes, ell)
    GY = _gauss_fields(Y, axes, ell)
    c = sigma ** 2 * (math.pi * ell ** 2 / 2) ** -1.5 * h ** 3
    if feat is None:
        return c * np.sum(GX.sum(0) * GY.sum(0))
    if feat[0] == "dot":
        A = fx.T @ GX  # (D, grid)
        B = fy.T @ GY
        return c * np.sum(A * B)
    _, lc, sc = feat
    flo = min(fx.min(), fy.min()) - 6 * lc
    fhi = max(fx.max(), fy.max()) + 6 * lc
    hr = lc / 3.0
    r = _grid(flo, fhi, hr)
    HX = np.exp(-((r[None, :] - fx[:, :1]) ** 2) / lc ** 2)  # (n, R)
    HY = np.exp(-((r[None, :] - fy[:, :1]) ** 2) / lc ** 2)
    A = np.einsum("iu,ir->ur", GX, HX)
    B = np.einsum("ju,jr->ur", GY, HY)
    cc = sc ** 2 * (math.pi * lc ** 2 / 2) ** -0.5 * hr
    return c * cc * np.sum(A * B)


def test_inner_product_geometric_by_quadrature():
    r = rng(1)
    X = r.uniform(-0.5, 0.5, size=(3, 3))
    Z = r.uniform(-0.5, 0.5, size=(4, 3))
    T = rand_T(r, 0.3, 0.2)
    ell, sigma = 0.3, 1.3
    ref = quad_F(X, transform(T, Z), ell, sigma)
    got = oracle.evaluate(X, Z, T, ell=ell, sigma=sigma)["F"]
    assert got == pytest.approx(ref, rel=1e-10)


def test_inner_product_se_feature_by_quadrature():
    r = rng(2)
    X = r.uniform(-0.4, 0.4, size=(3, 3))
    Z = r.uniform(-0.4, 0.4, size=(3, 3))
    fx = r.uniform(0, 1, size=(3, 1))
    fz = r.uniform(0, 1, size=(3, 1))
    T = rand_T(r, 0.2, 0.1)
    ell, sigma, lc, sc = 0.3, 0.9, 0.25, 1.7
    ref = quad_F(X, transform(T, Z), ell, sigma, fx, fz, feat=("se", lc, sc))
    got = oracle.evaluate(X, Z, T, FX=fx, FZ=fz, blocks=[("se", 1, lc, sc)], ell=ell, sigma=sigma)["F"]
    assert got == pytest.approx(ref, rel=1e-9)


def test_inner_product_dot_feature_by_quadrature():
    r = rng(3)
    X = r.uniform(-0.4, 0.4, size=(4, 3))
    Z = r.uniform(-0.4, 0.4, size=(3, 3))
    fx = r.dirichlet(np.ones(5), size=4)
    fz = r.dirichlet(np.ones(5), size=3)
    T = rand_T(r, 0.2, 0.1)
    ell, sigma = 0.25, 1.0
    ref = quad_F(X, transform(T, Z), ell, sigma, fx, fz, feat=("dot",))
    got = oracle.evaluate(X, Z, T, FX=fx, FZ=fz, blocks=[("dot", 5, 1.0, 1.0)], ell=ell, sigma=sigma)["F"]
    assert got == pytest.approx(ref, rel=1e-10)


def test_tensor_product_blocks_equal_kron():
    """Eq. (tensor_product): <u1 (x) u2, v1 (x) v2> = <u1,v1><u2,v2>."""
    r = rng(4)
    X = r.uniform(-1, 1, size=(6, 3))
    Z = r.uniform(-1, 1, size=(5, 3))
    a1, a2 = r.uniform(0, 1, size=(6, 2)), r.uniform(0, 1, size=(6, 3))
    b1, b2 = r.uniform(0, 1, size=(5, 2)), r.uniform(0, 1, size=(5, 3))
    T = rand_T(r)
    two = oracle.evaluate(X, Z, T, FX=np.hstack([a1, a2]), FZ=np.hstack([b1, b2]),
                          blocks=[("dot", 2, 1, 1), ("dot", 3, 1, 1)], ell=0.7)
    kx = np.array([np.kron(a1[i], a2[i]) for i in range(6)])
    kz = np.array([np.kron(b1[j], b2[j]) for j in range(5)])
    one = oracle.evaluate(X, Z, T, FX=kx, FZ=kz, blocks=[("dot", 6, 1, 1)], ell=0.7)
    assert two["F"] == pytest.approx(one["F"], rel=1e-13)
    np.testing.assert_allclose(two["g"], one["g"], rtol=1e-12, atol=1e-14)


def test_geometric_only_equals_unit_labels():
    """Eq. (geometric_only): labels identically 1 reduce to the plain kernel sum."""
    r = rng(5)
    X = r.uniform(-1, 1, size=(7, 3))
    Z = r.uniform(-1, 1, size=(9, 3))
    T = rand_T(r)
    a = oracle.evaluate(X, Z, T, ell=0.5)
    b = oracle.evaluate(X, Z, T, FX=np.ones((7, 1)), FZ=np.ones((9, 1)), blocks=[("dot", 1, 1, 1)], ell=0.5)
    assert a["F"] == pytest.approx(b["F"], rel=1e-14)


# ---------------------------------------------------------------------------
# 2. the cutoff: the pair set is the k-d tree's ball query
# ---------------------------------------------------------------------------

def test_cutoff_pair_set_matches_kdtree():
    r = rng(6)
    X = r.uniform(-2, 2, size=(400, 3))
    Z = r.uniform(-2, 2, size=(500, 3))
    T = rand_T(r, 0.3, 0.3)
    ell, cm = 0.2, 3.0
    res = oracle.evaluate(X, Z, T, ell=ell, cutoff_mult=cm)
    Y = transform(T, Z)
    n_tree = sum(len(v) for v in cKDTree(Y).query_ball_point(X, cm * ell))
    assert res["npairs"] == n_tree
    # the pairs left out are exactly the ones beyond the radius: their kernel
    # values make up the difference to the dense sum
    dense = oracle.evaluate(X, Z, T, ell=ell)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    far = np.exp(-d2[d2 > (cm * ell) ** 2] / (2 * ell ** 2)).sum()
    assert dense["F"] - res["F"] == pytest.approx(far, rel=1e-9, abs=1e-12)


def test_band_census_by_brute_force():
    """The census of pairs near the cutoff radius (the pair-count tolerance of
    the GPU parity tests) counts the squared distances in [lo, hi] as numpy
    does."""
    r = rng(62)
    X = r.uniform(-1, 1, size=(300, 3))
    Z = r.uniform(-1, 1, size=(280, 3))
    T = rand_T(r, 0.3, 0.2)
    d2 = ((X[:, None, :] - transform(T, Z)[None, :, :]) ** 2).sum(-1)
    for lo, hi in ((0.25, 0.36), (0.0, 0.01), (1.0, 1.0 + 1e-3)):
        assert oracle.count_band(X, Z, T, lo, hi) == int(((d2 >= lo) & (d2 <= hi)).sum())
    assert oracle.count_band(X, Z, T, 0.0, 100.0) == 300 * 280


def test_results_do_not_depend_on_the_thread_count():
    """The oracle keeps per-point partial sums and adds them in point order,
    so F, the gradient, F'', the input gradients and a registration are
    bitwise the same on 1 and on several threads."""
    r, X, Z, FX, FZ = _cloud_pair(63, 200, 180)
    T = rand_T(r, 0.2, 0.2)
    kw = dict(FX=FX, FZ=FZ, blocks=BLOCKS, ell=0.4, cutoff_mult=2.5)
    default = oracle.num_threads()
    a = oracle.evaluate(X, Z, T, nthreads=1, direction=np.ones(6), **kw)
    b = oracle.evaluate(X, Z, T, nthreads=4, direction=np.ones(6), **kw)
    assert a["F"] == b["F"] and np.array_equal(a["g"], b["g"]) and a["Fpp"] == b["Fpp"]
    ga = oracle.backward(X, Z, T, nthreads=1, **kw)
    gb = oracle.backward(X, Z, T, nthreads=4, **kw)
    for k in ("dX", "dZ", "dFX", "dFZ"):
        assert np.array_equal(ga[k], gb[k]), k
    assert ga["dell"] == gb["dell"]
    Ta, _, tra = oracle.register(X, Z, np.eye(4), nthreads=1, max_iters=5, **kw)
    Tb, _, trb = oracle.register(X, Z, np.eye(4), nthreads=3, max_iters=5, **kw)
    assert np.array_equal(Ta, Tb) and np.array_equal(tra, trb)
    oracle.evaluate(X[:1], Z[:1], T, nthreads=default, **kw)   # the thread count is process-wide: put it back
    assert oracle.num_threads() == default


def test_empty_clouds_give_zero():
    X = np.zeros((0, 3))
    Z = np.ones((5, 3))
    res = oracle.evaluate(X, Z, np.eye(4), ell=0.3)
    assert res["F"] == 0 and res["npairs"] == 0 and not np.any(res["g"])
    assert oracle.indicator(X, Z, np.eye(4), ell=0.3) == 0.0


# ---------------------------------------------------------------------------
# 3. invariants
# ---------------------------------------------------------------------------

BLOCKS = [("se", 3, 0.4, 1.1), ("dot", 4, 1.0, 1.0)]


def _cloud_pair(seed, n=30, m=25):
    r = rng(seed)
    X = r.uniform(-1, 1, size=(n, 3))
    Z = r.uniform(-1, 1, size=(m, 3))
    FX = np.hstack([r.uniform(0, 1, size=(n, 3)), r.dirichlet(np.ones(4), size=n)])
    FZ = np.hstack([r.uniform(0, 1, size=(m, 3)), r.dirichlet(np.ones(4), size=m)])
    return r, X, Z, FX, FZ


@pytest.mark.parametrize("cm", [0.0, 2.5])
def test_symmetry(cm):
    """<f_X, T f_Z> = <f_Z, T^-1 f_X> (the inner product and c_ij are symmetric)."""
    r, X, Z, FX, FZ = _cloud_pair(7)
    T = rand_T(r)
    a = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=0.4, cutoff_mult=cm, sigma=1.2)
    b = oracle.evaluate(Z, X, np.linalg.inv(T), FX=FZ, FZ=FX, blocks=BLOCKS, ell=0.4, cutoff_mult=cm, sigma=1.2)
    assert a["F"] == pytest.approx(b["F"], rel=1e-12)
    assert a["npairs"] == b["npairs"]


def test_rigid_invariance():
    """F(GX, GZ, G T G^-1) = F(X, Z, T) for any rigid G."""
    r, X, Z, FX, FZ = _cloud_pair(8)
    T = rand_T(r)
    G = rand_T(r, 2.0, 5.0)
    a = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=0.4)
    b = oracle.evaluate(transform(G, X), transform(G, Z), G @ T @ np.linalg.inv(G), FX=FX, FZ=FZ,
                        blocks=BLOCKS, ell=0.4)
    assert a["F"] == pytest.approx(b["F"], rel=1e-11)
    assert oracle.indicator(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=0.4) == pytest.approx(
        oracle.indicator(transform(G, X), transform(G, Z), G @ T @ np.linalg.inv(G), FX=FX, FZ=FZ,
                         blocks=BLOCKS, ell=0.4), rel=1e-11)


@pytest.mark.parametrize("cm", [0.0, 3.0])
def test_zero_gradient_identical_clouds(cm):
    """Z = X, T = I: every pair (i, j) has its mirror (j, i), so g = 0."""
    r, X, _, FX, _ = _cloud_pair(9)
    res = oracle.evaluate(X, X, np.eye(4), FX=FX, FZ=FX, blocks=BLOCKS, ell=0.4, cutoff_mult=cm)
    assert np.abs(res["g"]).max() < 1e-12 * max(1.0, res["F"])


def test_cauchy_schwarz():
    """Dense mode: F(X,Z,T)^2 <= F(X,X,I) F(Z,Z,I), equality for Z = X, T = I."""
    r, X, Z, FX, FZ = _cloud_pair(10)
    kw = dict(blocks=BLOCKS, ell=0.5)
    fxx = oracle.evaluate(X, X, np.eye(4), FX=FX, FZ=FX, **kw)["F"]
    fzz = oracle.evaluate(Z, Z, np.eye(4), FX=FZ, FZ=FZ, **kw)["F"]
    for _ in range(5):
        T = rand_T(r)
        f = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, **kw)["F"]
        assert f * f <= fxx * fzz * (1 + 1e-12)
    G = rand_T(r)
    f_same = oracle.evaluate(X, transform(G, X), np.linalg.inv(G), FX=FX, FZ=FX, **kw)["F"]
    assert f_same == pytest.approx(fxx, rel=1e-12)


def test_remark_norm_sqrt_n():
    """Remark (Sec. III-C): k -> delta and c_ii = 1 give |f_X| = sqrt(|X|), so
    the indicator of a cloud with itself tends to 1 as l shrinks below the
    point spacing."""
    r = rng(11)
    X = r.uniform(-1, 1, size=(50, 3))
    vals = [oracle.indicator(X, X, np.eye(4), ell=ell) for ell in (0.2, 0.05, 0.01, 0.002)]
    assert vals[0] > vals[1] > vals[2] >= vals[3]
    assert vals[-1] == pytest.approx(1.0, abs=1e-12)
    assert math.sqrt(oracle.evaluate(X, X, np.eye(4), ell=0.002)["F"]) == pytest.approx(math.sqrt(50), rel=1e-12)


def test_cosine_by_quadrature():
    """Eq. (indicator): the cosine of the embedded functions, each inner
    product taken by quadrature of the Gaussian fields (independent of the
    oracle's double sum)."""
    r = rng(30)
    X = r.uniform(-0.5, 0.5, size=(4, 3))
    Z = r.uniform(-0.5, 0.5, size=(3, 3))
    T = rand_T(r, 0.3, 0.2)
    ell = 0.3
    Y = transform(T, Z)
    ref = quad_F(X, Y, ell, 1.0) / math.sqrt(quad_F(X, X, ell, 1.0) * quad_F(Y, Y, ell, 1.0))
    assert oracle.cosine(X, Z, T, ell=ell, sigma=1.7) == pytest.approx(ref, rel=1e-10)


def test_cosine_bounds_and_remark():
    """Dense mode: |cos| <= 1 with equality for Z = G X, T = G^-1; with
    l below the point spacing (the Remark, Sec. III-C) the exact cosine and
    the indicator of Eq. (indicator_actual) coincide."""
    r, X, Z, FX, FZ = _cloud_pair(31)
    kw = dict(blocks=BLOCKS, ell=0.5)
    for _ in range(4):
        c = oracle.cosine(X, Z, rand_T(r), FX=FX, FZ=FZ, **kw)
        assert abs(c) <= 1.0 + 1e-12
    G = rand_T(r)
    assert oracle.cosine(X, transform(G, X), np.linalg.inv(G), FX=FX, FZ=FX, **kw) == pytest.approx(1.0, abs=1e-12)
    P = r.uniform(-1, 1, size=(40, 3))
    Q = P + r.normal(size=P.shape) * 1e-4
    assert oracle.cosine(P, Q, np.eye(4), ell=1e-3) == pytest.approx(oracle.indicator(P, Q, np.eye(4), ell=1e-3),
                                                                     rel=1e-9)


def test_indicator_peaks_at_zero_error():
    """Fig. 3 (Sec. III-C): rotating or translating a cloud away from itself
    lowers the indicator, and the maximum is at zero error."""
    p = scenes.cube_pair(n=600)
    X, F = p.X.astype(np.float64), p.FX.astype(np.float64)
    kw = dict(FX=F, FZ=F, blocks=p.blocks, ell=0.1)
    base = oracle.indicator(X, X, np.eye(4), **kw)
    axis = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    prev = base
    for deg in (1, 2, 4, 8, 16):
        T = expm_se3(np.concatenate([axis * math.radians(deg), np.zeros(3)]))
        cur = oracle.indicator(X, X, T, **kw)
        assert cur < prev
        prev = cur
    prev = base
    for d in (0.02, 0.05, 0.1, 0.2, 0.4):
        T = expm_se3(np.concatenate([np.zeros(3), axis * d]))
        cur = oracle.indicator(X, X, T, **kw)
        assert cur < prev
        prev = cur


# ---------------------------------------------------------------------------
# 4. the se(3) gradient and the second derivative by finite differences
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("with_feat", [False, True])
def test_gradient_central_differences(with_feat):
    r, X, Z, FX, FZ = _cloud_pair(12, 20, 18)
    T = rand_T(r, 0.3, 0.3)
    kw = dict(ell=0.45, sigma=1.3)
    if with_feat:
        kw.update(FX=FX, FZ=FZ, blocks=BLOCKS)
    g = oracle.evaluate(X, Z, T, **kw)["g"]
    eps = 1e-5
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = eps
        fp = oracle.evaluate(X, Z, expm_se3(e) @ T, **kw)["F"]
        fm = oracle.evaluate(X, Z, expm_se3(-e) @ T, **kw)["F"]
        fd[k] = (fp - fm) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-6 * np.linalg.norm(g)


@pytest.mark.parametrize("cut", [False, True])
def test_derivatives_in_extended_precision(cut):
    """F, its se(3) gradient and the second derivative along the gradient
    against the double sum written out in 30-digit arithmetic, differentiated
    by mpmath (the pose perturbed on the left through the 4x4 matrix
    exponential), on a tiny cloud pair with both kinds of feature block.
    With a cutoff, no pair lies within 5 % of its radius, so the pair set is
    the same throughout the differentiation."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    r = rng(60)
    n, m = 5, 4
    X = r.uniform(-0.4, 0.4, (n, 3))
    Z = r.uniform(-0.4, 0.4, (m, 3))
    FX = np.hstack([r.uniform(0, 1, (n, 3)), r.dirichlet(np.ones(4), n)])
    FZ = np.hstack([r.uniform(0, 1, (m, 3)), r.dirichlet(np.ones(4), m)])
    blocks = [("se", 3, 0.3, 1.2), ("dot", 4, 1.0, 1.0)]
    ell, sigma = 0.35, 1.1
    T = rand_T(r, 0.2, 0.2)
    mp = mpmath.mpf
    T0 = mpmath.matrix(T.tolist())
    Xm = [[mp(v) for v in row] for row in X]
    Zm = [mpmath.matrix([mp(v) for v in row] + [1]) for row in Z]
    c = [[mp(1.2) ** 2 * mpmath.exp(-sum((mp(a) - mp(b)) ** 2 for a, b in zip(FX[i, :3], FZ[j, :3]))
                                      / (2 * mp(0.3) ** 2))
          * sum(mp(a) * mp(b) for a, b in zip(FX[i, 3:], FZ[j, 3:])) for j in range(m)] for i in range(n)]
    Y = transform(T, Z)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    cm = 0.0
    inside = np.ones((n, m), bool)
    if cut:   # the first cutoff multiple with every pair at least 5 % away from the radius
        cm = next(k for k in np.arange(1.0, 3.01, 0.1)
                  if np.all(np.abs(np.sqrt(d2) / (k * ell) - 1.0) > 0.05))
        inside = d2 <= (cm * ell) ** 2
        assert 0 < inside.sum() < n * m

    def hat_mp(xi):
        w, v = xi[:3], xi[3:]
        return mpmath.matrix([[0, -w[2], w[1], v[0]], [w[2], 0, -w[0], v[1]], [-w[1], w[0], 0, v[2]],
                              [0, 0, 0, 0]])

    def F(xi):
        Tx = mpmath.expm(hat_mp(xi)) * T0
        s = mp(0)
        for j in range(m):
            y = Tx * Zm[j]
            for i in range(n):
                if inside[i, j]:
                    e2 = sum((Xm[i][q] - y[q]) ** 2 for q in range(3))
                    s += mp(sigma) ** 2 * mpmath.exp(-e2 / (2 * mp(ell) ** 2)) * c[i][j]
        return s

    def along(k):
        return lambda h: F([h if q == k else mp(0) for q in range(6)])

    g_ref = np.array([float(mpmath.diff(along(k), 0)) for k in range(6)])
    kw = dict(FX=FX, FZ=FZ, blocks=blocks, ell=ell, sigma=sigma, cutoff_mult=cm)
    res = oracle.evaluate(X, Z, T, **kw)
    assert res["F"] == pytest.approx(float(F([mp(0)] * 6)), rel=1e-13)
    assert res["npairs"] == int(inside.sum())
    assert np.abs(res["g"] - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
    d = res["g"]
    fpp_ref = float(mpmath.diff(lambda h: F([h * mp(a) for a in d]), 0, 2))
    fpp = oracle.evaluate(X, Z, T, direction=d, **kw)["Fpp"]
    assert fpp == pytest.approx(fpp_ref, rel=1e-11)


def test_second_derivative_along_direction():
    r, X, Z, FX, FZ = _cloud_pair(13, 20, 18)
    T = rand_T(r, 0.3, 0.3)
    kw = dict(FX=FX, FZ=FZ, blocks=BLOCKS, ell=0.45)
    for _ in range(3):
        xi = r.normal(size=6)
        res = oracle.evaluate(X, Z, T, direction=xi, **kw)
        eps = 1e-4
        f0 = res["F"]
        fp = oracle.evaluate(X, Z, expm_se3(eps * xi) @ T, **kw)["F"]
        fm = oracle.evaluate(X, Z, expm_se3(-eps * xi) @ T, **kw)["F"]
        fd2 = (fp - 2 * f0 + fm) / eps ** 2
        assert res["Fpp"] == pytest.approx(fd2, rel=2e-5, abs=1e-6 * abs(f0))
        # first derivative along xi is g . xi
        fd1 = (fp - fm) / (2 * eps)
        assert float(res["g"] @ xi) == pytest.approx(fd1, rel=1e-6)


# ---------------------------------------------------------------------------
# 5. SE(3) exponential / logarithm
# ---------------------------------------------------------------------------

def test_se3_exp_matches_expm():
    r = rng(14)
    for scale in (1e-8, 1e-5, 9e-4, 1.1e-3, 0.1, 1.0, 2.5):
        for _ in range(4):
            xi = r.normal(size=6) * scale
            T = oracle.se3_exp(xi)
            np.testing.assert_allclose(T, expm_se3(xi), rtol=0, atol=1e-14 * max(1.0, np.abs(xi).max()))
            assert np.linalg.det(T[:3, :3]) == pytest.approx(1.0, abs=1e-13)


def test_se3_log_inverts_exp():
    r = rng(15)
    for scale in (1e-9, 1e-6, 1e-3, 0.3, 2.0):
        for _ in range(4):
            xi = r.normal(size=6) * scale
            if np.linalg.norm(xi[:3]) > 3.0:
                continue
            back = oracle.se3_log(oracle.se3_exp(xi))
            np.testing.assert_allclose(back, xi, rtol=1e-9, atol=1e-15)
    T = rand_T(r)
    np.testing.assert_allclose(oracle.se3_exp(oracle.se3_log(T)), T, atol=1e-13)


def test_se3_exp_in_extended_precision():
    """The closed form and its small-angle series against the matrix
    exponential of the 4x4 twist in 40-digit arithmetic, at angles on both
    sides of the series' switch and with a long translation, so that an error
    in a series term (a few parts in 1e14 of the result) exceeds rounding."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    r = rng(16)
    for th in (1e-6, 3e-4, 9.9e-4, 1.01e-3, 0.05, 0.099, 0.101, 1.3, 3.0):
        for _ in range(3):
            axis = r.normal(size=3)
            axis /= np.linalg.norm(axis)
            v = r.normal(size=3)
            v *= 1e4 / np.linalg.norm(v)
            xi = np.concatenate([axis * th, v])
            ref = mpmath.expm(mpmath.matrix(hat(xi).tolist()))
            ref = np.array([[float(ref[i, j]) for j in range(4)] for i in range(4)])
            T = oracle.se3_exp(xi)
            np.testing.assert_allclose(T[:3, :3], ref[:3, :3], rtol=0, atol=8e-16)
            np.testing.assert_allclose(T[:3, 3], ref[:3, 3], rtol=0, atol=2e-15 * 1e4)


def test_se3_log_in_extended_precision():
    """The logarithm of a pose against the matrix logarithm of the same
    (rounded) pose in 40-digit arithmetic, on both sides of its series switch."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    r = rng(17)
    for th in (1e-6, 9.9e-4, 1.01e-3, 0.05, 1.3, 2.5):
        for _ in range(3):
            axis = r.normal(size=3)
            axis /= np.linalg.norm(axis)
            v = r.normal(size=3)
            v *= 1e2 / np.linalg.norm(v)
            E = mpmath.expm(mpmath.matrix(hat(np.concatenate([axis * th, v])).tolist()))
            T = np.array([[float(E[i, j]) for j in range(4)] for i in range(4)])
            L = mpmath.logm(mpmath.matrix(T.tolist()))
            ref = np.array([float(L[2, 1]), float(L[0, 2]), float(L[1, 0]),
                            float(L[0, 3]), float(L[1, 3]), float(L[2, 3])])
            got = oracle.se3_log(T)
            np.testing.assert_allclose(got[:3], ref[:3], rtol=0, atol=4e-15)
            np.testing.assert_allclose(got[3:], ref[3:], rtol=0, atol=4e-14 * 1e2)


def test_se3_small_angle_branch_continuous():
    axis = np.array([0.48, -0.6, 0.64])
    v = np.array([0.3, 0.1, -0.2])
    lo = oracle.se3_exp(np.concatenate([axis * (1e-3 * (1 - 1e-9)), v]))
    hi = oracle.se3_exp(np.concatenate([axis * (1e-3 * (1 + 1e-9)), v]))
    np.testing.assert_allclose(lo, hi, atol=1e-14)


# ---------------------------------------------------------------------------
# 6. registration end point: recovery of a known transform
# ---------------------------------------------------------------------------

def test_recovery_of_known_transform():
    """Z = T_gt X with the same points: the dense F attains its maximum at
    T_gt^-1 (Cauchy-Schwarz), and the ascent converges there."""
    p = scenes.cube_pair(n=300, seed=77)
    T_out, info, trace = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.3,
                                         max_iters=400, step_tol_rot=1e-9, step_tol_trans=1e-9)
    assert info["status"] == 0
    err = oracle.se3_log(np.linalg.inv(p.T_true) @ T_out)
    assert np.linalg.norm(err[:3]) < 1e-6 and np.linalg.norm(err[3:]) < 1e-6
    # the objective never decreases along the way
    F = trace[:, 1]
    assert np.all(np.diff(F) > -1e-9 * F[:-1])


def test_replay_reproduces_annealing_decisions():
    p = scenes.cube_pair(n=200, seed=78)
    kw = dict(FX=p.FX, FZ=p.FZ, blocks=p.blocks, ell=0.5, ell_min=0.2, cutoff_mult=3.0, anneal=True,
              max_iters=40, indicator_tol=5e-3)
    T1, info1, tr1 = oracle.register(p.X, p.Z, np.eye(4), **kw)
    assert tr1[:, 8].sum() > 0  # some decays happened
    T2, info2, tr2 = oracle.register(p.X, p.Z, np.eye(4), replay=tr1[:, 8].astype(int), **kw)
    np.testing.assert_array_equal(tr1, tr2)
    np.testing.assert_array_equal(T1, T2)
    # the lengthscale only shrinks, by the decay factor, never below the floor
    ells = tr1[:, 0]
    assert np.all(np.diff(ells) <= 0) and ells.min() >= 0.2
    steps = ells[1:][np.diff(ells) < 0] / ells[:-1][np.diff(ells) < 0]
    assert np.all((np.abs(steps - 0.98) < 1e-12) | (ells[1:][np.diff(ells) < 0] == 0.2))


# ---------------------------------------------------------------------------
# 7. gradients with respect to points, features and the lengthscale
# ---------------------------------------------------------------------------

def test_backward_central_differences():
    r, X, Z, FX, FZ = _cloud_pair(21, 14, 12)
    T = rand_T(r, 0.2, 0.2)
    kw = dict(blocks=BLOCKS, ell=0.5, sigma=1.1)
    g = oracle.backward(X, Z, T, FX=FX, FZ=FZ, **kw)

    def F(X_=X, Z_=Z, FX_=FX, FZ_=FZ, ell=0.5):
        return oracle.evaluate(X_, Z_, T, FX=FX_, FZ=FZ_, blocks=BLOCKS, ell=ell, sigma=1.1)["F"]

    eps = 1e-6
    for (i, a) in [(0, 0), (3, 1), (7, 2)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, a] += eps
        Xm[i, a] -= eps
        assert g["dX"][i, a] == pytest.approx((F(X_=Xp) - F(X_=Xm)) / (2 * eps), rel=1e-6, abs=1e-9)
    for (j, a) in [(1, 0), (5, 2)]:
        Zp, Zm = Z.copy(), Z.copy()
        Zp[j, a] += eps
        Zm[j, a] -= eps
        assert g["dZ"][j, a] == pytest.approx((F(Z_=Zp) - F(Z_=Zm)) / (2 * eps), rel=1e-6, abs=1e-9)
    for (i, a) in [(2, 0), (4, 2), (6, 3), (9, 5)]:   # squared-exponential and inner-product entries
        Fp, Fm = FX.copy(), FX.copy()
        Fp[i, a] += eps
        Fm[i, a] -= eps
        assert g["dFX"][i, a] == pytest.approx((F(FX_=Fp) - F(FX_=Fm)) / (2 * eps), rel=1e-6, abs=1e-9)
    for (j, a) in [(0, 1), (3, 4)]:
        Fp, Fm = FZ.copy(), FZ.copy()
        Fp[j, a] += eps
        Fm[j, a] -= eps
        assert g["dFZ"][j, a] == pytest.approx((F(FZ_=Fp) - F(FZ_=Fm)) / (2 * eps), rel=1e-6, abs=1e-9)
    assert g["dell"] == pytest.approx((F(ell=0.5 + eps) - F(ell=0.5 - eps)) / (2 * eps), rel=1e-6)


def test_backward_in_extended_precision():
    """Every input gradient (points, both clouds' squared-exponential and
    inner-product feature entries, the lengthscale) against mpmath's
    derivative of the double sum written out in 30-digit arithmetic, on a
    tiny dense pair."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    mp = mpmath.mpf
    r, X, Z, FX, FZ = _cloud_pair(61, 5, 4)
    T = rand_T(r, 0.2, 0.2)
    ell0, sigma = 0.5, 1.1
    Rm = [[mp(T[a, b]) for b in range(3)] for a in range(3)]
    tm = [mp(T[a, 3]) for a in range(3)]
    (_, d_se, l_se, s_se), (_, d_dot, _, _) = BLOCKS
    base = dict(X=[[mp(v) for v in row] for row in X], Z=[[mp(v) for v in row] for row in Z],
                FX=[[mp(v) for v in row] for row in FX], FZ=[[mp(v) for v in row] for row in FZ], ell=mp(ell0))

    def F(a):
        s = mp(0)
        for j, z in enumerate(a["Z"]):
            y = [sum(Rm[q][b] * z[b] for b in range(3)) + tm[q] for q in range(3)]
            v = a["FZ"][j]
            for i, x in enumerate(a["X"]):
                u = a["FX"][i]
                e2 = sum((x[q] - y[q]) ** 2 for q in range(3))
                c = mp(s_se) ** 2 * mpmath.exp(-sum((u[q] - v[q]) ** 2 for q in range(d_se)) / (2 * mp(l_se) ** 2))
                c *= sum(u[q] * v[q] for q in range(d_se, d_se + d_dot))
                s += mp(sigma) ** 2 * mpmath.exp(-e2 / (2 * a["ell"] ** 2)) * c
        return s

    def deriv(key, i=None, k=None):
        def f(h):
            a = dict(base)
            if key == "ell":
                a["ell"] = base["ell"] + h
            else:
                rows = [list(row) for row in base[key]]
                rows[i][k] += h
                a[key] = rows
            return F(a)
        return float(mpmath.diff(f, 0))

    g = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=ell0, sigma=sigma)
    for key, arr in (("X", "dX"), ("Z", "dZ"), ("FX", "dFX"), ("FZ", "dFZ")):
        ref = np.array([[deriv(key, i, k) for k in range(len(base[key][0]))] for i in range(len(base[key]))])
        assert np.abs(g[arr] - ref).max() <= 1e-12 * np.abs(ref).max(), arr
    assert g["dell"] == pytest.approx(deriv("ell"), rel=1e-12)


def test_backward_translation_invariance():
    """Moving both clouds together leaves F unchanged: sum dX + R sum dZ = 0."""
    r, X, Z, FX, FZ = _cloud_pair(22, 20, 17)
    T = rand_T(r, 0.3, 0.3)
    g = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=BLOCKS, ell=0.4, cutoff_mult=2.5)
    total = g["dX"].sum(0) + g["dZ"].sum(0) @ T[:3, :3].T
    assert np.abs(total).max() < 1e-10 * max(1.0, np.abs(g["dX"]).max())


def test_sequence_recovers_exact_motions():
    """Odometry chaining (Sec. V-A): frames that are exact rigid copies of one
    cloud; each registration recovers the true relative motion (dense F is
    maximal there, Cauchy-Schwarz) and the absolute poses are their products."""
    r = rng(40)
    W = r.uniform(-1.0, 1.0, size=(250, 3))
    C = [np.eye(4)]
    for _ in range(3):
        C.append(C[-1] @ rand_T(r, 0.05, 0.05))
    frames = [(transform(np.linalg.inv(Ck), W), None) for Ck in C]
    T_rel, T_abs, infos = oracle.register_sequence(frames, 0.3, ell=0.3, max_iters=300)
    for k in range(3):
        truth = np.linalg.inv(C[k]) @ C[k + 1]
        assert np.abs(T_rel[k] - truth).max() < 1e-5
        assert np.abs(T_abs[k + 1] - C[k + 1]).max() < 1e-5
        assert infos[k]["status"] == 0


def test_feature_cutoff_by_brute_force():
    """Sec. III-B's sparsity in feature space, as the optional feature cutoff:
    F equals the numpy double sum over the pairs inside both cutoffs (the
    colour distance of every squared-exponential block within the cutoff
    times its scale); a cutoff wide enough to keep every pair changes
    nothing."""
    r = rng(50)
    X = r.uniform(-0.6, 0.6, size=(40, 3))
    Z = r.uniform(-0.6, 0.6, size=(35, 3))
    FX = np.concatenate([r.uniform(0, 1, size=(40, 3)), r.dirichlet(np.ones(4), size=40)], axis=1)
    FZ = np.concatenate([r.uniform(0, 1, size=(35, 3)), r.dirichlet(np.ones(4), size=35)], axis=1)
    blocks = [("se", 3, 0.25, 1.3), ("dot", 4, 1.0, 1.0)]
    T = rand_T(r, 0.2, 0.1)
    ell, cm, fm = 0.3, 2.5, 1.5
    Y = transform(T, Z)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    c2 = ((FX[:, None, :3] - FZ[None, :, :3]) ** 2).sum(-1)
    keep = (d2 <= (cm * ell) ** 2) & (c2 <= (fm * 0.25) ** 2)
    w = np.exp(-d2 / (2 * ell ** 2)) * 1.3 ** 2 * np.exp(-c2 / (2 * 0.25 ** 2)) * (FX[:, None, 3:] * FZ[None, :, 3:]).sum(-1)
    ref = (w * keep).sum()
    got = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, feat_cutoff_mult=fm)
    assert got["F"] == pytest.approx(ref, rel=1e-12)
    assert got["npairs"] == int(keep.sum()) and 0 < keep.sum() < (d2 <= (cm * ell) ** 2).sum()
    wide = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, feat_cutoff_mult=100.0)
    plain = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm)
    assert wide["F"] == plain["F"] and wide["npairs"] == plain["npairs"]
    # the input gradients use the same pair set: central differences of F
    g = oracle.backward(X, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, feat_cutoff_mult=fm)
    eps = 1e-6
    Xp, Xm = X.copy(), X.copy()
    Xp[3, 1] += eps
    Xm[3, 1] -= eps
    fd = (oracle.evaluate(Xp, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, feat_cutoff_mult=fm)["F"]
          - oracle.evaluate(Xm, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, feat_cutoff_mult=fm)["F"]) / (2 * eps)
    assert g["dX"][3, 1] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_feature_cutoff_leaves_inner_product_blocks_uncut():
    """The feature cutoff applies to squared-exponential blocks alone: with an
    inner-product block whose vectors lie far apart (off the simplex, so that
    most distances exceed any radius the cutoff would give them), F and the
    pair count equal the numpy double sum cut on the colour block only."""
    r = rng(52)
    X = r.uniform(-0.5, 0.5, size=(36, 3))
    Z = r.uniform(-0.5, 0.5, size=(33, 3))
    FX = np.concatenate([r.uniform(0, 1, size=(36, 2)), r.uniform(0, 4, size=(36, 3))], axis=1)
    FZ = np.concatenate([r.uniform(0, 1, size=(33, 2)), r.uniform(0, 4, size=(33, 3))], axis=1)
    blocks = [("se", 2, 0.3, 1.0), ("dot", 3, 1.0, 1.0)]
    T = rand_T(r, 0.1, 0.05)
    ell, cm, fm = 0.4, 3.0, 1.2
    Y = transform(T, Z)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    c2 = ((FX[:, None, :2] - FZ[None, :, :2]) ** 2).sum(-1)
    p2 = ((FX[:, None, 2:] - FZ[None, :, 2:]) ** 2).sum(-1)
    keep = (d2 <= (cm * ell) ** 2) & (c2 <= (fm * 0.3) ** 2)
    assert (p2[keep] > (fm * 1.0) ** 2).mean() > 0.5      # a cut on the inner-product block would bite
    w = np.exp(-d2 / (2 * ell ** 2)) * np.exp(-c2 / (2 * 0.3 ** 2)) * (FX[:, None, 2:] * FZ[None, :, 2:]).sum(-1)
    got = oracle.evaluate(X, Z, T, FX=FX, FZ=FZ, blocks=blocks, ell=ell, cutoff_mult=cm, feat_cutoff_mult=fm)
    assert got["F"] == pytest.approx((w * keep).sum(), rel=1e-12)
    assert got["npairs"] == int(keep.sum())


def test_feature_cutoff_input_gradients_by_central_differences():
    """The oracle's input gradients with the feature cutoff (the pair set held
    fixed) against central differences of its F, for a point of Z and for a
    colour and a label entry of X and of Z; each perturbed point is chosen
    with no colour distance near the cutoff radius, so the pair set does not
    change between the two evaluations."""
    r = rng(51)
    X = r.uniform(-0.5, 0.5, size=(30, 3))
    Z = r.uniform(-0.5, 0.5, size=(28, 3))
    FX = np.concatenate([r.uniform(0, 1, size=(30, 3)), r.dirichlet(np.ones(4), size=30)], axis=1)
    FZ = np.concatenate([r.uniform(0, 1, size=(28, 3)), r.dirichlet(np.ones(4), size=28)], axis=1)
    blocks = [("se", 3, 0.25, 1.2), ("dot", 4, 1.0, 1.0)]
    T = rand_T(r, 0.15, 0.1)
    kw = dict(blocks=blocks, ell=0.35, cutoff_mult=2.5, feat_cutoff_mult=1.4)
    rad = 1.4 * 0.25
    c = np.sqrt(((FX[:, None, :3] - FZ[None, :, :3]) ** 2).sum(-1))
    far = np.abs(c - rad) > 1e-3          # colour distances well away from the radius
    i = int(np.argmax(far.all(1)))        # a point of X with none near it
    j = int(np.argmax(far.all(0)))        # a point of Z with none near it
    assert far[i].all() and far[:, j].all()
    g = oracle.backward(X, Z, T, FX=FX, FZ=FZ, **kw)
    eps = 1e-6

    def F(Xa, Za, FXa, FZa):
        return oracle.evaluate(Xa, Za, T, FX=FXa, FZ=FZa, **kw)["F"]

    def fd(which, idx):
        arrs = [X.copy(), Z.copy(), FX.copy(), FZ.copy()]
        arrs[which][idx] += eps
        fp = F(*arrs)
        arrs[which][idx] -= 2 * eps
        fm = F(*arrs)
        return (fp - fm) / (2 * eps)

    assert g["dZ"][j, 2] == pytest.approx(fd(1, (j, 2)), rel=1e-6, abs=1e-9)
    assert g["dFX"][i, 1] == pytest.approx(fd(2, (i, 1)), rel=1e-6, abs=1e-9)   # colour
    assert g["dFX"][i, 4] == pytest.approx(fd(2, (i, 4)), rel=1e-6, abs=1e-9)   # label
    assert g["dFZ"][j, 0] == pytest.approx(fd(3, (j, 0)), rel=1e-6, abs=1e-9)   # colour


def test_cosine_and_its_lengthscale_derivative_in_extended_precision():
    """The exact indicator of Eq. (indicator) as a function of l, written out
    as its three double sums in 30-digit arithmetic, and its l-derivative by
    mpmath's differentiation: oracle.cosine_ell gives both (dense sums, both
    kinds of feature block, a pose that moves Z)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    r = rng(61)
    n, m = 5, 6
    X = r.uniform(-0.5, 0.5, (n, 3))
    Z = r.uniform(-0.5, 0.5, (m, 3))
    FX = np.hstack([r.uniform(0, 1, (n, 3)), r.dirichlet(np.ones(4), n)])
    FZ = np.hstack([r.uniform(0, 1, (m, 3)), r.dirichlet(np.ones(4), m)])
    blocks = [("se", 3, 0.3, 1.2), ("dot", 4, 1.0, 1.0)]
    sigma, ell = 1.1, 0.4
    T = rand_T(r, 0.2, 0.2)
    mp = mpmath.mpf

    def feat_k(u, v):
        return mp(1.2) ** 2 * mpmath.exp(-sum((mp(a) - mp(b)) ** 2 for a, b in zip(u[:3], v[:3])) /
                                         (2 * mp(0.3) ** 2)) * sum(mp(a) * mp(b) for a, b in zip(u[3:], v[3:]))

    def dsum(A, B, FA, FB, l):
        s = mp(0)
        for i in range(len(A)):
            for j in range(len(B)):
                e2 = sum((mp(A[i][q]) - mp(B[j][q])) ** 2 for q in range(3))
                s += mp(sigma) ** 2 * mpmath.exp(-e2 / (2 * l ** 2)) * feat_k(FA[i], FB[j])
        return s

    Y = transform(T, Z)

    def cos(l):
        return dsum(X, Y, FX, FZ, l) / mpmath.sqrt(dsum(X, X, FX, FX, l) * dsum(Z, Z, FZ, FZ, l))

    c_ref = float(cos(mp(ell)))
    d_ref = float(mpmath.diff(cos, mp(ell)))
    c, d = oracle.cosine_ell(X, Z, T, FX, FZ, ell=ell, blocks=blocks, sigma=sigma, cutoff_mult=0.0)
    assert c == pytest.approx(c_ref, rel=1e-13)
    assert c == pytest.approx(oracle.cosine(X, Z, T, FX, FZ, ell=ell, blocks=blocks, sigma=sigma), rel=1e-14)
    assert d == pytest.approx(d_ref, rel=1e-11)
    assert abs(d) > 1e-3   # the derivative is not trivially zero here


def test_cosine_grows_towards_its_large_lengthscale_limit():
    """Why the library offers dcos/dl for a caller's own objective but no
    built-in maximisation of the cosine over l: on independently sampled
    clouds at the true pose the cosine rises monotonically with l towards
    the limit of constant functions (every geometric kernel value 1), so it
    has no interior maximum to fix l by."""
    import scenes
    q = scenes.batch_pairs(n_pairs=1, n_range=(400, 400))[0]
    ells = np.geomspace(0.03, 3.0, 9)
    vals = [oracle.cosine_ell(q.X, q.Z, q.T_true, q.FX, q.FZ, ell=l, blocks=q.blocks, cutoff_mult=0.0)
            for l in ells]
    cs = np.array([v[0] for v in vals])
    ds = np.array([v[1] for v in vals])
    assert np.all(np.diff(cs) > 0) and np.all(ds > 0)
