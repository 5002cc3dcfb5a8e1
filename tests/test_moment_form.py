"""The per-query moment form used by the CUDA path equals the oracle's direct
per-pair form (gradient and second derivative), in exact FP64 arithmetic.

The CUDA sweep works in Z's frame: for each query x'_i = T^-1 x_i and each
pair (i, j) inside the cutoff it accumulates W = sum w, E = sum w e and
Q = sum w e e^T with e = z_j - x'_i.  Everything the step needs is linear in
these per-query moments, so per-query contributions can be summed in any
partition.  With lever arms p_i = x'_i - c about a fixed centre c, and
P = [p]_x, eight sums suffice (43 numbers):

  S_W, S_E, S_Q, S_PQ = sum P Q, S_PQP = sum P Q P, S_Wp, S_Wpp = sum W p p^T,
  S_Ep = sum E p^T.

From them the gradient and the Hessian of eta -> F(T exp(eta^)) in the
centred coordinates follow; the adjoint of T^-1 and the shift to the centre
map them to the left perturbation exp(xi^) T that the oracle uses.  This
test writes that algebra out in numpy and compares it with the oracle.
"""
import numpy as np
import pytest

import oracle


def skew(a):
    return np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])


def moment_stats(X, Z, FX, FZ, T, ell, cm, blocks, c):
    R, t = T[:3, :3], T[:3, 3]
    Xp = (X - t) @ R  # rows: R^T (x - t)
    S = dict(W=0.0, E=np.zeros(3), Q=np.zeros((3, 3)), PQ=np.zeros((3, 3)), PQP=np.zeros((3, 3)),
             Wp=np.zeros(3), Wpp=np.zeros((3, 3)), Ep=np.zeros((3, 3)))
    for i in range(X.shape[0]):
        e = Z - Xp[i]
        d2 = (e * e).sum(1)
        keep = np.ones_like(d2, dtype=bool) if cm <= 0 else d2 <= (cm * ell) ** 2
        w = np.exp(-d2 / (2 * ell ** 2))
        off = 0
        for kind, dim, scale, sig in blocks:
            u, v = FX[i, off:off + dim], FZ[:, off:off + dim]
            if kind == "se":
                w = w * sig ** 2 * np.exp(-((v - u) ** 2).sum(1) / (2 * scale ** 2))
            else:
                w = w * (v @ u)
            off += dim
        w = np.where(keep, w, 0.0)
        W = w.sum()
        E = (w[:, None] * e).sum(0)
        Q = (w[:, None, None] * e[:, :, None] * e[:, None, :]).sum(0)
        p = Xp[i] - c
        P = skew(p)
        S["W"] += W
        S["E"] += E
        S["Q"] += Q
        S["PQ"] += P @ Q
        S["PQP"] += P @ Q @ P
        S["Wp"] += W * p
        S["Wpp"] += W * np.outer(p, p)
        S["Ep"] += np.outer(E, p)
    return S


def assemble(S, T, ell, c):
    L2, L4 = ell ** 2, ell ** 4
    I = np.eye(3)
    ExP = np.array([S["Ep"][1, 2] - S["Ep"][2, 1], S["Ep"][2, 0] - S["Ep"][0, 2], S["Ep"][0, 1] - S["Ep"][1, 0]])
    g_c = np.concatenate([ExP / L2, -S["E"] / L2])
    Hww = -S["PQP"] / L4 - (np.trace(S["Wpp"]) * I - S["Wpp"]) / L2 \
        + 0.5 * (S["Ep"] + S["Ep"].T - 2 * np.trace(S["Ep"]) * I) / L2
    Hwv = S["PQ"] / L4 - skew(S["Wp"]) / L2 - 0.5 * skew(S["E"]) / L2
    Hvv = S["Q"] / L4 - S["W"] * I / L2
    H_c = np.block([[Hww, Hwv], [Hwv.T, Hvv]])
    # centred coordinates: xi_c = A eta,  A = [[I, 0], [-[c]x, I]]
    A = np.block([[I, np.zeros((3, 3))], [-skew(c), I]])
    # right perturbation eta = Ad_{T^-1} xi of the left perturbation xi
    R, t = T[:3, :3], T[:3, 3]
    Ad_inv = np.block([[R.T, np.zeros((3, 3))], [-R.T @ skew(t), R.T]])
    B = A @ Ad_inv
    return B.T @ g_c, B.T @ H_c @ B


CASES = [
    (0.0, []),
    (0.0, [("se", 3, 0.3, 1.2)]),
    (2.5, [("se", 3, 0.3, 1.0), ("dot", 4, 1.0, 1.0)]),
]


@pytest.mark.parametrize("cm,blocks", CASES)
def test_moment_form_matches_direct_form(cm, blocks):
    r = np.random.Generator(np.random.PCG64(31))
    n, m = 40, 35
    X = r.uniform(-1, 1, size=(n, 3)) + np.array([20.0, -5.0, 40.0])
    Z = r.uniform(-1, 1, size=(m, 3)) + np.array([19.5, -5.2, 40.3])
    D = sum(b[1] for b in blocks)
    FX = r.uniform(0, 1, size=(n, D))
    FZ = r.uniform(0, 1, size=(m, D))
    xi0 = np.concatenate([r.normal(size=3) * 0.05, r.normal(size=3) * 0.2])
    T = oracle.se3_exp(xi0)
    ell = 0.6
    c = 0.5 * (Z.min(0) + Z.max(0))
    S = moment_stats(X, Z, FX, FZ, T, ell, cm, blocks, c)
    g, H = assemble(S, T, ell, c)
    kw = dict(FX=FX if D else None, FZ=FZ if D else None, blocks=blocks, ell=ell, cutoff_mult=cm)
    ref = oracle.evaluate(X, Z, T, **kw)
    assert S["W"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(g, ref["g"], rtol=0, atol=1e-9 * np.abs(ref["g"]).max())
    for _ in range(4):
        d = r.normal(size=6)
        fpp = oracle.evaluate(X, Z, T, direction=d, **kw)["Fpp"]
        assert float(d @ H @ d) == pytest.approx(fpp, rel=1e-9)
    assert np.allclose(H, H.T, atol=1e-9 * np.abs(H).max())


def test_step_direction_from_the_centred_gradient_matches_the_oracles_rule():
    """The CUDA step takes the ascent direction in Z's centred coordinates,
    (w~, v~) = (gc_w / rho^2, gc_v) with gc the centred gradient the
    statistics give, and maps it to the left perturbation as
    (R w~, R v~ + p x R w~), p = R c + t; the oracle forms it from the
    origin-based gradient g as (h_w / rho^2, h_u + p x h_w / rho^2) with
    h = (g_w + g_v x p, g_v).  With c the centroid of Z both are the same
    vector, and F' = g . d equals |gc_w|^2 / rho^2 + |gc_v|^2."""
    r = np.random.Generator(np.random.PCG64(33))
    n, m = 30, 45
    X = r.uniform(-1, 1, size=(n, 3)) + np.array([20.0, -5.0, 40.0])
    Z = r.uniform(-1, 1, size=(m, 3)) + np.array([19.5, -5.2, 40.3])
    T = oracle.se3_exp(np.concatenate([r.normal(size=3) * 0.05, r.normal(size=3) * 0.2]))
    ell = 0.5
    c = Z.mean(axis=0)
    rho2 = np.mean(np.sum((Z - c) ** 2, axis=1)) + ell ** 2
    S = moment_stats(X, Z, np.zeros((n, 0)), np.zeros((m, 0)), T, ell, 0.0, [], c)
    g, _ = assemble(S, T, ell, c)
    ExP = np.array([S["Ep"][1, 2] - S["Ep"][2, 1], S["Ep"][2, 0] - S["Ep"][0, 2], S["Ep"][0, 1] - S["Ep"][1, 0]])
    gc_w, gc_v = ExP / ell ** 2, -S["E"] / ell ** 2
    R, t = T[:3, :3], T[:3, 3]
    p = R @ c + t
    wt, vt = gc_w / rho2, gc_v
    d_kernel = np.concatenate([R @ wt, R @ vt + np.cross(p, R @ wt)])
    hw = g[:3] + np.cross(g[3:], p)
    d_oracle = np.concatenate([hw / rho2, g[3:] + np.cross(p, hw / rho2)])
    np.testing.assert_allclose(d_kernel, d_oracle, rtol=0, atol=1e-10 * np.abs(d_oracle).max())
    assert float(g @ d_oracle) == pytest.approx(gc_w @ gc_w / rho2 + gc_v @ gc_v, rel=1e-10)
