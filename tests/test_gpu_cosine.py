"""The exact indicator of Eq. (indicator) (cvo_cosine) against the oracle.

Tolerance: the cosine is F / sqrt(F_XX F_ZZ); each of the three sums carries
the relative error 1e-5 of the inner product, so the ratio is held to
1e-5 + 1e-5 / 2 + 1e-5 / 2 = 2e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

COS_RTOL = 2e-5


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def sl(pair, n, seed):
    r = rng(seed)
    ix = r.permutation(len(pair.X))[:n]
    iz = r.permutation(len(pair.Z))[:n]
    return pair.X[ix], pair.Z[iz], pair.FX[ix], pair.FZ[iz]


@pytest.mark.parametrize("case", ["cube-dense", "street-cutoff", "room-bf16"])
def test_cosine_matches_oracle(case):
    if case == "cube-dense":
        p = scenes.cube_pair(n=1200)
        X, Z, FX, FZ = p.X, p.Z, p.FX, p.FZ
        kw = dict(blocks=p.blocks, ell=0.1, cutoff_mult=0.0)
        bf16 = False
    elif case == "street-cutoff":
        p = scenes.street_pair()
        X, Z, FX, FZ = sl(p, 4000, 1)
        kw = dict(blocks=p.blocks, ell=0.2, cutoff_mult=3.0)
        bf16 = False
    else:
        p = scenes.room_pair()
        X, Z, FX, FZ = sl(p, 5000, 2)
        kw = dict(blocks=p.blocks, ell=0.1, cutoff_mult=3.0)
        bf16 = True
    h = cvo.CVO(**kw)
    if bf16:
        fx = dev(FX).to(torch.bfloat16)
        fz = dev(FZ).to(torch.bfloat16)
        FX, FZ = scenes.bf16_round(FX), scenes.bf16_round(FZ)
    else:
        fx, fz = dev(FX), dev(FZ)
    for T in (p.T_true, np.eye(4)):
        got, norms = h.cosine(dev(X), dev(Z), T, fx, fz)
        ref = oracle.cosine(X, Z, T, FX=FX, FZ=FZ, **kw)
        assert got == pytest.approx(ref, rel=COS_RTOL)
        # the norms do not depend on T: passing them back gives the same cosine
        again, norms2 = h.cosine(dev(X), dev(Z), T, fx, fz, norms2=norms)
        assert again == got and norms2 == norms
        if kw["cutoff_mult"] <= 0:
            assert abs(got) <= 1.0 + 1e-6
    # the approximate indicator of Eq. (indicator_actual) is F / sqrt(N M)
    i_theta = h.metric(dev(X), dev(Z), p.T_true, fx, fz)
    c, norms = h.cosine(dev(X), dev(Z), p.T_true, fx, fz)
    assert c == pytest.approx(i_theta * math.sqrt(len(X) * len(Z) / (norms[0] * norms[1])), rel=1e-12)


def test_cosine_edge_cases():
    r = rng(3)
    X, _ = scenes.random_cloud(r, 300, 0, extent=0.5)
    h = cvo.CVO(blocks=[], ell=0.05, cutoff_mult=0.0)
    c, norms = h.cosine(dev(X), dev(X), np.eye(4))
    assert c == pytest.approx(1.0, rel=1e-6)
    c0, n0 = h.cosine(dev(X[:0]), dev(X), np.eye(4))
    assert c0 == 0.0 and n0[0] == 0.0
    with pytest.raises(cvo.CvoError):
        h.cosine(dev(X), dev(X), np.eye(4), norms2=(-1.0, 1.0))


@pytest.mark.parametrize("cm", [0.0, 3.0])
def test_cosine_lengthscale_derivative_matches_oracle(cm):
    """cvo_cosine_dell against the oracle's cosine_ell (Eq. indicator and its
    l-derivative), dense and with a cutoff, and through cosine_fn's autograd."""
    p = scenes.room_pair()
    sel = np.random.Generator(np.random.PCG64(41)).permutation(p.n)[:1500]
    X, Z, FX, FZ = p.X[sel], p.Z[sel], p.FX[sel], p.FZ[sel]
    T = p.T_true
    ell = 0.12
    with cvo.CVO(blocks=p.blocks, ell=ell, cutoff_mult=cm) as h:
        c, d = cvo.cvo_cosine_dell(h.h, dev(X), dev(Z), T, dev(FX), dev(FZ))
        lt = torch.tensor(ell, dtype=torch.float64, requires_grad=True)
        ct = cvo.cosine_fn(h, dev(X), dev(Z), T, dev(FX), dev(FZ), ell=lt)
        ct.backward()
    co, do = oracle.cosine_ell(X, Z, T, FX, FZ, ell=ell, blocks=p.blocks, cutoff_mult=cm)
    assert c == pytest.approx(co, rel=1e-5)
    # with a cutoff, a pair whose FP32 and FP64 distance tests disagree moves
    # dF/dl by at most w d^2 / l^3 <= e^-4.5 9 / l: none lie that close here
    if cm > 0:
        for A, B, TT in ((X, Z, T), (X, X, np.eye(4)), (Z, Z, np.eye(4))):
            rc2 = (cm * ell) ** 2
            assert oracle.count_band(A, B, TT, rc2 * (1 - 1e-5), rc2 * (1 + 1e-5)) == 0
    assert d == pytest.approx(do, rel=1e-4)
    assert ct.item() == pytest.approx(c, rel=1e-12) and lt.grad.item() == pytest.approx(d, rel=1e-12)
