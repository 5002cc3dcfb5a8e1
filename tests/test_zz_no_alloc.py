"""The allocation-free entry point (cvo_evaluate_dense_noalloc) agrees with the
ordinary cvo_evaluate on two calls in a row.

Some callers may not allocate device memory while they run (a real-time loop
with a budget fixed at start-up, a plugin inside an application that owns the
GPU's memory pool); this entry point serves them from a fixed array inside the
library.  It is called here through the C ABI with device inputs and a device
output buffer, and compared with the handle-based call within the tolerances
of the parity tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu


def _fn():
    lib = cvo.load_library()
    fn = lib.cvo_evaluate_dense_noalloc
    P = ctypes.POINTER
    fn.argtypes = [P(cvo.Params), ctypes.c_void_p, P(cvo.Cloud), P(cvo.Cloud), ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _cloud(xyz, feat):
    c = cvo.Cloud()
    c.xyz = xyz.data_ptr()
    c.n = xyz.shape[0]
    c.feat = feat.data_ptr() if feat is not None else None
    c.feat_dtype = 1 if (feat is not None and feat.dtype == torch.bfloat16) else 0
    c.on_device = 1
    return c


def noalloc_eval(params, X, Z, FX, FZ, T, out=None):
    """One call through the C ABI; out: a device buffer of sizeof(cvo_eval)
    bytes for the results (one is made when None)."""
    fn = _fn()
    if out is None:
        out = torch.zeros(ctypes.sizeof(cvo.Eval), dtype=torch.uint8, device="cuda")
    cx, cz = _cloud(X, FX), _cloud(Z, FZ)
    Tm = np.ascontiguousarray(T, dtype=np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data,
            ctypes.c_void_p(out.data_ptr()))
    if rc < 0:
        raise cvo.CvoError(rc, cvo.cvo_last_error())
    torch.cuda.synchronize()
    e = cvo.Eval.from_buffer_copy(out.cpu().numpy().tobytes())
    return dict(F=e.F, grad=np.array(e.grad[:]), hess=np.array(e.hess[:]).reshape(6, 6), i_theta=e.i_theta,
                pairs=e.pairs)


def _close(a, b, gterms):
    """The parity tests' tolerances: F and i_theta 1e-5 relative; gradient
    1e-4 |g| + 1e-7 G (G: sum of the magnitudes of the gradient's per-pair
    terms, the FP32 rounding floor); Hessian 1e-4 of its largest entry."""
    assert a["F"] == pytest.approx(b["F"], rel=1e-5)
    assert a["i_theta"] == pytest.approx(b["i_theta"], rel=1e-5)
    gtol = 1e-4 * np.linalg.norm(b["grad"]) + 1e-7 * gterms
    assert np.abs(a["grad"] - b["grad"]).max() <= gtol
    assert np.abs(a["hess"] - b["hess"]).max() <= 1e-4 * np.abs(b["hess"]).max()
    assert a["pairs"] == b["pairs"]


def test_noalloc_matches_evaluate_on_two_calls_in_a_row():
    r = np.random.Generator(np.random.PCG64(5))
    cases = []
    p = scenes.cube_pair(n=1500)
    cases.append((p, np.eye(4)))
    q = scenes.cube_pair(n=1100, seed=4242)
    ang = 0.03
    T = np.eye(4)
    T[:3, :3] = scenes.quat_rotation(r.normal(size=3), ang)
    T[:3, 3] = [0.02, -0.01, 0.03]
    cases.append((q, T))
    for pair, T in cases:
        kw = dict(blocks=pair.blocks, ell=0.1, cutoff_mult=0.0, sigma=1.2)
        X, Z = torch.tensor(pair.X, device="cuda"), torch.tensor(pair.Z, device="cuda")
        FX, FZ = torch.tensor(pair.FX, device="cuda"), torch.tensor(pair.FZ, device="cuda")
        got = noalloc_eval(cvo.make_params(**kw), X, Z, FX, FZ, T)
        with cvo.CVO(**kw) as h:
            ref = h.evaluate(X, Z, T, FX, FZ)
        gterms = oracle.evaluate(pair.X, pair.Z, T, FX=pair.FX, FZ=pair.FZ, **kw)["gscale"]
        _close(got, ref, gterms)


def test_noalloc_rejects_requests_beyond_its_limits():
    X = torch.zeros((16385, 3), device="cuda")
    Z = torch.zeros((10, 3), device="cuda")
    with pytest.raises(cvo.CvoError) as e:
        noalloc_eval(cvo.make_params(ell=0.1, cutoff_mult=0.0), X, Z, None, None, np.eye(4))
    assert e.value.status == cvo.Status.ERR_INVALID_ARG and "16384" in str(e.value)
    with pytest.raises(cvo.CvoError) as e:
        noalloc_eval(cvo.make_params(ell=0.1, cutoff_mult=3.0), Z, Z, None, None, np.eye(4))
    assert "dense" in str(e.value)


def test_noalloc_with_feature_cutoff_matches_oracle():
    """The feature-space cutoff reaches the allocation-free entry too: its F and
    pair count follow the oracle with the same cutoff (colours quantised to
    1/8, so no squared colour distance lies near the cutoff radius)."""
    p = scenes.cube_pair(n=1300, seed=61)
    F = (np.round(p.FX * 8.0) / 8.0).astype(np.float32)
    kw = dict(blocks=p.blocks, ell=0.1, cutoff_mult=0.0)
    T = np.eye(4)
    X, Z = torch.tensor(p.X, device="cuda"), torch.tensor(p.Z, device="cuda")
    Fd = torch.tensor(F, device="cuda")
    got = noalloc_eval(cvo.make_params(feat_cutoff_mult=1.6, **kw), X, Z, Fd, Fd, T)
    ref = oracle.evaluate(p.X, p.Z, T, FX=F, FZ=F, feat_cutoff_mult=1.6, **kw)
    full = oracle.evaluate(p.X, p.Z, T, FX=F, FZ=F, **kw)
    assert ref["npairs"] < full["npairs"]
    assert got["F"] == pytest.approx(ref["F"], rel=1e-5)
    assert got["pairs"] == ref["npairs"]


def test_noalloc_bfloat16_features_match_evaluate():
    """Features stored in bfloat16 take the same path as in cvo_evaluate."""
    p = scenes.cube_pair(n=1200, seed=77)
    kw = dict(blocks=p.blocks, ell=0.1, cutoff_mult=0.0)
    T = np.eye(4)
    T[:3, 3] = [0.01, 0.02, -0.015]
    X, Z = torch.tensor(p.X, device="cuda"), torch.tensor(p.Z, device="cuda")
    FX = torch.tensor(p.FX, device="cuda").to(torch.bfloat16)
    FZ = torch.tensor(p.FZ, device="cuda").to(torch.bfloat16)
    got = noalloc_eval(cvo.make_params(**kw), X, Z, FX, FZ, T)
    with cvo.CVO(**kw) as h:
        ref = h.evaluate(X, Z, T, FX, FZ)
    FXo, FZo = scenes.bf16_round(p.FX), scenes.bf16_round(p.FZ)
    gterms = oracle.evaluate(p.X, p.Z, T, FX=FXo, FZ=FZo, **kw)["gscale"]
    _close(got, ref, gterms)


def test_noalloc_allocates_nothing_after_the_first_call():
    """The promise of the entry point: once a first call has run on the
    device (which, under lazy module loading, may load the library's device
    code and its fixed array), a further call changes neither PyTorch's
    allocated bytes nor the device's free memory."""
    p = scenes.cube_pair(n=900, seed=78)
    kw = dict(blocks=p.blocks, ell=0.1, cutoff_mult=0.0)
    X, Z = torch.tensor(p.X, device="cuda"), torch.tensor(p.Z, device="cuda")
    FX, FZ = torch.tensor(p.FX, device="cuda"), torch.tensor(p.FZ, device="cuda")
    out = torch.zeros(ctypes.sizeof(cvo.Eval), dtype=torch.uint8, device="cuda")
    params = cvo.make_params(**kw)
    first = noalloc_eval(params, X, Z, FX, FZ, np.eye(4), out)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    second = noalloc_eval(params, X, Z, FX, FZ, np.eye(4), out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    assert second["F"] == first["F"] and np.array_equal(second["grad"], first["grad"])


def test_invalid_feature_block_rejected_by_both_entry_points():
    """A non-finite sigma or scale of a squared-exponential block is an
    invalid argument for cvo_create and for the allocation-free entry alike
    (not NaN results with CVO_OK)."""
    X = torch.zeros((8, 3), device="cuda")
    F = torch.zeros((8, 3), device="cuda")
    for bad in ([("se", 3, 0.2, float("nan"))], [("se", 3, float("inf"), 1.0)]):
        with pytest.raises(cvo.CvoError) as e:
            cvo.CVO(blocks=bad, ell=0.1, cutoff_mult=0.0)
        assert e.value.status == cvo.Status.ERR_INVALID_ARG
        with pytest.raises(cvo.CvoError) as e:
            noalloc_eval(cvo.make_params(blocks=bad, ell=0.1, cutoff_mult=0.0), X, X, F, F, np.eye(4))
        assert e.value.status == cvo.Status.ERR_INVALID_ARG and "feature block" in str(e.value)
