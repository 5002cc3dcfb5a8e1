"""FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never does, and this package
never imports the CUDA library.  The arithmetic lives in ``cvo_oracle.c``
(plain C, double precision, brute force over all point pairs, OpenMP over the
points of X); this module only marshals numpy arrays into it.

Pinned against the mathematics (tests/test_oracle_pins.py): the inner product
by quadrature of the Gaussian convolution identity and by the explicit tensor
product of Eq. (tensor_product); symmetry, rigid invariance, Cauchy-Schwarz,
the Remark of Sec. III-C, the gradient and second derivative by central finite
differences on se(3), the SE(3) exponential by the matrix exponential.
The step rule, its trust region and the left-composed update (a reading: the
paper names a step size without a rule and cites gradient ascent on the Lie
group) by closed-form Newton iterates on problems with a one-variable
objective along the ascent direction, and by the equivariance of the whole
registration under a common rigid motion (tests/test_oracle_step_rule.py).
The annealing trigger and the stopping rule (readings of Sec. IV) by
closed-form annealed trajectories of the same one-variable problems
(tests/test_oracle_anneal_pins.py); the registration's end point by recovery
of a known transform.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cvo_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libcvo_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_BLOCKS = 4
TRACE_STRIDE = 22
KIND = {"se": 0, "dot": 1}


class _Kernel(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_double), ("sigma", ctypes.c_double), ("cutoff_mult", ctypes.c_double),
                ("n_blocks", ctypes.c_int), ("dim", ctypes.c_int * MAX_BLOCKS),
                ("kind", ctypes.c_int * MAX_BLOCKS), ("scale", ctypes.c_double * MAX_BLOCKS),
                ("sigk", ctypes.c_double * MAX_BLOCKS), ("feat_cutoff_mult", ctypes.c_double)]


class _Cloud(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("xyz", ctypes.c_void_p), ("feat", ctypes.c_void_p)]


class _Reg(ctypes.Structure):
    _fields_ = [("ell_init", ctypes.c_double), ("ell_min", ctypes.c_double), ("decay", ctypes.c_double),
                ("indicator_tol", ctypes.c_double), ("max_iters", ctypes.c_int), ("anneal", ctypes.c_int),
                ("step_tol_rot", ctypes.c_double), ("step_tol_trans", ctypes.c_double),
                ("max_step_rot", ctypes.c_double), ("max_step_trans", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("ell_final", ctypes.c_double),
                ("F", ctypes.c_double), ("i_theta", ctypes.c_double), ("last_step_rot", ctypes.c_double),
                ("last_step_trans", ctypes.c_double), ("pairs_total", ctypes.c_longlong)]


def build(force: bool = False) -> str:
    """Compile cvo_oracle.c into a shared library (gcc, -O2, OpenMP, IEEE math)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_eval.restype = ctypes.c_int
        lib.orc_register.restype = ctypes.c_int
        lib.orc_se3_log.restype = ctypes.c_int
        lib.orc_count_band.restype = ctypes.c_longlong
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _kernel(blocks, ell, cutoff_mult, sigma, feat_cutoff_mult=0.0):
    k = _Kernel()
    k.ell = float(ell)
    k.sigma = float(sigma)
    k.cutoff_mult = float(cutoff_mult)
    k.feat_cutoff_mult = float(feat_cutoff_mult)
    k.n_blocks = len(blocks)
    if len(blocks) > MAX_BLOCKS:
        raise ValueError("at most 4 feature blocks")
    for b, (kind, dim, scale, sig) in enumerate(blocks):
        k.dim[b] = int(dim)
        k.kind[b] = KIND[kind]
        k.scale[b] = float(scale)
        k.sigk[b] = float(sig)
    return k


def _cloud(P, F, keep):
    P = _f64(P).reshape(-1, 3)
    keep.append(P)
    c = _Cloud()
    c.n = P.shape[0]
    c.xyz = P.ctypes.data
    if F is not None and np.asarray(F).size > 0:
        F = _f64(F).reshape(P.shape[0], -1)
        keep.append(F)
        c.feat = F.ctypes.data
    else:
        c.feat = None
    return c


def evaluate(X, Z, T, *, FX=None, FZ=None, blocks=(), ell, cutoff_mult=0.0, sigma=1.0,
             direction=None, nthreads=0, feat_cutoff_mult=0.0):
    """Brute-force F, its se(3) gradient (omega, v) and, when ``direction`` is
    given, the second derivative of t -> F(exp(t direction^) T) at t = 0.
    ``gscale`` is the sum of the norms of the gradient's per-pair terms.
    Inputs are upcast exactly to float64.  Returns a dict."""
    lib = _load()
    keep = []
    cx = _cloud(X, FX, keep)
    cz = _cloud(Z, FZ, keep)
    k = _kernel(list(blocks), ell, cutoff_mult, sigma, feat_cutoff_mult)
    Tm = _f64(T).reshape(4, 4)
    out = np.zeros(9)
    npairs = ctypes.c_longlong(0)
    d = None
    if direction is not None:
        d = _f64(direction).reshape(6)
    rc = lib.orc_eval(ctypes.byref(k), ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data_as(ctypes.c_void_p),
                      d.ctypes.data_as(ctypes.c_void_p) if d is not None else None,
                      out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(npairs), int(nthreads))
    if rc != 0:
        raise ValueError("orc_eval: invalid argument")
    return dict(F=out[0], g=out[1:7].copy(), Fpp=out[7], gscale=out[8], npairs=int(npairs.value))


def indicator(X, Z, T, **kw):
    """Eq. (indicator_actual): F / sqrt(|X| |Z|)."""
    n, m = np.asarray(X).reshape(-1, 3).shape[0], np.asarray(Z).reshape(-1, 3).shape[0]
    if n == 0 or m == 0:
        return 0.0
    return evaluate(X, Z, T, **kw)["F"] / np.sqrt(float(n) * float(m))


def cosine(X, Z, T, FX=None, FZ=None, **kw):
    """Eq. (indicator): the cosine of the angle between f_X and the moved f_Z,
    <f_X, f_Z'> / (|f_X| |f_Z'|); the norms are the same double sum of each
    cloud with itself at the identity (a rigid motion preserves the norm)."""
    n, m = np.asarray(X).reshape(-1, 3).shape[0], np.asarray(Z).reshape(-1, 3).shape[0]
    if n == 0 or m == 0:
        return 0.0
    I = np.eye(4)
    fxx = evaluate(X, X, I, FX=FX, FZ=FX, **kw)["F"]
    fzz = evaluate(Z, Z, I, FX=FZ, FZ=FZ, **kw)["F"]
    return evaluate(X, Z, T, FX=FX, FZ=FZ, **kw)["F"] / np.sqrt(fxx * fzz)


def count_band(X, Z, T, lo, hi):
    """Pairs whose squared distance lies in [lo, hi] (cutoff-boundary census)."""
    lib = _load()
    keep = []
    cx = _cloud(X, None, keep)
    cz = _cloud(Z, None, keep)
    Tm = _f64(T).reshape(4, 4)
    return int(lib.orc_count_band(ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_double(lo), ctypes.c_double(hi)))


def se3_exp(xi):
    lib = _load()
    xi = _f64(xi).reshape(6)
    T = np.zeros((4, 4))
    lib.orc_se3_exp(xi.ctypes.data_as(ctypes.c_void_p), T.ctypes.data_as(ctypes.c_void_p))
    return T


def se3_log(T):
    lib = _load()
    T = _f64(T).reshape(4, 4)
    xi = np.zeros(6)
    if lib.orc_se3_log(T.ctypes.data_as(ctypes.c_void_p), xi.ctypes.data_as(ctypes.c_void_p)) != 0:
        raise ValueError("se3_log: rotation angle too close to pi")
    return xi


def register(X, Z, T_init, *, FX=None, FZ=None, blocks=(), ell, ell_min=None, cutoff_mult=0.0, sigma=1.0,
             max_iters=50, anneal=False, decay=0.98, indicator_tol=1e-3, step_tol_rot=1e-5,
             step_tol_trans=1e-5, max_step_rot=0.1, max_step_trans=0.0, replay=None, nthreads=0,
             feat_cutoff_mult=0.0):
    """Registration loop (see cvo_oracle.c).  Returns (T_out, info dict, trace array)."""
    lib = _load()
    keep = []
    cx = _cloud(X, FX, keep)
    cz = _cloud(Z, FZ, keep)
    k = _kernel(list(blocks), ell, cutoff_mult, sigma, feat_cutoff_mult)
    r = _Reg(ell_init=float(ell), ell_min=float(ell if ell_min is None else ell_min), decay=float(decay),
             indicator_tol=float(indicator_tol), max_iters=int(max_iters), anneal=int(bool(anneal)),
             step_tol_rot=float(step_tol_rot), step_tol_trans=float(step_tol_trans),
             max_step_rot=float(max_step_rot), max_step_trans=float(max_step_trans))
    T0 = _f64(T_init).reshape(4, 4)
    Tout = np.zeros((4, 4))
    info = _Info()
    trace = np.zeros((max(int(max_iters), 1), TRACE_STRIDE))
    rp = None
    if replay is not None:
        rp = np.ascontiguousarray(np.asarray(replay, dtype=np.int32).reshape(-1))
        if rp.size < max_iters:
            rp = np.concatenate([rp, np.zeros(max_iters - rp.size, dtype=np.int32)])
    rc = lib.orc_register(ctypes.byref(k), ctypes.byref(r), ctypes.byref(cx), ctypes.byref(cz),
                          T0.ctypes.data_as(ctypes.c_void_p), Tout.ctypes.data_as(ctypes.c_void_p),
                          ctypes.byref(info), trace.ctypes.data_as(ctypes.c_void_p),
                          rp.ctypes.data_as(ctypes.c_void_p) if rp is not None else None, int(nthreads))
    if rc != 0:
        raise ValueError("orc_register: invalid argument")
    d = dict(iters=info.iters, status=info.status, ell_final=info.ell_final, F=info.F, i_theta=info.i_theta,
             last_step_rot=info.last_step_rot, last_step_trans=info.last_step_trans,
             pairs_total=int(info.pairs_total))
    return Tout, d, trace[: info.iters].copy()


def backward(X, Z, T, *, FX=None, FZ=None, blocks=(), ell, cutoff_mult=0.0, sigma=1.0, nthreads=0,
             feat_cutoff_mult=0.0):
    """Gradients of F with respect to X, Z (float64, (N,3), (M,3)), the
    features (N,D), (M,D) and the lengthscale, for the pairs inside the
    cutoff (see cvo_oracle.c).  Returns a dict."""
    lib = _load()
    lib.orc_backward.restype = ctypes.c_int
    keep = []
    cx = _cloud(X, FX, keep)
    cz = _cloud(Z, FZ, keep)
    k = _kernel(list(blocks), ell, cutoff_mult, sigma, feat_cutoff_mult)
    D = sum(int(b[1]) for b in blocks)
    Tm = _f64(T).reshape(4, 4)
    dX = np.zeros((cx.n, 3))
    dZ = np.zeros((cz.n, 3))
    dFX = np.zeros((cx.n, D))
    dFZ = np.zeros((cz.n, D))
    dell = ctypes.c_double(0.0)
    vp = ctypes.c_void_p
    rc = lib.orc_backward(ctypes.byref(k), ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data_as(vp),
                          dX.ctypes.data_as(vp), dFX.ctypes.data_as(vp) if D else None, dZ.ctypes.data_as(vp),
                          dFZ.ctypes.data_as(vp) if D else None, ctypes.byref(dell), int(nthreads))
    if rc != 0:
        raise ValueError("orc_backward: invalid argument")
    return dict(dX=dX, dZ=dZ, dFX=dFX, dFZ=dFZ, dell=dell.value)


def register_sequence(frames, ell_first, T_first=None, *, ell, **kw):
    """Frame-to-frame odometry (Sec. IV, V-A) with the oracle's registration:
    frame k+1 onto frame k, the first pair from T_first (identity) at
    lengthscale ell_first, each later pair from the previous relative motion
    at ell.  Returns (T_rel list, T_abs list, infos)."""
    T_rel, infos = [], []
    T_abs = [np.eye(4)]
    for k in range(len(frames) - 1):
        (X, FX), (Z, FZ) = frames[k], frames[k + 1]
        init = (np.eye(4) if T_first is None else np.asarray(T_first, np.float64)) if k == 0 else T_rel[-1]
        l0 = ell_first if k == 0 else ell
        T, info, _ = register(X, Z, init, FX=FX, FZ=FZ, ell=l0, **kw)
        T_rel.append(T)
        infos.append(info)
        T_abs.append(T_abs[-1] @ T)
    return T_rel, T_abs, infos


def cosine_ell(X, Z, T, FX=None, FZ=None, *, ell, **kw):
    """The exact indicator of Eq. (indicator) as a function of the
    lengthscale, and its derivative: cos(l) = F_XZ / sqrt(F_XX F_ZZ), the
    norms the double sum of each cloud with itself at the identity, and
        dcos/dl = cos (F'_XZ / F_XZ - (F'_XX / F_XX + F'_ZZ / F_ZZ) / 2)
    with F' = dF/dl of each sum (orc_backward's dell, the pair set held
    fixed).  Returns (cos, dcos/dl); an empty cloud gives (0, 0)."""
    n, m = np.asarray(X).reshape(-1, 3).shape[0], np.asarray(Z).reshape(-1, 3).shape[0]
    if n == 0 or m == 0:
        return 0.0, 0.0
    I = np.eye(4)
    terms = []
    for A, B, FA, FB, TT in ((X, Z, FX, FZ, T), (X, X, FX, FX, I), (Z, Z, FZ, FZ, I)):
        F = evaluate(A, B, TT, FX=FA, FZ=FB, ell=ell, **kw)["F"]
        dF = backward(A, B, TT, FX=FA, FZ=FB, ell=ell, **kw)["dell"]
        terms.append((F, dF))
    (fxz, dxz), (fxx, dxx), (fzz, dzz) = terms
    c = fxz / np.sqrt(fxx * fzz)
    return c, c * (dxz / fxz - 0.5 * (dxx / fxx + dzz / fzz))

